"""Planted mistakes in the oracle, each caught by the pins (CPU).

The oracle is only worth trusting if its pins can tell a correct oracle from
a plausibly wrong one.  Each mutation below plants one slip in the C oracle
(a flipped fill rule, a transposed eye rotation, a reversed depth test, a
quadratic disk kernel, the smaller sphere root, a dropped half-texel shift,
swapped principal-point coordinates); in each decision mode at least one pin
of tests/test_oracle_pins.py must then fail, and with the mutation removed
they all pass again.
"""
import pytest

import oracle
from tests import test_oracle_pins as pins


def _pin_checks(decisions):
    checks = [
        ("fill rule golden", lambda: pins.test_top_left_golden()),
        ("snap", lambda: pins.test_snap_matches_fp64_projection(decisions)),
        ("coverage", lambda: pins.test_coverage_matches_fp64_ray_triangle((-0.4, 0.45, 0.3), decisions)),
        ("depth winner", lambda: pins.test_depth_winner_is_nearest(decisions)),
        ("single view", lambda: pins.test_single_view_at_eye_reproduces_image(decisions)),
        ("single view, off-centre", lambda: pins.test_single_view_identity_nonsquare_offcentre(decisions)),
        ("closed-form weights", lambda: pins.test_weights_closed_form(decisions)),
        ("weights vanish outside", lambda: pins.test_weights_vanish_outside_disks(decisions)),
        ("selection brute force", lambda: pins.test_view_selection_matches_fp64_bruteforce(decisions)),
    ]
    if decisions == "fp64":
        checks.append(("fp64 snap", lambda: pins.test_fp64_snap_is_the_rounded_fp64_projection()))
    return checks


def _failing(decisions):
    failed = []
    for name, check in _pin_checks(decisions):
        try:
            check()
        except Exception:  # an assertion, or records missing altogether
            failed.append(name)
    return failed


@pytest.mark.parametrize("decisions", ["fp32", "fp64"])
@pytest.mark.parametrize("mutation", sorted(oracle.MUTATIONS))
def test_each_planted_mistake_fails_a_pin(mutation, decisions):
    try:
        oracle.set_mutation(mutation)
        failed = _failing(decisions)
    finally:
        oracle.set_mutation(None)
    assert failed, "no pin catches %s" % mutation


def test_the_correct_oracle_passes_every_pin():
    for decisions in ("fp32", "fp64"):
        assert _failing(decisions) == []
