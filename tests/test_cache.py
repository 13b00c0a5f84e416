"""The host-side page cache (lf_cache_*, the tile cache of Sec. 4.2.1 with the
per-frame budget of Sec. 7.2), on the CPU through the C ABI: a hand-traced
FIFO sequence, protection of the images a frame wants, the budget, argument
errors, and random frame sequences against a plain restatement of the policy."""
import numpy as np
import pytest

lfm = pytest.importorskip("paper_1810_08860_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def _reference(n_items, capacity, frames):
    """The policy restated: per frame, admit missing wanted items in order (at most
    `budget`), each into a free page or the page of the earliest-admitted item the
    frame does not want."""
    page_of = {}
    item_in = [None] * capacity
    admitted = [None] * capacity
    clock = 0
    out = []
    for wanted, budget in frames:
        want = set(wanted)
        ups = []
        for it in wanted:
            if len(ups) >= budget:
                break
            if it in page_of:
                continue
            free = [p for p in range(capacity) if item_in[p] is None]
            if free:
                page = free[0]
            else:
                cand = [p for p in range(capacity) if item_in[p] not in want]
                if not cand:
                    break
                page = min(cand, key=lambda p: admitted[p])
                del page_of[item_in[page]]
            item_in[page], admitted[page] = it, clock
            clock += 1
            page_of[it] = page
            ups.append((it, page))
        out.append((ups, [page_of.get(i, -1) for i in range(n_items)]))
    return out


def test_fifo_sequence_by_hand():
    c = lfm.PageCache(8, 3)
    assert c.frame([0, 1, 2], 8) == [(0, 0), (1, 1), (2, 2)]
    assert c.frame([3], 8) == [(3, 0)]            # the earliest admitted (0) goes
    assert c.frame([4, 1], 8) == [(4, 2)]         # 1 is wanted: 2 is the earliest other
    p = c.pages()
    assert p[1] == 1 and p[3] == 0 and p[4] == 2 and p[0] == -1 and p[2] == -1
    c.close()


def test_wanted_images_are_never_evicted_and_the_budget_holds():
    c = lfm.PageCache(10, 2)
    assert c.frame([0, 1, 2], 5) == [(0, 0), (1, 1)]   # 2 finds no page: the coarse level covers it
    assert c.frame([5, 6, 7], 1) == [(5, 0)]           # budget 1
    assert (c.pages() >= 0).sum() == 2
    assert c.frame([], 3) == []
    c.close()


def test_argument_errors():
    with pytest.raises(lfm.LFError):
        lfm.PageCache(0, 4)
    c = lfm.PageCache(4, 2)
    with pytest.raises(lfm.LFError):
        c.frame([4], 2)                                # id out of range
    with pytest.raises(lfm.LFError):
        c.frame([-1], 2)
    c.close()


def test_random_frames_match_the_policy():
    rng = np.random.default_rng(1)
    for trial in range(20):
        n, cap = int(rng.integers(2, 40)), int(rng.integers(1, 12))
        frames = []
        for _ in range(30):
            k = int(rng.integers(0, n + 1))
            wanted = rng.permutation(n)[:k].tolist()
            frames.append((wanted, int(rng.integers(0, 8))))
        c = lfm.PageCache(n, cap)
        for (wanted, budget), (ups, pages) in zip(frames, _reference(n, cap, frames)):
            assert c.frame(wanted, budget) == ups
            assert c.pages().tolist() == pages
        c.close()
