/*
 * lf_oracle.c - plain, slow CPU oracle for disk-blended light field rendering
 * with per-view geometry (Overbeck et al., TOG 2018: Sec. 4.1 Eq. 1-2, the
 * linear disk kernel of Sec. 4.1, the two-pass accumulate/normalise scheme of
 * Sec. 4.2 and the intra-image occlusion test of Sec. 4.2.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA renderer
 * never calls it and shares no code with it.
 *
 * What it computes, per eye pixel (i, j) (Eq. 1: one ray query per pixel):
 *   - the eye ray o + t e, e = ((i+1/2-cx)/fx, (j+1/2-cy)/fy, 1) in the eye
 *     frame, and its crossing p of the capture sphere (larger root);
 *   - for every view i whose disk contains p (|p - c_i| < r_i), the disk
 *     weight w_i = max(0, 1 - |p - c_i| / r_i) (linear falloff, Sec. 4.1);
 *   - the view's per-view mesh (G x G grid of depth-displaced vertices in the
 *     view's own camera frame, Sec. 4.5) rasterised into the eye with a
 *     1/256-pixel snapped, int64 edge-function rasteriser (top-left rule),
 *     near-clipped at z_near;
 *   - the intra-view depth test (Sec. 4.2.2): per (pixel, view) the fragment
 *     nearest the eye wins, ties to the lowest triangle id;
 *   - the winner's ray/plane hit projected into source view i and sampled
 *     bilinearly (the continuous sample I_i(s_i, t_i) of Eq. 2);
 *   - Eq. 2: sum_i w_i I_i / sum_i w_i, alpha 1; (0,0,0,0) where sum w = 0.
 *
 * Asymmetric oval disks (Sec. 4.4), when disk extents are given: disk i lies
 * in the plane through its centre c_i normal to view i's optical axis, its u
 * and v axes along the view's image x and y axes; (u, v) is where the eye ray
 * meets that plane (t >= 0), and the oval is the union of four quarter
 * ellipses with semi-axes e_u+, e_u- (for u >= 0, u < 0) and e_v+, e_v-:
 * rho^2 = (u / e_u)^2 + (v / e_v)^2, inside where rho^2 < 1, weight 1 - rho
 * (the linear falloff of Sec. 4.1 along each ray from the centre).  No sphere
 * crossing is involved in this mode.
 *
 * Precision.  Colour, weights, depths and texture coordinates are FP64.  The
 * discrete decisions - whether a vertex lies in front of the near plane, the
 * snapped vertex positions, which triangle wins the depth test, and whether p
 * lies inside a disk - are taken in one of two modes (orc_lightfield.decisions):
 *   ORC_DECIDE_FP64  the definition: the vertex goes to the eye through world
 *       coordinates, X_eye = R_eye^T (R_i X_cam + t_i - t_eye), in FP64 with no
 *       fused operations; the snap is llrint(256 (f x / z + c)) of the FP64
 *       projection; the clip point is interpolated in FP64; the depth winner is
 *       the smallest FP64 depth z = d / (n . e) of the parent triangle's plane
 *       (fragments with n . e = 0 or z <= 0 are dropped); disk membership is
 *       |p - c_i|^2 < r_i^2 in FP64 at the FP64 sphere crossing.
 *   ORC_DECIDE_FP32  the fast renderer's reading: the same decisions in FP32,
 *       with the operation order written below (the pose composition is FP64,
 *       rounded once to FP32), so that a float deciding an integer is decided in
 *       the same precision on both sides and the two can be compared bit for bit.
 * The two modes differ only where a quantity lies within FP32 rounding of a
 * decision boundary; orc_margins measures how close each (pixel, view) is.
 * Build with -ffp-contract=off so no multiply-add is fused behind the code's
 * back; every fused multiply-add below is an explicit fmaf().
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ types */

typedef struct {
  int32_t n_views, W, H, G;
  const double* poses;   /* n x 12: R row-major camera->world, then centre */
  const double* intr;    /* n x 4: fx, fy, cx, cy */
  const uint8_t* rgba;   /* n x H x W x 4 */
  const float* depth;    /* n x G x G, z-depth in the view's frame, row k then column j */
  const float* disk_c;   /* n x 3 world */
  const float* disk_r;   /* n */
  double sphere_c[3];
  double sphere_r;
  float z_near;
  int32_t pad;
  const float* disk_ext; /* n x 4 oval extents (+u, -u, +v, -v) in metres, or NULL: round disks */
  int32_t decisions;     /* ORC_DECIDE_FP32 or ORC_DECIDE_FP64 */
  int32_t pad2;
} orc_lightfield;

enum { ORC_DECIDE_FP32 = 0, ORC_DECIDE_FP64 = 1 };

typedef struct {
  double pose[12];
  double intr[4];
  int32_t W, H;
} orc_eye;

/* One (pixel, view) pair whose FP32 disk test says "inside". */
typedef struct {
  int32_t pixel;     /* index into the caller's pixel list */
  int32_t view;
  int32_t n_cover;   /* (sub-)triangles covering the pixel centre (edge test only) */
  int32_t winner;    /* parent triangle id of the depth-test winner, -1 if none */
  int32_t min_id, max_id;
  uint32_t id_hash;  /* xor of orc_mix32(parent id) over covering triangles */
  int32_t pad;
  double w;          /* FP64 disk weight */
  double s, t;       /* FP64 source coordinates of the winner (pixel-edge units) */
} orc_frag;

enum { ORC_STAT_TRI_KEPT = 0, ORC_STAT_TRI_CLIPPED, ORC_STAT_TRI_FAR, ORC_STAT_TRI_DEGENERATE,
       ORC_STAT_TRI_BEHIND, ORC_STAT_FRAG_COVER, ORC_STAT_FRAG_WIN, ORC_STAT_SRC_BEHIND,
       ORC_STAT_FRAG_OVERFLOW, ORC_N_STATS };

#define ORC_SNAP_LIMIT 536870912.0f /* 2^29 subpixel units: larger snapped values drop the triangle */

/* ------------------------------------------------------------------ helpers */

/* Planted mistakes for the pin tests (0: none).  Each code breaks one step of
   the method the way a plausible slip would, so the tests can show that some
   pin catches it:
     1 fill rule flipped           2 eye rotation transposed
     3 depth test reversed         4 quadratic disk kernel
     5 smaller sphere root         6 bilinear half-texel shift dropped
     7 cx and cy swapped in the eye projection */
static int g_mutation = 0;
void orc_set_mutation(int m) { g_mutation = m; }

uint32_t orc_mix32(uint32_t x) {
  /* murmur3 32-bit finaliser */
  x ^= x >> 16; x *= 0x85EBCA6Bu;
  x ^= x >> 13; x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

/* dot3 in the fixed FP32 order a0*b0 + (a1*b1 + a2*b2), fused as written. */
static float dot3f(const float a[3], const float b[3]) {
  return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

static int64_t floor_div(int64_t a, int64_t b) { /* b > 0 */
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) --q;
  return q;
}

/* The eye as the entry points see it: with mutation 2 its rotation transposed. */
static const orc_eye* orc_eye_used(const orc_eye* eye, orc_eye* tmp) {
  if (g_mutation != 2 || !eye) return eye;
  *tmp = *eye;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) tmp->pose[r * 3 + c] = eye->pose[c * 3 + r];
  return tmp;
}

/* ------------------------------------------------------------------ per-eye, per-view setup */

typedef struct {
  /* FP64 composition: X_eye = M X_cam + m  (M = R_eye^T R_i, m = R_eye^T (t_i - t_eye)) */
  double M[9], m[3];
  float Mf[9], mf[3];
  /* disk in sphere-centred FP32 coordinates for the inside decision */
  float cc[3], r2;
  double c64[3], r64;
  /* oval disk (Sec. 4.4) in the eye frame: plane normal n, axes x, y (columns of
     M), k = n.c', (u0, v0) = (x.c', y.c') with c' the disk centre; reciprocal
     extents (+u, -u) and (+v, -v).  FP32 for the decision, FP64 for the weight. */
  int oval;
  float on[3], ox[3], oy[3], ok, ou0, ov0, oru[2], orv[2];
  double on64[3], ox64[3], oy64[3], ok64, ou064, ov064, oru64[2], orv64[2];
} orc_viewpose;

/* A1: pose composition in FP64, fixed order, no fusion; then one rounding to FP32. */
static void orc_compose(const double* Re_pose, const double* Ri_pose, orc_viewpose* vp) {
  const double* Re = Re_pose;     /* eye R row-major, centre at [9..11] */
  const double* Ri = Ri_pose;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = Re[0 * 3 + r] * Ri[0 * 3 + c];
      s = s + Re[1 * 3 + r] * Ri[1 * 3 + c];
      s = s + Re[2 * 3 + r] * Ri[2 * 3 + c];
      vp->M[r * 3 + c] = s;
    }
  double d[3] = {Ri[9] - Re[9], Ri[10] - Re[10], Ri[11] - Re[11]};
  for (int r = 0; r < 3; ++r) {
    double s = Re[0 * 3 + r] * d[0];
    s = s + Re[1 * 3 + r] * d[1];
    s = s + Re[2 * 3 + r] * d[2];
    vp->m[r] = s;
  }
  for (int k = 0; k < 9; ++k) vp->Mf[k] = (float)vp->M[k];
  for (int k = 0; k < 3; ++k) vp->mf[k] = (float)vp->m[k];
}

/* ------------------------------------------------------------------ per-view mesh */

typedef struct {
  int32_t id;            /* parent triangle id */
  int64_t X[3], Y[3];    /* snapped, oriented so the signed area is positive */
  uint8_t tl[3];         /* edge k (v_k -> v_{k+1}) is top or left */
  uint8_t culled;        /* zero area or off screen: kept only for orc_margins, covers nothing */
  int32_t bx0, by0, bx1, by1; /* pixel-centre bounding box, clamped to the eye */
  float ia, ib, ic;      /* FP32 inverse-depth plane: 1/z = ia ex + ib ey + ic */
  double n64[3], d64;    /* FP64 plane of the parent: n . X = d */
} orc_tri;

typedef struct {
  int built;
  int32_t n_tri;
  orc_tri* tri;
} orc_mesh;

typedef struct {
  float x, y, z;         /* FP32 eye coordinates */
  int in;                /* z >= z_near, in the precision of the decision mode */
  int far;               /* snapped value beyond the 2^29 limit */
  int64_t SX, SY;        /* snapped 1/256-pixel coordinates (valid when in && !far) */
  double X64[3];         /* FP64 eye coordinates, through world coordinates */
} orc_vert;

/* FP64 snap of an eye-space point with z >= z_near: llrint(256 (f x / z + c)),
   round half to even (the default rounding mode). */
static int orc_snap64(double x, double y, double z, const double* K, int64_t* SX, int64_t* SY) {
  const double su = 256.0 * (K[0] * x / z + K[2]);
  const double sv = 256.0 * (K[1] * y / z + K[3]);
  if (!(fabs(su) < 536870912.0) || !(fabs(sv) < 536870912.0)) return 0;
  *SX = llrint(su);
  *SY = llrint(sv);
  return 1;
}

/* Snap an eye-space point (x, y, z) with z >= z_near to 1/256 pixel (FP32 reading). */
static int orc_snap(float x, float y, float z, float fx, float fy, float cx, float cy,
                    int64_t* SX, int64_t* SY) {
  float qx = x / z, qy = y / z;
  float u = fmaf(fx, qx, cx), v = fmaf(fy, qy, cy);
  float su = u * 256.0f, sv = v * 256.0f;
  if (!(fabsf(su) < ORC_SNAP_LIMIT) || !(fabsf(sv) < ORC_SNAP_LIMIT)) return 0;
  *SX = llrintf(su);
  *SY = llrintf(sv);
  return 1;
}

/* Top-left rule in a y-down screen for a positively oriented triangle. */
static int orc_top_left(int64_t ax, int64_t ay, int64_t bx, int64_t by) {
  const int tl = (ay == by && bx > ax) || (by < ay);
  return g_mutation == 1 ? !tl : tl;
}

/* Pixel-centre coverage of an oriented snapped triangle (exact int64). */
int orc_covers(const int64_t X[3], const int64_t Y[3], const uint8_t tl[3], int32_t i, int32_t j) {
  int64_t px = 256 * (int64_t)i + 128, py = 256 * (int64_t)j + 128;
  for (int k = 0; k < 3; ++k) {
    int k1 = (k + 1) % 3;
    int64_t E = (X[k1] - X[k]) * (py - Y[k]) - (Y[k1] - Y[k]) * (px - X[k]);
    if (!(E > 0 || (E == 0 && tl[k]))) return 0;
  }
  return 1;
}

/* Set up one snapped (sub-)triangle; returns 1 if kept. */
static int orc_setup_tri(orc_tri* t, int32_t id, const int64_t sx[3], const int64_t sy[3],
                         int W, int H) {
  int64_t X[3] = {sx[0], sx[1], sx[2]}, Y[3] = {sy[0], sy[1], sy[2]};
  t->id = id;
  t->culled = 1;
  for (int k = 0; k < 3; ++k) { t->X[k] = X[k]; t->Y[k] = Y[k]; }
  int64_t A = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
  if (A == 0) return 0;
  if (A < 0) {
    int64_t tx = X[1], ty = Y[1];
    X[1] = X[2]; Y[1] = Y[2]; X[2] = tx; Y[2] = ty;
  }
  int64_t minx = X[0], maxx = X[0], miny = Y[0], maxy = Y[0];
  for (int k = 1; k < 3; ++k) {
    if (X[k] < minx) minx = X[k];
    if (X[k] > maxx) maxx = X[k];
    if (Y[k] < miny) miny = Y[k];
    if (Y[k] > maxy) maxy = Y[k];
  }
  /* pixel centres 256 i + 128 inside [min, max] */
  int64_t i0 = floor_div(minx - 128 + 255, 256), i1 = floor_div(maxx - 128, 256);
  int64_t j0 = floor_div(miny - 128 + 255, 256), j1 = floor_div(maxy - 128, 256);
  if (i0 < 0) i0 = 0;
  if (j0 < 0) j0 = 0;
  if (i1 > W - 1) i1 = W - 1;
  if (j1 > H - 1) j1 = H - 1;
  for (int k = 0; k < 3; ++k) { t->X[k] = X[k]; t->Y[k] = Y[k]; }
  if (i0 > i1 || j0 > j1) return 0;
  t->culled = 0;
  for (int k = 0; k < 3; ++k) {
    int k1 = (k + 1) % 3;
    t->tl[k] = (uint8_t)orc_top_left(X[k], Y[k], X[k1], Y[k1]);
  }
  t->bx0 = (int32_t)i0; t->bx1 = (int32_t)i1; t->by0 = (int32_t)j0; t->by1 = (int32_t)j1;
  return 1;
}

/* Build the clipped, snapped, set-up triangle list of one view for one eye.
   keep_culled: also keep zero-area and off-screen sub-triangles (flagged
   culled, covering nothing) for orc_margins. */
static int orc_build_mesh(const orc_lightfield* lf, const orc_eye* eye, int view,
                          const orc_viewpose* vp, orc_mesh* mesh, int64_t* stats, int keep_culled) {
  const int G = lf->G, W = eye->W, H = eye->H;
  const int fp64 = lf->decisions == ORC_DECIDE_FP64;
  const double* K = lf->intr + (size_t)view * 4;
  const double* Ri = lf->poses + (size_t)view * 12;
  const double* Re = eye->pose;
  const float* dep = lf->depth + (size_t)view * G * G;
  const float fxe = (float)eye->intr[0], fye = (float)eye->intr[1];
  float cxe = (float)eye->intr[2], cye = (float)eye->intr[3];
  double Ksnap[4] = {eye->intr[0], eye->intr[1], eye->intr[2], eye->intr[3]};
  if (g_mutation == 7) {
    const float tf = cxe; cxe = cye; cye = tf;
    Ksnap[2] = eye->intr[3]; Ksnap[3] = eye->intr[2];
  }
  const float zn = lf->z_near;
  const double zn64 = (double)lf->z_near;
  orc_vert* V = (orc_vert*)malloc(sizeof(orc_vert) * (size_t)G * G);
  float* af = (float*)malloc(sizeof(float) * G);
  float* bf = (float*)malloc(sizeof(float) * G);
  double* a64 = (double*)malloc(sizeof(double) * G);
  double* b64 = (double*)malloc(sizeof(double) * G);
  int64_t cap = 4 * (int64_t)(G - 1) * (G - 1) + 4;
  mesh->tri = (orc_tri*)malloc(sizeof(orc_tri) * (size_t)cap);
  if (!V || !af || !bf || !a64 || !b64 || !mesh->tri) {
    free(V); free(af); free(bf); free(a64); free(b64); free(mesh->tri); mesh->tri = NULL;
    return 0;
  }
  /* Grid vertex (j, k) sits at source pixel-edge coordinates (j W/(G-1), k H/(G-1)). */
  for (int j = 0; j < G; ++j) {
    double s = ((double)j * (double)lf->W) / (double)(G - 1);
    a64[j] = (s - K[2]) / K[0];
    af[j] = (float)a64[j];
    double t = ((double)j * (double)lf->H) / (double)(G - 1);
    b64[j] = (t - K[3]) / K[1];
    bf[j] = (float)b64[j];
  }
  for (int k = 0; k < G; ++k)
    for (int j = 0; j < G; ++j) {
      orc_vert* v = &V[k * G + j];
      float z = dep[k * G + j];
      /* FP32 reading: X_cam = z (a_j, b_k, 1); X_eye = Mf X_cam + mf (fused in the fixed order) */
      float Xc[3] = {z * af[j], z * bf[k], z};
      float e[3];
      for (int r = 0; r < 3; ++r)
        e[r] = fmaf(vp->Mf[r * 3 + 0], Xc[0], fmaf(vp->Mf[r * 3 + 1], Xc[1], fmaf(vp->Mf[r * 3 + 2], Xc[2], vp->mf[r])));
      v->x = e[0]; v->y = e[1]; v->z = e[2];
      /* FP64 definition: X_world = R_i X_cam + t_i, X_eye = R_eye^T (X_world - t_eye), no fusion */
      double z64 = (double)z;
      double X64[3] = {z64 * a64[j], z64 * b64[k], z64};
      double d[3];
      for (int r = 0; r < 3; ++r) {
        double w = Ri[r * 3 + 0] * X64[0] + Ri[r * 3 + 1] * X64[1] + Ri[r * 3 + 2] * X64[2] + Ri[9 + r];
        d[r] = w - Re[9 + r];
      }
      for (int r = 0; r < 3; ++r) v->X64[r] = Re[0 * 3 + r] * d[0] + Re[1 * 3 + r] * d[1] + Re[2 * 3 + r] * d[2];
      v->far = 0;
      if (fp64) {
        v->in = (v->X64[2] >= zn64);
        if (v->in) v->far = !orc_snap64(v->X64[0], v->X64[1], v->X64[2], Ksnap, &v->SX, &v->SY);
      } else {
        v->in = (e[2] >= zn);
        if (v->in) v->far = !orc_snap(e[0], e[1], e[2], fxe, fye, cxe, cye, &v->SX, &v->SY);
      }
    }
  int32_t n = 0;
  for (int k = 0; k < G - 1; ++k)
    for (int j = 0; j < G - 1; ++j)
      for (int half = 0; half < 2; ++half) {
        int32_t id = 2 * (k * (G - 1) + j) + half;
        const orc_vert* tv[3];
        if (half == 0) { tv[0] = &V[k * G + j]; tv[1] = &V[k * G + j + 1]; tv[2] = &V[(k + 1) * G + j]; }
        else { tv[0] = &V[k * G + j + 1]; tv[1] = &V[(k + 1) * G + j + 1]; tv[2] = &V[(k + 1) * G + j]; }
        int n_in = tv[0]->in + tv[1]->in + tv[2]->in;
        if (n_in == 0) { stats[ORC_STAT_TRI_BEHIND]++; continue; }
        /* FP64 plane of the parent through its unsnapped vertices: n . X = d */
        double f1[3], f2[3], n64[3];
        for (int r = 0; r < 3; ++r) { f1[r] = tv[1]->X64[r] - tv[0]->X64[r]; f2[r] = tv[2]->X64[r] - tv[0]->X64[r]; }
        n64[0] = f1[1] * f2[2] - f1[2] * f2[1];
        n64[1] = f1[2] * f2[0] - f1[0] * f2[2];
        n64[2] = f1[0] * f2[1] - f1[1] * f2[0];
        double d64 = n64[0] * tv[0]->X64[0] + n64[1] * tv[0]->X64[1] + n64[2] * tv[0]->X64[2];
        float ia = 0.0f, ib = 0.0f, ic = 0.0f;
        if (!fp64) {
          /* FP32 inverse-depth plane of the parent triangle (original vertex order) */
          float e1[3] = {tv[1]->x - tv[0]->x, tv[1]->y - tv[0]->y, tv[1]->z - tv[0]->z};
          float e2[3] = {tv[2]->x - tv[0]->x, tv[2]->y - tv[0]->y, tv[2]->z - tv[0]->z};
          float nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
          float v0[3] = {tv[0]->x, tv[0]->y, tv[0]->z};
          float dd = dot3f(nn, v0);
          ia = nn[0] / dd; ib = nn[1] / dd; ic = nn[2] / dd;
          if (dd == 0.0f || !isfinite(ia) || !isfinite(ib) || !isfinite(ic)) { stats[ORC_STAT_TRI_DEGENERATE]++; continue; }
        }
        /* Near clip (Sutherland-Hodgman against z >= z_near), then fan. */
        int64_t px[4], py[4];
        int np = 0, far = 0;
        if (n_in == 3) {
          for (int q = 0; q < 3; ++q) { px[q] = tv[q]->SX; py[q] = tv[q]->SY; far |= tv[q]->far; }
          np = 3;
        } else {
          stats[ORC_STAT_TRI_CLIPPED]++;
          for (int q = 0; q < 3; ++q) {
            const orc_vert* a = tv[q];
            const orc_vert* b = tv[(q + 1) % 3];
            if (a->in) { px[np] = a->SX; py[np] = a->SY; far |= a->far; ++np; }
            if (a->in != b->in) {
              int ok;
              if (fp64) {
                double tt = (zn64 - a->X64[2]) / (b->X64[2] - a->X64[2]);
                double ix = a->X64[0] + tt * (b->X64[0] - a->X64[0]);
                double iy = a->X64[1] + tt * (b->X64[1] - a->X64[1]);
                ok = orc_snap64(ix, iy, zn64, Ksnap, &px[np], &py[np]);
              } else {
                float tt = (zn - a->z) / (b->z - a->z);
                float ix = fmaf(tt, b->x - a->x, a->x);
                float iy = fmaf(tt, b->y - a->y, a->y);
                ok = orc_snap(ix, iy, zn, fxe, fye, cxe, cye, &px[np], &py[np]);
              }
              if (!ok) far = 1;
              ++np;
            }
          }
        }
        if (far) { stats[ORC_STAT_TRI_FAR]++; continue; }
        for (int f = 0; f + 2 < np; ++f) {
          int64_t sx[3] = {px[0], px[f + 1], px[f + 2]}, sy[3] = {py[0], py[f + 1], py[f + 2]};
          orc_tri* t = &mesh->tri[n];
          int kept = orc_setup_tri(t, id, sx, sy, W, H);
          if (!kept && !keep_culled) continue;
          t->ia = ia; t->ib = ib; t->ic = ic;
          t->n64[0] = n64[0]; t->n64[1] = n64[1]; t->n64[2] = n64[2]; t->d64 = d64;
          ++n;
          if (kept) stats[ORC_STAT_TRI_KEPT]++;
        }
      }
  mesh->n_tri = n;
  mesh->built = 1;
  free(V); free(af); free(bf); free(a64); free(b64);
  return 1;
}

/* ------------------------------------------------------------------ per-pixel */

typedef struct {
  float ex, ey;          /* FP32 eye-frame ray (z = 1) */
  int has_p32;
  float p32[3];          /* FP32 sphere crossing, sphere-centred */
  double e64[3];
  int has_p64;
  double p64[3];         /* FP64 sphere crossing, world */
} orc_ray;

/* Eye ray and its crossing of the capture sphere (larger root). */
static void orc_pixel_ray(const orc_lightfield* lf, const orc_eye* eye, int32_t i, int32_t j, orc_ray* r) {
  const double* Re = eye->pose;
  /* FP32 decision path */
  float fx = (float)eye->intr[0], fy = (float)eye->intr[1], cx = (float)eye->intr[2], cy = (float)eye->intr[3];
  r->ex = ((float)i + 0.5f - cx) / fx;
  r->ey = ((float)j + 0.5f - cy) / fy;
  float Rf[9];
  for (int k = 0; k < 9; ++k) Rf[k] = (float)Re[k];
  float d[3];
  for (int k = 0; k < 3; ++k) d[k] = fmaf(Rf[k * 3 + 0], r->ex, fmaf(Rf[k * 3 + 1], r->ey, Rf[k * 3 + 2]));
  float o[3];
  for (int k = 0; k < 3; ++k) o[k] = (float)(Re[9 + k] - lf->sphere_c[k]);
  float R2 = (float)(lf->sphere_r * lf->sphere_r);
  float a = dot3f(d, d), b = dot3f(o, d), c = dot3f(o, o) - R2;
  float disc = b * b - a * c;
  r->has_p32 = 0;
  if (disc >= 0.0f) {
    float t = g_mutation == 5 ? (-sqrtf(disc) - b) / a : (sqrtf(disc) - b) / a;
    if (t >= 0.0f) {
      r->has_p32 = 1;
      for (int k = 0; k < 3; ++k) r->p32[k] = fmaf(t, d[k], o[k]);
    }
  }
  /* FP64 value path */
  r->e64[0] = ((double)i + 0.5 - eye->intr[2]) / eye->intr[0];
  r->e64[1] = ((double)j + 0.5 - eye->intr[3]) / eye->intr[1];
  r->e64[2] = 1.0;
  double dw[3], ow[3];
  for (int k = 0; k < 3; ++k) {
    dw[k] = Re[k * 3 + 0] * r->e64[0] + Re[k * 3 + 1] * r->e64[1] + Re[k * 3 + 2];
    ow[k] = Re[9 + k] - lf->sphere_c[k];
  }
  double A = dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2];
  double B = ow[0] * dw[0] + ow[1] * dw[1] + ow[2] * dw[2];
  double C = ow[0] * ow[0] + ow[1] * ow[1] + ow[2] * ow[2] - lf->sphere_r * lf->sphere_r;
  double D = B * B - A * C;
  r->has_p64 = 0;
  if (D >= 0.0) {
    double t = g_mutation == 5 ? (-B - sqrt(D)) / A : (-B + sqrt(D)) / A;
    if (t >= 0.0) {
      r->has_p64 = 1;
      for (int k = 0; k < 3; ++k) r->p64[k] = Re[9 + k] + t * dw[k];
    }
  }
}

/* Oval disk (Sec. 4.4), FP32 decision: rho^2 < 1 where the eye ray meets the
   disk plane at t >= 0.  Fixed order: each dot product with e = (ex, ey, 1) is
   fma(a0, ex, fma(a1, ey, a2)). */
static int orc_inside_oval(const orc_ray* r, const orc_viewpose* vp) {
  const float den = fmaf(vp->on[0], r->ex, fmaf(vp->on[1], r->ey, vp->on[2]));
  if (den == 0.0f) return 0;
  const float t = vp->ok / den;
  if (!(t >= 0.0f)) return 0;
  const float ue = fmaf(vp->ox[0], r->ex, fmaf(vp->ox[1], r->ey, vp->ox[2]));
  const float ve = fmaf(vp->oy[0], r->ex, fmaf(vp->oy[1], r->ey, vp->oy[2]));
  const float u = fmaf(t, ue, -vp->ou0), v = fmaf(t, ve, -vp->ov0);
  const float a = u * (u >= 0.0f ? vp->oru[0] : vp->oru[1]);
  const float b = v * (v >= 0.0f ? vp->orv[0] : vp->orv[1]);
  return fmaf(a, a, b * b) < 1.0f;
}

/* FP64 oval weight 1 - rho at the FP64 ray's plane hit. */
static double orc_weight_oval(const orc_ray* r, const orc_viewpose* vp) {
  const double* e = r->e64;
  const double den = vp->on64[0] * e[0] + vp->on64[1] * e[1] + vp->on64[2] * e[2];
  if (den == 0.0) return 0.0;
  const double t = vp->ok64 / den;
  if (t < 0.0) return 0.0;
  const double u = t * (vp->ox64[0] * e[0] + vp->ox64[1] * e[1] + vp->ox64[2] * e[2]) - vp->ou064;
  const double v = t * (vp->oy64[0] * e[0] + vp->oy64[1] * e[1] + vp->oy64[2] * e[2]) - vp->ov064;
  const double a = u * (u >= 0.0 ? vp->oru64[0] : vp->oru64[1]);
  const double b = v * (v >= 0.0 ? vp->orv64[0] : vp->orv64[1]);
  const double w = 1.0 - sqrt(a * a + b * b);
  return w > 0.0 ? w : 0.0;
}

/* Oval rho^2 in FP64 at the FP64 ray's plane hit (t >= 0); 2 when the ray
   does not meet the plane in front of the eye. */
static double orc_rho2_oval64(const orc_ray* r, const orc_viewpose* vp) {
  const double* e = r->e64;
  const double den = vp->on64[0] * e[0] + vp->on64[1] * e[1] + vp->on64[2] * e[2];
  if (den == 0.0) return 2.0;
  const double t = vp->ok64 / den;
  if (!(t >= 0.0)) return 2.0;
  const double u = t * (vp->ox64[0] * e[0] + vp->ox64[1] * e[1] + vp->ox64[2] * e[2]) - vp->ou064;
  const double v = t * (vp->oy64[0] * e[0] + vp->oy64[1] * e[1] + vp->oy64[2] * e[2]) - vp->ov064;
  const double a = u * (u >= 0.0 ? vp->oru64[0] : vp->oru64[1]);
  const double b = v * (v >= 0.0 ? vp->orv64[0] : vp->orv64[1]);
  return a * a + b * b;
}

/* Disk membership in the decision mode: |p - c_i|^2 < r_i^2 (FP32 with
   sphere-centred coordinates, or FP64 at the FP64 crossing), or the oval's
   rho^2 < 1. */
static int orc_inside(const orc_ray* r, const orc_viewpose* vp, int fp64) {
  if (fp64) {
    if (vp->oval) return orc_rho2_oval64(r, vp) < 1.0;
    if (!r->has_p64) return 0;
    double dx = r->p64[0] - vp->c64[0], dy = r->p64[1] - vp->c64[1], dz = r->p64[2] - vp->c64[2];
    return dx * dx + dy * dy + dz * dz < vp->r64 * vp->r64;
  }
  if (vp->oval) return orc_inside_oval(r, vp);
  if (!r->has_p32) return 0;
  float df[3] = {r->p32[0] - vp->cc[0], r->p32[1] - vp->cc[1], r->p32[2] - vp->cc[2]};
  return dot3f(df, df) < vp->r2;
}

/* FP64 linear disk kernel (Sec. 4.1): 1 at the centre, 0 at the rim. */
static double orc_weight(const orc_ray* r, const orc_viewpose* vp) {
  if (vp->oval) return orc_weight_oval(r, vp);
  if (!r->has_p64) return 0.0;
  double dx = r->p64[0] - vp->c64[0], dy = r->p64[1] - vp->c64[1], dz = r->p64[2] - vp->c64[2];
  double w = g_mutation == 4 ? 1.0 - (dx * dx + dy * dy + dz * dz) / (vp->r64 * vp->r64)
                             : 1.0 - sqrt(dx * dx + dy * dy + dz * dz) / vp->r64;
  return w > 0.0 ? w : 0.0;
}

/* Bilinear sample of view `view` at pixel-edge coordinates (s, t), clamp to edge, RGB / 255. */
static void orc_bilinear(const orc_lightfield* lf, int view, double s, double t, double rgb[3],
                         int32_t ti[4], int32_t tj[4]) {
  double u = s - 0.5, v = t - 0.5;
  if (g_mutation == 6) { u = s; v = t; }
  if (u < -1.0) u = -1.0;
  if (u > (double)lf->W) u = (double)lf->W;
  if (v < -1.0) v = -1.0;
  if (v > (double)lf->H) v = (double)lf->H;
  double fu = floor(u), fv = floor(v);
  double al = u - fu, be = v - fv;
  int i0 = (int)fu, j0 = (int)fv;
  int is[2] = {i0, i0 + 1}, js[2] = {j0, j0 + 1};
  for (int q = 0; q < 2; ++q) {
    if (is[q] < 0) is[q] = 0;
    if (is[q] > lf->W - 1) is[q] = lf->W - 1;
    if (js[q] < 0) js[q] = 0;
    if (js[q] > lf->H - 1) js[q] = lf->H - 1;
  }
  const uint8_t* img = lf->rgba + (size_t)view * lf->W * lf->H * 4;
  double wq[4] = {(1 - al) * (1 - be), al * (1 - be), (1 - al) * be, al * be};
  int qi[4] = {is[0], is[1], is[0], is[1]}, qj[4] = {js[0], js[0], js[1], js[1]};
  rgb[0] = rgb[1] = rgb[2] = 0.0;
  for (int q = 0; q < 4; ++q) {
    const uint8_t* px = img + ((size_t)qj[q] * lf->W + qi[q]) * 4;
    for (int c = 0; c < 3; ++c) rgb[c] += wq[q] * ((double)px[c] / 255.0);
    if (ti) { ti[q] = qi[q]; tj[q] = qj[q]; }
  }
}

/* ------------------------------------------------------------------ driver */

typedef struct {
  const orc_lightfield* lf;
  const orc_eye* eye;
  const orc_viewpose* vps;
  orc_mesh* meshes;
  const int32_t* pixels;
  int64_t n_pixels;
  double* out;
  orc_frag* frags;
  int32_t max_slots;
  int32_t* n_slots;
  uint64_t* texel_bits; /* optional bitset over all views' texels */
  int64_t next;
  int64_t stats[ORC_N_STATS];
  pthread_mutex_t mu;
} orc_job;

static void orc_shade_pixel(orc_job* job, int64_t pidx, int64_t* stats) {
  const orc_lightfield* lf = job->lf;
  const orc_eye* eye = job->eye;
  int32_t i, j;
  if (job->pixels) { i = job->pixels[2 * pidx]; j = job->pixels[2 * pidx + 1]; }
  else { i = (int32_t)(pidx % eye->W); j = (int32_t)(pidx / eye->W); }
  orc_ray ray;
  orc_pixel_ray(lf, eye, i, j, &ray);
  const int fp64 = lf->decisions == ORC_DECIDE_FP64;
  const double* Re = eye->pose;
  double acc[3] = {0, 0, 0}, wsum = 0.0;
  int32_t slots = 0;
  for (int v = 0; v < lf->n_views; ++v) {
    const orc_viewpose* vp = &job->vps[v];
    if (!orc_inside(&ray, vp, fp64)) continue;
    const orc_mesh* mesh = &job->meshes[v];
    int32_t n_cover = 0, winner = -1, min_id = 0x7fffffff, max_id = -1;
    uint32_t hash = 0;
    float best = 0.0f;
    double best_z = 0.0;
    const orc_tri* wt = NULL;
    for (int32_t q = 0; q < mesh->n_tri; ++q) {
      const orc_tri* t = &mesh->tri[q];
      if (t->culled) continue;
      if (i < t->bx0 || i > t->bx1 || j < t->by0 || j > t->by1) continue;
      if (!orc_covers(t->X, t->Y, t->tl, i, j)) continue;
      ++n_cover;
      if (t->id < min_id) min_id = t->id;
      if (t->id > max_id) max_id = t->id;
      hash ^= orc_mix32((uint32_t)t->id);
      /* Intra-view depth test: the nearest fragment wins, ties to the lower id. */
      if (fp64) {
        double ne = t->n64[0] * ray.e64[0] + t->n64[1] * ray.e64[1] + t->n64[2] * ray.e64[2];
        if (ne == 0.0) continue;
        double z = t->d64 / ne;
        const int nearer = g_mutation == 3 ? z > best_z : z < best_z;
        if (z > 0.0 && isfinite(z) && (winner < 0 || nearer || (z == best_z && t->id < winner))) {
          best_z = z; winner = t->id; wt = t;
        }
      } else {
        /* FP32 1/z; the list is in id order, so a tie keeps the earlier (lower) id */
        float iz = fmaf(t->ia, ray.ex, fmaf(t->ib, ray.ey, t->ic));
        const int nearer = g_mutation == 3 ? iz < best : iz > best;
        if (iz > 0.0f && (winner < 0 || nearer)) { best = iz; winner = t->id; wt = t; }
      }
    }
    stats[ORC_STAT_FRAG_COVER] += n_cover;
    double w = orc_weight(&ray, vp);
    double s = NAN, tt = NAN;
    if (wt) {
      stats[ORC_STAT_FRAG_WIN]++;
      /* FP64 ray/plane hit of the winner, X_eye = z e, taken through world
         coordinates into source view v (Eq. 2's I_i(s_i, t_i)). */
      double ne = wt->n64[0] * ray.e64[0] + wt->n64[1] * ray.e64[1] + wt->n64[2] * ray.e64[2];
      double z = wt->d64 / ne;
      const double* Ri = lf->poses + (size_t)v * 12;
      double Xe[3] = {z * ray.e64[0], z * ray.e64[1], z * ray.e64[2]};
      double X[3];
      for (int r = 0; r < 3; ++r)
        X[r] = Re[r * 3 + 0] * Xe[0] + Re[r * 3 + 1] * Xe[1] + Re[r * 3 + 2] * Xe[2] + Re[9 + r] - Ri[9 + r];
      double Xs[3];
      for (int r = 0; r < 3; ++r) Xs[r] = Ri[0 * 3 + r] * X[0] + Ri[1 * 3 + r] * X[1] + Ri[2 * 3 + r] * X[2];
      const double* K = lf->intr + (size_t)v * 4;
      if (Xs[2] > 0.0) {
        s = K[0] * Xs[0] / Xs[2] + K[2];
        tt = K[1] * Xs[1] / Xs[2] + K[3];
        double rgb[3];
        int32_t ti[4], tj[4];
        orc_bilinear(lf, v, s, tt, rgb, ti, tj);
        for (int c = 0; c < 3; ++c) acc[c] += w * rgb[c];
        wsum += w;
        if (job->texel_bits) {
          size_t base = (size_t)v * lf->W * lf->H;
          for (int q = 0; q < 4; ++q) {
            size_t bit = base + (size_t)tj[q] * lf->W + ti[q];
            __atomic_fetch_or(&job->texel_bits[bit >> 6], 1ULL << (bit & 63), __ATOMIC_RELAXED);
          }
        }
      } else {
        stats[ORC_STAT_SRC_BEHIND]++;
      }
    }
    if (job->frags) {
      if (slots < job->max_slots) {
        orc_frag* f = &job->frags[pidx * job->max_slots + slots];
        f->pixel = (int32_t)pidx; f->view = v; f->n_cover = n_cover; f->winner = winner;
        f->min_id = n_cover ? min_id : -1; f->max_id = max_id; f->id_hash = hash; f->pad = 0;
        f->w = w; f->s = s; f->t = tt;
      } else {
        stats[ORC_STAT_FRAG_OVERFLOW]++;
      }
    }
    ++slots;
  }
  if (job->n_slots) job->n_slots[pidx] = slots;
  double* o = job->out + pidx * 4;
  if (wsum > 0.0) {
    o[0] = acc[0] / wsum; o[1] = acc[1] / wsum; o[2] = acc[2] / wsum; o[3] = 1.0;
  } else {
    o[0] = o[1] = o[2] = o[3] = 0.0;
  }
}

static void* orc_worker(void* arg) {
  orc_job* job = (orc_job*)arg;
  int64_t st[ORC_N_STATS];
  memset(st, 0, sizeof(st));
  for (;;) {
    int64_t p0 = __atomic_fetch_add(&job->next, 64, __ATOMIC_RELAXED);
    if (p0 >= job->n_pixels) break;
    int64_t p1 = p0 + 64 < job->n_pixels ? p0 + 64 : job->n_pixels;
    for (int64_t p = p0; p < p1; ++p) orc_shade_pixel(job, p, st);
  }
  pthread_mutex_lock(&job->mu);
  for (int k = 0; k < ORC_N_STATS; ++k) job->stats[k] += st[k];
  pthread_mutex_unlock(&job->mu);
  return NULL;
}

static void orc_run_threads(orc_job* job, int n_threads) {
  job->next = 0;
  if (n_threads <= 1) { orc_worker(job); return; }
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  int started = 0;
  for (int k = 0; k < n_threads; ++k) {
    if (pthread_create(&th[k], NULL, orc_worker, job) != 0) break;
    ++started;
  }
  if (started == 0) orc_worker(job);
  for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
}

static void orc_init_viewposes(const orc_lightfield* lf, const orc_eye* eye, orc_viewpose* vps) {
  for (int v = 0; v < lf->n_views; ++v) {
    orc_viewpose* vp = &vps[v];
    orc_compose(eye->pose, lf->poses + (size_t)v * 12, vp);
    for (int k = 0; k < 3; ++k) {
      vp->cc[k] = (float)((double)lf->disk_c[v * 3 + k] - lf->sphere_c[k]);
      vp->c64[k] = (double)lf->disk_c[v * 3 + k];
    }
    vp->r2 = lf->disk_r[v] * lf->disk_r[v];
    vp->r64 = (double)lf->disk_r[v];
    vp->oval = lf->disk_ext != NULL;
    if (vp->oval) {
      /* axes: the columns of M = R_eye^T R_i; the disk centre in the eye frame in FP64 */
      const double* Re = eye->pose;
      double dc[3], cp[3];
      for (int k = 0; k < 3; ++k) dc[k] = (double)lf->disk_c[v * 3 + k] - Re[9 + k];
      for (int r = 0; r < 3; ++r) {
        double s = Re[0 * 3 + r] * dc[0];
        s = s + Re[1 * 3 + r] * dc[1];
        s = s + Re[2 * 3 + r] * dc[2];
        cp[r] = s;
      }
      for (int k = 0; k < 3; ++k) {
        vp->ox64[k] = vp->M[k * 3 + 0];
        vp->oy64[k] = vp->M[k * 3 + 1];
        vp->on64[k] = vp->M[k * 3 + 2];
        vp->ox[k] = vp->Mf[k * 3 + 0];
        vp->oy[k] = vp->Mf[k * 3 + 1];
        vp->on[k] = vp->Mf[k * 3 + 2];
      }
      vp->ok64 = vp->on64[0] * cp[0] + vp->on64[1] * cp[1] + vp->on64[2] * cp[2];
      vp->ou064 = vp->ox64[0] * cp[0] + vp->ox64[1] * cp[1] + vp->ox64[2] * cp[2];
      vp->ov064 = vp->oy64[0] * cp[0] + vp->oy64[1] * cp[1] + vp->oy64[2] * cp[2];
      vp->ok = (float)vp->ok64;
      vp->ou0 = (float)vp->ou064;
      vp->ov0 = (float)vp->ov064;
      const float* ext = lf->disk_ext + (size_t)v * 4;
      vp->oru64[0] = 1.0 / (double)ext[0];
      vp->oru64[1] = 1.0 / (double)ext[1];
      vp->orv64[0] = 1.0 / (double)ext[2];
      vp->orv64[1] = 1.0 / (double)ext[3];
      for (int k = 0; k < 2; ++k) {
        vp->oru[k] = (float)vp->oru64[k];
        vp->orv[k] = (float)vp->orv64[k];
      }
    }
  }
}

typedef struct {
  const orc_lightfield* lf;
  const orc_eye* eye;
  const int32_t* pixels;
  int64_t n_pixels;
  const orc_viewpose* vps;
  uint8_t* active;
  int64_t next;
} orc_sel_job;

static void* orc_sel_worker(void* arg) {
  orc_sel_job* job = (orc_sel_job*)arg;
  const int nv = job->lf->n_views;
  for (;;) {
    int64_t p0 = __atomic_fetch_add(&job->next, 256, __ATOMIC_RELAXED);
    if (p0 >= job->n_pixels) break;
    int64_t p1 = p0 + 256 < job->n_pixels ? p0 + 256 : job->n_pixels;
    for (int64_t p = p0; p < p1; ++p) {
      int32_t i, j;
      if (job->pixels) { i = job->pixels[2 * p]; j = job->pixels[2 * p + 1]; }
      else { i = (int32_t)(p % job->eye->W); j = (int32_t)(p / job->eye->W); }
      orc_ray ray;
      orc_pixel_ray(job->lf, job->eye, i, j, &ray);
      for (int v = 0; v < nv; ++v)
        if (!job->active[v] && orc_inside(&ray, &job->vps[v], job->lf->decisions == ORC_DECIDE_FP64))
          __atomic_store_n(&job->active[v], (uint8_t)1, __ATOMIC_RELAXED);
    }
  }
  return NULL;
}

/*
 * View selection: active[v] = 1 iff some listed pixel's sphere crossing lies
 * inside disk v (the set of views Eq. 2 sums over with nonzero weight).
 * pixels: NULL for every pixel of the eye, else n_pixels (i, j) pairs.
 */
int orc_select_views(const orc_lightfield* lf, const orc_eye* eye, const int32_t* pixels,
                     int64_t n_pixels, uint8_t* active, int n_threads) {
  orc_eye eye_tmp;
  eye = orc_eye_used(eye, &eye_tmp);
  orc_viewpose* vps = (orc_viewpose*)calloc((size_t)lf->n_views, sizeof(orc_viewpose));
  if (!vps) return 1;
  orc_init_viewposes(lf, eye, vps);
  memset(active, 0, (size_t)lf->n_views);
  orc_sel_job job = {lf, eye, pixels, pixels ? n_pixels : (int64_t)eye->W * eye->H, vps, active, 0};
  if (n_threads <= 1) orc_sel_worker(&job);
  else {
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    int started = 0;
    for (int k = 0; k < n_threads; ++k) {
      if (pthread_create(&th[k], NULL, orc_sel_worker, &job) != 0) break;
      ++started;
    }
    if (started == 0) orc_sel_worker(&job);
    for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
  }
  free(vps);
  return 0;
}

/*
 * Render listed pixels of one eye (Eq. 1-2).
 *   pixels     NULL for every pixel in row-major order, else n_pixels (i, j) pairs
 *   out_rgba   n_pixels x 4 doubles
 *   frags      optional n_pixels x max_slots records, n_slots[p] = records for pixel p
 *   texel_bits optional bitset of n_views*W*H bits marking the texels read by
 *              winners' bilinear footprints (caller zeroes it)
 *   stats      optional ORC_N_STATS counters
 * Returns 0 on success, 1 on allocation failure, 2 on bad arguments.
 */
int orc_render(const orc_lightfield* lf, const orc_eye* eye, const int32_t* pixels, int64_t n_pixels,
               double* out_rgba, orc_frag* frags, int32_t max_slots, int32_t* n_slots,
               uint64_t* texel_bits, int64_t* stats, int n_threads) {
  orc_eye eye_tmp;
  eye = orc_eye_used(eye, &eye_tmp);
  if (!lf || !eye || !out_rgba || lf->n_views < 0 || lf->G < 2 || eye->W <= 0 || eye->H <= 0) return 2;
  if (!pixels) n_pixels = (int64_t)eye->W * eye->H;
  orc_viewpose* vps = (orc_viewpose*)calloc((size_t)lf->n_views + 1, sizeof(orc_viewpose));
  orc_mesh* meshes = (orc_mesh*)calloc((size_t)lf->n_views + 1, sizeof(orc_mesh));
  uint8_t* need = (uint8_t*)calloc((size_t)lf->n_views + 1, 1);
  if (!vps || !meshes || !need) { free(vps); free(meshes); free(need); return 1; }
  orc_init_viewposes(lf, eye, vps);
  /* Only views whose disk holds some listed pixel contribute (Eq. 2 terms with w > 0). */
  orc_sel_job sj = {lf, eye, pixels, n_pixels, vps, need, 0};
  orc_sel_worker(&sj);
  orc_job job;
  memset(&job, 0, sizeof(job));
  int rc = 0;
  for (int v = 0; v < lf->n_views; ++v)
    if (need[v] && !orc_build_mesh(lf, eye, v, &vps[v], &meshes[v], job.stats, 0)) { rc = 1; break; }
  if (rc == 0) {
    job.lf = lf; job.eye = eye; job.vps = vps; job.meshes = meshes; job.pixels = pixels;
    job.n_pixels = n_pixels; job.out = out_rgba; job.frags = frags; job.max_slots = max_slots;
    job.n_slots = n_slots; job.texel_bits = texel_bits;
    pthread_mutex_init(&job.mu, NULL);
    orc_run_threads(&job, n_threads);
    pthread_mutex_destroy(&job.mu);
    if (stats) memcpy(stats, job.stats, sizeof(job.stats));
  }
  for (int v = 0; v < lf->n_views; ++v) free(meshes[v].tri);
  free(vps); free(meshes); free(need);
  return rc;
}

/*
 * All covering fragments of one (pixel, view): parent ids, FP32 inverse depth
 * (the depth-test key) and FP64 eye-space depth of the ray/plane hit.
 * Returns the number written (<= cap), or -1 on error.
 */
int orc_pixel_fragments(const orc_lightfield* lf, const orc_eye* eye, int32_t i, int32_t j, int32_t view,
                        int32_t* ids, float* inv_z, double* z64, int32_t cap) {
  orc_eye eye_tmp;
  eye = orc_eye_used(eye, &eye_tmp);
  if (view < 0 || view >= lf->n_views) return -1;
  orc_viewpose vp;
  memset(&vp, 0, sizeof(vp));
  orc_compose(eye->pose, lf->poses + (size_t)view * 12, &vp);
  orc_mesh mesh;
  memset(&mesh, 0, sizeof(mesh));
  int64_t st[ORC_N_STATS];
  memset(st, 0, sizeof(st));
  if (!orc_build_mesh(lf, eye, view, &vp, &mesh, st, 0)) return -1;
  orc_ray ray;
  orc_pixel_ray(lf, eye, i, j, &ray);
  int n = 0;
  for (int32_t q = 0; q < mesh.n_tri; ++q) {
    const orc_tri* t = &mesh.tri[q];
    if (i < t->bx0 || i > t->bx1 || j < t->by0 || j > t->by1) continue;
    if (!orc_covers(t->X, t->Y, t->tl, i, j)) continue;
    if (n < cap) {
      ids[n] = t->id;
      double ne = t->n64[0] * ray.e64[0] + t->n64[1] * ray.e64[1] + t->n64[2] * ray.e64[2];
      z64[n] = t->d64 / ne;
      inv_z[n] = lf->decisions == ORC_DECIDE_FP64 ? (float)(ne / t->d64)
                                                  : fmaf(t->ia, ray.ex, fmaf(t->ib, ray.ey, t->ic));
    }
    ++n;
  }
  free(mesh.tri);
  return n < cap ? n : cap;
}

/*
 * Snapped, clipped, oriented triangles of one view for one eye (for pins).
 * Writes up to cap rows of: id, X0, Y0, X1, Y1, X2, Y2 (int64).  Returns the
 * count, or -1 on error.
 */
int64_t orc_view_triangles(const orc_lightfield* lf, const orc_eye* eye, int32_t view,
                           int64_t* rows, int64_t cap, int64_t* stats) {
  orc_eye eye_tmp;
  eye = orc_eye_used(eye, &eye_tmp);
  if (view < 0 || view >= lf->n_views) return -1;
  orc_viewpose vp;
  memset(&vp, 0, sizeof(vp));
  orc_compose(eye->pose, lf->poses + (size_t)view * 12, &vp);
  orc_mesh mesh;
  memset(&mesh, 0, sizeof(mesh));
  int64_t st[ORC_N_STATS];
  memset(st, 0, sizeof(st));
  if (!orc_build_mesh(lf, eye, view, &vp, &mesh, st, 0)) return -1;
  int64_t n = mesh.n_tri < cap ? mesh.n_tri : cap;
  for (int64_t q = 0; q < n; ++q) {
    const orc_tri* t = &mesh.tri[q];
    int64_t* r = rows + q * 7;
    r[0] = t->id;
    for (int k = 0; k < 3; ++k) { r[1 + 2 * k] = t->X[k]; r[2 + 2 * k] = t->Y[k]; }
  }
  if (stats) memcpy(stats, st, sizeof(st));
  free(mesh.tri);
  return n;
}

/*
 * Coverage of pixel (i, j) by the snapped triangle (sx, sy) in any winding:
 * orient, classify edges, test (for pins).  Returns -1 for zero area.
 */
int orc_cover_raw(const int64_t sx[3], const int64_t sy[3], int32_t i, int32_t j) {
  orc_tri t;
  memset(&t, 0, sizeof(t));
  int64_t X[3] = {sx[0], sx[1], sx[2]}, Y[3] = {sy[0], sy[1], sy[2]};
  int64_t A = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
  if (A == 0) return -1;
  if (A < 0) {
    int64_t tx = X[1], ty = Y[1];
    X[1] = X[2]; Y[1] = Y[2]; X[2] = tx; Y[2] = ty;
  }
  uint8_t tl[3];
  for (int k = 0; k < 3; ++k) {
    int k1 = (k + 1) % 3;
    tl[k] = (uint8_t)orc_top_left(X[k], Y[k], X[k1], Y[k1]);
  }
  return orc_covers(X, Y, tl, i, j);
}

/* Distance in subpixels from point (px, py) to segment a-b (exact inputs, FP64). */
static double orc_seg_dist(double px, double py, double ax, double ay, double bx, double by) {
  const double dx = bx - ax, dy = by - ay;
  const double L2 = dx * dx + dy * dy;
  double t = L2 > 0.0 ? ((px - ax) * dx + (py - ay) * dy) / L2 : 0.0;
  if (t < 0.0) t = 0.0;
  if (t > 1.0) t = 1.0;
  const double ex = ax + t * dx - px, ey = ay + t * dy - py;
  return sqrt(ex * ex + ey * ey);
}

/*
 * How close each listed (pixel, view) lies to the boundaries of the three
 * decisions, with the meshes and crossings of the light field's decision mode:
 *   out[3k+0]  disk: |p - c| / r - 1 for round disks, rho - 1 for ovals
 *              (negative inside); NaN when the ray has no crossing
 *   out[3k+1]  coverage: distance in subpixels from the pixel centre to the
 *              nearest edge of any snapped sub-triangle of the view - zero-area
 *              ones included - whose snapped box, grown by one pixel, holds
 *              the centre; +inf when there is none
 *   out[3k+2]  depth: (z2 - z1) / z1 for the two nearest covering parent
 *              triangles by FP64 depth (z > 0); +inf with fewer than two
 * pv lists n triples (i, j, view).  A difference between the two decision
 * modes at a (pixel, view) is explained when one of these is within the
 * rounding of FP32.  Returns 0, 1 on allocation failure, 2 on bad arguments.
 */
int orc_margins(const orc_lightfield* lf, const orc_eye* eye, const int32_t* pv, int64_t n, double* out) {
  orc_eye eye_tmp;
  eye = orc_eye_used(eye, &eye_tmp);
  if (!lf || !eye || (!pv && n > 0) || !out) return 2;
  orc_viewpose* vps = (orc_viewpose*)calloc((size_t)lf->n_views + 1, sizeof(orc_viewpose));
  orc_mesh* meshes = (orc_mesh*)calloc((size_t)lf->n_views + 1, sizeof(orc_mesh));
  if (!vps || !meshes) { free(vps); free(meshes); return 1; }
  orc_init_viewposes(lf, eye, vps);
  int rc = 0;
  int64_t st[ORC_N_STATS];
  for (int64_t k = 0; k < n && rc == 0; ++k) {
    const int32_t i = pv[3 * k], j = pv[3 * k + 1], v = pv[3 * k + 2];
    double* o = out + 3 * k;
    if (v < 0 || v >= lf->n_views) { rc = 2; break; }
    orc_ray ray;
    orc_pixel_ray(lf, eye, i, j, &ray);
    const orc_viewpose* vp = &vps[v];
    if (vp->oval) {
      const double r2 = orc_rho2_oval64(&ray, vp);
      o[0] = r2 >= 2.0 ? NAN : sqrt(r2) - 1.0;
    } else if (ray.has_p64) {
      double dx = ray.p64[0] - vp->c64[0], dy = ray.p64[1] - vp->c64[1], dz = ray.p64[2] - vp->c64[2];
      o[0] = sqrt(dx * dx + dy * dy + dz * dz) / vp->r64 - 1.0;
    } else {
      o[0] = NAN;
    }
    if (!meshes[v].built) {
      memset(st, 0, sizeof(st));
      if (!orc_build_mesh(lf, eye, v, vp, &meshes[v], st, 1)) { rc = 1; break; }
    }
    const orc_mesh* m = &meshes[v];
    const double cx = 256.0 * i + 128.0, cy = 256.0 * j + 128.0;
    double edge = INFINITY, z1 = INFINITY, z2 = INFINITY;
    int32_t id1 = -1;
    for (int32_t q = 0; q < m->n_tri; ++q) {
      const orc_tri* t = &m->tri[q];
      int64_t mnx = t->X[0], mxx = t->X[0], mny = t->Y[0], mxy = t->Y[0];
      for (int c = 1; c < 3; ++c) {
        if (t->X[c] < mnx) mnx = t->X[c];
        if (t->X[c] > mxx) mxx = t->X[c];
        if (t->Y[c] < mny) mny = t->Y[c];
        if (t->Y[c] > mxy) mxy = t->Y[c];
      }
      if (cx < (double)mnx - 256.0 || cx > (double)mxx + 256.0 || cy < (double)mny - 256.0 || cy > (double)mxy + 256.0)
        continue;
      for (int c = 0; c < 3; ++c) {
        const int c1 = (c + 1) % 3;
        const double d = orc_seg_dist(cx, cy, (double)t->X[c], (double)t->Y[c], (double)t->X[c1], (double)t->Y[c1]);
        if (d < edge) edge = d;
      }
      if (t->culled || !orc_covers(t->X, t->Y, t->tl, i, j)) continue;
      const double ne = t->n64[0] * ray.e64[0] + t->n64[1] * ray.e64[1] + t->n64[2] * ray.e64[2];
      if (ne == 0.0) continue;
      const double z = t->d64 / ne;
      if (!(z > 0.0) || !isfinite(z)) continue;
      if (t->id == id1) continue;  /* the other sub-triangle of the nearest parent */
      if (z < z1) { z2 = z1; z1 = z; id1 = t->id; }
      else if (z < z2) { z2 = z; }
    }
    o[1] = edge;
    o[2] = isfinite(z2) ? (z2 - z1) / z1 : INFINITY;
  }
  for (int v = 0; v < lf->n_views; ++v) free(meshes[v].tri);
  free(vps);
  free(meshes);
  return rc;
}
