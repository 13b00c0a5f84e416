/*
 * lfscene.c - seeded synthetic inputs for the disk-blended light field renderer.
 *
 * This is input generation only: it ray-casts an analytic scene (textured
 * Lambertian spheres inside a textured backdrop sphere, or planes) from a set
 * of pinhole cameras, producing the RGBA8 source photographs and the per-view
 * depth grids that play the role of the paper's captured images and
 * multiview-stereo depth maps (Sec. 3, Sec. 4.5).  It holds none of the
 * rendering method's arithmetic (no blending, no rasterisation, no disks);
 * both the FP64 oracle and the CUDA library consume its output bytes.
 *
 * Camera convention: pose = (R, t) with R the row-major 3x3 camera->world
 * rotation (columns are the camera axes in world coordinates) and t the
 * centre of projection in world coordinates.  Camera x points right, y down,
 * z forward.  Pixel (i, j) covers [i, i+1) x [j, j+1); its centre is
 * (i + 0.5, j + 0.5).
 *
 * Primitive record (LFS_PRIM_STRIDE doubles each):
 *   [0]      kind: 0 = sphere seen from outside, 1 = backdrop sphere seen from
 *            inside, 2 = infinite plane
 *   [1..3]   sphere centre / a point on the plane
 *   [4]      radius (kinds 0, 1)
 *   [5..7]   plane normal (kind 2, need not be unit length)
 *   [8..10]  albedo colour A (linear RGB in [0, 1])
 *   [11..13] albedo colour B
 *   [14]     checker period in metres (0 = constant colour A)
 *   [15]     value-noise cell size in metres (0 = no noise)
 *   [16]     value-noise amplitude in [0, 1]
 *   [17]     ambient term in [0, 1]
 * Shading: radiance = albedo * (ambient + (1 - ambient) * max(0, n . l)) with
 * n the surface normal facing the ray origin and l the unit light direction.
 * No shadows, so the light field is view independent (Lambertian).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LFS_PRIM_STRIDE 20

typedef struct {
  const double* prims;
  int n_prims;
  double light[3];
  int n_cams;
  const double* poses; /* n_cams x 12 */
  const double* intr;  /* n_cams x 4: fx, fy, cx, cy */
  int W, H;
  uint8_t* out_rgba;   /* n_cams x H x W x 4, or NULL */
  float* out_pixdepth; /* n_cams x H x W, or NULL */
  int G;
  float* out_grid;     /* n_cams x G x G, or NULL */
  int64_t n_items;
  int64_t next;        /* work counter, advanced atomically */
} lfs_job;

static uint64_t lfs_hash3(int64_t x, int64_t y, int64_t z) {
  uint64_t h = (uint64_t)x * 0x9E3779B97F4A7C15ULL;
  h ^= (uint64_t)y * 0xC2B2AE3D27D4EB4FULL + 0x165667B19E3779F9ULL + (h << 6) + (h >> 2);
  h ^= (uint64_t)z * 0x85EBCA77C2B2AE63ULL + 0x27D4EB2F165667C5ULL + (h << 6) + (h >> 2);
  /* SplitMix64 finaliser */
  h ^= h >> 30; h *= 0xBF58476D1CE4E5B9ULL;
  h ^= h >> 27; h *= 0x94D049BB133111EBULL;
  h ^= h >> 31;
  return h;
}

static double lfs_lattice(int64_t x, int64_t y, int64_t z) {
  return (double)(lfs_hash3(x, y, z) >> 11) * 0x1.0p-53;
}

static double lfs_smooth(double t) { return t * t * (3.0 - 2.0 * t); }

/* Trilinear value noise in [0, 1) with smoothstep weights. */
static double lfs_noise(double x, double y, double z) {
  double fx = floor(x), fy = floor(y), fz = floor(z);
  int64_t ix = (int64_t)fx, iy = (int64_t)fy, iz = (int64_t)fz;
  double ux = lfs_smooth(x - fx), uy = lfs_smooth(y - fy), uz = lfs_smooth(z - fz);
  double c[2][2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int d = 0; d < 2; ++d) c[a][b][d] = lfs_lattice(ix + a, iy + b, iz + d);
  double x00 = c[0][0][0] + (c[1][0][0] - c[0][0][0]) * ux;
  double x10 = c[0][1][0] + (c[1][1][0] - c[0][1][0]) * ux;
  double x01 = c[0][0][1] + (c[1][0][1] - c[0][0][1]) * ux;
  double x11 = c[0][1][1] + (c[1][1][1] - c[0][1][1]) * ux;
  double y0 = x00 + (x10 - x00) * uy;
  double y1 = x01 + (x11 - x01) * uy;
  return y0 + (y1 - y0) * uz;
}

/* Albedo of primitive q at local position (x, y, z) (relative to its anchor). */
static void lfs_albedo(const double* q, double x, double y, double z, double rgb[3]) {
  int use_b = 0;
  if (q[14] > 0.0) {
    double p = q[14];
    int64_t s = (int64_t)floor(x / p) + (int64_t)floor(y / p) + (int64_t)floor(z / p);
    use_b = (int)(s & 1);
  }
  const double* col = use_b ? q + 11 : q + 8;
  double m = 1.0;
  if (q[15] > 0.0) {
    double n = lfs_noise(x / q[15], y / q[15], z / q[15]);
    m = 1.0 - q[16] + q[16] * n;
  }
  rgb[0] = col[0] * m;
  rgb[1] = col[1] * m;
  rgb[2] = col[2] * m;
}

/* Nearest positive hit along o + t d (d need not be unit).  Returns t, or -1. */
static double lfs_trace(const lfs_job* job, const double o[3], const double d[3], double rgb[3]) {
  double best_t = INFINITY;
  int best = -1;
  double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  for (int k = 0; k < job->n_prims; ++k) {
    const double* q = job->prims + (size_t)k * LFS_PRIM_STRIDE;
    int kind = (int)q[0];
    double t = -1.0;
    if (kind == 0 || kind == 1) {
      double oc[3] = {o[0] - q[1], o[1] - q[2], o[2] - q[3]};
      double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
      double c = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - q[4] * q[4];
      double disc = b * b - dd * c;
      if (disc < 0.0) continue;
      double sq = sqrt(disc);
      double t0 = (-b - sq) / dd, t1 = (-b + sq) / dd;
      if (kind == 0) t = (t0 > 1e-9) ? t0 : ((t1 > 1e-9) ? t1 : -1.0);
      else t = (t1 > 1e-9) ? t1 : -1.0;
    } else {
      double nd = q[5] * d[0] + q[6] * d[1] + q[7] * d[2];
      if (nd == 0.0) continue;
      double num = q[5] * (q[1] - o[0]) + q[6] * (q[2] - o[1]) + q[7] * (q[3] - o[2]);
      t = num / nd;
      if (!(t > 1e-9)) t = -1.0;
    }
    if (t > 0.0 && t < best_t) { best_t = t; best = k; }
  }
  if (best < 0) { rgb[0] = rgb[1] = rgb[2] = 0.0; return -1.0; }
  const double* q = job->prims + (size_t)best * LFS_PRIM_STRIDE;
  double X[3] = {o[0] + best_t * d[0], o[1] + best_t * d[1], o[2] + best_t * d[2]};
  double n[3];
  int kind = (int)q[0];
  if (kind == 0 || kind == 1) {
    n[0] = X[0] - q[1]; n[1] = X[1] - q[2]; n[2] = X[2] - q[3];
  } else {
    n[0] = q[5]; n[1] = q[6]; n[2] = q[7];
  }
  double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  n[0] /= nl; n[1] /= nl; n[2] /= nl;
  if (n[0] * d[0] + n[1] * d[1] + n[2] * d[2] > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
  double alb[3];
  lfs_albedo(q, X[0] - q[1], X[1] - q[2], X[2] - q[3], alb);
  double ndl = n[0] * job->light[0] + n[1] * job->light[1] + n[2] * job->light[2];
  double shade = q[17] + (1.0 - q[17]) * (ndl > 0.0 ? ndl : 0.0);
  rgb[0] = alb[0] * shade; rgb[1] = alb[1] * shade; rgb[2] = alb[2] * shade;
  return best_t;
}

static uint8_t lfs_to_u8(double v) {
  if (!(v > 0.0)) return 0;
  if (v >= 1.0) return 255;
  return (uint8_t)floor(v * 255.0 + 0.5);
}

/* One work item = one image row of one camera, or one grid row. */
static void lfs_do_item(lfs_job* job, int64_t item) {
  int64_t img_items = (int64_t)job->n_cams * job->H;
  int cam, row, is_grid = 0;
  if (item < img_items) { cam = (int)(item / job->H); row = (int)(item % job->H); }
  else { item -= img_items; cam = (int)(item / job->G); row = (int)(item % job->G); is_grid = 1; }
  const double* P = job->poses + (size_t)cam * 12;
  const double* K = job->intr + (size_t)cam * 4;
  const double o[3] = {P[9], P[10], P[11]};
  double rgb[3];
  if (!is_grid) {
    double yc = ((double)row + 0.5 - K[3]) / K[1];
    for (int i = 0; i < job->W; ++i) {
      double xc = ((double)i + 0.5 - K[2]) / K[0];
      double d[3] = {P[0] * xc + P[1] * yc + P[2], P[3] * xc + P[4] * yc + P[5], P[6] * xc + P[7] * yc + P[8]};
      double t = lfs_trace(job, o, d, rgb);
      size_t pix = ((size_t)cam * job->H + row) * job->W + i;
      if (job->out_rgba) {
        uint8_t* px = job->out_rgba + pix * 4;
        px[0] = lfs_to_u8(rgb[0]); px[1] = lfs_to_u8(rgb[1]); px[2] = lfs_to_u8(rgb[2]); px[3] = 255;
      }
      if (job->out_pixdepth) job->out_pixdepth[pix] = (float)(t > 0.0 ? t : 1e4);
    }
  } else {
    int G = job->G;
    double tt = (double)row * (double)job->H / (double)(G - 1);
    double yc = (tt - K[3]) / K[1];
    for (int j = 0; j < G; ++j) {
      double ss = (double)j * (double)job->W / (double)(G - 1);
      double xc = (ss - K[2]) / K[0];
      double d[3] = {P[0] * xc + P[1] * yc + P[2], P[3] * xc + P[4] * yc + P[5], P[6] * xc + P[7] * yc + P[8]};
      double t = lfs_trace(job, o, d, rgb);
      /* d has unit z in the camera frame, so t is the z-depth. */
      job->out_grid[((size_t)cam * G + row) * G + j] = (float)(t > 0.0 ? t : 1e4);
    }
  }
}

static void* lfs_worker(void* arg) {
  lfs_job* job = (lfs_job*)arg;
  for (;;) {
    int64_t item = __atomic_fetch_add(&job->next, 1, __ATOMIC_RELAXED);
    if (item >= job->n_items) break;
    lfs_do_item(job, item);
  }
  return NULL;
}

/*
 * Ray-cast n_cams cameras of W x H pixels.  Any output may be NULL.
 * out_grid receives the z-depth at the G x G mesh vertices (j, k) placed at
 * pixel-edge coordinates (j W / (G-1), k H / (G-1)).  Returns 0 on success.
 */
int lfs_render(const double* prims, int n_prims, const double* light, int n_cams,
               const double* poses, const double* intr, int W, int H,
               uint8_t* out_rgba, float* out_pixdepth, int G, float* out_grid, int n_threads) {
  if (n_prims <= 0 || n_cams < 0 || W <= 0 || H <= 0) return 1;
  if (out_grid && G < 2) return 1;
  lfs_job job;
  memset(&job, 0, sizeof(job));
  job.prims = prims; job.n_prims = n_prims;
  double ln = sqrt(light[0] * light[0] + light[1] * light[1] + light[2] * light[2]);
  job.light[0] = light[0] / ln; job.light[1] = light[1] / ln; job.light[2] = light[2] / ln;
  job.n_cams = n_cams; job.poses = poses; job.intr = intr; job.W = W; job.H = H;
  job.out_rgba = out_rgba; job.out_pixdepth = out_pixdepth; job.G = G; job.out_grid = out_grid;
  /* Items 0 .. n_cams*H-1 are image rows, the rest are grid rows. */
  int64_t img_rows = (int64_t)n_cams * H;
  job.n_items = img_rows + (out_grid ? (int64_t)n_cams * G : 0);
  job.next = (out_rgba || out_pixdepth) ? 0 : img_rows;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if (n_threads == 1) { lfs_worker(&job); return 0; }
  pthread_t th[256];
  int started = 0;
  for (int k = 0; k < n_threads; ++k) {
    if (pthread_create(&th[k], NULL, lfs_worker, &job) != 0) break;
    ++started;
  }
  if (started == 0) lfs_worker(&job);
  for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
  return 0;
}
