// lf_setup.cu - per-view and per-triangle set-up kernels.
//
//   grid_tables_kernel   once per mesh build: per-view ray directions of the
//                        grid columns/rows, a_j = (j W/(G-1) - cx)/fx, b_k likewise.
//   view_setup_kernel    per call, one thread per (eye, view): FP64 composition
//                        of the view's camera->eye transform, its source
//                        projection, disk constants, and a conservative screen
//                        footprint of the disk, which is OR-ed into per-tile view
//                        masks (the culling of disks against the eye, Sec. 4.2.1).
//   tri_setup_kernel     per call, one CTA per (eye, view) with a non-empty
//                        footprint: vertex transform and 1/256-pixel snap, near
//                        clip, int64 triangle set-up and footprint culling, written
//                        as one contiguous segment in triangle-id order.
//
// Every float operation that feeds an integer decision (snapped position, depth
// winner, disk membership) uses explicit round-to-nearest intrinsics in a fixed
// order, so the decision is the same on any compiler setting.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "lf_internal.h"
#include "lf_launch.h"

namespace lfk {

// ------------------------------------------------------------------ small helpers

__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0, float b1, float b2) {
  return __fmaf_rn(a0, b0, __fmaf_rn(a1, b1, __fmul_rn(a2, b2)));
}

__device__ __forceinline__ bool snap_rn(float x, float y, float z, float fx, float fy, float cx, float cy,
                                        int32_t& sx, int32_t& sy) {
  float qx = __fdiv_rn(x, z), qy = __fdiv_rn(y, z);
  float u = __fmaf_rn(fx, qx, cx), v = __fmaf_rn(fy, qy, cy);
  float su = __fmul_rn(u, 256.0f), sv = __fmul_rn(v, 256.0f);
  const float lim = (float)kSnapLimit;
  if (!(fabsf(su) < lim) || !(fabsf(sv) < lim)) return false;
  sx = __float2int_rn(su);  // |su| < 2^29: the 32-bit round-to-nearest-even conversion is exact
  sy = __float2int_rn(sv);
  return true;
}

__device__ __forceinline__ int64_t floor_div256_up(int64_t a) {  // ceil(a / 256)
  return (a + 255) >> 8;
}

// ------------------------------------------------------------------ grid tables

__global__ void grid_tables_kernel(const ViewStatic* __restrict__ views, int n_views, int src_w, int src_h,
                                   int G, float* __restrict__ a, float* __restrict__ b) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_views * G) return;
  int v = (int)(idx / G), j = (int)(idx % G);
  const ViewStatic& V = views[v];
  double s = __ddiv_rn(__dmul_rn((double)j, (double)src_w), (double)(G - 1));
  double t = __ddiv_rn(__dmul_rn((double)j, (double)src_h), (double)(G - 1));
  a[idx] = __double2float_rn(__ddiv_rn(__dsub_rn(s, V.cx), V.fx));
  b[idx] = __double2float_rn(__ddiv_rn(__dsub_rn(t, V.cy), V.fy));
}

cudaError_t launch_grid_tables(const ViewStatic* views, int n_views, int src_w, int src_h, int G, float* a,
                               float* b, cudaStream_t s) {
  int64_t n = (int64_t)n_views * G;
  grid_tables_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(views, n_views, src_w, src_h, G, a, b);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ texture conversion

__global__ void convert_textures_kernel(const uchar4* __restrict__ src, void* __restrict__ dst, int64_t n,
                                        int fmt, const float* __restrict__ view_scale, int64_t per_view) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; idx < n; idx += stride) {
    uchar4 c = src[idx];
    float r = __fdiv_rn((float)c.x, 255.0f), g = __fdiv_rn((float)c.y, 255.0f), bl = __fdiv_rn((float)c.z, 255.0f);
    if (fmt == LF_TEX_F32) {
      reinterpret_cast<float4*>(dst)[idx] = make_float4(r, g, bl, 1.0f);
    } else if (fmt == LF_TEX_BF16) {
      __nv_bfloat162 lo = __floats2bfloat162_rn(r, g);
      __nv_bfloat162 hi = __floats2bfloat162_rn(bl, 1.0f);
      uint2 pk;
      pk.x = *reinterpret_cast<uint32_t*>(&lo);
      pk.y = *reinterpret_cast<uint32_t*>(&hi);
      reinterpret_cast<uint2*>(dst)[idx] = pk;
    } else if (fmt == LF_TEX_FP8E4M3) {
      float inv = __frcp_rn(view_scale[idx / per_view]);
      __nv_fp8x4_e4m3 q(make_float4(__fmul_rn(r, inv), __fmul_rn(g, inv), __fmul_rn(bl, inv), 0.0f));
      reinterpret_cast<__nv_fp8x4_storage_t*>(dst)[idx] = q.__x;
    }
  }
}

cudaError_t launch_convert_textures(const uint8_t* src, void* dst, int64_t n_texels, int fmt,
                                    const float* view_scale, int64_t texels_per_view, cudaStream_t s) {
  int64_t blocks = (n_texels + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  convert_textures_kernel<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const uchar4*>(src), dst, n_texels,
                                                          fmt, view_scale, texels_per_view);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ per-view reductions

__global__ void view_scale_kernel(const uchar4* __restrict__ src, int64_t per_view, float* __restrict__ scale,
                                  ViewStatic* __restrict__ views) {
  __shared__ int s_max;
  if (threadIdx.x == 0) s_max = 1;
  __syncthreads();
  const uchar4* p = src + (int64_t)blockIdx.x * per_view;
  int m = 1;
  for (int64_t i = threadIdx.x; i < per_view; i += blockDim.x) {
    uchar4 c = p[i];
    m = max(m, max((int)c.x, max((int)c.y, (int)c.z)));
  }
  atomicMax(&s_max, m);
  __syncthreads();
  if (threadIdx.x == 0) {
    float sc = __fdiv_rn(__fdiv_rn((float)s_max, 255.0f), 448.0f);
    scale[blockIdx.x] = sc;
    views[blockIdx.x].tex_scale = sc;
  }
}

cudaError_t launch_view_scale(const uint8_t* rgba8, int n_views, int64_t per_view, float* scale, ViewStatic* views,
                              cudaStream_t s) {
  view_scale_kernel<<<n_views, 256, 0, s>>>(reinterpret_cast<const uchar4*>(rgba8), per_view, scale, views);
  return cudaGetLastError();
}

__global__ void depth_offsets_kernel(const float* __restrict__ depth, int per_view, __half* __restrict__ dst,
                                     ViewStatic* __restrict__ views) {
  __shared__ float s_min[256];
  const float* p = depth + (int64_t)blockIdx.x * per_view;
  float m = INFINITY;
  for (int i = threadIdx.x; i < per_view; i += blockDim.x) m = fminf(m, p[i]);
  s_min[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s_min[threadIdx.x] = fminf(s_min[threadIdx.x], s_min[threadIdx.x + o]);
    __syncthreads();
  }
  const float z0 = s_min[0];
  if (threadIdx.x == 0) views[blockIdx.x].depth_origin = z0;
  __half* q = dst + (int64_t)blockIdx.x * per_view;
  for (int i = threadIdx.x; i < per_view; i += blockDim.x) q[i] = __float2half_rn(__fsub_rn(p[i], z0));
}

cudaError_t launch_depth_offsets(const float* depth, int n_views, int per_view, void* dst_half, ViewStatic* views,
                                 cudaStream_t s) {
  depth_offsets_kernel<<<n_views, 256, 0, s>>>(depth, per_view, static_cast<__half*>(dst_half), views);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ view set-up

// Range of x/z over forward rays (z > 0) that meet a ball of radius rho whose
// centre projects to (c, cz) in the plane of one image axis and the optical
// axis: the directions within asin(rho/L) of the centre's direction, clipped to
// the forward half-plane.  Returns false when no forward ray meets it; an
// infinite bound is returned as +-inf.  FP32 is enough: the caller pads the
// ball and the pixel range, and the result only culls.
__device__ bool axis_extent(float c, float cz, float rho, float& lo, float& hi) {
  const float half_pi = 1.57079632679f;
  const float L2 = c * c + cz * cz;
  if (L2 <= rho * rho * 1.0001f) {  // the eye's projection lies inside the ball's
    lo = -INFINITY;
    hi = INFINITY;
    return true;
  }
  const float th = atan2f(c, cz), de = asinf(fminf(1.0f, rho * rsqrtf(L2)) ) + 1e-5f;
  const float a = fmaxf(th - de, -half_pi), b = fminf(th + de, half_pi);
  if (!(a < b)) return false;
  lo = (a <= -half_pi + 1e-4f) ? -INFINITY : tanf(a);
  hi = (b >= half_pi - 1e-4f) ? INFINITY : tanf(b);
  return true;
}

// Pixel-index range [i0, i1] whose centres' x/z lies in [lo, hi], padded by two pixels.
__device__ void pixel_range(float lo, float hi, float f, float c, int n, int& i0, int& i1) {
  const float u0 = f * lo + c, u1 = f * hi + c;
  i0 = (int)fmaxf(-1.0f, fminf((float)n, floorf(u0 - 0.5f) - 2.0f));
  i1 = (int)fmaxf(-1.0f, fminf((float)n, ceilf(u1 - 0.5f) + 2.0f));
}

constexpr int kViewsPerSetupBlock = 16;
constexpr int kViewSetupThreads = 128;
constexpr int kViewSetupSlices = 8;  // blocks sharing one group of views' (view, tile) cone tests

// A block takes 16 views of one eye.  Threads 0-15 do the per-view set-up
// (FP64 composition, FP32 shading map and disk constants, conservative
// footprint); then all threads test every (view, tile) pair of the block's
// footprints and OR the view's bit into the masks of the tiles it can reach.
// The tile test compares cones from the eye: a pixel whose sphere crossing
// lies in the disk has its ray within asin(rho/|c|) of the direction to the
// disk centre c, and every pixel ray of a tile lies within (half diagonal)/f
// of the tile's centre ray (rays through image points s apart differ by at
// most s/f in angle), so a tile is skipped only when the two cones are apart.
__global__ void __launch_bounds__(kViewSetupThreads) view_setup_kernel(FrameArgs A) {
  __shared__ float s_dir[kViewsPerSetupBlock][4];   // unit direction to the disk centre, cos of the cone limit
  __shared__ int s_off[kViewsPerSetupBlock + 1];   // exclusive prefix of the footprints' tile counts
  __shared__ int s_tile[kViewsPerSetupBlock][3];    // footprint: first tile column and row, tile columns
  const int e = blockIdx.y;
  const int v0 = blockIdx.x * kViewsPerSetupBlock;
  const EyeParams& E = A.eyes[e];
  const float tile_half_diag = 0.5f * sqrtf((float)(A.tile_w * A.tile_w + A.tile_h * A.tile_h));
  const float alpha_tile = tile_half_diag / fminf((float)E.fx, (float)E.fy);
  const bool writer = blockIdx.z == 0;  // the other slices only share the cone tests
  // Triangle set-up may launch now: it waits for this grid to complete before
  // it reads anything the grid writes.
  griddep_wait();
  griddep_release();
  if (writer && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    // the frame's counters start at zero (no kernel before this one uses them)
    *A.pool_counter = 0ull;
    *A.error_word = 0u;
    *A.work_counter = 0;
    *A.bin_offsets_counter = 0ull;
    *A.bin_entries_counter = 0ull;
  }
  if (writer && blockIdx.x == 0 && threadIdx.x == 0) {
    // the eye's FP32 decision constants, each rounded once from FP64
    EyeFloat& F = A.eyes_f[e];
    for (int k = 0; k < 9; ++k) F.R[k] = __double2float_rn(E.R[k]);
    for (int k = 0; k < 3; ++k) F.o[k] = __double2float_rn(__dsub_rn(E.t[k], A.sphere_c[k]));
    F.fx = __double2float_rn(E.fx); F.fy = __double2float_rn(E.fy);
    F.cx = __double2float_rn(E.cx); F.cy = __double2float_rn(E.cy);
    F.R2 = __double2float_rn(__dmul_rn(A.sphere_r, A.sphere_r));
    F.pad[0] = F.pad[1] = F.pad[2] = 0.0f;
  }
  int n_tiles = 0;  // tiles of this thread's view's footprint (threads 0-15)
  if (threadIdx.x < kViewsPerSetupBlock) {
    const int v = v0 + threadIdx.x;
    int bb[4] = {1, 1, 0, 0};
    float dir[4] = {0.f, 0.f, 1.f, 2.f};
    if (v < A.n_views) {
      const ViewStatic& V = A.views[v];
      if (writer) {
      A.active[(int64_t)e * A.n_views + v] = 0;  // set by the raster when a pixel sees the view
      ViewRec& R = A.vrecs[(int64_t)e * A.n_views + v];
      // A1: M = R_eye^T R_i, m = R_eye^T (t_i - t_eye) in FP64, fixed order, no fusion.
      double M[9], m[3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double s = __dmul_rn(E.R[0 * 3 + r], V.R[0 * 3 + c]);
          s = __dadd_rn(s, __dmul_rn(E.R[1 * 3 + r], V.R[1 * 3 + c]));
          s = __dadd_rn(s, __dmul_rn(E.R[2 * 3 + r], V.R[2 * 3 + c]));
          M[r * 3 + c] = s;
        }
      const double d[3] = {__dsub_rn(V.t[0], E.t[0]), __dsub_rn(V.t[1], E.t[1]), __dsub_rn(V.t[2], E.t[2])};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        double s = __dmul_rn(E.R[0 * 3 + r], d[0]);
        s = __dadd_rn(s, __dmul_rn(E.R[1 * 3 + r], d[1]));
        s = __dadd_rn(s, __dmul_rn(E.R[2 * 3 + r], d[2]));
        m[r] = s;
      }
      float Mc[9], mc[3];
#pragma unroll
      for (int k = 0; k < 9; ++k) R.Mf[k] = Mc[k] = __double2float_rn(M[k]);
#pragma unroll
      for (int k = 0; k < 3; ++k) R.Mf[9 + k] = mc[k] = __double2float_rn(m[k]);

      // Source projection for shading: h = K_i' M^T (Kinv_e [x, y, 1] - m / z), with
      // K_i' using (cx - 1/2, cy - 1/2) so h.x/h.z is the bilinear coordinate u = s - 1/2.
      // FP32 from the composition: it only places texture samples.
      const float Ki[9] = {(float)V.fx, 0.f, (float)(V.cx - 0.5), 0.f, (float)V.fy, (float)(V.cy - 0.5),
                           0.f, 0.f, 1.f};
      const float ifx = 1.0f / (float)E.fx, ify = 1.0f / (float)E.fy;
      const float Ke[9] = {ifx, 0.f, -(float)E.cx * ifx, 0.f, ify, -(float)E.cy * ify, 0.f, 0.f, 1.f};
      float KM[9];  // Ki M^T
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
          KM[r * 3 + c] = Ki[r * 3 + 0] * Mc[c * 3 + 0] + Ki[r * 3 + 1] * Mc[c * 3 + 1] + Ki[r * 3 + 2] * Mc[c * 3 + 2];
      for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c)
          R.Hm[r * 3 + c] = KM[r * 3 + 0] * Ke[0 * 3 + c] + KM[r * 3 + 1] * Ke[1 * 3 + c] + KM[r * 3 + 2] * Ke[2 * 3 + c];
        R.Hm[9 + r] = -(KM[r * 3 + 0] * mc[0] + KM[r * 3 + 1] * mc[1] + KM[r * 3 + 2] * mc[2]);
      }

      // Disk (Sec. 4.1): centre relative to the sphere centre in FP32, r^2.
      for (int k = 0; k < 3; ++k) R.cc[k] = __double2float_rn(__dsub_rn((double)V.disk_c[k], A.sphere_c[k]));
      R.cc[3] = __fmul_rn(V.disk_r, V.disk_r);
      R.inv_r = __frcp_rn(V.disk_r);
      if (A.disk_mode == 1) {
        // Oval disk (Sec. 4.4): its plane's normal and axes are the columns of M; the
        // centre in the eye frame and the dot products in FP64, fixed order, each
        // rounded once.
        const double dcw[3] = {__dsub_rn((double)V.disk_c[0], E.t[0]), __dsub_rn((double)V.disk_c[1], E.t[1]),
                               __dsub_rn((double)V.disk_c[2], E.t[2])};
        double cp[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          double s = __dmul_rn(E.R[0 * 3 + r], dcw[0]);
          s = __dadd_rn(s, __dmul_rn(E.R[1 * 3 + r], dcw[1]));
          s = __dadd_rn(s, __dmul_rn(E.R[2 * 3 + r], dcw[2]));
          cp[r] = s;
        }
        auto dotc = [&](int col) {
          return __dadd_rn(__dadd_rn(__dmul_rn(M[0 * 3 + col], cp[0]), __dmul_rn(M[1 * 3 + col], cp[1])),
                           __dmul_rn(M[2 * 3 + col], cp[2]));
        };
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          R.ov_x[k] = Mc[k * 3 + 0];
          R.ov_y[k] = Mc[k * 3 + 1];
          R.ov_n[k] = Mc[k * 3 + 2];
        }
        R.ov_k = __double2float_rn(dotc(2));
        R.ov_u0 = __double2float_rn(dotc(0));
        R.ov_v0 = __double2float_rn(dotc(1));
        R.ov_ru[0] = __double2float_rn(__ddiv_rn(1.0, (double)V.disk_ext[0]));
        R.ov_ru[1] = __double2float_rn(__ddiv_rn(1.0, (double)V.disk_ext[1]));
        R.ov_rv[0] = __double2float_rn(__ddiv_rn(1.0, (double)V.disk_ext[2]));
        R.ov_rv[1] = __double2float_rn(__ddiv_rn(1.0, (double)V.disk_ext[3]));
      }
      // the view's texels: its page in a two-level frame, else its slice of the texture array
      const int tb = A.tex_format == LF_TEX_F32 ? 16 : A.tex_format == LF_TEX_BF16 ? 8 : 4;
      R.tex = A.tex_table ? A.tex_table[v]
                          : static_cast<const char*>(A.textures) + (int64_t)v * A.src_w * A.src_h * tb;
      R.tri_base = 0;
      R.bin_off = -1;
      R.big_base = 0;
      R.big_count = 0;
      R.tri_count = 0;
      }

      // Conservative footprint: a pixel whose sphere crossing can fall inside the
      // disk has a forward ray passing within r of c_i, so it lies in the screen
      // extent of the ball of radius r (padded) about c_i.
      float cw[3], ce[3];
      for (int k = 0; k < 3; ++k) cw[k] = (float)((double)V.disk_c[k] - E.t[k]);
      for (int r = 0; r < 3; ++r)
        ce[r] = (float)E.R[0 * 3 + r] * cw[0] + (float)E.R[1 * 3 + r] * cw[1] + (float)E.R[2 * 3 + r] * cw[2];
      // an oval lies in the disk of its largest extent about c_i, in its plane
      const float r_out = A.disk_mode == 1 ? fmaxf(fmaxf(V.disk_ext[0], V.disk_ext[1]),
                                                    fmaxf(V.disk_ext[2], V.disk_ext[3]))
                                           : V.disk_r;
      const float rho = r_out * 1.001f + 1e-4f;
      float xlo, xhi, ylo, yhi;
      if (axis_extent(ce[0], ce[2], rho, xlo, xhi) && axis_extent(ce[1], ce[2], rho, ylo, yhi)) {
        int x0, x1, y0, y1;
        pixel_range(xlo, xhi, (float)E.fx, (float)E.cx, E.W, x0, x1);
        pixel_range(ylo, yhi, (float)E.fy, (float)E.cy, E.H, y0, y1);
        x0 = max(x0, 0); y0 = max(y0, 0);
        x1 = min(x1, E.W - 1); y1 = min(y1, E.H - 1);
        if (x0 <= x1 && y0 <= y1) { bb[0] = x0; bb[1] = y0; bb[2] = x1; bb[3] = y1; }
      }
      if (writer) {
        ViewRec& R = A.vrecs[(int64_t)e * A.n_views + v];
        R.bb[0] = bb[0]; R.bb[1] = bb[1]; R.bb[2] = bb[2]; R.bb[3] = bb[3];
      }
      // cone of the ball seen from the eye, widened by a tile's angular radius
      const float L = sqrtf(ce[0] * ce[0] + ce[1] * ce[1] + ce[2] * ce[2]);
      if (L > rho) {
        const float lim = asinf(rho / L) + alpha_tile + 1e-4f;
        dir[0] = ce[0] / L; dir[1] = ce[1] / L; dir[2] = ce[2] / L;
        dir[3] = lim < 3.14159f ? cosf(lim) : -2.0f;
      } else {
        dir[3] = -2.0f;  // the eye is inside the ball: every tile of the footprint
      }
    }
    for (int k = 0; k < 4; ++k) s_dir[threadIdx.x][k] = dir[k];
    int tx0 = 0, ty0 = 0, ntx = 1;
    if (bb[0] <= bb[2] && bb[1] <= bb[3]) {
      tx0 = bb[0] / A.tile_w;
      ty0 = bb[1] / A.tile_h;
      ntx = bb[2] / A.tile_w - tx0 + 1;
      n_tiles = ntx * (bb[3] / A.tile_h - ty0 + 1);
    }
    s_tile[threadIdx.x][0] = tx0;
    s_tile[threadIdx.x][1] = ty0;
    s_tile[threadIdx.x][2] = ntx;
  }
  // the footprints' tile counts, scanned by warp 0 (which holds threads 0-15)
  if (threadIdx.x < 32) {
    int incl = n_tiles;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)threadIdx.x >= o) incl += y;
    }
    if (threadIdx.x < kViewsPerSetupBlock) s_off[threadIdx.x] = incl - n_tiles;
    if (threadIdx.x == kViewsPerSetupBlock - 1) s_off[kViewsPerSetupBlock] = incl;
  }
  __syncthreads();
  const int total = s_off[kViewsPerSetupBlock];
  const float fx = (float)E.fx, fy = (float)E.fy, cx = (float)E.cx, cy = (float)E.cy;
  for (int f = threadIdx.x + blockIdx.z * kViewSetupThreads; f < total; f += kViewSetupThreads * kViewSetupSlices) {
    int k = 0;  // the view whose range [s_off[k], s_off[k + 1]) holds f
#pragma unroll
    for (int step = kViewsPerSetupBlock / 2; step > 0; step >>= 1)
      if (s_off[k + step] <= f) k += step;
    const int q = f - s_off[k];
    const int ntx = s_tile[k][2];
    const int tx = s_tile[k][0] + q % ntx, ty = s_tile[k][1] + q / ntx;
    // centre ray of the tile's pixel-centre rectangle
    const float xc = (float)(tx * A.tile_w) + 0.5f * (float)(A.tile_w - 1) + 0.5f;
    const float yc = (float)(ty * A.tile_h) + 0.5f * (float)(A.tile_h - 1) + 0.5f;
    const float rx = (xc - cx) / fx, ry = (yc - cy) / fy;
    const float inv = rsqrtf(rx * rx + ry * ry + 1.0f);
    const float cosang = (rx * s_dir[k][0] + ry * s_dir[k][1] + s_dir[k][2]) * inv;
    if (cosang < s_dir[k][3]) continue;
    const int v = v0 + k;
    const int64_t tile = (int64_t)E.tile_base + (int64_t)ty * E.tiles_x + tx;
    atomicOr(&A.tile_masks[tile * A.mask_words + (v >> 5)], 1u << (v & 31));
  }
}

cudaError_t launch_view_setup(const FrameArgs& a, cudaStream_t s) {
  dim3 grid((a.n_views + kViewsPerSetupBlock - 1) / kViewsPerSetupBlock, a.n_eyes, kViewSetupSlices);
  view_setup_kernel<<<grid, kViewSetupThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ triangle set-up

struct VtxSmem {
  float* x;
  float* y;
  float* z;
  uint8_t* oc;  // outcode: bit0..3 left/right/above/below the padded footprint, bit4 behind z_near
};

constexpr uint8_t kOcBehind = 16;

struct SetupCtx {
  float fx, fy, cx, cy, zn;
  int W, H;
  int bb0, bb1, bb2, bb3;
};

// Orient, classify and bound one snapped sub-triangle; false if culled.
__device__ bool setup_sub(const int32_t* sx, const int32_t* sy, const SetupCtx& C, TriRec& t, int32_t& tl) {
  int64_t X0 = sx[0], Y0 = sy[0], X1 = sx[1], Y1 = sy[1], X2 = sx[2], Y2 = sy[2];
  int64_t A = (X1 - X0) * (Y2 - Y0) - (Y1 - Y0) * (X2 - X0);
  if (A == 0) return false;
  if (A < 0) {
    int64_t tx = X1, ty = Y1;
    X1 = X2; Y1 = Y2; X2 = tx; Y2 = ty;
  }
  int64_t minx = min(X0, min(X1, X2)), maxx = max(X0, max(X1, X2));
  int64_t miny = min(Y0, min(Y1, Y2)), maxy = max(Y0, max(Y1, Y2));
  int64_t i0 = floor_div256_up(minx - 128), i1 = (maxx - 128) >> 8;
  int64_t j0 = floor_div256_up(miny - 128), j1 = (maxy - 128) >> 8;
  i0 = max(i0, (int64_t)C.bb0);
  j0 = max(j0, (int64_t)C.bb1);
  i1 = min(i1, (int64_t)C.bb2);
  j1 = min(j1, (int64_t)C.bb3);
  if (i0 > i1 || j0 > j1) return false;
  t.bx0 = (int16_t)i0; t.by0 = (int16_t)j0; t.bx1 = (int16_t)i1; t.by1 = (int16_t)j1;
  t.x[0] = (int32_t)X0; t.y[0] = (int32_t)Y0;
  t.x[1] = (int32_t)X1; t.y[1] = (int32_t)Y1;
  t.x[2] = (int32_t)X2; t.y[2] = (int32_t)Y2;
  const int64_t X[3] = {X0, X1, X2}, Y[3] = {Y0, Y1, Y2};
  tl = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int k1 = (k + 1) % 3;
    const bool f = (Y[k] == Y[k1] && X[k1] > X[k]) || (Y[k1] < Y[k]);
    tl |= (int)f << k;
  }
  return true;
}

// Set up parent triangle `id` from vertex slots q0, q1, q2; writes up to two
// records into out[] and returns how many were kept.  The decisions (snap,
// clip, orientation, fill rule) are taken exactly as the oracle takes them;
// the outcode test only drops triangles that lie wholly outside the padded
// disk footprint, whose pixels never see this view.
__device__ __forceinline__ int setup_parent(int id, int q0, int q1, int q2, const VtxSmem& S, const SetupCtx& C,
                                            TriRec* out) {
  const uint8_t o0 = S.oc[q0], o1 = S.oc[q1], o2 = S.oc[q2];
  if (o0 & o1 & o2) return 0;  // all behind, or all beyond one side of the footprint
  const int n_in = ((o0 & kOcBehind) == 0) + ((o1 & kOcBehind) == 0) + ((o2 & kOcBehind) == 0);
  const float x0 = S.x[q0], y0 = S.y[q0], z0 = S.z[q0];
  const float x1 = S.x[q1], y1 = S.y[q1], z1 = S.z[q1];
  const float x2 = S.x[q2], y2 = S.y[q2], z2 = S.z[q2];
  // FP32 inverse-depth plane of the parent (original vertex order), fixed order.
  const float e1x = __fsub_rn(x1, x0), e1y = __fsub_rn(y1, y0), e1z = __fsub_rn(z1, z0);
  const float e2x = __fsub_rn(x2, x0), e2y = __fsub_rn(y2, y0), e2z = __fsub_rn(z2, z0);
  const float nx = __fsub_rn(__fmul_rn(e1y, e2z), __fmul_rn(e1z, e2y));
  const float ny = __fsub_rn(__fmul_rn(e1z, e2x), __fmul_rn(e1x, e2z));
  const float nz = __fsub_rn(__fmul_rn(e1x, e2y), __fmul_rn(e1y, e2x));
  const float dd = dot3_rn(nx, ny, nz, x0, y0, z0);
  const float ia = __fdiv_rn(nx, dd), ib = __fdiv_rn(ny, dd), ic = __fdiv_rn(nz, dd);
  if (dd == 0.0f || !isfinite(ia) || !isfinite(ib) || !isfinite(ic)) return 0;
  int32_t px[4], py[4];
  int np = 0;
  if (n_in == 3) {
    if (!snap_rn(x0, y0, z0, C.fx, C.fy, C.cx, C.cy, px[0], py[0])) return 0;
    if (!snap_rn(x1, y1, z1, C.fx, C.fy, C.cx, C.cy, px[1], py[1])) return 0;
    if (!snap_rn(x2, y2, z2, C.fx, C.fy, C.cx, C.cy, px[2], py[2])) return 0;
    np = 3;
  } else {
    // Sutherland-Hodgman against z >= z_near, walking v0 -> v1 -> v2 -> v0.
    const float vx[3] = {x0, x1, x2}, vy[3] = {y0, y1, y2}, vz[3] = {z0, z1, z2};
    const bool in[3] = {(o0 & kOcBehind) == 0, (o1 & kOcBehind) == 0, (o2 & kOcBehind) == 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int k1 = (k + 1) % 3;
      if (in[k]) {
        if (!snap_rn(vx[k], vy[k], vz[k], C.fx, C.fy, C.cx, C.cy, px[np], py[np])) return 0;
        ++np;
      }
      if (in[k] != in[k1]) {
        const float tt = __fdiv_rn(__fsub_rn(C.zn, vz[k]), __fsub_rn(vz[k1], vz[k]));
        const float ix = __fmaf_rn(tt, __fsub_rn(vx[k1], vx[k]), vx[k]);
        const float iy = __fmaf_rn(tt, __fsub_rn(vy[k1], vy[k]), vy[k]);
        if (!snap_rn(ix, iy, C.zn, C.fx, C.fy, C.cx, C.cy, px[np], py[np])) return 0;
        ++np;
      }
    }
  }
  int n = 0;
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    if (f + 2 >= np) break;
    const int32_t sx[3] = {px[0], px[f + 1], px[f + 2]}, sy[3] = {py[0], py[f + 1], py[f + 2]};
    int32_t tl;
    TriRec& t = out[n];
    if (!setup_sub(sx, sy, C, t, tl)) continue;
    t.ia = ia; t.ib = ib; t.ic = ic;
    t.id_tl = (id << 3) | tl;
    ++n;
  }
  return n;
}

// Block-wide exclusive scan of small non-negative counts (blockDim.x multiple of 32).
__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  int base = 0;
  total = 0;
  for (int w = 0; w < nw; ++w) {
    int c = s_warp[w];
    if (w < warp) base += c;
    total += c;
  }
  __syncthreads();
  return base + x - v;
}

// ------------------------------------------------------------------ binning

// Bins one (eye, view)'s n set-up triangles (pool records tri_base ..
// tri_base + n - 1, written by this block) into the screen tiles of its
// footprint box; the triangle set-up block calls it once its records are
// written.  Per tile the bin holds pool indices of the triangles whose pixel
// box overlaps it, in no particular order (the per-view depth decision does
// not depend on order); triangles whose box spans more than A.bin_max_tiles
// tiles go to the view's list of big ones, which every tile of the view scans
// (only the static-scratch render caps it).  Offsets and cursors live in the
// offset pool: [ntiles + 1 absolute entry offsets][ntiles cursors]; the
// per-tile counts and cursors use `cnt` (cnt_cap ints of shared memory) when
// the footprint fits, else the pool's cursor half.
template <int BLOCK>
__device__ void bin_view(const FrameArgs& A, ViewRec& R, int n, int tri_base, int* cnt_smem, int cnt_cap,
                         int* s_warp) {
  __shared__ long long s_off, s_ent;
  __shared__ int s_big;
  const int tw = A.tile_w, th = A.tile_h;
  const int tx0 = R.bb[0] / tw, ty0 = R.bb[1] / th;
  const int ntx = R.bb[2] / tw - tx0 + 1, nty = R.bb[3] / th - ty0 + 1;
  const int nt = ntx * nty;
  if (threadIdx.x == 0) {
    const unsigned long long o = atomicAdd(A.bin_offsets_counter, (unsigned long long)(2 * nt + 1));
    s_off = ((long long)o + 2 * nt + 1 <= A.bin_offsets_capacity) ? (long long)o : -1;
    if (s_off < 0) atomicOr(A.error_word, kErrPoolOverflow);
    s_big = 0;
  }
  __syncthreads();
  if (s_off < 0) return;
  int* offs = A.bin_offsets + s_off;
  int* curs = offs + nt + 1;
  int* cnt = nt <= cnt_cap ? cnt_smem : curs;  // counts, then cursors
  for (int k = threadIdx.x; k < nt; k += BLOCK) cnt[k] = 0;
  __syncthreads();
  const TriRec* tris = A.pool + tri_base;
  auto span = [&](int t, int& x0, int& y0, int& x1, int& y1) {
    const int2 bb = *reinterpret_cast<const int2*>(tris + t);
    x0 = max((int)(int16_t)(bb.x & 0xffff) / tw - tx0, 0);
    y0 = max((bb.x >> 16) / th - ty0, 0);
    x1 = min((int)(int16_t)(bb.y & 0xffff) / tw - tx0, ntx - 1);
    y1 = min((bb.y >> 16) / th - ty0, nty - 1);
  };
  int my_big = 0;
  for (int t = threadIdx.x; t < n; t += BLOCK) {
    int x0, y0, x1, y1;
    span(t, x0, y0, x1, y1);
    if (x0 > x1 || y0 > y1) continue;
    if ((x1 - x0 + 1) * (y1 - y0 + 1) > A.bin_max_tiles) { ++my_big; continue; }
    for (int y = y0; y <= y1; ++y)
      for (int x = x0; x <= x1; ++x) atomicAdd(&cnt[y * ntx + x], 1);
  }
  if (my_big) atomicAdd(&s_big, my_big);
  __syncthreads();
  // exclusive scan of the counts in place; each thread owns a contiguous run
  const int per = (nt + BLOCK - 1) / BLOCK;
  const int r0 = threadIdx.x * per, r1 = min(r0 + per, nt);
  int run = 0;
  for (int k = r0; k < r1; ++k) run += cnt[k];
  int total;
  int o = block_exclusive_scan(run, s_warp, total);
  if (threadIdx.x == 0) {
    const int need = total + s_big;
    const unsigned long long b = atomicAdd(A.bin_entries_counter, (unsigned long long)need);
    s_ent = ((long long)b + need <= A.bin_entries_capacity) ? (long long)b : -1;
    if (s_ent < 0) atomicOr(A.error_word, kErrPoolOverflow);
  }
  __syncthreads();
  const long long ent = s_ent;
  if (ent < 0) return;
  for (int k = r0; k < r1; ++k) {
    const int c = cnt[k];
    offs[k] = (int)(ent + o);
    cnt[k] = (int)(ent + o);  // cursor
    o += c;
  }
  if (threadIdx.x == 0) {
    offs[nt] = (int)(ent + total);
    s_big = 0;
  }
  __syncthreads();
  const int big_base = (int)(ent + total);
  for (int t = threadIdx.x; t < n; t += BLOCK) {
    int x0, y0, x1, y1;
    span(t, x0, y0, x1, y1);
    if (x0 > x1 || y0 > y1) continue;
    const int idx = tri_base + t;
    if ((x1 - x0 + 1) * (y1 - y0 + 1) > A.bin_max_tiles) {
      A.bin_entries[big_base + atomicAdd(&s_big, 1)] = idx;
      continue;
    }
    for (int y = y0; y <= y1; ++y)
      for (int x = x0; x <= x1; ++x) A.bin_entries[atomicAdd(&cnt[y * ntx + x], 1)] = idx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    R.bin_off = (int32_t)s_off;
    R.btx0 = (int16_t)tx0; R.bty0 = (int16_t)ty0;
    R.bntx = (int16_t)ntx; R.bnty = (int16_t)nty;
    R.big_base = big_base;
    R.big_count = s_big;
  }
}

// Shared-memory row stride of the vertex arrays: >= G and = 4 (mod 32), so
// the 4x4 cells of a cluster read 16 different banks.
__host__ __device__ inline int vertex_row_stride(int G) { return G + ((36 - G % 32) % 32); }

// One CTA per (eye, view) whose disk footprint reaches the eye.  Per band of
// grid rows: (1) the band's vertices go to eye space with outcodes against the
// padded footprint; (2) warps walk the 4x4-cell clusters, skip clusters whose
// vertices all lie beyond one side (or behind the eye), and append the
// triangles that pass their own outcode test to a candidate list; (3) all
// threads share the candidates for the full set-up (snap, clip, orientation,
// fill rule).  With the whole grid in one band (the usual case) one atomic
// reserves an upper bound of the view's records and one pass writes them;
// with several bands pass 1 counts the records, one atomic reserves the
// view's segment and pass 2 writes them.  The order inside a segment does not matter:
// the raster's depth decision within a view is order-independent.  Then the
// block bins its records into the screen tiles (bin_view), the shared memory
// of the vertex arrays holding the per-tile counts.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 3) tri_setup_kernel(FrameArgs A, int band_rows, int cnt_cap) {
  constexpr int NW = BLOCK / 32;
  const int v = blockIdx.x, e = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the view set-up has completed (it wrote the view records read below); the
  // raster may then launch, and waits for this grid before it reads the bins
  griddep_wait();
  griddep_release();
  ViewRec& R = A.vrecs[(int64_t)e * A.n_views + v];
  const int bb0 = R.bb[0], bb1 = R.bb[1], bb2 = R.bb[2], bb3 = R.bb[3];
  if (bb0 > bb2 || bb1 > bb3) return;  // disk footprint misses the eye
  // a two-level frame sets up only the views the eye draws
  if (A.enable_bits && !((A.enable_bits[(int64_t)e * A.mask_words + (v >> 5)] >> (v & 31)) & 1u)) return;
  const EyeParams& E = A.eyes[e];
  const EyeFloat& EF = A.eyes_f[e];
  const int G = A.G;
  extern __shared__ __align__(16) unsigned char smem[];
  const int RS = vertex_row_stride(G);
  const int nv_band = (band_rows + 1) * RS;
  const int n_cell = G - 1;
  VtxSmem S;
  S.x = reinterpret_cast<float*>(smem);
  S.y = S.x + nv_band;
  S.z = S.y + nv_band;
  uint16_t* s_cand = reinterpret_cast<uint16_t*>(S.z + nv_band);  // candidate triangles of the band
  S.oc = reinterpret_cast<uint8_t*>(s_cand + 2 * n_cell * band_rows);
  __shared__ int s_warp[NW];
  __shared__ int s_ncand, s_pos, s_ntwo;
  __shared__ long long s_tri_base;

  SetupCtx C;
  C.fx = EF.fx; C.fy = EF.fy; C.cx = EF.cx; C.cy = EF.cy;
  C.zn = A.z_near; C.W = E.W; C.H = E.H;
  C.bb0 = bb0; C.bb1 = bb1; C.bb2 = bb2; C.bb3 = bb3;
  // outcode planes in the form fx*x <op> (edge - cx) * z, padded by 2 pixels
  const float oxl = (float)bb0 - 2.0f - C.cx, oxr = (float)bb2 + 3.0f - C.cx;
  const float oyt = (float)bb1 - 2.0f - C.cy, oyb = (float)bb3 + 3.0f - C.cy;
  float Mf[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) Mf[k] = R.Mf[k];
  const float* ta = A.tables.a + (int64_t)v * G;
  const float* tb = A.tables.b + (int64_t)v * G;
  const ViewStatic& V = A.views[v];
  const int ncl = (n_cell + kClusterCells - 1) / kClusterCells;  // clusters per side
  const int n_bands = (n_cell + band_rows - 1) / band_rows;

  // q / G without an integer division: (q + 1/2) / G is at least 1/(2G) away
  // from an integer and the float product errs by under 3e-5 for q < 2^17.
  const float inv_G = 1.0f / (float)G;
  const float inv_ncl = 1.0f / (float)ncl;
  auto load_band = [&](int k0, int k1) {  // vertex rows k0 .. k1 inclusive
    const int nq = (k1 - k0 + 1) * G;
#pragma unroll 4
    for (int q = threadIdx.x; q < nq; q += BLOCK) {
      const int kq = (int)(((float)q + 0.5f) * inv_G);
      const int k = k0 + kq, j = q - kq * G;
      const int64_t gi = ((int64_t)v * G + k) * G + j;
      float z;
      if (A.mesh_format == LF_MESH_F16_OFFSET)
        z = __fadd_rn(V.depth_origin, __half2float(reinterpret_cast<const __half*>(A.depth)[gi]));
      else
        z = __ldg(reinterpret_cast<const float*>(A.depth) + gi);
      const float X = __fmul_rn(z, __ldg(ta + j)), Y = __fmul_rn(z, __ldg(tb + k)), Z = z;
      const float ex = __fmaf_rn(Mf[0], X, __fmaf_rn(Mf[1], Y, __fmaf_rn(Mf[2], Z, Mf[9])));
      const float ey = __fmaf_rn(Mf[3], X, __fmaf_rn(Mf[4], Y, __fmaf_rn(Mf[5], Z, Mf[10])));
      const float ez = __fmaf_rn(Mf[6], X, __fmaf_rn(Mf[7], Y, __fmaf_rn(Mf[8], Z, Mf[11])));
      uint8_t oc = kOcBehind;
      if (ez >= C.zn) {
        const float ux = C.fx * ex, uy = C.fy * ey;
        oc = (uint8_t)((ux < oxl * ez ? 1 : 0) | (ux > oxr * ez ? 2 : 0) | (uy < oyt * ez ? 4 : 0) |
                       (uy > oyb * ez ? 8 : 0));
      }
      const int slot = kq * RS + j;
      S.x[slot] = ex; S.y[slot] = ey; S.z[slot] = ez;
      S.oc[slot] = oc;
    }
  };
  // vertex slots of band-local triangle (kk, j, half)
  auto tri_slots = [&](int kk, int j, int half, int& q0, int& q1, int& q2) {
    const int r0 = kk * RS;
    if (half == 0) { q0 = r0 + j; q1 = r0 + j + 1; q2 = r0 + RS + j; }
    else { q0 = r0 + j + 1; q1 = r0 + RS + j + 1; q2 = r0 + RS + j; }
  };
  // Warps walk the band's clusters; surviving triangles join the candidate list.
  auto gather = [&](int k0, int k1) {
    if (threadIdx.x == 0) s_ncand = s_ntwo = 0;
    __syncthreads();
    const int cy0 = k0 / kClusterCells, cy1 = (k1 + kClusterCells - 1) / kClusterCells;
    const int c0 = cy0 * ncl, c1 = cy1 * ncl;
    for (int c = c0 + warp; c < c1; c += NW) {
      const int cl_y = (int)(((float)c + 0.5f) * inv_ncl), cl_x = c - cl_y * ncl;
      // AND of the outcodes of the cluster's (up to) 5 x 5 vertices: a bit set
      // here is set on every vertex of every triangle of the cluster
      uint32_t oca = 0xffu;
      if (lane < 25) {
        const int k = min(cl_y * kClusterCells + lane / 5, n_cell), j = min(cl_x * kClusterCells + lane % 5, n_cell);
        oca = S.oc[(k - k0) * RS + j];
      }
      if (__reduce_and_sync(0xffffffffu, oca) != 0u) continue;
      const int cell = lane >> 1, half = lane & 1;
      const int j = cl_x * kClusterCells + (cell & 3), k = cl_y * kClusterCells + (cell >> 2);
      bool keep = false, two = false;
      if (j < n_cell && k < k1) {
        int q0, q1, q2;
        tri_slots(k - k0, j, half, q0, q1, q2);
        const uint8_t o0 = S.oc[q0], o1 = S.oc[q1], o2 = S.oc[q2];
        keep = (o0 & o1 & o2) == 0;
        // exactly two vertices in front of the near plane: clipping may give two sub-triangles
        two = keep && ((o0 & kOcBehind) == 0) + ((o1 & kOcBehind) == 0) + ((o2 & kOcBehind) == 0) == 2;
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, keep);
      const uint32_t bal2 = __ballot_sync(0xffffffffu, two);
      if (lane == 0 && bal2) atomicAdd(&s_ntwo, __popc(bal2));
      int base = 0;
      if (lane == 0 && bal) base = atomicAdd(&s_ncand, __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (keep) s_cand[base + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)((((k - k0) * n_cell + j) << 1) | half);
    }
    __syncthreads();
  };
  auto setup_cand = [&](int k0, int code, TriRec* tmp) -> int {
    const int half = code & 1, cell = code >> 1;
    const int kk = (int)(((float)cell + 0.5f) / (float)n_cell);
    const int j = cell - kk * n_cell;
    int q0, q1, q2;
    tri_slots(kk, j, half, q0, q1, q2);
    const int id = 2 * ((k0 + kk) * n_cell + j) + half;
    return setup_parent(id, q0, q1, q2, S, C, tmp);
  };

  if (n_bands == 1) {
    // The whole grid in one band: one pass.  The view reserves an upper bound of
    // its records (one per candidate, two for a candidate with exactly two
    // vertices in front of the near plane), then writes the records it keeps
    // compactly from the start of the reservation.
    __syncthreads();
    load_band(0, n_cell);
    __syncthreads();
    gather(0, n_cell);
    const int nc = s_ncand;
    if (threadIdx.x == 0) {
      const int bound = nc + s_ntwo;
      long long tb_ = -1;
      if (bound > 0) {
        const unsigned long long b = atomicAdd(A.pool_counter, (unsigned long long)bound);
        if ((long long)b + bound <= A.pool_capacity) tb_ = (long long)b;
        else atomicOr(A.error_word, kErrPoolOverflow);
      }
      s_tri_base = tb_;
      s_pos = 0;
    }
    __syncthreads();
    const long long tri_base = s_tri_base;
    if (tri_base < 0) return;
    for (int i = threadIdx.x; i < nc; i += BLOCK) {
      TriRec tmp[2];
      const int n = setup_cand(0, s_cand[i], tmp);
      if (n) {
        const int pos = atomicAdd(&s_pos, n);
        for (int k = 0; k < n; ++k) A.pool[tri_base + pos + k] = tmp[k];
      }
    }
    __syncthreads();  // the block's records are written and visible to all its threads
    const int total = s_pos;
    if (threadIdx.x == 0) {
      R.tri_base = (int32_t)tri_base;
      R.tri_count = total;
    }
    if (total > 0) bin_view<BLOCK>(A, R, total, (int)tri_base, reinterpret_cast<int*>(smem), cnt_cap, s_warp);
    return;
  }

  // Several bands: pass 1 counts the kept records, pass 2 writes them.
  int my_count = 0;
  for (int bnd = 0; bnd < n_bands; ++bnd) {
    const int k0 = bnd * band_rows, k1 = min(k0 + band_rows, n_cell);
    __syncthreads();
    load_band(k0, k1);
    __syncthreads();
    gather(k0, k1);
    const int nc = s_ncand;
    for (int i = threadIdx.x; i < nc; i += BLOCK) {
      TriRec tmp[2];
      my_count += setup_cand(k0, s_cand[i], tmp);
    }
  }
  int total;
  block_exclusive_scan(my_count, s_warp, total);
  if (threadIdx.x == 0) {
    long long tb_ = -1;
    if (total > 0) {
      const unsigned long long b = atomicAdd(A.pool_counter, (unsigned long long)total);
      if ((long long)b + total <= A.pool_capacity) tb_ = (long long)b;
      else atomicOr(A.error_word, kErrPoolOverflow);
    }
    s_tri_base = tb_;
    s_pos = 0;
    R.tri_base = tb_ < 0 ? 0 : (int32_t)tb_;
    R.tri_count = tb_ < 0 ? 0 : total;
  }
  __syncthreads();
  const long long tri_base = s_tri_base;
  if (tri_base < 0) return;
  // Pass 2: write the records.
  for (int bnd = 0; bnd < n_bands; ++bnd) {
    const int k0 = bnd * band_rows, k1 = min(k0 + band_rows, n_cell);
    __syncthreads();
    load_band(k0, k1);
    __syncthreads();
    gather(k0, k1);
    const int nc = s_ncand;
    for (int i = threadIdx.x; i < nc; i += BLOCK) {
      TriRec tmp[2];
      const int n = setup_cand(k0, s_cand[i], tmp);
      if (n) {
        const int pos = atomicAdd(&s_pos, n);
        for (int k = 0; k < n; ++k) A.pool[tri_base + pos + k] = tmp[k];
      }
    }
  }
  __syncthreads();  // the block's records are written and visible to all its threads
  bin_view<BLOCK>(A, R, total, (int)tri_base, reinterpret_cast<int*>(smem), cnt_cap, s_warp);
}

constexpr int kSetupBlock = 256;
constexpr size_t kVtxBytes = 13;  // x, y, z (4 B each) + outcode

// Cell rows per band: the whole grid when it fits (vertex arrays plus a 16-bit
// candidate per triangle), else a multiple of the cluster size.
static int setup_band_rows(int G, size_t smem_limit) {
  const size_t per_row = kVtxBytes * (size_t)vertex_row_stride(G) + 2 * 2 * (size_t)(G - 1);
  int rows = (int)((smem_limit - kVtxBytes * (size_t)vertex_row_stride(G)) / per_row);
  rows = min(rows, 32767 / max(1, G - 1));  // band-local triangle codes fit 16 bits
  if (rows >= G - 1) return G - 1;
  rows = (rows / kClusterCells) * kClusterCells;
  return rows < kClusterCells ? kClusterCells : rows;
}

cudaError_t launch_tri_setup(const FrameArgs& a, cudaStream_t s, bool pdl) {
  const size_t limit = 96 * 1024;
  cudaError_t err = ensure_dynamic_smem(reinterpret_cast<const void*>(tri_setup_kernel<kSetupBlock>), (int)limit + 64);
  if (err != cudaSuccess) return err;
  const int rows = setup_band_rows(a.G, limit);
  const size_t vtx = (size_t)(rows + 1) * vertex_row_stride(a.G) * kVtxBytes + 2 * 2 * (size_t)(a.G - 1) * rows + 64;
  // the binning counts reuse the vertex arrays' shared memory: at least kBinSmemTiles ints
  const size_t bytes = std::max(vtx, sizeof(int) * (size_t)kBinSmemTiles);
  const int cnt_cap = (int)(bytes / sizeof(int));
  dim3 grid(a.n_views, a.n_eyes);
  return launch_kernel(tri_setup_kernel<kSetupBlock>, grid, dim3(kSetupBlock), bytes, s, pdl, a, rows, cnt_cap);
}

}  // namespace lfk
