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

#include "lf_internal.h"

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
  sx = (int32_t)__float2ll_rn(su);
  sy = (int32_t)__float2ll_rn(sv);
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

// x/z extent of a ball (centre (c, cz), radius rho) seen from the origin, in
// the plane spanned by one image axis and the optical axis.  Returns false
// when the ball lies entirely behind the eye; sets unbounded when it crosses
// the eye plane or contains the eye.
__device__ bool ball_extent(double c, double cz, double rho, double& lo, double& hi, bool& unbounded) {
  unbounded = false;
  if (cz < -rho) return false;
  double L2 = c * c + cz * cz - rho * rho;
  if (cz <= rho || L2 <= 0.0) {
    unbounded = true;
    return true;
  }
  double L = sqrt(L2);
  double den = cz * cz - rho * rho;
  lo = (c * cz - rho * L) / den;
  hi = (c * cz + rho * L) / den;
  return true;
}

__global__ void view_setup_kernel(FrameArgs A) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  int e = blockIdx.y;
  if (v >= A.n_views) return;
  const EyeParams& E = A.eyes[e];
  const ViewStatic& V = A.views[v];
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
  double d[3] = {__dsub_rn(V.t[0], E.t[0]), __dsub_rn(V.t[1], E.t[1]), __dsub_rn(V.t[2], E.t[2])};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    double s = __dmul_rn(E.R[0 * 3 + r], d[0]);
    s = __dadd_rn(s, __dmul_rn(E.R[1 * 3 + r], d[1]));
    s = __dadd_rn(s, __dmul_rn(E.R[2 * 3 + r], d[2]));
    m[r] = s;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) R.Mf[k] = __double2float_rn(M[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k) R.Mf[9 + k] = __double2float_rn(m[k]);

  // Source projection for shading: h = K_i' M^T (Kinv_e [x, y, 1] - m / z), with
  // K_i' using (cx - 1/2, cy - 1/2) so h.x/h.z is the bilinear coordinate u = s - 1/2.
  double Ki[9] = {V.fx, 0.0, V.cx - 0.5, 0.0, V.fy, V.cy - 0.5, 0.0, 0.0, 1.0};
  double Ke[9] = {1.0 / E.fx, 0.0, -E.cx / E.fx, 0.0, 1.0 / E.fy, -E.cy / E.fy, 0.0, 0.0, 1.0};
  double KM[9];  // Ki M^T
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) KM[r * 3 + c] = Ki[r * 3 + 0] * M[c * 3 + 0] + Ki[r * 3 + 1] * M[c * 3 + 1] + Ki[r * 3 + 2] * M[c * 3 + 2];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c)
      R.Hm[r * 3 + c] = (float)(KM[r * 3 + 0] * Ke[0 * 3 + c] + KM[r * 3 + 1] * Ke[1 * 3 + c] + KM[r * 3 + 2] * Ke[2 * 3 + c]);
    R.Hm[9 + r] = (float)(-(KM[r * 3 + 0] * m[0] + KM[r * 3 + 1] * m[1] + KM[r * 3 + 2] * m[2]));
  }

  // Disk (Sec. 4.1): centre relative to the sphere centre in FP32, r^2.
  for (int k = 0; k < 3; ++k) R.cc[k] = __double2float_rn(__dsub_rn((double)V.disk_c[k], A.sphere_c[k]));
  R.cc[3] = __fmul_rn(V.disk_r, V.disk_r);
  R.inv_r = __frcp_rn(V.disk_r);
  R.seg_base = 0;
  R.seg_count = 0;

  // Conservative footprint: every pixel whose sphere crossing can fall inside
  // the disk sees a ray passing within r of c_i, so it lies in the screen
  // extent of the ball of radius r (slightly inflated) about c_i.
  double cw[3] = {(double)V.disk_c[0] - E.t[0], (double)V.disk_c[1] - E.t[1], (double)V.disk_c[2] - E.t[2]};
  double ce[3];
  for (int r = 0; r < 3; ++r) ce[r] = E.R[0 * 3 + r] * cw[0] + E.R[1 * 3 + r] * cw[1] + E.R[2 * 3 + r] * cw[2];
  double rho = (double)V.disk_r * (1.0 + 1e-4) + 1e-5;
  double xlo, xhi, ylo, yhi;
  bool ux, uy;
  int bx0 = 0, by0 = 0, bx1 = E.W - 1, by1 = E.H - 1;
  bool vis = ball_extent(ce[0], ce[2], rho, xlo, xhi, ux) && ball_extent(ce[1], ce[2], rho, ylo, yhi, uy);
  if (vis) {
    if (!ux) {
      double u0 = E.fx * xlo + E.cx, u1 = E.fx * xhi + E.cx;
      bx0 = (int)fmax(-1.0, floor(u0 - 0.5) - 1.0);
      bx1 = (int)fmin((double)E.W, ceil(u1 - 0.5) + 1.0);
    }
    if (!uy) {
      double v0 = E.fy * ylo + E.cy, v1 = E.fy * yhi + E.cy;
      by0 = (int)fmax(-1.0, floor(v0 - 0.5) - 1.0);
      by1 = (int)fmin((double)E.H, ceil(v1 - 0.5) + 1.0);
    }
    bx0 = max(bx0, 0);
    by0 = max(by0, 0);
    bx1 = min(bx1, E.W - 1);
    by1 = min(by1, E.H - 1);
    if (bx0 > bx1 || by0 > by1) vis = false;
  }
  if (!vis) {
    R.bb[0] = 1; R.bb[1] = 1; R.bb[2] = 0; R.bb[3] = 0;
    return;
  }
  R.bb[0] = bx0; R.bb[1] = by0; R.bb[2] = bx1; R.bb[3] = by1;
  int tx0 = bx0 / A.tile_w, tx1 = bx1 / A.tile_w, ty0 = by0 / A.tile_h, ty1 = by1 / A.tile_h;
  uint32_t bit = 1u << (v & 31);
  int word = v >> 5;
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) {
      int64_t tile = (int64_t)E.tile_base + (int64_t)ty * E.tiles_x + tx;
      atomicOr(&A.tile_masks[tile * A.mask_words + word], bit);
    }
}

cudaError_t launch_view_setup(const FrameArgs& a, cudaStream_t s) {
  dim3 grid((a.n_views + 127) / 128, a.n_eyes);
  view_setup_kernel<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ triangle set-up

struct VtxSmem {
  float* x;
  float* y;
  float* z;
  int32_t* sx;
  int32_t* sy;
  uint8_t* fl;  // bit0: z >= z_near, bit1: snapped beyond the limit
};

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
  int64_t X[3] = {X0, X1, X2}, Y[3] = {Y0, Y1, Y2};
  tl = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int k1 = (k + 1) % 3;
    bool f = (Y[k] == Y[k1] && X[k1] > X[k]) || (Y[k1] < Y[k]);
    tl |= (int)f << k;
  }
  return true;
}

// Set up parent triangle `id` (vertex slots q0, q1, q2 in smem); writes up to two
// records into out[] and returns how many were kept.
__device__ int setup_parent(int id, int q0, int q1, int q2, const VtxSmem& S, const SetupCtx& C, TriRec* out) {
  int q[3] = {q0, q1, q2};
  int in0 = S.fl[q0] & 1, in1 = S.fl[q1] & 1, in2 = S.fl[q2] & 1;
  int n_in = in0 + in1 + in2;
  if (n_in == 0) return 0;
  // cheap reject: all vertices in front and the snapped bbox misses the footprint
  if (n_in == 3) {
    if ((S.fl[q0] | S.fl[q1] | S.fl[q2]) & 2) return 0;
    int32_t mnx = min(S.sx[q0], min(S.sx[q1], S.sx[q2])), mxx = max(S.sx[q0], max(S.sx[q1], S.sx[q2]));
    int32_t mny = min(S.sy[q0], min(S.sy[q1], S.sy[q2])), mxy = max(S.sy[q0], max(S.sy[q1], S.sy[q2]));
    // pixel centre 256 i + 128 within [mn, mx]
    if (mxx < 256 * C.bb0 + 128 || mnx > 256 * C.bb2 + 128 || mxy < 256 * C.bb1 + 128 || mny > 256 * C.bb3 + 128)
      return 0;
  }
  // FP32 inverse-depth plane of the parent (original vertex order), fixed order.
  float e1x = __fsub_rn(S.x[q1], S.x[q0]), e1y = __fsub_rn(S.y[q1], S.y[q0]), e1z = __fsub_rn(S.z[q1], S.z[q0]);
  float e2x = __fsub_rn(S.x[q2], S.x[q0]), e2y = __fsub_rn(S.y[q2], S.y[q0]), e2z = __fsub_rn(S.z[q2], S.z[q0]);
  float nx = __fsub_rn(__fmul_rn(e1y, e2z), __fmul_rn(e1z, e2y));
  float ny = __fsub_rn(__fmul_rn(e1z, e2x), __fmul_rn(e1x, e2z));
  float nz = __fsub_rn(__fmul_rn(e1x, e2y), __fmul_rn(e1y, e2x));
  float dd = dot3_rn(nx, ny, nz, S.x[q0], S.y[q0], S.z[q0]);
  float ia = __fdiv_rn(nx, dd), ib = __fdiv_rn(ny, dd), ic = __fdiv_rn(nz, dd);
  if (dd == 0.0f || !isfinite(ia) || !isfinite(ib) || !isfinite(ic)) return 0;
  int32_t px[4], py[4];
  int np = 0;
  bool far = false;
  if (n_in == 3) {
    for (int k = 0; k < 3; ++k) { px[k] = S.sx[q[k]]; py[k] = S.sy[q[k]]; }
    np = 3;
  } else {
    for (int k = 0; k < 3; ++k) {
      int a = q[k], b = q[(k + 1) % 3];
      bool ain = S.fl[a] & 1, bin = S.fl[b] & 1;
      if (ain) {
        px[np] = S.sx[a]; py[np] = S.sy[a];
        far |= (S.fl[a] & 2) != 0;
        ++np;
      }
      if (ain != bin) {
        float tt = __fdiv_rn(__fsub_rn(C.zn, S.z[a]), __fsub_rn(S.z[b], S.z[a]));
        float ix = __fmaf_rn(tt, __fsub_rn(S.x[b], S.x[a]), S.x[a]);
        float iy = __fmaf_rn(tt, __fsub_rn(S.y[b], S.y[a]), S.y[a]);
        if (!snap_rn(ix, iy, C.zn, C.fx, C.fy, C.cx, C.cy, px[np], py[np])) far = true;
        ++np;
      }
    }
  }
  if (far) return 0;
  int n = 0;
  for (int f = 0; f + 2 < np; ++f) {
    int32_t sx[3] = {px[0], px[f + 1], px[f + 2]}, sy[3] = {py[0], py[f + 1], py[f + 2]};
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

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) tri_setup_kernel(FrameArgs A, int band_rows) {
  const int v = blockIdx.x, e = blockIdx.y;
  ViewRec& R = A.vrecs[(int64_t)e * A.n_views + v];
  const int bb0 = R.bb[0], bb1 = R.bb[1], bb2 = R.bb[2], bb3 = R.bb[3];
  if (bb0 > bb2 || bb1 > bb3) return;  // disk footprint misses the eye
  const EyeParams& E = A.eyes[e];
  const int G = A.G;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nv_band = (band_rows + 1) * G;
  VtxSmem S;
  S.x = reinterpret_cast<float*>(smem);
  S.y = S.x + nv_band;
  S.z = S.y + nv_band;
  S.sx = reinterpret_cast<int32_t*>(S.z + nv_band);
  S.sy = S.sx + nv_band;
  S.fl = reinterpret_cast<uint8_t*>(S.sy + nv_band);
  __shared__ int s_warp[BLOCK / 32];
  __shared__ long long s_base;

  SetupCtx C;
  C.fx = __double2float_rn(E.fx); C.fy = __double2float_rn(E.fy);
  C.cx = __double2float_rn(E.cx); C.cy = __double2float_rn(E.cy);
  C.zn = A.z_near; C.W = E.W; C.H = E.H;
  C.bb0 = bb0; C.bb1 = bb1; C.bb2 = bb2; C.bb3 = bb3;
  float Mf[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) Mf[k] = R.Mf[k];
  const float* ta = A.tables.a + (int64_t)v * G;
  const float* tb = A.tables.b + (int64_t)v * G;
  const ViewStatic& V = A.views[v];
  const int n_cell_rows = G - 1;
  const int n_bands = (n_cell_rows + band_rows - 1) / band_rows;

  auto load_band = [&](int k0, int k1) {  // vertex rows k0 .. k1 inclusive
    int nrow = k1 - k0 + 1;
    for (int q = threadIdx.x; q < nrow * G; q += BLOCK) {
      int k = k0 + q / G, j = q % G;
      int64_t gi = ((int64_t)v * G + k) * G + j;
      float z;
      if (A.mesh_format == LF_MESH_F16_OFFSET)
        z = __fadd_rn(V.depth_origin, __half2float(reinterpret_cast<const __half*>(A.depth)[gi]));
      else
        z = reinterpret_cast<const float*>(A.depth)[gi];
      float X = __fmul_rn(z, ta[j]), Y = __fmul_rn(z, tb[k]), Z = z;
      float ex = __fmaf_rn(Mf[0], X, __fmaf_rn(Mf[1], Y, __fmaf_rn(Mf[2], Z, Mf[9])));
      float ey = __fmaf_rn(Mf[3], X, __fmaf_rn(Mf[4], Y, __fmaf_rn(Mf[5], Z, Mf[10])));
      float ez = __fmaf_rn(Mf[6], X, __fmaf_rn(Mf[7], Y, __fmaf_rn(Mf[8], Z, Mf[11])));
      uint8_t fl = 0;
      int32_t sx = 0, sy = 0;
      if (ez >= C.zn) {
        fl = 1;
        if (!snap_rn(ex, ey, ez, C.fx, C.fy, C.cx, C.cy, sx, sy)) fl |= 2;
      }
      S.x[q] = ex; S.y[q] = ey; S.z[q] = ez;
      S.sx[q] = sx; S.sy[q] = sy; S.fl[q] = fl;
    }
  };

  // Pass 1 counts kept records; pass 2 writes them in id order.
  int my_count = 0;
  for (int bnd = 0; bnd < n_bands; ++bnd) {
    int k0 = bnd * band_rows, k1 = min(k0 + band_rows, n_cell_rows);
    __syncthreads();
    load_band(k0, k1);
    __syncthreads();
    int n_tri = 2 * (G - 1) * (k1 - k0);
    for (int q = threadIdx.x; q < n_tri; q += BLOCK) {
      int cell = q >> 1, half = q & 1;
      int kk = cell / (G - 1), j = cell % (G - 1);
      int id = 2 * ((k0 + kk) * (G - 1) + j) + half;
      int r0 = kk * G;
      TriRec tmp[2];
      if (half == 0) my_count += setup_parent(id, r0 + j, r0 + j + 1, r0 + G + j, S, C, tmp);
      else my_count += setup_parent(id, r0 + j + 1, r0 + G + j + 1, r0 + G + j, S, C, tmp);
    }
  }
  int total;
  block_exclusive_scan(my_count, s_warp, total);
  if (threadIdx.x == 0) {
    long long base = -1;
    if (total > 0) {
      unsigned long long b = atomicAdd(A.pool_counter, (unsigned long long)total);
      if ((long long)b + total <= A.pool_capacity) base = (long long)b;
      else atomicOr(A.error_word, kErrPoolOverflow);
    }
    s_base = base;
    R.seg_base = base < 0 ? 0 : (int32_t)base;
    R.seg_count = base < 0 ? 0 : total;
  }
  __syncthreads();
  const long long base = s_base;
  if (base < 0) return;
  long long run = 0;
  for (int bnd = 0; bnd < n_bands; ++bnd) {
    int k0 = bnd * band_rows, k1 = min(k0 + band_rows, n_cell_rows);
    if (n_bands > 1) {
      __syncthreads();
      load_band(k0, k1);
      __syncthreads();
    }
    int n_tri = 2 * (G - 1) * (k1 - k0);
    for (int q0 = 0; q0 < n_tri; q0 += BLOCK) {
      int q = q0 + threadIdx.x;
      TriRec tmp[2];
      int n = 0;
      if (q < n_tri) {
        int cell = q >> 1, half = q & 1;
        int kk = cell / (G - 1), j = cell % (G - 1);
        int id = 2 * ((k0 + kk) * (G - 1) + j) + half;
        int r0 = kk * G;
        if (half == 0) n = setup_parent(id, r0 + j, r0 + j + 1, r0 + G + j, S, C, tmp);
        else n = setup_parent(id, r0 + j + 1, r0 + G + j + 1, r0 + G + j, S, C, tmp);
      }
      int chunk_total;
      int off = block_exclusive_scan(n, s_warp, chunk_total);
      for (int k = 0; k < n; ++k) A.pool[base + run + off + k] = tmp[k];
      run += chunk_total;
    }
  }
}

constexpr int kSetupBlock = 256;
constexpr size_t kVtxBytes = 21;  // x, y, z, sx, sy (4 B each) + flags

static int setup_band_rows(int G, size_t smem_limit) {
  int rows = (int)(smem_limit / (kVtxBytes * (size_t)G)) - 1;
  if (rows > G - 1) rows = G - 1;
  if (rows < 1) rows = 1;
  return rows;
}

cudaError_t launch_tri_setup(const FrameArgs& a, cudaStream_t s) {
  const size_t limit = 160 * 1024;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t err = cudaFuncSetAttribute(tri_setup_kernel<kSetupBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)limit + 64);
    if (err != cudaSuccess) return err;
    attr_done = true;
  }
  int rows = setup_band_rows(a.G, limit);
  size_t bytes = (size_t)(rows + 1) * a.G * kVtxBytes + 64;
  dim3 grid(a.n_views, a.n_eyes);
  tri_setup_kernel<kSetupBlock><<<grid, kSetupBlock, bytes, s>>>(a, rows);
  return cudaGetLastError();
}

}  // namespace lfk
