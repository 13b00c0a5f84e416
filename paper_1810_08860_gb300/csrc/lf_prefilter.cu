// lf_prefilter.cu - Eq. 5 of the light field prefilter (Sec. 5.1): per pixel
// (s', t') of one source view, the Monte Carlo ratio
//     sum_j rho_j sigma_j Lbar_j / sum_j rho_j sigma_j
// over samples j, each a point o_j on the view's disk and an offset (ds, dt)
// of the Lanczos-2 pixel basis.  The ray of sample j leaves o_j toward X, the
// point where image point (s' + ds, t' + dt) lands on the view's own mesh.
// All rays of a sample share o_j, so the host renders Lbar for them as one
// pinhole view at o_j (the method itself, on the dense model); this kernel
// reads that render at X's projection with a bilinear filter on colour
// premultiplied by the render's alpha, so pixels no dense view covers add no
// weight.  FP32 values throughout; the only decision is den > 0.
#include <cuda_fp16.h>

#include "lf_prefilter.h"

namespace lfk {

namespace {

__device__ __forceinline__ float4 load_pm(const float4* __restrict__ img, int Ws, int x, int y) {
  const float4 c = __ldg(img + (int64_t)y * Ws + x);
  return make_float4(c.x * c.w, c.y * c.w, c.z * c.w, c.w);
}

__device__ __forceinline__ float grid_depth(const PrefilterArgs& A, int k, int j, float z0) {
  const int64_t gi = ((int64_t)A.view * A.G + k) * A.G + j;
  if (A.mesh_format == LF_MESH_F16_OFFSET)
    return z0 + __half2float(reinterpret_cast<const __half*>(A.depth)[gi]);
  return __ldg(reinterpret_cast<const float*>(A.depth) + gi);
}

__global__ void __launch_bounds__(256) prefilter_accumulate_kernel(PrefilterArgs A) {
  const int px = blockIdx.x * 16 + (threadIdx.x & 15);
  const int py = blockIdx.y * 16 + (threadIdx.x >> 4);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && *A.dense_error) atomicOr(A.error, *A.dense_error);
  if (px >= A.W || py >= A.H) return;
  const int G = A.G;
  const float* ta = A.tab_a + (int64_t)A.view * G;
  const float* tb = A.tab_b + (int64_t)A.view * G;
  const float z0 = A.views[A.view].depth_origin;
  const float gsx = (float)(G - 1) / (float)A.W, gsy = (float)(G - 1) / (float)A.H;
  float nr = 0.f, ng = 0.f, nb = 0.f, den = 0.f;
  for (int j = 0; j < A.n_samples; ++j) {
    const float4 smp = __ldg(A.sample + j);
    const float2 off = __ldg(A.offset + j);
    // the image point, clamped to the rectangle the mesh spans
    const float s = fminf(fmaxf((float)px + 0.5f + off.x, 0.0f), (float)A.W);
    const float t = fminf(fmaxf((float)py + 0.5f + off.y, 0.0f), (float)A.H);
    const float gx = s * gsx, gy = t * gsy;
    const int cj = min(max((int)floorf(gx), 0), G - 2), ck = min(max((int)floorf(gy), 0), G - 2);
    const bool upper = (gx - (float)cj) + (gy - (float)ck) > 1.0f;  // beyond the (j+1,k)-(j,k+1) diagonal
    // the holding triangle's vertices in the view's camera frame
    const int ja = upper ? cj + 1 : cj, ka = ck;          // v0: (j,k) or (j+1,k)
    const int jb = cj + 1, kb = upper ? ck + 1 : ck;      // v1: (j+1,k) or (j+1,k+1)
    const int jc = cj, kc = ck + 1;                       // v2: (j,k+1)
    const float za = grid_depth(A, ka, ja, z0), zb = grid_depth(A, kb, jb, z0), zc = grid_depth(A, kc, jc, z0);
    const float3 v0 = make_float3(za * __ldg(ta + ja), za * __ldg(tb + ka), za);
    const float3 v1 = make_float3(zb * __ldg(ta + jb), zb * __ldg(tb + kb), zb);
    const float3 v2 = make_float3(zc * __ldg(ta + jc), zc * __ldg(tb + kc), zc);
    const float3 e1 = make_float3(v1.x - v0.x, v1.y - v0.y, v1.z - v0.z);
    const float3 e2 = make_float3(v2.x - v0.x, v2.y - v0.y, v2.z - v0.z);
    const float3 n = make_float3(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
    const float ex = (s - A.cx) / A.fx, ey = (t - A.cy) / A.fy;
    const float ne = n.x * ex + n.y * ey + n.z;
    if (ne == 0.0f) continue;
    const float z = (n.x * v0.x + n.y * v0.y + n.z * v0.z) / ne;
    // X seen from the sample's aperture point (the render shares the view's rotation)
    const float xx = z * ex - smp.x, xy = z * ey - smp.y, xz = z - smp.z;
    if (!(xz > 0.0f)) continue;
    const float u = fminf(fmaxf(A.fxs * (xx / xz) + A.cxs - 0.5f, -1.0f), (float)A.Ws);
    const float v = fminf(fmaxf(A.fys * (xy / xz) + A.cys - 0.5f, -1.0f), (float)A.Hs);
    const float fu = floorf(u), fv = floorf(v);
    const float al = u - fu, be = v - fv;
    const int i0 = min(max((int)fu, 0), A.Ws - 1), i1 = min(max((int)fu + 1, 0), A.Ws - 1);
    const int j0 = min(max((int)fv, 0), A.Hs - 1), j1 = min(max((int)fv + 1, 0), A.Hs - 1);
    const float4* img = A.renders + (int64_t)j * A.Ws * A.Hs;
    const float4 c00 = load_pm(img, A.Ws, i0, j0), c10 = load_pm(img, A.Ws, i1, j0);
    const float4 c01 = load_pm(img, A.Ws, i0, j1), c11 = load_pm(img, A.Ws, i1, j1);
    const float w00 = (1.f - al) * (1.f - be), w10 = al * (1.f - be), w01 = (1.f - al) * be, w11 = al * be;
    const float w = smp.w;
    nr += w * (w00 * c00.x + w10 * c10.x + w01 * c01.x + w11 * c11.x);
    ng += w * (w00 * c00.y + w10 * c10.y + w01 * c01.y + w11 * c11.y);
    nb += w * (w00 * c00.z + w10 * c10.z + w01 * c01.z + w11 * c11.z);
    den += w * (w00 * c00.w + w10 * c10.w + w01 * c01.w + w11 * c11.w);
  }
  float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
  if (den > 0.0f) {
    const float inv = 1.0f / den;
    o = make_float4(nr * inv, ng * inv, nb * inv, 1.0f);
  }
  A.out[(int64_t)py * A.W + px] = o;
}

}  // namespace

cudaError_t launch_prefilter_accumulate(const PrefilterArgs& a, cudaStream_t s) {
  if (a.W <= 0 || a.H <= 0) return cudaSuccess;
  dim3 grid((a.W + 15) / 16, (a.H + 15) / 16);
  prefilter_accumulate_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lfk
