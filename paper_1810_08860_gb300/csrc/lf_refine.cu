// lf_refine.cu - the learned refinement y = x + f(x) applied to a normalised
// render (a learned image-space stand-in for the offline projection of Sec. 5,
// Eq. 4-5): three 3x3 convolutions 3->32->32->3 with ReLU, zero padding.
//
// Training kernels (this file): the per-CTA partial-sum reduction of the
// weight gradients (a fixed order: deterministic), the count of valid pixels,
// Adam (Kingma & Ba 2015, Algorithm 1) on FP32 master weights, and
// pack_weights_kernel (the BF16 operand layouts of every layer).  The GEMMs of
// training and of the per-layer path (convolutions forward and backward, the
// loss epilogue, weight and bias gradients) run on tcgen05 in
// lf_refine_conv_tc.cu; the fused inference kernel is in lf_refine_tc.cu.
//
// Layouts.  Images: n x H x W x 4 FP32 (RGBA).  Hidden activations and their
// gradients: n x H x W x 32 BF16.  Parameters: the flat FP32 vector
// W1[32][3][3][3], b1[32], W2[32][32][3][3], b2[32], W3[3][32][3][3], b3[3].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "lf_internal.h"
#include "lf_launch.h"

namespace lfk {

// grad[base + i] = sum over the CTA rows b of partial[b][i], in a fixed order:
// eight interleaved sums (rows k, k + 8, k + 16, .. for k < 8) added pairwise.
// 256 threads: 8 row phases x 32 consecutive outputs.
__global__ void reduce_partials_kernel(const float* __restrict__ partial, int n_rows, int seg,
                                       float* __restrict__ grad) {
  __shared__ float part[8][32];
  const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (i < seg)
    for (int b = k; b < n_rows; b += 8) s += partial[(size_t)b * seg + i];
  part[k][lane] = s;
  __syncthreads();
  if (k == 0 && i < seg)
    grad[i] = ((part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane])) +
              ((part[4][lane] + part[5][lane]) + (part[6][lane] + part[7][lane]));
}

// Number of pixels valid (alpha > 0) in both the input and the target.
__global__ void count_valid_kernel(const float4* __restrict__ x, const float4* __restrict__ t, int64_t n,
                                   int* __restrict__ count) {
  int c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += (x[i].w > 0.f && t[i].w > 0.f) ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// Adam on the FP32 master weights; omb = 1 - beta (rounded once from the
// exact value), c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t).
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float beta1, float beta2, float omb1,
                            float omb2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = __fadd_rn(__fmul_rn(beta1, m[i]), __fmul_rn(omb1, gi));
  const float vi = __fadd_rn(__fmul_rn(beta2, v[i]), __fmul_rn(__fmul_rn(omb2, gi), gi));
  m[i] = mi;
  v[i] = vi;
  const float den = __fadd_rn(__fsqrt_rn(__fmul_rn(vi, c2)), eps);
  p[i] = __fsub_rn(p[i], __fmul_rn(lr, __fdiv_rn(__fmul_rn(mi, c1), den)));
}

// BF16 operand layouts of every layer from the FP32 parameters.
//   w1f[32 o][32 k']      k' = tap * 3 + c < 27: W1[o][c][tap]
//   w2f[9][32 o][32 c]    W2[o][c][tap]
//   w3f[9][8 o][32 c]     W3[o][c][tap], o < 3
//   w3b[32 c][32 k']      k' = tap * 3 + o < 27: W3[o][c][8 - tap]   (through layer 3's input)
//   w2b[9][32 c][32 o]    W2[o][c][8 - tap]                         (through layer 2's input)
//   then the fused kernel's B operands, K-major groups g of 8 channels:
//   L1 [dy][g][o][8] over the pair-packed input (x[q-1], x[q]) | (x[q+1], x[q+2]),
//   four channels R, G, B, 1 per position: kernel column kx = 2g + (e >= 4),
//   b1 at the constant 1 of the centre tap; L2 [dy][kc][g][kx*32 + o][8] and
//   L3 [dy][kc][g][kx*4 + o][8] (kernel columns stacked along N) with input
//   channel c = kc*16 + g*8 + e.  b2 and b3 are read in FP32 by the fused kernel.
__global__ void pack_weights_kernel(const float* __restrict__ prm, __nv_bfloat16* __restrict__ w) {
  constexpr int n1 = 32 * 32, n2 = 9 * 32 * 32, n3 = 9 * 8 * 32, n3b = 32 * 32, n2b = 9 * 32 * 32;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float v = 0.f;
  if (i < n1) {
    const int o = i >> 5, k = i & 31;
    if (k < 27) v = prm[kRefineOffW1 + o * 27 + (k % 3) * 9 + k / 3];
  } else if (i < n1 + n2) {
    const int j = i - n1, tap = j >> 10, o = (j >> 5) & 31, c = j & 31;
    v = prm[kRefineOffW2 + (o * 32 + c) * 9 + tap];
  } else if (i < n1 + n2 + n3) {
    const int j = i - n1 - n2, tap = j >> 8, o = (j >> 5) & 7, c = j & 31;
    if (o < 3) v = prm[kRefineOffW3 + (o * 32 + c) * 9 + tap];
  } else if (i < n1 + n2 + n3 + n3b) {
    const int j = i - n1 - n2 - n3, c = j >> 5, k = j & 31;
    if (k < 27) v = prm[kRefineOffW3 + ((k % 3) * 32 + c) * 9 + (8 - k / 3)];
  } else if (i < n1 + n2 + n3 + n3b + n2b) {
    const int j = i - n1 - n2 - n3 - n3b, tap = j >> 10, c = (j >> 5) & 31, o = j & 31;
    v = prm[kRefineOffW2 + (o * 32 + c) * 9 + (8 - tap)];
  } else if (i < kPackTc + 1536) {  // L1 [dy][g][o][e]: tap kx = 2g + e/4, channel e%4
    const int j = i - kPackTc, dy = j / 512, g = (j / 256) & 1, o = (j >> 3) & 31, e = j & 7;
    const int kx = 2 * g + (e >> 2), c = e & 3;
    if (kx < 3 && c < 3) v = prm[kRefineOffW1 + o * 27 + c * 9 + dy * 3 + kx];
    else if (kx == 1 && c == 3 && dy == 1) v = prm[kRefineOffB1 + o];  // b1 meets the constant input channel
  } else if (i < kPackTc + 1536 + 9216) {  // L2 [dy][kc][g][n = kx*32 + o][e], c = kc*16 + g*8 + e
    const int j = i - kPackTc - 1536, dy = j / 3072, kc = (j / 1536) & 1, g = (j / 768) & 1, n = (j >> 3) % 96;
    const int c = kc * 16 + g * 8 + (j & 7), kx = n >> 5, o = n & 31;
    v = prm[kRefineOffW2 + (o * 32 + c) * 9 + dy * 3 + kx];
  } else if (i < kRefinePackedElems) {  // L3 [dy][kc][g][n = kx*4 + o][e], o < 3
    const int j = i - kPackTc - 1536 - 9216, dy = j / 512, kc = (j / 256) & 1, g = (j / 128) & 1, n = (j >> 3) & 15;
    const int c = kc * 16 + g * 8 + (j & 7), kx = n >> 2, o = n & 3;
    if (o < 3 && kx < 3) v = prm[kRefineOffW3 + (o * 32 + c) * 9 + dy * 3 + kx];
  } else {
    return;
  }
  w[i] = __float2bfloat16_rn(v);
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_refine_reduce(const float* partial, int n_rows, int seg, float* grad, cudaStream_t s) {
  reduce_partials_kernel<<<(seg + 31) / 32, 256, 0, s>>>(partial, n_rows, seg, grad);
  return cudaGetLastError();
}

cudaError_t launch_refine_count(const float* x, const float* t, int64_t n_pix, int* count, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((n_pix + 255) / 256, 1024);
  count_valid_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(reinterpret_cast<const float4*>(x),
                                                             reinterpret_cast<const float4*>(t), n_pix, count);
  return cudaGetLastError();
}

cudaError_t launch_refine_adam(float* p, float* m, float* v, const float* g, int n, float lr, double beta1,
                               double beta2, float eps, float c1, float c2, cudaStream_t s) {
  adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(p, m, v, g, n, lr, (float)beta1, (float)beta2, (float)(1.0 - beta1),
                                              (float)(1.0 - beta2), eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_refine_pack(const float* params, __nv_bfloat16* w, cudaStream_t s) {
  pack_weights_kernel<<<(kRefinePackedElems + 255) / 256, 256, 0, s>>>(params, w);
  return cudaGetLastError();
}

}  // namespace lfk
