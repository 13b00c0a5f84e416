// lf_refine.cu - the learned refinement y = x + f(x) applied to a normalised
// render (a learned image-space stand-in for the offline projection of Sec. 5,
// Eq. 4-5): three 3x3 convolutions 3->32->32->3 with ReLU, zero padding.
//
// Training kernels (this file): BF16 tensor-core (mma.sync m16n8k16) implicit
// GEMMs over 32x8-pixel output tiles with FP32 accumulation,
//   conv_mma_kernel   forward layers, backward through a layer's input (the
//                     same correlation with flipped, transposed weights), and a
//                     fused loss / dL/dr epilogue;
//   wgrad_kernel      weight and bias gradients, per-CTA partial sums reduced
//                     in a fixed order (deterministic);
//   adam_kernel       Adam (Kingma & Ba 2015, Algorithm 1) on FP32 master weights;
//   pack_weights_kernel  the BF16 operand layouts of every layer.
// The fused inference kernel (tcgen05 / TMEM) is in lf_refine_tc.cu.
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

namespace {

constexpr int kRTW = 32, kRTH = 8;                   // output tile: 8 warps x one 32-pixel row
constexpr int kHaloW = kRTW + 2, kHaloH = kRTH + 2;  // input tile with the 1-pixel ring
constexpr int kRowB = 80;                            // shared bytes per pixel row of 32 BF16 (+16: no bank conflicts)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}

// D += A(16x16, row) * B(16x8, col), BF16 operands, FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Stage the (kRTH+2) x (kRTW+2) input ring of a 32-channel BF16 map (zeros
// outside the image) as rows of kRowB bytes.
__device__ __forceinline__ void stage_halo32(unsigned char* s, const __nv_bfloat16* src, int img, int H, int W,
                                             int x0, int y0, int tid, int nthreads) {
  for (int i = tid; i < kHaloW * kHaloH * 4; i += nthreads) {
    const int pix = i >> 2, ch = i & 3;
    const int gy = y0 - 1 + pix / kHaloW, gx = x0 - 1 + pix % kHaloW;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gy >= 0 && gy < H && gx >= 0 && gx < W)
      v = reinterpret_cast<const uint4*>(src + (((size_t)img * H + gy) * W + gx) * 32)[ch];
    *reinterpret_cast<uint4*>(s + pix * kRowB + ch * 16) = v;
  }
}

// Stage the im2col rows of a 3-channel FP32 RGBA map for the tile's 256
// output pixels: k = tap * 3 + c (tap = ky * 3 + kx reads (y + ky - 1,
// x + kx - 1)), 27 used of 32, zeros outside the image.  One thread per pixel.
__device__ __forceinline__ void stage_im2col3(unsigned char* s, const float* src, int img, int H, int W, int x0,
                                              int y0, int p) {
  const int py = p >> 5, px = p & 31;
  float v[32];
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int gy = y0 + py + tap / 3 - 1, gx = x0 + px + tap % 3 - 1;
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gy >= 0 && gy < H && gx >= 0 && gx < W) t = reinterpret_cast<const float4*>(src)[((size_t)img * H + gy) * W + gx];
    v[tap * 3 + 0] = t.x;
    v[tap * 3 + 1] = t.y;
    v[tap * 3 + 2] = t.z;
  }
#pragma unroll
  for (int k = 27; k < 32; ++k) v[k] = 0.f;
  uint4* dst = reinterpret_cast<uint4*>(s + p * kRowB);
#pragma unroll
  for (int c = 0; c < 4; ++c)
    dst[c] = make_uint4(pack_bf16x2(v[8 * c + 0], v[8 * c + 1]), pack_bf16x2(v[8 * c + 2], v[8 * c + 3]),
                        pack_bf16x2(v[8 * c + 4], v[8 * c + 5]), pack_bf16x2(v[8 * c + 6], v[8 * c + 7]));
}

}  // namespace

// ------------------------------------------------------------------ convolution

// out[p][o] = sum_{tap, c} Wt[tap][o][c] * in[p + off(tap)][c]: M = 256 tile
// pixels (warp w owns output row w, two m16 tiles), N = COUT, K = 32 per tap.
// IN = kConvInRGBA takes the 3 channels of an FP32 RGBA map through im2col
// (one K = 32 "tap"); kConvInBF16 a 32-channel BF16 map, nine taps.
template <int IN, int COUT, int EPI>
__global__ void __launch_bounds__(256) conv_mma_kernel(RefineConvArgs A) {
  extern __shared__ __align__(16) unsigned char sm[];
  constexpr int NT = COUT / 8;
  constexpr int TAPS = IN == kConvInRGBA ? 1 : 9;
  unsigned char* s_w = sm;
  unsigned char* s_in = sm + TAPS * COUT * kRowB;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int img = blockIdx.z, x0 = blockIdx.x * kRTW, y0 = blockIdx.y * kRTH;
  const int H = A.H, W = A.W;

  for (int i = tid; i < TAPS * COUT * 4; i += 256)
    *reinterpret_cast<uint4*>(s_w + (i >> 2) * kRowB + (i & 3) * 16) = reinterpret_cast<const uint4*>(A.wt)[i];
  if (IN == kConvInBF16) stage_halo32(s_in, A.src_h, img, H, W, x0, y0, tid, 256);
  else stage_im2col3(s_in, A.src_f, img, H, W, x0, y0, tid);
  __syncthreads();

  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[mt][nt][i] = 0.f;

  const int mi = lane >> 3, r8 = lane & 7;
#pragma unroll 1
  for (int tap = 0; tap < TAPS; ++tap) {
    const int ky = tap / 3, kx = tap % 3;
#pragma unroll
    for (int kc = 0; kc < 32; kc += 16) {
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int px = mt * 16 + (mi & 1) * 8 + r8;
        const int pixel = IN == kConvInBF16 ? (warp + ky) * kHaloW + px + kx : warp * 32 + px;
        ldsm_x4(smem_u32(s_in + pixel * kRowB + (kc + (mi >> 1) * 8) * 2), a[mt]);
      }
      if (NT == 1) {
        uint32_t b0, b1;
        const int m2 = (lane >> 3) & 1;
        ldsm_x2(smem_u32(s_w + (tap * COUT + r8) * kRowB + (kc + m2 * 8) * 2), b0, b1);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][0], a[mt], b0, b1);
      } else {
#pragma unroll
        for (int np = 0; np < NT; np += 2) {
          uint32_t b[4];
          const int nrow = (np + (mi >> 1)) * 8 + r8;
          ldsm_x4(smem_u32(s_w + (tap * COUT + nrow) * kRowB + (kc + (mi & 1) * 8) * 2), b);
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            mma_bf16(acc[mt][np], a[mt], b[0], b[1]);
            mma_bf16(acc[mt][np + 1], a[mt], b[2], b[3]);
          }
        }
      }
    }
  }

  // Epilogue: acc[mt][nt][h*2 + j] is pixel mt*16 + lane/4 + 8h of the warp's
  // row, channel nt*8 + (lane%4)*2 + j.
  const int gy = y0 + warp;
  float lsum = 0.f;
  float scale = 0.f;
  if (EPI == kEpiLoss) {
    const int cnt = *A.count;
    scale = cnt > 0 ? 1.0f / (3.0f * (float)cnt) : 0.f;
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gx = x0 + mt * 16 + (lane >> 2) + 8 * h;
      if (gy >= H || gx >= W) continue;
      const size_t pix = ((size_t)img * H + gy) * W + gx;
      if (EPI == kEpiRelu || EPI == kEpiMask) {
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int ch = nt * 8 + (lane & 3) * 2;
          float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
          if (EPI == kEpiRelu) {
            v0 = fmaxf(v0 + A.bias[ch], 0.f);
            v1 = fmaxf(v1 + A.bias[ch + 1], 0.f);
          } else {
            const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(A.mask + pix * 32 + ch);
            if (!(__bfloat162float(m.x) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(m.y) > 0.f)) v1 = 0.f;
          }
          *reinterpret_cast<uint32_t*>(A.out_h + pix * 32 + ch) = pack_bf16x2(v0, v1);
        }
      } else {  // kEpiResid / kEpiLoss: three output channels in n-tile 0
        const int q = lane & 3;  // q = 0: channels 0, 1; q = 1: channel 2 (and alpha)
        if (q > 1) continue;
        const float4 x = reinterpret_cast<const float4*>(A.x)[pix];
        const float xc0 = q == 0 ? x.x : x.z, xc1 = x.y;
        const float r0 = acc[mt][0][2 * h] + A.bias[2 * q];
        const float y0v = xc0 + r0;
        float y1v = 0.f;
        if (q == 0) y1v = xc1 + (acc[mt][0][2 * h + 1] + A.bias[1]);
        if (EPI == kEpiResid) {
          const bool valid = x.w > 0.f;
          float2 o;
          o.x = valid ? y0v : 0.f;
          o.y = valid ? (q == 0 ? y1v : 1.f) : 0.f;
          reinterpret_cast<float2*>(A.out_f + pix * 4)[q] = o;
        } else {
          const float4 t = reinterpret_cast<const float4*>(A.target)[pix];
          const bool valid = x.w > 0.f && t.w > 0.f;
          const float d0 = valid ? y0v - (q == 0 ? t.x : t.z) : 0.f;
          const float d1 = (valid && q == 0) ? y1v - t.y : 0.f;
          lsum += d0 * d0 + d1 * d1;
          reinterpret_cast<float2*>(A.out_f + pix * 4)[q] = make_float2(2.f * scale * d0, 2.f * scale * d1);
        }
      }
    }
  }
  if (EPI == kEpiLoss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0 && lsum != 0.f) atomicAdd(A.loss, lsum * scale);
  }
}

// ------------------------------------------------------------------ weight gradients

// dW[o][c][tap] = sum_p g[p][o] * a[p + off(tap)][c] and db[o] = sum_p g[p][o]
// over a tile's 256 output pixels, accumulated over the CTA's tiles (a
// persistent loop) and written as one partial row per CTA.
//   MODE 1: g = dL/dz1 (32-ch BF16), a = im2col of the network input (K' = 27
//           of 32: one "tap"); 8 warps, warp w takes the pixels of row w and the
//           warps' sums are added at the end.  Row: W1 (864) then b1 (32).
//   MODE 2: g = dL/dz2 (32-ch BF16), a = a1; 9 warps, warp = tap.  W2, b2.
//   MODE 3: g = dL/dr (FP32 RGBA, 3 channels, padded to 16), a = a2; 9 warps.  W3, b3.
// M = output channels (A = g^T, loaded transposed), N = input channels (B = the
// shifted input rows, loaded transposed), K = pixels.
template <int MODE>
__global__ void __launch_bounds__(MODE == 1 ? 256 : 288) wgrad_kernel(RefineWgradArgs A) {
  constexpr int NTHREADS = MODE == 1 ? 256 : 288;
  constexpr int MT = MODE == 3 ? 1 : 2;              // m16 tiles of output channels
  constexpr int GROW = MODE == 3 ? 48 : kRowB;       // shared bytes per g row
  constexpr int COUT = MODE == 3 ? 3 : 32;
  constexpr int SEG = MODE == 1 ? 864 + 32 : (MODE == 2 ? 9216 + 32 : 864 + 3);
  extern __shared__ __align__(16) unsigned char sm[];
  unsigned char* s_g = sm;
  unsigned char* s_a = sm + 256 * GROW;
  __shared__ float s_bias[9][32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int H = A.H, W = A.W;
  const int mi = lane >> 3, r8 = lane & 7;

  float acc[MT][4][4];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[mt][nt][i] = 0.f;
  float bsum = 0.f;
  const int bch = tid & 31, bgrp = tid >> 5;  // bias: channel, pixel group

#pragma unroll 1
  for (int tile = blockIdx.x; tile < A.n_tiles; tile += gridDim.x) {
    const int img = tile / (A.tiles_x * A.tiles_y);
    const int rem = tile - img * A.tiles_x * A.tiles_y;
    const int y0 = (rem / A.tiles_x) * kRTH, x0 = (rem % A.tiles_x) * kRTW;
    __syncthreads();  // the previous tile's operands are no longer read
    if (MODE == 3) {
      for (int p = tid; p < 256; p += NTHREADS) {
        const int gy = y0 + (p >> 5), gx = x0 + (p & 31);
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gy < H && gx < W) t = reinterpret_cast<const float4*>(A.g_f)[((size_t)img * H + gy) * W + gx];
        uint4* d = reinterpret_cast<uint4*>(s_g + p * GROW);
        d[0] = make_uint4(pack_bf16x2(t.x, t.y), pack_bf16x2(t.z, 0.f), 0u, 0u);
        d[1] = make_uint4(0u, 0u, 0u, 0u);
      }
    } else {
      for (int i = tid; i < 256 * 4; i += NTHREADS) {
        const int p = i >> 2, ch = i & 3;
        const int gy = y0 + (p >> 5), gx = x0 + (p & 31);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gy < H && gx < W) v = reinterpret_cast<const uint4*>(A.g_h + (((size_t)img * H + gy) * W + gx) * 32)[ch];
        *reinterpret_cast<uint4*>(s_g + p * GROW + ch * 16) = v;
      }
    }
    if (MODE == 1) stage_im2col3(s_a, A.x, img, H, W, x0, y0, tid);
    else stage_halo32(s_a, A.a_h, img, H, W, x0, y0, tid, NTHREADS);
    __syncthreads();

    // bias: sum of g over the tile's pixels
    if (bch < COUT) {
      const int ngrp = NTHREADS / 32;
      for (int p = bgrp; p < 256; p += ngrp)
        bsum += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(s_g + p * GROW + bch * 2));
    }

    const int ky = MODE == 1 ? 0 : warp / 3, kx = MODE == 1 ? 0 : warp % 3;
    const int s0 = MODE == 1 ? warp * 2 : 0, s1 = MODE == 1 ? warp * 2 + 2 : 16;
#pragma unroll 1
    for (int s = s0; s < s1; ++s) {  // 16-pixel K steps: row s/2, columns (s%2)*16 ..
      const int py = s >> 1, px0 = (s & 1) * 16;
      uint32_t a[MT][4];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int p = py * 32 + px0 + (mi >> 1) * 8 + r8;
        ldsm_x4_t(smem_u32(s_g + p * GROW + (mt * 16 + (mi & 1) * 8) * 2), a[mt]);
      }
#pragma unroll
      for (int np = 0; np < 4; np += 2) {
        uint32_t b[4];
        const int pp = px0 + (mi & 1) * 8 + r8;
        const int row = MODE == 1 ? py * 32 + pp : (py + ky) * kHaloW + pp + kx;
        ldsm_x4_t(smem_u32(s_a + row * kRowB + (np + (mi >> 1)) * 16), b);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          mma_bf16(acc[mt][np], a[mt], b[0], b[1]);
          mma_bf16(acc[mt][np + 1], a[mt], b[2], b[3]);
        }
      }
    }
  }

  // ---- write this CTA's partial row
  float* out = A.partial + (size_t)blockIdx.x * SEG;
  __syncthreads();
  s_bias[bgrp][bch] = bsum;
  if (MODE == 1) {
    float* red = reinterpret_cast<float*>(sm);  // [8 warps][32 o][32 k']
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int o = mt * 16 + (lane >> 2) + 8 * (i >> 1), k = nt * 8 + (lane & 3) * 2 + (i & 1);
          red[(warp * 32 + o) * 32 + k] = acc[mt][nt][i];
        }
    __syncthreads();
    for (int e = tid; e < 32 * 27; e += NTHREADS) {
      const int o = e / 27, k = e % 27;
      float s = 0.f;
      for (int w = 0; w < 8; ++w) s += red[(w * 32 + o) * 32 + k];
      out[o * 27 + (k % 3) * 9 + k / 3] = s;  // k = tap * 3 + c -> W1[o][c][tap]
    }
  } else {
    const int tap = warp;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int o = mt * 16 + (lane >> 2) + 8 * (i >> 1), c = nt * 8 + (lane & 3) * 2 + (i & 1);
          if (o < COUT) out[(o * 32 + c) * 9 + tap] = acc[mt][nt][i];
        }
    __syncthreads();
  }
  __syncthreads();
  if (tid < COUT) {
    float s = 0.f;
    for (int g = 0; g < NTHREADS / 32; ++g) s += s_bias[g][tid];
    out[SEG - COUT + tid] = s;
  }
}

// grad[base + i] = sum over CTAs b (in order) of partial[b][i].
__global__ void reduce_partials_kernel(const float* __restrict__ partial, int n_rows, int seg,
                                       float* __restrict__ grad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < seg; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < n_rows; ++b) s += partial[(size_t)b * seg + i];
    grad[i] = s;
  }
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

namespace {

template <int IN, int COUT, int EPI>
cudaError_t launch_conv_t(const RefineConvArgs& a, cudaStream_t s) {
  const int taps = IN == kConvInRGBA ? 1 : 9;
  const int in_bytes = IN == kConvInRGBA ? 256 * kRowB : kHaloW * kHaloH * kRowB;
  const int smem = taps * COUT * kRowB + in_bytes;
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(conv_mma_kernel<IN, COUT, EPI>), smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.W + kRTW - 1) / kRTW, (a.H + kRTH - 1) / kRTH, a.n);
  conv_mma_kernel<IN, COUT, EPI><<<grid, 256, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_wgrad_t(const RefineWgradArgs& a, cudaStream_t s) {
  const int g_bytes = 256 * (MODE == 3 ? 48 : kRowB);
  const int a_bytes = MODE == 1 ? 256 * kRowB : kHaloW * kHaloH * kRowB;
  int smem = g_bytes + a_bytes;
  if (MODE == 1 && smem < 8 * 32 * 32 * 4) smem = 8 * 32 * 32 * 4;  // the cross-warp reduction reuses it
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(wgrad_kernel<MODE>), smem);
  if (e != cudaSuccess) return e;
  wgrad_kernel<MODE><<<a.n_ctas, MODE == 1 ? 256 : 288, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_refine_conv(int in_mode, int cout, int epi, const RefineConvArgs& a, cudaStream_t s) {
  if (in_mode == kConvInRGBA && cout == 32 && epi == kEpiRelu) return launch_conv_t<kConvInRGBA, 32, kEpiRelu>(a, s);
  if (in_mode == kConvInRGBA && cout == 32 && epi == kEpiMask) return launch_conv_t<kConvInRGBA, 32, kEpiMask>(a, s);
  if (in_mode == kConvInBF16 && cout == 32 && epi == kEpiRelu) return launch_conv_t<kConvInBF16, 32, kEpiRelu>(a, s);
  if (in_mode == kConvInBF16 && cout == 32 && epi == kEpiMask) return launch_conv_t<kConvInBF16, 32, kEpiMask>(a, s);
  if (in_mode == kConvInBF16 && cout == 8 && epi == kEpiResid) return launch_conv_t<kConvInBF16, 8, kEpiResid>(a, s);
  if (in_mode == kConvInBF16 && cout == 8 && epi == kEpiLoss) return launch_conv_t<kConvInBF16, 8, kEpiLoss>(a, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_refine_wgrad(int mode, const RefineWgradArgs& a, cudaStream_t s) {
  if (mode == 1) return launch_wgrad_t<1>(a, s);
  if (mode == 2) return launch_wgrad_t<2>(a, s);
  if (mode == 3) return launch_wgrad_t<3>(a, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_refine_reduce(const float* partial, int n_rows, int seg, float* grad, cudaStream_t s) {
  reduce_partials_kernel<<<(seg + 255) / 256, 256, 0, s>>>(partial, n_rows, seg, grad);
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
