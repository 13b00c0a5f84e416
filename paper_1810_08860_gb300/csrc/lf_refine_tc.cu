// lf_refine_tc.cu - fused inference of the learned refinement y = x + f(x)
// (three 3x3 convolutions 3->32->32->3, ReLU, zero padding; the learned
// stand-in for the offline projection of Sec. 5, Eq. 4-5) on the
// fifth-generation tensor cores: tcgen05.mma from shared memory into TMEM.
//
// One persistent CTA per SM loops over output tiles of 26 x 30 pixels.  The
// tile's input is held as a 32 x 36 halo of positions q = 32*hy + hx (3-pixel
// ring), and every layer is computed over a contiguous range of q as an
// implicit GEMM whose A rows are the positions themselves: the 3x3 tap
// (dy, dx) is the same operand shifted by 32*dy + dx rows.  Rows whose taps
// wrap across a halo row are computed but never read by a needed output.
//   layer 1: 9 M-tiles of 128 positions, per tap one K = 16 MMA (3 real input
//            channels), N = 32;
//   layer 2: 8 M-tiles, per tap two K = 16 MMAs, N = 32;
//   layer 3: 8 M-tiles, per tap two K = 16 MMAs, N = 16 (3 real outputs).
// After each layer all 8 warps read the accumulators (tcgen05.ld, warp w sees
// TMEM lanes 32*(w%4) ..), add the bias, apply ReLU, zero positions outside
// the image (the next layer's zero padding) and store BF16 back to shared
// memory for the next layer.  The residual add uses the FP32 input from global
// memory.  One thread issues the MMAs and commits them to an mbarrier; every
// wait is bounded and reports through an error flag instead of hanging.
//
// Shared-memory operands use the K-major layout without swizzling: a position
// (row) holds 8 channels in 16 contiguous bytes, rows follow each other every
// 16 bytes (8-row core matrices 128 bytes apart), and each further group of 8
// channels starts kGroupB bytes later.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lf_internal.h"

namespace lfk {

namespace {

constexpr int kHW = 32, kHH = 36;                    // halo tile (positions)
constexpr int kTW = kHW - 6, kTH = kHH - 6;          // 26 x 30 output pixels
constexpr int kRows = 1280;                          // positions held per buffer (10 x 128)
constexpr int kGroupB = kRows * 16;                  // bytes per group of 8 channels
constexpr int kBufB = 4 * kGroupB;                   // 32 channels
constexpr int kW1B = 9 * 1024, kW2B = 9 * 2048, kW3B = 9 * 1024;
constexpr int kWB = kW1B + kW2B + kW3B;              // 36,864 bytes of BF16 weights
constexpr int kSmemBytes = 2 * kBufB + kWB + 64;
constexpr int kStart1 = kHW + 1, kTiles1 = 9;        // layer 1 rows [33, 1185)
constexpr int kStart2 = 2 * (kHW + 1), kTiles2 = 8;  // layer 2 rows [66, 1090)
constexpr int kStart3 = 3 * (kHW + 1), kTiles3 = 8;  // layer 3 rows [99, 1123)
constexpr uint32_t kTmemCols = 512;
constexpr int kThreads = 256;
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance
// between channel groups (K), sbo = between 8-row core matrices (M or N).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t addr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t addr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ int tap_shift(int tap) { return (tap / 3 - 1) * kHW + (tap % 3 - 1); }

struct FusedArgs {
  int32_t n, H, W, tiles_x, tiles_y, n_tiles;
  const float* in;
  float* out;
  const float* bias;             // b1 (32), b2 (32), b3 (3) at their parameter offsets
  const __nv_bfloat16* wtc;      // w1t [9][2][32][8], w2t [9][4][32][8], w3t [9][4][16][8]
  int32_t* error;                // set to 1 if a wait gave up
};

// Hidden-layer epilogue: accumulators of M-tile rows -> bias, ReLU, zero
// outside the image -> BF16 rows of `dst` (4 groups of 8 channels).
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem, int start, int n_mtiles, const float* bias,
                                                unsigned char* dst, int x0, int y0, int H, int W) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3;
  for (int mt = warp >> 2; mt < n_mtiles; mt += 2) {
    const int q = start + mt * 128 + quarter * 32 + lane;
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(mt * 32), v);
    if (q >= kRows) continue;
    const int hy = q >> 5, hx = q & 31;
    const int gy = y0 - 3 + hy, gx = x0 - 3 + hx;
    const bool inside = hy < kHH && gy >= 0 && gy < H && gx >= 0 && gx < W;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = g * 8 + 2 * j;
        const float a = inside ? fmaxf(v[c] + bias[c], 0.f) : 0.f;
        const float b = inside ? fmaxf(v[c + 1] + bias[c + 1], 0.f) : 0.f;
        w[j] = pack2(a, b);
      }
      *reinterpret_cast<uint4*>(dst + g * kGroupB + q * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) refine_fused_kernel(FusedArgs A) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* buf0 = sm;          // x (group 0), then a2
  unsigned char* buf1 = sm + kBufB;  // a1
  unsigned char* wts = sm + 2 * kBufB;
  uint64_t* bar = reinterpret_cast<uint64_t*>(wts + kWB);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wts + kWB + 8);
  __shared__ int s_abort;
  __shared__ float s_bias[67];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // Both activation buffers start at zero (rows never written stay finite),
  // then the weights and biases.
  for (int i = tid; i < 2 * kBufB / 16; i += kThreads) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < kWB / 16; i += kThreads)
    reinterpret_cast<uint4*>(wts)[i] = reinterpret_cast<const uint4*>(A.wtc)[i];
  if (tid < 32) s_bias[tid] = A.bias[kRefineOffB1 + tid];
  else if (tid < 64) s_bias[tid] = A.bias[kRefineOffB2 + tid - 32];
  else if (tid < 67) s_bias[tid] = A.bias[kRefineOffB3 + tid - 64];
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t s0 = su32(buf0), s1 = su32(buf1), sw = su32(wts);
  const int H = A.H, W = A.W;
  uint32_t phase = 0;

  for (int tile = blockIdx.x; tile < A.n_tiles; tile += gridDim.x) {
    const int per_img = A.tiles_x * A.tiles_y;
    const int img = tile / per_img, rem = tile - img * per_img;
    const int y0 = (rem / A.tiles_x) * kTH, x0 = (rem % A.tiles_x) * kTW;
    const float4* in = reinterpret_cast<const float4*>(A.in) + (size_t)img * H * W;

    // ---- stage x (3 channels + zeros) into group 0 of buf0
    for (int q = tid; q < kRows; q += kThreads) {
      const int hy = q >> 5, hx = q & 31;
      const int gy = y0 - 3 + hy, gx = x0 - 3 + hx;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (hy < kHH && gy >= 0 && gy < H && gx >= 0 && gx < W) v = in[(size_t)gy * W + gx];
      *reinterpret_cast<uint4*>(buf0 + q * 16) = make_uint4(pack2(v.x, v.y), pack2(v.z, 0.f), 0u, 0u);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();

    // ---- layer 1: A = x rows (group 0; group 1 is multiplied by zero weights)
    if (tid == 0) {
      tc_after_sync();
      for (int mt = 0; mt < kTiles1; ++mt)
        for (int tap = 0; tap < 9; ++tap) {
          const int q = kStart1 + mt * 128 + tap_shift(tap);
          mma(tmem + mt * 32, smem_desc(s0 + q * 16, kGroupB, 128), smem_desc(sw + tap * 1024, 512, 128),
              instr_desc(128, 32), tap > 0);
        }
      commit(bar);
    }
    bool ok = __all_sync(0xffffffffu, wait_phase(bar, phase));
    phase ^= 1u;
    if (!ok) s_abort = 1;
    tc_after_sync();
    if (ok) hidden_epilogue(tmem, kStart1, kTiles1, s_bias, buf1, x0, y0, H, W);
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    if (s_abort) break;

    // ---- layer 2: A = a1 (buf1), two K halves of 16 channels
    if (tid == 0) {
      tc_after_sync();
      for (int mt = 0; mt < kTiles2; ++mt)
        for (int tap = 0; tap < 9; ++tap)
          for (int kc = 0; kc < 2; ++kc) {
            const int q = kStart2 + mt * 128 + tap_shift(tap);
            mma(tmem + mt * 32, smem_desc(s1 + kc * 2 * kGroupB + q * 16, kGroupB, 128),
                smem_desc(sw + kW1B + tap * 2048 + kc * 1024, 512, 128), instr_desc(128, 32), (tap | kc) != 0);
          }
      commit(bar);
    }
    ok = __all_sync(0xffffffffu, wait_phase(bar, phase));
    phase ^= 1u;
    if (!ok) s_abort = 1;
    tc_after_sync();
    if (ok) hidden_epilogue(tmem, kStart2, kTiles2, s_bias + 32, buf0, x0, y0, H, W);
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    if (s_abort) break;

    // ---- layer 3: A = a2 (buf0), N = 16 (3 real outputs)
    if (tid == 0) {
      tc_after_sync();
      for (int mt = 0; mt < kTiles3; ++mt)
        for (int tap = 0; tap < 9; ++tap)
          for (int kc = 0; kc < 2; ++kc) {
            const int q = kStart3 + mt * 128 + tap_shift(tap);
            mma(tmem + mt * 16, smem_desc(s0 + kc * 2 * kGroupB + q * 16, kGroupB, 128),
                smem_desc(sw + kW1B + kW2B + tap * 1024 + kc * 512, 256, 128), instr_desc(128, 16),
                (tap | kc) != 0);
          }
      commit(bar);
    }
    ok = __all_sync(0xffffffffu, wait_phase(bar, phase));
    phase ^= 1u;
    if (!ok) s_abort = 1;
    tc_after_sync();
    if (ok) {
      const int quarter = warp & 3;
      float4* out = reinterpret_cast<float4*>(A.out) + (size_t)img * H * W;
      for (int mt = warp >> 2; mt < kTiles3; mt += 2) {
        const int q = kStart3 + mt * 128 + quarter * 32 + lane;
        float r[4];
        tmem_ld4(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(mt * 16), r);
        const int hy = q >> 5, hx = q & 31;
        if (hy < 3 || hy >= 3 + kTH || hx < 3 || hx >= 3 + kTW) continue;
        const int gy = y0 - 3 + hy, gx = x0 - 3 + hx;
        if (gy >= H || gx >= W) continue;
        const float4 x = in[(size_t)gy * W + gx];
        float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x.w > 0.f) {
          y.x = x.x + (r[0] + s_bias[64]);
          y.y = x.y + (r[1] + s_bias[65]);
          y.z = x.z + (r[2] + s_bias[66]);
          y.w = 1.f;
        }
        out[(size_t)gy * W + gx] = y;
      }
    }
    tc_before_sync();
    __syncthreads();  // the next tile overwrites buf0 and the accumulators
    if (s_abort) break;
  }

  if (tid == 0 && s_abort) atomicOr(A.error, 1);
  __syncthreads();
  if (warp == 0) {
    tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

}  // namespace

cudaError_t launch_refine_fused(int32_t n, int32_t w, int32_t h, const float* in, float* out, const float* params,
                                const __nv_bfloat16* packed, int sm_count, int32_t* error, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(refine_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  FusedArgs a;
  a.n = n;
  a.H = h;
  a.W = w;
  a.tiles_x = (w + kTW - 1) / kTW;
  a.tiles_y = (h + kTH - 1) / kTH;
  a.n_tiles = a.tiles_x * a.tiles_y * n;
  a.in = in;
  a.out = out;
  a.bias = params;
  a.wtc = packed + kPackTc;
  a.error = error;
  if (a.n_tiles == 0) return cudaSuccess;
  const int grid = a.n_tiles < sm_count ? a.n_tiles : sm_count;
  refine_fused_kernel<<<grid, kThreads, kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lfk
