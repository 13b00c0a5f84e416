// lf_refine_tc.cu - fused inference of the learned refinement y = x + f(x)
// (three 3x3 convolutions 3->32->32->3, ReLU, zero padding; the learned
// stand-in for the offline projection of Sec. 5, Eq. 4-5) on the
// fifth-generation tensor cores: tcgen05.mma from shared memory into TMEM.
//
// One persistent CTA per SM loops over output tiles of 26 x 30 pixels.  A
// tile's input is a 32 x 36 halo of positions q = 32*hy + hx (3-pixel ring);
// each halo row is exactly 32 positions, i.e. one warp quadrant of TMEM lanes.
// Every layer is an implicit GEMM over M-tiles of 128 positions (4 halo rows):
//   D[q][kx*C + o] = sum_{ky, c} a[q + 32*(ky-1)][c] * W[o][c][ky][kx]
// so the three kernel rows are three shifted A operands (MMAs accumulating
// into one D) and the three kernel columns are stacked along N; the epilogue
// finishes the convolution with two warp shuffles,
//   out[q][o] = D[q-1][0*C + o] + D[q][1*C + o] + D[q+1][2*C + o].
// Per M-tile: layer 1 (3 input channels padded to K = 16, N = 96) 3 MMAs,
// layer 2 (K = 32, N = 96) 6 MMAs, layer 3 (K = 32, N = 16, 3 real outputs
// per kernel column) 6 MMAs.  The biases ride on the MMAs: the input carries a
// constant 1 in channel 3 that meets b1 in the centre weights, and layers 2
// and 3 add one MMA of a constant-1 operand against a bias block.
//
// Roles: lane 0 of warps 16 and 17 issues the MMAs (even and odd M-tiles) into a
// ring of 5 TMEM slots of 96 columns, committing each M-tile to the slot's
// "full" mbarrier; warps 0-15 (four groups of 4 taking M-tiles in turn; warp
// w reads TMEM lanes 32*(w%4) ..) wait on "full", read the accumulators, release the slot on its
// "empty" mbarrier, combine the kernel columns, apply ReLU, zero positions outside the image
// (the next layer's zero padding) and store BF16 rows for the next layer.  A
// "layer done" mbarrier lets the issuer start a layer once every row of the
// previous one is in shared memory.  At the end each issuing thread commits to
// its own "drain" mbarrier and waits for it, so no MMA it issued is still
// running when the CTA deallocates its tensor memory, also after an abort.  The next tile's FP32 halo streams into a
// staging buffer with cp.async while the current tile computes; the residual
// add uses FP32 inputs loaded into registers while layer 3 runs.  Every wait
// is bounded and reports through an error flag instead of hanging.
//
// Shared-memory operands use the K-major layout without swizzling: a position
// (row) holds 8 channels in 16 contiguous bytes, rows follow every 16 bytes
// (8-row core matrices 128 bytes apart), and each further group of 8 channels
// starts kGroupB bytes later.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lf_internal.h"
#include "lf_launch.h"

namespace lfk {

namespace {

constexpr int kHW = 32, kHH = 36;            // halo tile (positions)
constexpr int kTW = kHW - 6, kTH = kHH - 6;  // 26 x 30 output pixels
constexpr int kRows = 1280;                  // positions held per buffer (10 x 128)
constexpr int kGroupB = kRows * 16;          // bytes per group of 8 channels
constexpr int kBufB = 4 * kGroupB;           // 32 channels
// B operands: per kernel row (and K half) a block of 2 groups x N rows x 16 B
constexpr int kW1Blk = 2 * 96 * 16, kW2Blk = 2 * 96 * 16, kW3Blk = 2 * 16 * 16;
constexpr int kW1B = 3 * kW1Blk, kW2B = 6 * kW2Blk, kW3B = 6 * kW3Blk;
constexpr int kB2Blk = 2 * 96 * 16, kB3Blk = 2 * 16 * 16;  // b2, b3 against the constant-1 operand
constexpr int kWB = kW1B + kW2B + kW3B + kB2Blk + kB3Blk;  // 34,304 bytes
constexpr int kOnesB = 2 * 128 * 16;         // A operand: channel 0 = 1 on 128 rows
constexpr int kXsB = kHH * kHW * 16;         // FP32 RGBA halo of the next tile
constexpr int kSlots = 5, kSlotCols = 96;    // TMEM ring
constexpr int kNumBars = 2 * kSlots + 3;     // full[5], empty[5], layer_done, drain[2]
constexpr int kSmemBytes = 2 * kBufB + kWB + kOnesB + kXsB + kNumBars * 8 + 8;
constexpr int kStart1 = 32, kTiles1 = 9;     // layer 1 rows [32, 1184): halo rows 1..36
constexpr int kStart2 = 64, kTiles2 = 8;     // layer 2 rows [64, 1088): halo rows 2..33
constexpr int kStart3 = 96, kTiles3 = 8;     // layer 3 rows [96, 1120): halo rows 3..34
constexpr uint32_t kTmemCols = 512;
constexpr int kEpiWarps = 16;                // epilogue warps: 4 groups of 4 (one warp per TMEM lane quadrant)
constexpr int kEpiGroups = kEpiWarps / 4;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = kEpiThreads + 64;   // + two MMA warps
// which wait ran out of time (bit 0: the CTA aborted)
constexpr int kErrIssuerLayer = 2, kErrIssuerSlot = 4, kErrEpilogueFull = 8, kErrDrain = 16;
// The drain wait is not cut short by a small configured limit: MMAs that are
// still running when their issuer gives up finish in microseconds, and the
// tensor memory must not be freed under them.
constexpr uint64_t kDrainNs = 2000000000ull;

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

__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of `bar` with the given parity.  Returns 0 once it
// completed, 2 once limit_ns of wall time (%globaltimer) have passed without
// it, 1 at once when another warp already gave up (abort_flag may be null: the
// wait then ignores aborts).  The first probe does not block.
__device__ __forceinline__ int wait_phase_status(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                                 uint64_t limit_ns) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  if (done) return 0;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (done) return 0;
    if (abort_flag && (it & 15) == 0 && *abort_flag) return 1;
    if (global_ns() - t0 >= limit_ns) return 2;
  }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Barrier among the epilogue warps only (named barrier 1).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

struct FusedArgs {
  int32_t n, H, W, tiles_x, tiles_y, n_tiles;
  const float* in;
  float* out;
  const __nv_bfloat16* wtc;  // B operands: L1, L2, L3 blocks
  int32_t* error;            // set to 1 if a wait gave up
  uint64_t wait_ns;          // bound on each mbarrier wait
};

__device__ __forceinline__ void tile_origin(const FusedArgs& A, int tile, int& img, int& x0, int& y0) {
  const int per_img = A.tiles_x * A.tiles_y;
  img = tile / per_img;
  const int rem = tile - img * per_img;
  y0 = (rem / A.tiles_x) * kTH;
  x0 = (rem % A.tiles_x) * kTW;
}

// Epilogue threads start copying a tile's FP32 RGBA halo into xs (zeros outside the image).
__device__ __forceinline__ void prefetch_halo(uint32_t xs, const FusedArgs& A, int tile) {
  int img, x0, y0;
  tile_origin(A, tile, img, x0, y0);
  const float4* in = reinterpret_cast<const float4*>(A.in) + (size_t)img * A.H * A.W;
  for (int q = threadIdx.x; q < kHH * kHW; q += kEpiThreads) {
    const int gy = y0 - 3 + (q >> 5), gx = x0 - 3 + (q & 31);
    const bool ok = gy >= 0 && gy < A.H && gx >= 0 && gx < A.W;
    cp_async16(xs + q * 16, ok ? static_cast<const void*>(in + (size_t)gy * A.W + gx) : static_cast<const void*>(in),
               ok ? 16u : 0u);
  }
  cp_async_commit();
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) refine_fused_kernel(FusedArgs A) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* buf0 = sm;          // x (group 0), then a2
  unsigned char* buf1 = sm + kBufB;  // a1
  unsigned char* wts = sm + 2 * kBufB;
  unsigned char* ones = wts + kWB;
  unsigned char* xs = ones + kOnesB;
  uint64_t* full = reinterpret_cast<uint64_t*>(xs + kXsB);
  uint64_t* empty = full + kSlots;
  uint64_t* layer_done = empty + kSlots;
  uint64_t* drain = layer_done + 1;  // one per issuing thread
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 2);
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool issuer = warp >= kEpiWarps;

  // Both activation buffers start at zero (rows never written stay finite),
  // then the weights and the constant-1 operand; the first tile's halo is already on its way.
  if (!issuer && blockIdx.x < A.n_tiles) prefetch_halo(su32(xs), A, blockIdx.x);
  for (int i = tid; i < 2 * kBufB / 16; i += kThreads) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < kWB / 16; i += kThreads)
    reinterpret_cast<uint4*>(wts)[i] = reinterpret_cast<const uint4*>(A.wtc)[i];
  for (int i = tid; i < kOnesB / 16; i += kThreads)  // row i (group 0): channel 0 = 1; group 1: zeros
    reinterpret_cast<uint4*>(ones)[i] = make_uint4(i < 128 ? 0x3F80u : 0u, 0u, 0u, 0u);
  if (tid == 0) {
    s_abort = 0;
    for (int b = 0; b < kSlots; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(full + b)), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(empty + b)), "r"(4));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(layer_done)), "r"(kEpiWarps));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(drain + 0)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(drain + 1)), "r"(1));
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
  const int H = A.H, W = A.W;

  if (issuer) {
    // ------------------------------------------------------------ MMA warps (lane 0 of each)
    // Warp 8 issues the even M-tiles, warp 9 the odd ones, so two threads keep
    // the tensor core fed; descriptors are precomputed and only their start
    // address (in 16-byte units, the low field) moves.
    if (lane == 0) {
      const int parity = warp - kEpiWarps;
      const uint64_t a0 = smem_desc(su32(buf0), kGroupB, 128), a1 = smem_desc(su32(buf1), kGroupB, 128);
      const uint64_t a_ones = smem_desc(su32(ones), 128 * 16, 128);
      const uint32_t sw = su32(wts);
      const uint64_t b2bias = smem_desc(sw + kW1B + kW2B + kW3B, 96 * 16, 128);
      const uint64_t b3bias = smem_desc(sw + kW1B + kW2B + kW3B + kB2Blk, 16 * 16, 128);
      uint64_t b1d[3], b2d[6], b3d[6];
#pragma unroll
      for (int k = 0; k < 3; ++k) b1d[k] = smem_desc(sw + k * kW1Blk, 96 * 16, 128);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        b2d[k] = smem_desc(sw + kW1B + k * kW2Blk, 96 * 16, 128);
        b3d[k] = smem_desc(sw + kW1B + kW2B + k * kW3Blk, 16 * 16, 128);
      }
      constexpr uint64_t kHalf = 2 * kGroupB / 16;  // second K half of 16 channels, in 16-byte units
      uint32_t done_phase = 0;
      int c = 0;
      bool ok = true;
      auto wait_layer = [&]() {
        if (ok) {
          const int w = wait_phase_status(layer_done, done_phase, &s_abort, A.wait_ns);
          if (w == 2) atomicOr(A.error, kErrIssuerLayer);
          ok = w == 0;
        }
        done_phase ^= 1u;
        tc_after_sync();
      };
      // M-tile c: wait for its slot to be released, return the slot's first column.
      auto slot_col = [&]() -> uint32_t {
        const int slot = c % kSlots;
        if (ok) {
          const int w = wait_phase_status(empty + slot, ((uint32_t)(c / kSlots) & 1u) ^ 1u, &s_abort, A.wait_ns);
          if (w == 2) atomicOr(A.error, kErrIssuerSlot);
          ok = w == 0;
        }
        tc_after_sync();
        return tmem + (uint32_t)(slot * kSlotCols);
      };
      for (int tile = blockIdx.x; tile < A.n_tiles; tile += gridDim.x) {
        wait_layer();  // x of this tile is in buf0
        for (int m = 0; m < kTiles1; ++m, ++c) {
          if ((c & 1) != parity || !ok) continue;
          const uint32_t d = slot_col();
          if (!ok) continue;
          const uint64_t a = a0 + (uint64_t)(kStart1 - 32 + m * 128);
          mma(d, a, b1d[0], instr_desc(128, 96), 0);
          mma(d, a + 32, b1d[1], instr_desc(128, 96), 1);
          mma(d, a + 64, b1d[2], instr_desc(128, 96), 1);
          commit(full + c % kSlots);
        }
        wait_layer();  // every a1 row is written
        for (int m = 0; m < kTiles2; ++m, ++c) {
          if ((c & 1) != parity || !ok) continue;
          const uint32_t d = slot_col();
          if (!ok) continue;
          const uint64_t a = a1 + (uint64_t)(kStart2 - 32 + m * 128);
#pragma unroll
          for (int dy = 0; dy < 3; ++dy) {
            mma(d, a + 32 * dy, b2d[2 * dy], instr_desc(128, 96), dy > 0);
            mma(d, a + 32 * dy + kHalf, b2d[2 * dy + 1], instr_desc(128, 96), 1);
          }
          mma(d, a_ones, b2bias, instr_desc(128, 96), 1);
          commit(full + c % kSlots);
        }
        wait_layer();  // every a2 row is written
        for (int m = 0; m < kTiles3; ++m, ++c) {
          if ((c & 1) != parity || !ok) continue;
          const uint32_t d = slot_col();
          if (!ok) continue;
          const uint64_t a = a0 + (uint64_t)(kStart3 - 32 + m * 128);
#pragma unroll
          for (int dy = 0; dy < 3; ++dy) {
            mma(d, a + 32 * dy, b3d[2 * dy], instr_desc(128, 16), dy > 0);
            mma(d, a + 32 * dy + kHalf, b3d[2 * dy + 1], instr_desc(128, 16), 1);
          }
          mma(d, a_ones, b3bias, instr_desc(128, 16), 1);
          commit(full + c % kSlots);
        }
      }
      if (!ok) s_abort = 1;
      // Drain: the commit arrives once every MMA this thread issued has completed.
      // Waited for even after an abort (the abort flag does not cut it short), so
      // the tensor memory is never deallocated under a running MMA.
      commit(drain + parity);
      if (wait_phase_status(drain + parity, 0u, nullptr, A.wait_ns > kDrainNs ? A.wait_ns : kDrainNs) == 2)
        atomicOr(A.error, kErrDrain);
    }
  } else {
    // ---------------------------------------------------------------- epilogue warps
    const int quarter = warp & 3, group = warp >> 2;  // group g takes the M-tiles with c % kEpiGroups == g
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    int c = 0;          // the same running M-tile counter as the MMA warp
    bool ok = true;
    auto acquire = [&]() -> uint32_t {  // wait for M-tile c's accumulators (lane 0 polls)
      const int slot = c % kSlots;
      int got = 1;
      if (lane == 0) {
        const int w = wait_phase_status(full + slot, (uint32_t)(c / kSlots) & 1u, &s_abort, A.wait_ns);
        if (w == 2) atomicOr(A.error, kErrEpilogueFull);
        got = w == 0;
      }
      ok = __shfl_sync(0xffffffffu, got, 0) != 0;
      if (!ok) s_abort = 1;
      tc_after_sync();
      return tmem + lane_base + (uint32_t)(slot * kSlotCols);
    };
    auto release = [&]() {  // the slot's accumulators are in registers
      tmem_wait_ld();
      tc_before_sync();
      __syncwarp();
      if (lane == 0) arrive(empty + c % kSlots);
    };
    auto layer_finished = [&]() {  // this warp's shared-memory rows are visible to the MMAs
      fence_async_smem();
      __syncwarp();
      if (lane == 0) arrive(layer_done);
    };
    // A hidden layer: M-tiles of rows start + 128 m into dst (BF16, 4 groups).
    auto hidden = [&](int start, int n_mtiles, unsigned char* dst, int x0, int y0) {
      for (int m = 0; m < n_mtiles; ++m, ++c) {
        if (c % kEpiGroups != group || __any_sync(0xffffffffu, s_abort != 0)) continue;
        const uint32_t t = acquire();
        if (!ok) continue;
        const int q = start + m * 128 + quarter * 32 + lane;  // halo row q / 32, column lane
        const int gy = y0 - 3 + (q >> 5), gx = x0 - 3 + lane;
        const bool inside = (q >> 5) < kHH && gy >= 0 && gy < H && gx >= 0 && gx < W;
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // output channels 16h .. 16h + 15
          float d0[16], d1[16], d2[16];
          tmem_ld16(t + 0 * 32 + 16 * h, d0);
          tmem_ld16(t + 1 * 32 + 16 * h, d1);
          tmem_ld16(t + 2 * 32 + 16 * h, d2);
          if (h == 1) release();  // waits for the loads, then frees the slot for the MMA warps
          else tmem_wait_ld();
          uint32_t w[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int k = 2 * j + e;
              const float left = __shfl_up_sync(0xffffffffu, d0[k], 1);     // kernel column 0 reads q - 1
              const float right = __shfl_down_sync(0xffffffffu, d2[k], 1);  // kernel column 2 reads q + 1
              v[e] = fmaxf(left + d1[k] + right, 0.f);  // the bias came with the MMAs
            }
            w[j] = inside ? pack2(v[0], v[1]) : 0u;
          }
          if (q < kRows) {
            *reinterpret_cast<uint4*>(dst + (2 * h) * kGroupB + q * 16) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4*>(dst + (2 * h + 1) * kGroupB + q * 16) = make_uint4(w[4], w[5], w[6], w[7]);
          }
        }
      }
    };

    for (int tile = blockIdx.x; tile < A.n_tiles; tile += gridDim.x) {
      int img, x0, y0;
      tile_origin(A, tile, img, x0, y0);
      const float4* in = reinterpret_cast<const float4*>(A.in) + (size_t)img * H * W;
      // ---- x: FP32 halo (prefetched) -> BF16 group 0 of buf0, then the next halo starts
      cp_async_wait_all();
      epi_sync();  // every halo row landed; the previous tile's layer-3 MMAs are complete
      for (int q = tid; q < kHH * kHW; q += kEpiThreads) {
        const float4 v = reinterpret_cast<const float4*>(xs)[q];
        *reinterpret_cast<uint4*>(buf0 + q * 16) = make_uint4(pack2(v.x, v.y), pack2(v.z, 1.f), 0u, 0u);
      }
      layer_finished();  // layer 1 may start
      epi_sync();        // xs is free
      if (tile + (int)gridDim.x < A.n_tiles) prefetch_halo(su32(xs), A, tile + gridDim.x);

      hidden(kStart1, kTiles1, buf1, x0, y0);
      layer_finished();
      hidden(kStart2, kTiles2, buf0, x0, y0);
      layer_finished();

      // ---- layer 3 and the residual; the FP32 inputs of this warp's outputs load meanwhile.
      // Layer-3 M-tile m has counter c + m; this group owns m = first + kEpiGroups * j.
      const int first = (group - c % kEpiGroups + kEpiGroups) % kEpiGroups;
      constexpr int kOwn = kTiles3 / kEpiGroups;
      float4 xr[kOwn];
      int oidx[kOwn];
#pragma unroll
      for (int j = 0; j < kOwn; ++j) {
        const int m = first + kEpiGroups * j;
        const int hy = (kStart3 >> 5) + 4 * m + quarter;
        const int gy = y0 - 3 + hy, gx = x0 - 3 + lane;
        const bool out_ok = hy < 3 + kTH && lane >= 3 && lane < 3 + kTW && gy < H && gx < W;
        oidx[j] = out_ok ? gy * W + gx : -1;
        xr[j] = out_ok ? in[(size_t)gy * W + gx] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      float4* out = reinterpret_cast<float4*>(A.out) + (size_t)img * H * W;
      const int c3 = c;  // counter of layer 3's first M-tile
#pragma unroll
      for (int j = 0; j < kOwn; ++j) {
        c = c3 + first + kEpiGroups * j;
        if (__any_sync(0xffffffffu, s_abort != 0)) continue;
        const uint32_t t = acquire();
        if (!ok) continue;
        float d[16];
        tmem_ld16(t, d);
        release();
        float r[3];
#pragma unroll
        for (int o = 0; o < 3; ++o) {
          const float left = __shfl_up_sync(0xffffffffu, d[o], 1);
          const float right = __shfl_down_sync(0xffffffffu, d[8 + o], 1);
          r[o] = left + d[4 + o] + right;
        }
        if (oidx[j] >= 0) {
          const float4 x = xr[j];
          float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
          if (x.w > 0.f) {
            y.x = x.x + r[0];
            y.y = x.y + r[1];
            y.z = x.z + r[2];
            y.w = 1.f;
          }
          out[oidx[j]] = y;
        }
      }
      c = c3 + kTiles3;
    }
    cp_async_wait_all();
  }

  tc_before_sync();
  __syncthreads();
  if (tid == 0 && s_abort) atomicOr(A.error, 1);
  if (warp == 0) {
    tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

cudaError_t launch_refine_fused(int32_t n, int32_t w, int32_t h, const float* in, float* out, const float* params,
                                const __nv_bfloat16* packed, int sm_count, int32_t* error, uint64_t wait_ns,
                                cudaStream_t s) {
  (void)params;  // the biases are packed with the weights
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(refine_fused_kernel), kSmemBytes);
  if (e != cudaSuccess) return e;
  FusedArgs a;
  a.n = n;
  a.H = h;
  a.W = w;
  a.tiles_x = (w + kTW - 1) / kTW;
  a.tiles_y = (h + kTH - 1) / kTH;
  a.n_tiles = a.tiles_x * a.tiles_y * n;
  a.in = in;
  a.out = out;
  a.wtc = packed + kPackTc;
  a.error = error;
  a.wait_ns = wait_ns;
  if (a.n_tiles == 0) return cudaSuccess;
  const int grid = a.n_tiles < sm_count ? a.n_tiles : sm_count;
  refine_fused_kernel<<<grid, kThreads, kSmemBytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lfk
