// lf_refine_tc.cu - fused inference of the learned refinement y = x + f(x)
// (three 3x3 convolutions 3->32->32->3, ReLU, zero padding; the learned
// stand-in for the offline projection of Sec. 5, Eq. 4-5) on the
// fifth-generation tensor cores: tcgen05.mma from shared memory into TMEM.
//
// One persistent CTA per SM loops over output tiles of 26 x 30 pixels.  A
// tile's input is a 32 x 36 halo of positions q = 32*hy + hx (3-pixel ring);
// each halo row is exactly 32 positions, one warp quadrant of TMEM lanes.
// Every layer is an implicit GEMM over M-tiles of 128 positions (4 halo rows).
// Layers 1 and 2 run the whole 3x3 window in the MMAs, N = 32 outputs:
//   D[q][o] = sum_{ky, kx, c} a[q + 32*(ky-1) + (kx-1)][c] * W[o][c][ky][kx],
// each tap a shifted A operand (a position is 16 bytes per 8 channels, so a
// shift moves the descriptor's start).  Layer 1's input is pair-packed:
// position s holds (x[s], x[s+1]) as 8 channels (R, G, B, 1 twice), and its A
// descriptor puts the second K group two positions on, so one K = 16 MMA
// covers kernel columns -1..+2 (the last with zero weights): one MMA per
// kernel row.  Layer 2 takes 18 MMAs (9 taps x 2 halves of 32 channels).
// Layer 3 (3 outputs) stacks the kernel columns along N = 16 and finishes
// with two warp shuffles per output:
//   out[q][o] = D[q-1][o] + D[q][4 + o] + D[q+1][8 + o].
// Measured on GB300, an M = 128, K = 16 MMA costs about max(45, 0.55 N)
// cycles, so stacking layer 2's columns along N (N = 96) would take fewer
// tensor cycles, but finishing them costs 64 shuffles and 64 adds per
// position in the epilogue, which then bounds the kernel; with full windows
// the epilogue is a TMEM load, the bias, ReLU with BF16 packing (one cvt per
// pair) and four stores.  b1 meets the constant-1 input channel in the MMAs;
// b2 and b3 are added in FP32 by the epilogue.
//
// Roles: lane 0 of warps 16-19 issues the MMAs (issuer i takes the M-tiles
// whose running number c has c % 4 == i) into a ring of 16 TMEM slots of 32
// columns, committing each M-tile to a "full" mbarrier; warps 0-15 form four
// groups of 4 (group g takes c % 4 == g; warp w reads TMEM lanes 32*(w%4) ..)
// that wait on "full", read the accumulators, release the slot on an "empty"
// mbarrier and store BF16 rows for the next layer (zero outside the image: the
// next layer's zero padding).  Slot c % 16 thus always belongs to one issuer
// and one group, so each ring mbarrier has one waiter taking its phases in
// order and arrivals that come in phase order (a parity wait cannot tell a
// phase from the one two phases earlier).
//
// Schedule: a tile's 25 M-tiles follow one fixed order (kSchedule) that the
// issuers and the groups both walk, so the layers overlap.  Per-M-tile
// "ready" mbarriers carry the dependencies: layer-2 M-tile m waits for
// layer-1 M-tiles m-1, m and m+1 (its window reads rows of m and m+1 and one
// position of m-1, and its output overwrites input rows that m-1..m+1 read),
// layer-3 M-tile m for layer-2 M-tiles m and m+1.  The order leaves tensor work
// between a producer and its consumer to hide the epilogue.  At a tile
// boundary every group has taken all 25 M-tiles (so every MMA of the tile is
// complete) before the next tile's input overwrites buffer 0.
//
// The next tile's FP32 halo streams into a staging buffer with one tiled TMA
// copy (cp.async.bulk.tensor over a tensor map of the input, zeros outside the
// image) while the current tile computes; the residual add uses FP32 inputs loaded into
// registers before layer 3's accumulators are read.  Every wait is bounded
// (%globaltimer) and reports through an error flag instead of hanging; at the
// end each issuer commits to its own "drain" mbarrier and waits for it, so no
// MMA is running when the CTA frees its tensor memory, also after an abort.
//
// Shared-memory operands use the K-major layout without swizzling: a position
// (row) holds 8 channels in 16 contiguous bytes, rows follow every 16 bytes
// (8-row core matrices 128 bytes apart), and each further group of 8 channels
// starts kGroupB bytes later (layer 1's input: 32 bytes later, see above).
#include <cuda.h>  // CUtensorMap and its enums (the encoder is reached through the runtime)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lf_internal.h"
#include "lf_launch.h"

namespace lfk {

namespace {

constexpr int kHW = 32, kHH = 36;            // halo tile (positions)
constexpr int kTW = kHW - 6, kTH = kHH - 6;  // 26 x 30 output pixels
// Positions held per buffer (row r of a buffer holds position base + r):
//   x   (pair-packed layer-1 input, two buffers) read [-1, 1217), base 0
//   a1  (buffer 1) written [32, 1184), read [31, 1121), base 32
//   a2  (buffer 2) written [64, 1088), read [64, 1152), base 64 (rows never written stay zero)
// A read one row before a buffer (an output column that is never used) meets
// finite data: the weights or the previous buffer.
constexpr int kRowsX = 1220, kRows1 = 1152, kRows2 = 1088;
constexpr int kBase1 = 32, kBase2 = 64;
constexpr int kGroup1B = kRows1 * 16, kGroup2B = kRows2 * 16;  // bytes per group of 8 channels
constexpr int kXB = kRowsX * 16, kBuf1B = 4 * kGroup1B, kBuf2B = 4 * kGroup2B;
// B operands, K-major [2 K groups][N rows][16 B]:
//   layer 1 per kernel row ky (pair-packed taps kx = -1..+2, N = 32),
//   layer 2 per (ky, half of the 32 input channels) (N = 96: kx*32 + o),
//   layer 3 per (ky, half) (N = 16: kx*4 + o).
constexpr int kW1Blk = 2 * 32 * 16, kW2Blk = 2 * 96 * 16, kW3Blk = 2 * 16 * 16;
constexpr int kW1B = 3 * kW1Blk, kW2B = 6 * kW2Blk, kW3B = 6 * kW3Blk;
constexpr int kWB = kW1B + kW2B + kW3B;  // 24,576 bytes
static_assert(kWB == 2 * (kRefinePackedElems - kPackTc), "the packed operands are the shared-memory image");
constexpr int kXsB = kHH * kHW * 16;         // FP32 RGBA halo of the next tile
constexpr int kBiasB = 48 * 4;               // b2[32], b3[3]
constexpr int kSlots = 5, kSlotCols = 96;    // TMEM ring
constexpr int kIssuers = 4;                  // MMA warps
constexpr int kRing = 20;                    // ring mbarriers, indexed by c % kRing
constexpr int kEpiWarps = 16;                // epilogue warps: 4 groups of 4 (one warp per TMEM lane quadrant)
constexpr int kEpiGroups = kEpiWarps / 4;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kLoaderWarp = kEpiWarps + kIssuers;  // stages each tile's input
constexpr int kThreads = kEpiThreads + 32 * kIssuers + 32;
static_assert(kRing % kSlots == 0 && kRing % kEpiGroups == 0 && kRing % kIssuers == 0 && kEpiGroups == kIssuers,
              "each ring mbarrier belongs to one slot, one epilogue group and one issuer");
constexpr int kStart1 = 32, kTiles1 = 9;     // layer 1 rows [32, 1184): halo rows 1..36
constexpr int kStart2 = 64, kTiles2 = 8;     // layer 2 rows [64, 1088): halo rows 2..33
constexpr int kStart3 = 96, kTiles3 = 8;     // layer 3 rows [96, 1120): halo rows 3..34
// full[20], empty[20], x_ready[2], drain[4], ready1[9], ready2[8], done3[8], l1done[2], xs_full
constexpr int kNumBars = 2 * kRing + 2 + kIssuers + kTiles1 + kTiles2 + kTiles3 + 2 + 1;
constexpr int kSmemBytes = kWB + 2 * kXB + kBuf1B + kBuf2B + kXsB + kBiasB + kNumBars * 8 + 16;
static_assert(kSmemBytes <= 227 * 1024, "fits one CTA's shared memory");
constexpr uint32_t kTmemCols = 512;
static_assert(kSlots * kSlotCols <= (int)kTmemCols, "the ring fits the tensor memory");
// A CTA's tiles run as a pipeline: period k issues layers 2 and 3 of its tile
// k-1 together with layer 1 of its tile k (entries layer << 4 | m), so the
// tensor core does not wait at tile boundaries.  An entry (code << 4 | m)
// holds the layer in the code's low two bits and the count of M-tiles less one
// above them: layer 1 runs in triples (three 32-column accumulators fill a
// slot) and layer 3 in pairs, so the ring's per-entry handshakes are shared.  A period issues all of layer 2 first, then alternates layer 3
// with the next tile's layer 1, so every
// consumer comes at least seven M-tiles after its producers (the epilogue of
// one M-tile takes longer than several M-tiles of tensor work); the first
// period has only layer 1, the last no layer 1.
constexpr int kLenFirst = 3, kLenMid = 15, kLenLast = 12;
constexpr int kOffMid = kLenFirst, kOffLast = kLenFirst + kLenMid;
__device__ __constant__ const uint8_t kSchedule[kLenFirst + kLenMid + kLenLast] = {
    0x90, 0x93, 0x96,  // first
    0x20, 0x21, 0x22, 0x23, 0x24, 0x25, 0x26, 0x27, 0x70, 0x90, 0x72, 0x93, 0x74, 0x96, 0x76,  // middle
    0x20, 0x21, 0x22, 0x23, 0x24, 0x25, 0x26, 0x27, 0x70, 0x72, 0x74, 0x76};  // last
// which wait ran out of time (bit 0: the CTA aborted)
constexpr int kErrIssuerLayer = 2, kErrIssuerSlot = 4, kErrEpilogueFull = 8, kErrDrain = 16, kErrLoader = 32;
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
__device__ __forceinline__ void tmem_ld32(uint32_t addr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// max(lo, 0) and max(hi, 0) rounded to BF16 (nearest even), lo in the low half.
__device__ __forceinline__ uint32_t relu_pack2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}


struct FusedArgs {
  int32_t n, H, W, tiles_x, tiles_y, n_tiles;
  const float* in;
  float* out;                // image i at out + i * H * W * 4 ...
  float* out1;               // ... except image 1 at out1 when set (a stereo pair's two buffers)
  const __nv_bfloat16* wtc;  // B operands: L1, L2, L3 blocks
  const float* prm;          // FP32 parameters (b2, b3 read from here)
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

// The loader's lane 0 starts the tiled TMA copy of a tile's FP32 RGBA halo
// (4 channels x 32 positions x 36 rows of the tensor map over the input; zeros
// where the box leaves the image) into xs; it completes on xs_full with its
// byte count.  The loader's earlier reads of xs are ordered before the copy.
__device__ __forceinline__ void load_halo(const CUtensorMap* tmap, uint32_t xs, uint64_t* xs_full, const FusedArgs& A,
                                          int tile) {
  int img, x0, y0;
  tile_origin(A, tile, img, x0, y0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(xs_full)), "r"(kXsB) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::
          "r"(xs), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(0), "r"(x0 - 3), "r"(y0 - 3), "r"(img), "r"(su32(xs_full))
      : "memory");
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) refine_fused_kernel(FusedArgs A, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(1024) unsigned char sm[];
  // The weights come first: layer 1's first window reaches one position before
  // the x buffer (an output column that is never used) and reads finite weights there.
  unsigned char* wts = sm;
  unsigned char* xb = wts + kWB;       // x, pair-packed: tile j of this CTA in xb + (j % 2) * kXB
  unsigned char* buf1 = xb + 2 * kXB;  // a1
  unsigned char* buf2 = buf1 + kBuf1B;  // a2
  unsigned char* xs = buf2 + kBuf2B;
  float* bias = reinterpret_cast<float*>(xs + kXsB);  // b2[32], b3[3]
  uint64_t* full = reinterpret_cast<uint64_t*>(xs + kXsB + kBiasB);
  uint64_t* empty = full + kRing;
  uint64_t* x_ready = empty + kRing;    // x of tile j is in xb + (j % 2) * kXB: x_ready[j % 2]
  uint64_t* drain = x_ready + 2;        // one per issuer
  uint64_t* ready1 = drain + kIssuers;  // layer-1 M-tile m is in buffer 1 (four arrivals)
  uint64_t* ready2 = ready1 + kTiles1;  // layer-2 M-tile m is in buffer 2
  uint64_t* done3 = ready2 + kTiles2;   // layer-3 M-tile m has read buffer 2
  uint64_t* l1done = done3 + kTiles3;   // every layer-1 M-tile of tile j is complete: l1done[j % 2]
  uint64_t* xs_full = l1done + 2;       // the TMA copy of a tile's halo landed in xs
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(xs_full + 1);
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool issuer = warp >= kEpiWarps && warp < kLoaderWarp;

  // The x and activation buffers start at zero (rows never written stay finite),
  // then the weights and biases; the first tile's halo is already on its way.
  for (int i = tid; i < (2 * kXB + kBuf1B + kBuf2B) / 16; i += kThreads)
    reinterpret_cast<uint4*>(xb)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < kWB / 16; i += kThreads)
    reinterpret_cast<uint4*>(wts)[i] = reinterpret_cast<const uint4*>(A.wtc)[i];
  if (tid < 32) bias[tid] = A.prm[kRefineOffB2 + tid];
  else if (tid < 35) bias[tid] = A.prm[kRefineOffB3 + tid - 32];
  if (tid == 0) {
    s_abort = 0;
    for (int b = 0; b < kRing; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(full + b)), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(empty + b)), "r"(4));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(x_ready + b)), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(l1done + b)), "r"(4 * kTiles1));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(xs_full)), "r"(1));
    for (int b = 0; b < kIssuers; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(drain + b)), "r"(1));
    for (int b = 0; b < kTiles1 + kTiles2 + kTiles3; ++b)  // ready1, ready2, done3: one group's four warps
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(ready1 + b)), "r"(4));
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
  // Launched as a programmatic dependent of the render, the set-up above (weights
  // and biases, written long before the render began) overlaps the end of the
  // raster; its output, this kernel's input, is read only past this wait.
  griddep_wait();

  // Tiles of this CTA: blockIdx.x + j * gridDim.x, j < n_own; periods k = 0 .. n_own.
  const int n_own = blockIdx.x < A.n_tiles ? (A.n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  auto period = [&](int k, int& off, int& len) {
    if (k == 0) off = 0, len = kLenFirst;
    else if (k == n_own) off = kOffLast, len = kLenLast;
    else off = kOffMid, len = kLenMid;
  };
  if (issuer) {
    // ------------------------------------------------------------ MMA warps (lane 0 of each)
    // Descriptors are precomputed; only their start address (in 16-byte
    // units, the low field) moves with the M-tile and the tap.
    if (lane == 0) {
      const int me = warp - kEpiWarps;
      const uint32_t sw = su32(wts);
      // pair-packed x: K group 1 two positions on; a1, a2 descriptors address position 0
      const uint64_t ax0 = smem_desc(su32(xb), 32, 128), ax1 = smem_desc(su32(xb) + kXB, 32, 128);
      const uint64_t a1d = smem_desc(su32(buf1) - kBase1 * 16, kGroup1B, 128);
      const uint64_t a2d = smem_desc(su32(buf2) - kBase2 * 16, kGroup2B, 128);
      const uint64_t b1d = smem_desc(sw, 32 * 16, 128);
      const uint64_t b2d = smem_desc(sw + kW1B, 96 * 16, 128);
      const uint64_t b3d = smem_desc(sw + kW1B + kW2B, 16 * 16, 128);
      constexpr uint64_t kHalf1 = 2 * kGroup1B / 16, kHalf2 = 2 * kGroup2B / 16;  // second 16 channels
      constexpr uint32_t kId32 = instr_desc(128, 32), kId96 = instr_desc(128, 96), kId16 = instr_desc(128, 16);
      int c = 0;
      bool ok = true;
      // A barrier completed once per tile; parity = the tile's index in this CTA, mod 2.
      auto wait_tile = [&](uint64_t* bar, uint32_t parity) {
        if (ok) {
          const int w = wait_phase_status(bar, parity, &s_abort, A.wait_ns);
          if (w == 2) atomicOr(A.error, kErrIssuerLayer);
          ok = w == 0;
        }
      };
      // M-tile c: wait until M-tile c - kSlots has released the slot, return the slot's first column.
      auto slot_col = [&]() -> uint32_t {
        if (ok && c >= kSlots) {
          const int p = c - kSlots;
          const int w = wait_phase_status(empty + p % kRing, (uint32_t)(p / kRing) & 1u, &s_abort, A.wait_ns);
          if (w == 2) atomicOr(A.error, kErrIssuerSlot);
          ok = w == 0;
        }
        tc_after_sync();
        return tmem + (uint32_t)((c % kSlots) * kSlotCols);
      };
      for (int k = 0; k <= n_own; ++k) {
        int off, len;
        period(k, off, len);
        // parities of the tiles k (layer 1), k - 1 (layers 2, 3) and k - 2
        const uint32_t pu = (uint32_t)k & 1u, pt = pu ^ 1u, pp = pu;
        bool x_seen = false;
        const int c0 = c;
        for (int i = (me - c0 % kIssuers + kIssuers) % kIssuers; i < len; i += kIssuers) {
          c = c0 + i;
          if (!ok) break;
          const int code = kSchedule[off + i] >> 4, m = kSchedule[off + i] & 15;
          const int layer = code & 3, cnt = 1 + (code >> 2);  // M-tiles m .. m + cnt - 1
          if (layer == 1) {
            if (!x_seen) wait_tile(x_ready + (k & 1), (uint32_t)(k >> 1) & 1u);  // x of tile k is in its xb
            x_seen = true;
            // a1 rows it overwrites: layer-2 M-tiles m-1 .. m+cnt of tile k-1 have read them
            if (k > 0)
              for (int j = m - 1; j <= m + cnt; ++j)
                if (j >= 0 && j < kTiles2) wait_tile(ready2 + j, pt);
          } else if (layer == 2) {
            // a1 rows it reads (layer-1 M-tiles m-1 .. m+1 of tile k-1) are written
            for (int j = m - 1; j <= m + 1; ++j)
              if (j >= 0) wait_tile(ready1 + j, pt);
            // a2 rows it overwrites: layer-3 M-tiles m-1, m of tile k-2 have read them
            if (k > 1) {
              if (m > 0) wait_tile(done3 + m - 1, pp);
              wait_tile(done3 + m, pp);
            }
          } else {  // a2 rows it reads (layer-2 M-tiles m .. m+cnt of tile k-1) are written
            for (int j = m; j <= m + cnt; ++j)
              if (j < kTiles2) wait_tile(ready2 + j, pt);
          }
          if (!ok) break;
          const uint32_t d = slot_col();
          if (!ok) break;
          if (layer == 1) {
            // output position p = kStart1 + 128 m + r; kernel row ky starts at p + 32 (ky - 1) - 1
            const uint64_t a = ((k & 1) ? ax1 : ax0) + (uint64_t)(int64_t)(kStart1 - 33 + 128 * m);
            for (int s = 0; s < cnt; ++s) {  // M-tile m + s into columns 32 s ..
#pragma unroll
              for (int ky = 0; ky < 3; ++ky)
                mma(d + 32 * s, a + 128 * s + 32 * ky, b1d + (uint64_t)(ky * (kW1Blk / 16)), kId32, ky > 0);
            }
          } else if (layer == 2) {
            const uint64_t a = a1d + (uint64_t)(kStart2 - 32 + 128 * m);
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {  // kernel row ky reads p + 32 (ky - 1); columns along N
#pragma unroll
              for (int h = 0; h < 2; ++h)
                mma(d, a + 32 * ky + h * kHalf1, b2d + (uint64_t)((2 * ky + h) * (kW2Blk / 16)), kId96, ky > 0 || h > 0);
            }
          } else {
            const uint64_t a = a2d + (uint64_t)(kStart3 - 32 + 128 * m);
            for (int s = 0; s < cnt; ++s) {  // M-tile m + s into columns 16 s ..
#pragma unroll
              for (int ky = 0; ky < 3; ++ky) {
#pragma unroll
                for (int h = 0; h < 2; ++h)
                  mma(d + 16 * s, a + 128 * s + 32 * ky + h * kHalf2, b3d + (uint64_t)((2 * ky + h) * (kW3Blk / 16)),
                      kId16, ky > 0 || h > 0);
              }
            }
          }
          commit(full + c % kRing);
        }
        c = c0 + len;
        if (!ok) break;
      }
      if (!ok) s_abort = 1;
      // Drain: the commit arrives once every MMA this thread issued has completed.
      // Waited for even after an abort (the abort flag does not cut it short), so
      // the tensor memory is never deallocated under a running MMA.
      commit(drain + me);
      if (wait_phase_status(drain + me, 0u, nullptr, A.wait_ns > kDrainNs ? A.wait_ns : kDrainNs) == 2)
        atomicOr(A.error, kErrDrain);
    }
  } else if (warp == kLoaderWarp) {
    // ---------------------------------------------------------------- input loader
    // Tile j's FP32 halo (a TMA copy into xs) -> pair-packed BF16 in
    // xb + (j % 2) * kXB, once that buffer's last reader, layer 1 of tile
    // j - 2, is complete; then tile j + 1's halo starts streaming into xs.
    bool ok = true;
    int pending = -1;  // the tile whose copy into xs was issued and not yet waited for
    if (n_own > 0) {
      if (lane == 0) load_halo(&tmap, su32(xs), xs_full, A, blockIdx.x);
      pending = 0;
    }
    for (int j = 0; j < n_own && ok; ++j) {
      if (j >= 2) {
        int got = 1;
        if (lane == 0) {
          const int w = wait_phase_status(l1done + (j & 1), (uint32_t)((j - 2) >> 1) & 1u, &s_abort, A.wait_ns);
          if (w == 2) atomicOr(A.error, kErrLoader);
          got = w == 0;
        }
        ok = __shfl_sync(0xffffffffu, got, 0) != 0;
        if (!ok) {
          s_abort = 1;
          break;
        }
      }
      int landed = 1;
      if (lane == 0) {
        const int w = wait_phase_status(xs_full, (uint32_t)j & 1u, &s_abort, A.wait_ns);
        if (w == 2) atomicOr(A.error, kErrLoader);
        landed = w == 0;
      }
      ok = __shfl_sync(0xffffffffu, landed, 0) != 0;
      if (!ok) {
        s_abort = 1;
        break;
      }
      pending = -1;
      unsigned char* dst = xb + (j & 1) * kXB;
      for (int q = lane; q < kHH * kHW; q += 32) {
        const float4 v0 = reinterpret_cast<const float4*>(xs)[q];
        const float4 v1 = q + 1 < kHH * kHW ? reinterpret_cast<const float4*>(xs)[q + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<uint4*>(dst + q * 16) =
            make_uint4(pack2(v0.x, v0.y), pack2(v0.z, 1.f), pack2(v1.x, v1.y), pack2(v1.z, 1.f));
      }
      fence_async_smem();  // the rows are visible to the MMAs
      __syncwarp();        // and every lane has read xs
      if (lane == 0) arrive(x_ready + (j & 1));  // layer 1 of tile j may start
      if (j + 1 < n_own) {
        if (lane == 0) load_halo(&tmap, su32(xs), xs_full, A, blockIdx.x + (j + 1) * gridDim.x);
        pending = j + 1;
      }
    }
    // after an abort, a copy still in flight lands before the CTA can leave
    if (lane == 0 && pending >= 0 &&
        wait_phase_status(xs_full, (uint32_t)pending & 1u, nullptr, A.wait_ns > kDrainNs ? A.wait_ns : kDrainNs) == 2)
      atomicOr(A.error, kErrDrain);
  } else {
    // ---------------------------------------------------------------- epilogue warps
    const int quarter = warp & 3, group = warp >> 2;  // group g takes the M-tiles with c % kEpiGroups == g
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    int c = 0;  // the same running M-tile counter as the MMA warps
    bool ok = true;
    auto acquire = [&]() -> uint32_t {  // wait for M-tile c's accumulators (lane 0 polls)
      int got = 1;
      if (lane == 0) {
        const int w = wait_phase_status(full + c % kRing, (uint32_t)(c / kRing) & 1u, &s_abort, A.wait_ns);
        if (w == 2) atomicOr(A.error, kErrEpilogueFull);
        got = w == 0;
      }
      ok = __shfl_sync(0xffffffffu, got, 0) != 0;
      if (!ok) s_abort = 1;
      tc_after_sync();
      return tmem + lane_base + (uint32_t)((c % kSlots) * kSlotCols);
    };
    auto release = [&]() {  // the slot's accumulators are in registers
      tmem_wait_ld();
      tc_before_sync();
      __syncwarp();
      if (lane == 0) arrive(empty + c % kRing);
    };
    auto published = [&](uint64_t* bar) {  // this warp's shared-memory rows are visible to the MMAs
      fence_async_smem();
      __syncwarp();
      if (lane == 0) arrive(bar);
    };
    // Hidden-layer M-tile m, accumulators at TMEM address t, as BF16 into rows
    // start + 128 m of dst (4 groups of 8 channels, group_b bytes apart), zero
    // outside the image; the slot is released after the loads when `last`.
    // Layer 1 (full windows): ReLU(D).  Layer 2 (kernel columns along
    // N): ReLU(D[q-1][o] + D[q][32 + o] + D[q+1][64 + o] + b2[o]), the
    // neighbouring positions taken from the neighbouring lanes (columns 0 and
    // 31 of the halo get a wrong neighbour; they are never used).
    auto hidden = [&](uint32_t t, int start, int m, unsigned char* dst, int base, int group_b, int rows, int x0,
                      int y0, bool stacked, bool last) {
      const int q = start + m * 128 + quarter * 32 + lane;  // halo row q / 32, column lane
      const int gy = y0 - 3 + (q >> 5), gx = x0 - 3 + lane;
      const bool inside = (q >> 5) < kHH && gy >= 0 && gy < H && gx >= 0 && gx < W;
      unsigned char* row = dst + (q - base) * 16;
      const bool keep = q - base < rows;
      if (!stacked) {
        float v[32];
        tmem_ld32(t, v);
        if (last) release();  // waits for the load, then frees the slot for the MMA warps
        else tmem_wait_ld();
        uint32_t w[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) w[j] = inside ? relu_pack2(v[2 * j], v[2 * j + 1]) : 0u;
        if (keep) {
#pragma unroll
          for (int g = 0; g < 4; ++g)
            *reinterpret_cast<uint4*>(row + g * group_b) = make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
        }
        return;
      }
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
            v[e] = left + d1[k] + right + bias[16 * h + k];
          }
          w[j] = inside ? relu_pack2(v[0], v[1]) : 0u;
        }
        if (keep) {
          *reinterpret_cast<uint4*>(row + (2 * h) * group_b) = make_uint4(w[0], w[1], w[2], w[3]);
          *reinterpret_cast<uint4*>(row + (2 * h + 1) * group_b) = make_uint4(w[4], w[5], w[6], w[7]);
        }
      }
    };

    for (int k = 0; k <= n_own; ++k) {
      int off, len;
      period(k, off, len);
      int ux0 = 0, uy0 = 0, tx0 = 0, ty0 = 0, img = 0;
      if (k > 0) tile_origin(A, blockIdx.x + (k - 1) * gridDim.x, img, tx0, ty0);
      const float4* in = reinterpret_cast<const float4*>(A.in) + (size_t)img * H * W;  // tile k - 1
      float4* out = (img == 1 && A.out1) ? reinterpret_cast<float4*>(A.out1)
                                         : reinterpret_cast<float4*>(A.out) + (size_t)img * H * W;
      if (k < n_own) {
        int uimg;
        tile_origin(A, blockIdx.x + k * gridDim.x, uimg, ux0, uy0);
      }

      // ---- the period's M-tiles in the issuers' order; group g takes those with c % 4 == g
      const int c0 = c;
      for (int i = (group - c0 % kEpiGroups + kEpiGroups) % kEpiGroups; i < len && ok; i += kEpiGroups) {
        c = c0 + i;
        if (__any_sync(0xffffffffu, s_abort != 0)) break;
        const int code = kSchedule[off + i] >> 4, m = kSchedule[off + i] & 15;
        const int layer = code & 3, cnt = 1 + (code >> 2);  // M-tiles m .. m + cnt - 1, one slot
        if (layer == 1) {
          const uint32_t t = acquire();
          if (!ok) break;
          for (int s = 0; s < cnt; ++s) {
            hidden(t + 32 * s, kStart1, m + s, buf1, kBase1, kGroup1B, kRows1, ux0, uy0, false, s + 1 == cnt);
            published(ready1 + m + s);
            if (lane == 0) arrive(l1done + (k & 1));  // its MMAs (readers of x) are complete
          }
          continue;
        }
        if (layer == 2) {
          const uint32_t t = acquire();
          if (!ok) break;
          hidden(t, kStart2, m, buf2, kBase2, kGroup2B, kRows2, tx0, ty0, true, true);
          published(ready2 + m);
          continue;
        }
        // layer 3 of tile k-1 and the residual: this warp's rows of the entry's
        // M-tiles; their FP32 inputs load first
        float4 x[2];
        int pix[2];
        for (int s = 0; s < 2; ++s) {
          const int hy = (kStart3 >> 5) + 4 * (m + s) + quarter;
          const int gy = ty0 - 3 + hy, gx = tx0 - 3 + lane;
          const bool out_ok = s < cnt && hy < 3 + kTH && lane >= 3 && lane < 3 + kTW && gy < H && gx < W;
          pix[s] = out_ok ? gy * W + gx : -1;
          x[s] = out_ok ? in[(size_t)gy * W + gx] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const uint32_t t = acquire();
        if (!ok) break;
        for (int s = 0; s < cnt; ++s) {
          float d[16];
          tmem_ld16(t + 16 * s, d);
          if (s + 1 == cnt) {
            release();
            __syncwarp();
            if (lane == 0)
              for (int j = 0; j < cnt; ++j) arrive(done3 + m + j);  // their MMAs (the readers of buffer 2) are complete
          } else {
            tmem_wait_ld();
          }
          float r[3];
#pragma unroll
          for (int o = 0; o < 3; ++o) {
            const float left = __shfl_up_sync(0xffffffffu, d[o], 1);       // kernel column 0 reads q - 1
            const float right = __shfl_down_sync(0xffffffffu, d[8 + o], 1);  // kernel column 2 reads q + 1
            r[o] = left + d[4 + o] + right + bias[32 + o];
          }
          if (pix[s] >= 0) {
            float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
            if (x[s].w > 0.f) {
              y.x = x[s].x + r[0];
              y.y = x[s].y + r[1];
              y.z = x[s].z + r[2];
              y.w = 1.f;
            }
            out[pix[s]] = y;
          }
        }
      }
      c = c0 + len;
    }
  }

  tc_before_sync();
  __syncthreads();
  if (tid == 0 && s_abort) atomicOr(A.error, 1);
  if (warp == 0) {
    tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

cudaError_t launch_refine_fused(int32_t n, int32_t w, int32_t h, const float* in, float* out, float* out1,
                                const float* params, const __nv_bfloat16* packed, int sm_count, int32_t* error,
                                uint64_t wait_ns, cudaStream_t s, bool pdl) {
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
  a.out1 = n > 1 ? out1 : nullptr;
  a.wtc = packed + kPackTc;
  a.prm = params;
  a.error = error;
  a.wait_ns = wait_ns;
  if (a.n_tiles == 0) return cudaSuccess;
  // The input as a 4-D tensor (4 channels, W, H, n) for the halo copies: a 16-byte aligned base,
  // row and image strides of W * 16 and W * H * 16 bytes.
  if ((reinterpret_cast<uintptr_t>(in) & 15u) != 0) return cudaErrorInvalidValue;
  const EncodeTiled enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tmap;
  const cuuint64_t dims[4] = {4, (cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)n};
  const cuuint64_t strides[3] = {16, (cuuint64_t)w * 16, (cuuint64_t)w * h * 16};
  const cuuint32_t box[4] = {4, (cuuint32_t)kHW, (cuuint32_t)kHH, 1};
  const cuuint32_t step[4] = {1, 1, 1, 1};
  if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(in), dims, strides, box, step,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int grid = a.n_tiles < sm_count ? a.n_tiles : sm_count;
  return launch_kernel(refine_fused_kernel, dim3(grid), dim3(kThreads), kSmemBytes, s, pdl, a, tmap);
}

}  // namespace lfk
