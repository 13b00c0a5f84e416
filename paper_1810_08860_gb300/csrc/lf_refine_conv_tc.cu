// lf_refine_conv_tc.cu - the refinement's training GEMMs on the fifth-
// generation tensor cores (tcgen05.mma from shared memory into TMEM): the
// single-layer convolutions (forward layers of training and of the per-layer
// inference path, the backward pass through a layer's input as the same
// correlation with flipped, transposed weights, the fused residual / loss
// epilogues) and the weight and bias gradients (wgrad_tc_kernel, below).  The network
// is the learned stand-in for the offline projection of Sec. 5, Eq. 4-5:
// y = x + conv3x3(32->3) . ReLU . conv3x3(32->32) . ReLU . conv3x3(3->32) (x).
//
// out[p][o] = sum_{tap, c} W[tap][o][c] * in[p + off(tap)][c], tap = 3 ky + kx
// reading (y + ky - 1, x + kx - 1), zero outside the image.
//
// Persistent CTAs of four warps; output tiles of 30 x 16 pixels over a halo
// of 32 positions x 18 rows, positions q = 32 hy + hx, so a halo row is one
// TMEM lane quadrant and a tap is an A operand shifted by 32 (ky - 1) + kx - 1
// positions (a descriptor start 16 bytes per position on).  Four M-tiles of
// 128 positions (4 halo rows each) per tile, N = the output channels (32, or
// 16 for the 3-output layer).  32-channel BF16 inputs: two K = 16 MMAs per tap,
// 18 per M-tile.  3-channel FP32 RGBA inputs are staged pair-packed (position
// s holds x[s] and x[s+1] as R, G, B, 0 twice) and the A descriptor puts the
// second K group two positions on, so one MMA covers kernel columns -1..+2 of
// a kernel row: 3 MMAs per M-tile.  Output columns 0 and 31 of the halo see a
// wrapped neighbour and are never stored.
//
// Per tile: the halo is staged (zeros outside the image), one thread issues
// the tile's MMAs and commits to an mbarrier, every warp waits (bounded by
// wait_ns, an error word on give-up), reads its lane quadrant of each M-tile's
// accumulators with tcgen05.ld and runs the epilogue.  Halos arrive by TMA: a
// 32-channel BF16 halo by one tiled copy per group of 8 channels straight into
// the MMA operand layout, the next tile's copy issued as soon as the current
// tile's MMAs have read the buffer (it lands during the epilogue); a 3-channel
// FP32 RGBA halo into a staging buffer that the four warps convert to BF16
// pairs, the next tile's copy issued as soon as they have read it (it lands
// during the MMAs and the epilogue).  Four CTAs share an SM, so one CTA's MMAs
// overlap another's staging and epilogue.
//
// Shared-memory operands use the K-major layout without swizzling: a position
// (row) holds 8 channels in 16 contiguous bytes, rows follow every 16 bytes
// (8-row core matrices 128 bytes apart), and each further group of 8 channels
// starts kCGroupB bytes later.  The weights arrive in the packed layouts of
// pack_weights_kernel (rows of 32 K values per output) and are rearranged into
// core-matrix blocks when a CTA loads them.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "lf_internal.h"
#include "lf_launch.h"

namespace lfk {

namespace {

constexpr int kCTW = 30, kCTH = 16;              // output tile
constexpr int kCHW = 32, kCHH = kCTH + 2;         // halo: 32 positions x 18 rows
constexpr int kCMT = kCTH / 4;                    // M-tiles of 128 positions per tile
constexpr int kCPos = kCHH * kCHW;                // 576 positions
constexpr int kCGuard = 2;                        // positions before and after (reads reach one beyond)
constexpr int kCGroupB = ((kCPos + 2 * kCGuard) * 16 + 127) / 128 * 128;  // bytes per group of 8 channels
constexpr int kCXOff = 128 - kCGuard * 16;        // halo position 0 of each group starts 128-byte aligned
constexpr int kCHaloTx = 4 * kCPos * 16;          // bytes of a tile's four TMA copies (32-channel halo)
constexpr int kCXsB = kCPos * 16;                 // a tile's FP32 RGBA halo (3-channel input), one TMA copy
constexpr int kCThreads = 128;
constexpr int kCPerSM = 4;                        // CTAs per SM: 4 x 128 TMEM columns
constexpr uint32_t kCTmemCols = 128;
constexpr uint64_t kCDrainNs = 2000000000ull;     // the teardown's wait for issued MMAs

__device__ __forceinline__ uint32_t c_su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t c_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f16, FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t c_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void c_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void c_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(c_su32(bar))
               : "memory");
}

// 0 once the phase of `bar` with this parity completed, 2 after limit_ns of
// %globaltimer without it.
__device__ __forceinline__ int c_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  uint32_t done;
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(c_su32(bar)), "r"(parity)
        : "memory");
    if (done) return 0;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (it == 0) t0 = t;
    else if (t - t0 >= limit_ns) return 2;
  }
}

__device__ __forceinline__ void c_tmem_ld16(uint32_t addr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Tile `tile`'s 32-channel BF16 halo by TMA: one tiled copy per group g of 8
// channels (a box of 8 channels x 32 positions x 18 rows of the 5-D tensor map
// {8, 4, W, H, n} over the map; zeros where the box leaves the image) into the
// group's operand rows, completing on `bar` with the copies' byte count.
__device__ __forceinline__ void c_load_halo(const CUtensorMap* tmap, uint32_t sx0, uint64_t* bar, int img, int x0,
                                            int y0) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(c_su32(bar)), "r"(kCHaloTx) : "memory");
#pragma unroll
  for (int g = 0; g < 4; ++g)
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
        "[%7];" ::"r"(sx0 + g * kCGroupB),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(0), "r"(g), "r"(x0 - 1), "r"(y0 - 1), "r"(img), "r"(c_su32(bar))
        : "memory");
}

// Tile `tile`'s FP32 RGBA halo by TMA: one tiled copy (4 channels x 32
// positions x 18 rows of the 4-D tensor map {4, W, H, n}; zeros outside the
// image) into the staging buffer xs, completing on `bar`.  Earlier reads of xs
// by this CTA's threads are ordered before the copy by a barrier and the
// proxy fence.
__device__ __forceinline__ void c_load_rgba(const CUtensorMap* tmap, uint32_t xs, uint64_t* bar, int img, int x0,
                                            int y0) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(c_su32(bar)), "r"(kCXsB) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::
          "r"(xs), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(0), "r"(x0 - 1), "r"(y0 - 1), "r"(img),
      "r"(c_su32(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t c_pack(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

}  // namespace

template <int IN, int COUT, int EPI>
__global__ void __launch_bounds__(kCThreads, kCPerSM)
    conv_tc_kernel(RefineConvArgs A, const __grid_constant__ CUtensorMap tmap) {
  constexpr int N = COUT < 16 ? 16 : COUT;                 // MMA N (the 3-output layer pads to 16)
  constexpr int NB = IN == kConvInBF16 ? 18 : 3;           // B blocks: (tap, half) or kernel row
  constexpr int kBlkB = 2 * N * 16;
  constexpr int kWBytes = NB * kBlkB;
  constexpr int G = IN == kConvInBF16 ? 4 : 1;             // channel groups in the halo
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char* sw = sm;
  unsigned char* sx = sm + kWBytes + kCXOff;  // group g, position p: sx + g * kCGroupB + (p + kCGuard) * 16
  constexpr int kXsOff = (kWBytes + kCXOff + G * kCGroupB + 127) / 128 * 128;
  unsigned char* xs = sm + kXsOff;             // 3-channel input: the FP32 RGBA halo as it landed
  constexpr int kBarOff = IN == kConvInBF16 ? kWBytes + kCXOff + G * kCGroupB : kXsOff + kCXsB;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kBarOff);     // the tile's MMAs completed
  uint64_t* xbar = bar + 1;                                         // the tile's TMA halo landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  __shared__ float s_bias[32];
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int H = A.H, W = A.W;

  // Weights into core-matrix blocks: block b, K group g, row n at sw + b * kBlkB + (g * N + n) * 16.
  for (int i = tid; i < NB * 2 * N; i += kCThreads) {
    const int b = i / (2 * N), g = (i / N) & 1, n = i % N;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (n < COUT) {
      if (IN == kConvInBF16) {  // packed [tap][n][32]: block b = 2 tap + half
        v = *reinterpret_cast<const uint4*>(A.wt + ((size_t)(b >> 1) * COUT + n) * 32 + 16 * (b & 1) + 8 * g);
      } else {  // packed [n][32], k = tap * 3 + c; block b = ky, element e: kx = 2g + e / 4, c = e % 4
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint32_t half2 = 0;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int e = 2 * j + h, kx = 2 * g + (e >> 2), c = e & 3;
            uint32_t bits = 0;
            if (kx < 3 && c < 3) bits = *reinterpret_cast<const uint16_t*>(A.wt + n * 32 + (b * 3 + kx) * 3 + c);
            half2 |= bits << (16 * h);
          }
          w[j] = half2;
        }
        v = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    *reinterpret_cast<uint4*>(sw + b * kBlkB + (g * N + n) * 16) = v;
  }
  for (int i = tid; i < G * kCGroupB / 16; i += kCThreads)  // the guard rows stay zero
    reinterpret_cast<uint4*>(sx)[i] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeros, to the tensor core and TMA
  if (tid < 32) s_bias[tid] = (EPI == kEpiRelu || (EPI != kEpiMask && tid < 3)) ? A.bias[tid] : 0.f;
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(c_su32(bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(c_su32(xbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(c_su32(tslot)),
                 "r"(kCTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  float loss_scale = 0.f;
  if (EPI == kEpiLoss) {
    const int cnt = *A.count;
    loss_scale = cnt > 0 ? 1.0f / (3.0f * (float)cnt) : 0.f;
  }
  const int tiles_x = (W + kCTW - 1) / kCTW, tiles_y = (H + kCTH - 1) / kCTH;
  const int n_tiles = tiles_x * tiles_y * A.n;
  // tile -> image and output origin (the halo starts one row and one column before)
  auto origin = [&](int tile, int& img, int& x0, int& y0) {
    img = tile / (tiles_x * tiles_y);
    const int rem = tile - img * tiles_x * tiles_y;
    y0 = (rem / tiles_x) * kCTH;
    x0 = (rem % tiles_x) * kCTW;
  };
  const uint32_t sx0 = c_su32(sx) + kCGuard * 16;  // halo position 0 of group 0 (128-byte aligned)
  uint32_t phase = 0, xphase = 0;
  bool issued = false;        // an MMA commit of this CTA may still be outstanding
  bool halo_pending = false;  // thread 0: a TMA halo copy may still be landing
  if (tid == 0 && (int)blockIdx.x < n_tiles) {
    int img, x0, y0;
    origin(blockIdx.x, img, x0, y0);
    if (IN == kConvInBF16) c_load_halo(&tmap, sx0, xbar, img, x0, y0);
    else c_load_rgba(&tmap, c_su32(xs), xbar, img, x0, y0);
    halo_pending = true;
  }
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    int img, x0, y0;
    origin(tile, img, x0, y0);

    // ---- stage the halo
    if (IN == kConvInBF16) {  // issued before this tile (above, or during the previous epilogue)
      if (tid == 0) {
        if (c_wait(xbar, xphase, A.wait_ns) != 0) {
          atomicOr(A.error, 1024);
          s_abort = 1;
        } else {
          xphase ^= 1u;
          halo_pending = false;
        }
      }
    } else {  // every thread waits for the staged FP32 halo, then converts its positions
      if (c_wait(xbar, xphase, A.wait_ns) != 0) {
        atomicOr(A.error, 1024);
        s_abort = 1;
      } else {
        xphase ^= 1u;
        if (tid == 0) halo_pending = false;
      }
      __syncthreads();
      if (!s_abort) {
        const float4* xf = reinterpret_cast<const float4*>(xs);
        for (int p = tid; p < kCPos; p += kCThreads) {
          const float4 v0 = xf[p], v1 = p + 1 < kCPos ? xf[p + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
          *reinterpret_cast<uint4*>(sx + (p + kCGuard) * 16) =
              make_uint4(c_pack(v0.x, v0.y), c_pack(v0.z, 0.f), c_pack(v1.x, v1.y), c_pack(v1.z, 0.f));
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (s_abort) break;  // the halo copy's wait gave up
    // the warps have read the staged FP32 halo: the next tile's copy lands during the MMAs
    if (IN == kConvInRGBA && tid == 0 && tile + (int)gridDim.x < n_tiles) {
      int nimg, nx0, ny0;
      origin(tile + gridDim.x, nimg, nx0, ny0);
      c_load_rgba(&tmap, c_su32(xs), xbar, nimg, nx0, ny0);
      halo_pending = true;
    }

    // ---- the tile's MMAs: M-tile m holds output positions 32 (4m + 1) + r, r < 128
    if (tid == 0) {
      const uint32_t sxa = c_su32(sx) + kCGuard * 16;  // position 0
      const uint64_t ad = c_desc(sxa, IN == kConvInBF16 ? kCGroupB : 32, 128);
      const uint64_t bd = c_desc(c_su32(sw), N * 16, 128);
      constexpr uint32_t id = c_idesc(128, N);
      for (int m = 0; m < kCMT; ++m) {
        const uint32_t d = tmem + (uint32_t)(m * N);
        if (IN == kConvInBF16) {
#pragma unroll
          for (int t = 0; t < 9; ++t) {  // tap t = 3 ky + kx starts at 32 (4m + ky) + kx - 1
#pragma unroll
            for (int h = 0; h < 2; ++h)
              c_mma(d, ad + (uint64_t)(int64_t)(32 * (4 * m + t / 3) + t % 3 - 1) + (uint64_t)(h * (2 * kCGroupB / 16)),
                    bd + (uint64_t)((2 * t + h) * (kBlkB / 16)), id, t > 0 || h > 0);
          }
        } else {
#pragma unroll
          for (int ky = 0; ky < 3; ++ky)  // kernel row ky: pairs from 32 (4m + ky) - 1
            c_mma(d, ad + (uint64_t)(int64_t)(32 * (4 * m + ky) - 1), bd + (uint64_t)(ky * (kBlkB / 16)), id, ky > 0);
        }
      }
      c_commit(bar);
    }
    issued = true;
    if (lane == 0 && c_wait(bar, phase, A.wait_ns) != 0) {
      atomicOr(A.error, 64);
      s_abort = 1;
    }
    __syncthreads();  // every warp has waited: the abort decision is the same for the whole CTA
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (s_abort) break;
    issued = false;
    phase ^= 1u;
    // the MMAs have read the halo: the next tile's copy lands during this epilogue
    if (IN == kConvInBF16 && tid == 0 && tile + (int)gridDim.x < n_tiles) {
      int nimg, nx0, ny0;
      origin(tile + gridDim.x, nimg, nx0, ny0);
      c_load_halo(&tmap, sx0, xbar, nimg, nx0, ny0);
      halo_pending = true;
    }

    // ---- epilogue: warp w reads lanes 32w.. (halo row 4m + 1 + w, column lane) of each M-tile
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const int gx = x0 + lane - 1;
    float lsum = 0.f;
    for (int m = 0; m < kCMT; ++m) {
      const int gy = y0 + 4 * m + warp;
      const bool store = lane >= 1 && lane <= kCTW && gy < H && gx < W;
      const size_t pix = ((size_t)img * H + (store ? gy : 0)) * W + (store ? gx : 0);
      const uint32_t t = tmem + lane_base + (uint32_t)(m * N);
      if (EPI == kEpiRelu || EPI == kEpiMask) {
        float v0[16], v1[16];
        c_tmem_ld16(t, v0);
        c_tmem_ld16(t + 16, v1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!store) continue;
        float v[32];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          v[k] = v0[k];
          v[16 + k] = v1[k];
        }
        uint32_t w[16];
        if (EPI == kEpiRelu) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            w[j] = c_pack(fmaxf(v[2 * j] + s_bias[2 * j], 0.f), fmaxf(v[2 * j + 1] + s_bias[2 * j + 1], 0.f));
        } else {
          const uint4* mk = reinterpret_cast<const uint4*>(A.mask + pix * 32);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint4 mq = mk[q];
            const uint32_t mw[4] = {mq.x, mq.y, mq.z, mq.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const __nv_bfloat162 mm = *reinterpret_cast<const __nv_bfloat162*>(&mw[j]);
              const int k = 8 * q + 2 * j;
              w[4 * q + j] = c_pack(__bfloat162float(mm.x) > 0.f ? v[k] : 0.f, __bfloat162float(mm.y) > 0.f ? v[k + 1] : 0.f);
            }
          }
        }
        uint4* dst = reinterpret_cast<uint4*>(A.out_h + pix * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
      } else {  // kEpiResid / kEpiLoss: outputs 0..2
        float v[16];
        c_tmem_ld16(t, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!store) continue;
        const float4 x = reinterpret_cast<const float4*>(A.x)[pix];
        const float r0 = v[0] + s_bias[0], r1 = v[1] + s_bias[1], r2 = v[2] + s_bias[2];
        if (EPI == kEpiResid) {
          const bool valid = x.w > 0.f;
          reinterpret_cast<float4*>(A.out_f)[pix] =
              valid ? make_float4(x.x + r0, x.y + r1, x.z + r2, 1.f) : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
          const float4 tg = reinterpret_cast<const float4*>(A.target)[pix];
          const bool valid = x.w > 0.f && tg.w > 0.f;
          const float d0 = valid ? (x.x + r0) - tg.x : 0.f;
          const float d1 = valid ? (x.y + r1) - tg.y : 0.f;
          const float d2 = valid ? (x.z + r2) - tg.z : 0.f;
          lsum += d0 * d0 + d1 * d1 + d2 * d2;
          reinterpret_cast<float4*>(A.out_f)[pix] =
              make_float4(2.f * loss_scale * d0, 2.f * loss_scale * d1, 2.f * loss_scale * d2, 0.f);
        }
      }
    }
    if (EPI == kEpiLoss) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
      if (lane == 0 && lsum != 0.f) atomicAdd(A.loss, lsum * loss_scale);
    }
    // every warp has read the accumulators and the halo before the next tile overwrites them
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }

  // A wait that gave up may leave MMAs running: wait for them before the tensor memory is freed.
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && issued && s_abort && c_wait(bar, phase, kCDrainNs) != 0) atomicOr(A.error, 128);
  // and for a halo copy still landing (a wait that gave up) before the shared memory is released
  if (tid == 0 && halo_pending && c_wait(xbar, xphase, kCDrainNs) != 0) atomicOr(A.error, 2048);
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCTmemCols));
  }
}

namespace {

template <int IN, int COUT, int EPI>
cudaError_t launch_conv_tc_t(const RefineConvArgs& a, cudaStream_t s) {
  constexpr int N = COUT < 16 ? 16 : COUT;
  constexpr int kW = (IN == kConvInBF16 ? 18 : 3) * 2 * N * 16;
  constexpr int used = IN == kConvInBF16 ? kW + kCXOff + 4 * kCGroupB + 24
                                         : (kW + kCXOff + kCGroupB + 127) / 128 * 128 + kCXsB + 24;
  // At least 54 KB: no more than kCPerSM CTAs share an SM, so their tensor memory (128 columns each)
  // always fits and no CTA waits in tcgen05.alloc for another persistent CTA to finish.
  constexpr int smem = used < 54 * 1024 ? 54 * 1024 : used;
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(conv_tc_kernel<IN, COUT, EPI>), smem);
  if (e != cudaSuccess) return e;
  const int n_tiles = ((a.W + kCTW - 1) / kCTW) * ((a.H + kCTH - 1) / kCTH) * a.n;
  if (n_tiles == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  // The halo copies' tensor map, over a 16-byte aligned base.  32-channel input: a 5-D tensor
  // {8 channels, 4 groups, W, H, n} of BF16, with group, position, row and image strides of 16,
  // 64, W * 64 and W * H * 64 bytes.  3-channel input: a 4-D tensor {4 channels, W, H, n} of FP32
  // RGBA, strides 16, W * 16 and W * H * 16 bytes.
  CUtensorMap tmap;
  std::memset(&tmap, 0, sizeof(tmap));
  const EncodeTiled enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  if (IN == kConvInBF16) {
    if ((reinterpret_cast<uintptr_t>(a.src_h) & 15u) != 0) return cudaErrorInvalidValue;
    const cuuint64_t dims[5] = {8, 4, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.n};
    const cuuint64_t strides[4] = {16, 64, (cuuint64_t)a.W * 64, (cuuint64_t)a.W * a.H * 64};
    const cuuint32_t box[5] = {8, 1, (cuuint32_t)kCHW, (cuuint32_t)kCHH, 1};
    const cuuint32_t step[5] = {1, 1, 1, 1, 1};
    if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(a.src_h), dims, strides, box,
            step, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  } else {
    if ((reinterpret_cast<uintptr_t>(a.src_f) & 15u) != 0) return cudaErrorInvalidValue;
    const cuuint64_t dims[4] = {4, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.n};
    const cuuint64_t strides[3] = {16, (cuuint64_t)a.W * 16, (cuuint64_t)a.W * a.H * 16};
    const cuuint32_t box[4] = {4, (cuuint32_t)kCHW, (cuuint32_t)kCHH, 1};
    const cuuint32_t step[4] = {1, 1, 1, 1};
    if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(a.src_f), dims, strides, box, step,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  const int grid = n_tiles < sms * kCPerSM ? n_tiles : sms * kCPerSM;
  conv_tc_kernel<IN, COUT, EPI><<<grid, kCThreads, smem, s>>>(a, tmap);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_refine_conv(int in_mode, int cout, int epi, const RefineConvArgs& a, cudaStream_t s) {
  if (in_mode == kConvInRGBA && cout == 32 && epi == kEpiRelu) return launch_conv_tc_t<kConvInRGBA, 32, kEpiRelu>(a, s);
  if (in_mode == kConvInRGBA && cout == 32 && epi == kEpiMask) return launch_conv_tc_t<kConvInRGBA, 32, kEpiMask>(a, s);
  if (in_mode == kConvInBF16 && cout == 32 && epi == kEpiRelu) return launch_conv_tc_t<kConvInBF16, 32, kEpiRelu>(a, s);
  if (in_mode == kConvInBF16 && cout == 32 && epi == kEpiMask) return launch_conv_tc_t<kConvInBF16, 32, kEpiMask>(a, s);
  if (in_mode == kConvInBF16 && cout == 8 && epi == kEpiResid) return launch_conv_tc_t<kConvInBF16, 8, kEpiResid>(a, s);
  if (in_mode == kConvInBF16 && cout == 8 && epi == kEpiLoss) return launch_conv_tc_t<kConvInBF16, 8, kEpiLoss>(a, s);
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ weight gradients
//
// dW[o][c][tap] = sum_p g[p][o] a[p + off(tap)][c], db[o] = sum_p g[p][o]
// (g = dL/dz of the layer's output, a = the layer's input), as one GEMM
// D[(tap, c)][o] over K = pixels: M = 9 x 32 rows of shifted input channels
// plus a row of ones, whose product with g is the bias gradient (modes 2, 3:
// 289 rows in three M-tiles of 128; mode 1, the 3-channel input: 28 rows in
// one), N = the output channels (32; 3 padded to 16 in mode 3).  Both operands
// are K-major, so a CTA transposes each 64-pixel chunk (32 x 2 outputs) into
// shared memory: ldmatrix.trans turns an 8-position x 8-channel block of a
// staged 32-channel map into one channel's 8 consecutive pixels spread over four
// lanes, i.e. one 16-byte operand row.  The accumulators stay in TMEM over all
// of a CTA's chunks; the CTA then writes its partial row, and the rows are
// summed in a fixed order afterwards (deterministic).
//   MODE 1: g = dL/dz1 (BF16, 32), a = the network input (FP32 RGBA, 3).  W1, b1.
//   MODE 2: g = dL/dz2 (BF16, 32), a = a1 (BF16, 32).                        W2, b2.
//   MODE 3: g = dL/dr  (FP32 RGBA, 3), a = a2 (BF16, 32).                    W3, b3.

namespace {

constexpr int kWPx = 64;                         // pixels per chunk: 32 x 2 outputs
constexpr int kWHW = 34, kWHH = 4;               // input halo of a chunk
constexpr int kWRowB = 80;                       // staged 32-channel rows (64 B + 16 B: no bank conflicts)
constexpr int kWThreads = 128;

__device__ __forceinline__ void c_ldsm_x4_t(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}

}  // namespace

template <int MODE>
__global__ void __launch_bounds__(kWThreads) wgrad_tc_kernel(RefineWgradArgs A) {
  constexpr int MR = MODE == 1 ? 128 : 384;                     // A rows (M), zero beyond the data
  constexpr int MT = MR / 128;
  constexpr int ONES = MODE == 1 ? 27 : 288;                    // the row of ones (bias gradient)
  constexpr int N = MODE == 3 ? 16 : 32;
  constexpr int COUT = MODE == 3 ? 3 : 32;
  constexpr int SEG = MODE == 1 ? 864 + 32 : (MODE == 2 ? 9216 + 32 : 864 + 3);
  constexpr int kLboA = MR * 16, kLboB = N * 16;                // bytes between 8-pixel K groups
  constexpr int kAB = 8 * kLboA, kBB = 8 * kLboB;               // 64 pixels = 8 K groups
  constexpr int kHaloB = kWHW * kWHH * kWRowB;                  // modes 2, 3: 32-channel input halo
  constexpr int kGB = kWPx * kWRowB;                            // modes 1, 2: 32-channel g
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char* sa = sm;                 // A: [8 K groups][MR rows][16 B]
  unsigned char* sb = sa + kAB;           // B: [8 K groups][N rows][16 B]
  unsigned char* sh = sb + kBB;           // staged input halo (FP32 RGBA in mode 1)
  unsigned char* sg = sh + kHaloB;        // staged g (FP32 RGBA in mode 3)
  uint64_t* bar = reinterpret_cast<uint64_t*>(sg + kGB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int H = A.H, W = A.W;

  for (int i = tid; i < (kAB + kBB) / 16; i += kWThreads) reinterpret_cast<uint4*>(sa)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int j = tid; j < 8; j += kWThreads)  // the row of ones
    *reinterpret_cast<uint4*>(sa + j * kLboA + ONES * 16) = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(c_su32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(c_su32(tslot)),
                 "r"(kCTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  const int cx = (W + 31) / 32, cy = (H + 1) / 2, n_chunks = cx * cy * A.n;
  // A chunk's g (its 64 pixels) and input halo, zeros outside the image, travel
  // through registers: chunk k + 1 is loaded while chunk k's MMAs run, and
  // stored into the staging buffers once chunk k's transposes have read them.
  constexpr int GI = MODE == 3 ? 1 : 2;  // g items (16 bytes) per thread
  constexpr int HI = MODE == 1 ? 2 : 5;  // halo items per thread
  uint4 gr[GI], hr[HI];
  auto load = [&](int chunk) {
    const int img = chunk / (cx * cy), rem = chunk - img * cx * cy;
    const int y0 = (rem / cx) * 2, x0 = (rem % cx) * 32;  // output origin; halo at (y0-1, x0-1)
#pragma unroll
    for (int k = 0; k < GI; ++k) {
      const int i = tid + k * kWThreads;
      gr[k] = make_uint4(0u, 0u, 0u, 0u);
      if (MODE == 3) {
        const int gy = y0 + (i >> 5), gx = x0 + (i & 31);
        if (i < kWPx && gy < H && gx < W)
          gr[k] = reinterpret_cast<const uint4*>(A.g_f)[((size_t)img * H + gy) * W + gx];
      } else {
        const int p = i >> 2, q = i & 3, gy = y0 + (p >> 5), gx = x0 + (p & 31);
        if (gy < H && gx < W) gr[k] = reinterpret_cast<const uint4*>(A.g_h + (((size_t)img * H + gy) * W + gx) * 32)[q];
      }
    }
#pragma unroll
    for (int k = 0; k < HI; ++k) {
      const int i = tid + k * kWThreads;
      hr[k] = make_uint4(0u, 0u, 0u, 0u);
      if (MODE == 1) {
        const int gy = y0 - 1 + i / kWHW, gx = x0 - 1 + i % kWHW;
        if (i < kWHW * kWHH && gy >= 0 && gy < H && gx >= 0 && gx < W)
          hr[k] = reinterpret_cast<const uint4*>(A.x)[((size_t)img * H + gy) * W + gx];
      } else {
        const int P = i >> 2, q = i & 3, gy = y0 - 1 + P / kWHW, gx = x0 - 1 + P % kWHW;
        if (P < kWHW * kWHH && gy >= 0 && gy < H && gx >= 0 && gx < W)
          hr[k] = reinterpret_cast<const uint4*>(A.a_h + (((size_t)img * H + gy) * W + gx) * 32)[q];
      }
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int k = 0; k < GI; ++k) {
      const int i = tid + k * kWThreads;
      if (MODE == 3) {
        if (i < kWPx) reinterpret_cast<uint4*>(sg)[i] = gr[k];
      } else {
        *reinterpret_cast<uint4*>(sg + (i >> 2) * kWRowB + (i & 3) * 16) = gr[k];
      }
    }
#pragma unroll
    for (int k = 0; k < HI; ++k) {
      const int i = tid + k * kWThreads;
      if (MODE == 1) {
        if (i < kWHW * kWHH) reinterpret_cast<uint4*>(sh)[i] = hr[k];
      } else if ((i >> 2) < kWHW * kWHH) {
        *reinterpret_cast<uint4*>(sh + (i >> 2) * kWRowB + (i & 3) * 16) = hr[k];
      }
    }
  };
  uint32_t phase = 0;
  bool issued = false, any = false;
  if (blockIdx.x < n_chunks) {
    load(blockIdx.x);
    store();
    if (blockIdx.x + gridDim.x < n_chunks) load(blockIdx.x + gridDim.x);
  }
  for (int chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x) {
    __syncthreads();  // this chunk's staged g and halo are visible; the previous chunk's MMAs completed

    // ---- A rows (tap, c) and B rows o, K group j = pixels 8j .. 8j + 7 (py = j / 4, px = 8 (j % 4) ..)
    if (MODE == 1) {  // rows tap * 3 + c from the FP32 halo
      for (int i = tid; i < 27 * 8; i += kWThreads) {
        const int row = i >> 3, j = i & 7, tap = row / 3, c = row % 3;
        const int base = (j / 4 + tap / 3) * kWHW + (j % 4) * 8 + tap % 3;
        const float* hf = reinterpret_cast<const float*>(sh);
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) w[e] = c_pack(hf[(base + 2 * e) * 4 + c], hf[(base + 2 * e + 1) * 4 + c]);
        *reinterpret_cast<uint4*>(sa + j * kLboA + row * 16) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    } else {  // 9 taps x 4 channel groups x 8 K groups of 8x8 blocks, four per ldmatrix
      for (int i = warp; i < 9 * 4 * 8 / 4; i += kWThreads / 32) {
        const int mat = lane >> 3, r = lane & 7, b = 4 * i + mat;
        const int tap = b >> 5, cg = (b >> 3) & 3, j = b & 7;
        const int P = (j / 4 + tap / 3) * kWHW + (j % 4) * 8 + tap % 3 + r;
        uint32_t v[4];
        c_ldsm_x4_t(c_su32(sh + P * kWRowB + cg * 16), v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int bk = 4 * i + k, tk = bk >> 5, ck = (bk >> 3) & 3, jk = bk & 7;
          *reinterpret_cast<uint32_t*>(sa + jk * kLboA + (tk * 32 + ck * 8 + (lane >> 2)) * 16 + (lane & 3) * 4) = v[k];
        }
      }
    }
    if (MODE == 3) {  // rows o < 3 from the FP32 g
      for (int i = tid; i < 3 * 8; i += kWThreads) {
        const int o = i >> 3, j = i & 7;
        const float* gf = reinterpret_cast<const float*>(sg);
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) w[e] = c_pack(gf[(8 * j + 2 * e) * 4 + o], gf[(8 * j + 2 * e + 1) * 4 + o]);
        *reinterpret_cast<uint4*>(sb + j * kLboB + o * 16) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    } else {  // 4 channel groups x 8 K groups of 8x8 blocks
      for (int i = warp; i < 4 * 8 / 4; i += kWThreads / 32) {
        const int mat = lane >> 3, r = lane & 7, b = 4 * i + mat;
        const int cg = b >> 3, j = b & 7;
        uint32_t v[4];
        c_ldsm_x4_t(c_su32(sg + (8 * j + r) * kWRowB + cg * 16), v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int bk = 4 * i + k, ck = bk >> 3, jk = bk & 7;
          *reinterpret_cast<uint32_t*>(sb + jk * kLboB + (ck * 8 + (lane >> 2)) * 16 + (lane & 3) * 4) = v[k];
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // ---- D[m-tile][o] += A[rows][64 px] B[o][64 px]
    if (tid == 0) {
      const uint64_t ad = c_desc(c_su32(sa), kLboA, 128), bd = c_desc(c_su32(sb), kLboB, 128);
      constexpr uint32_t id = c_idesc(128, N);
      for (int m = 0; m < MT; ++m) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)  // K = 16: two 8-pixel groups
          c_mma(tmem + (uint32_t)(m * N), ad + (uint64_t)(m * 128 * 16 / 16) + (uint64_t)(kk * 2 * kLboA / 16),
                bd + (uint64_t)(kk * 2 * kLboB / 16), id, (any || kk > 0) ? 1u : 0u);
      }
      c_commit(bar);
    }
    issued = true;
    any = true;
    // the staging buffers are free (the transposes read them before the barrier above):
    // the next chunk moves in while this one's MMAs run, and the one after starts loading
    if (chunk + gridDim.x < n_chunks) {
      store();
      if (chunk + 2 * gridDim.x < n_chunks) load(chunk + 2 * gridDim.x);
    }
    if (lane == 0 && c_wait(bar, phase, A.wait_ns) != 0) {
      atomicOr(A.error, 256);
      s_abort = 1;
    }
    __syncthreads();  // the whole CTA takes the same decision
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (s_abort) break;
    issued = false;
    phase ^= 1u;
  }

  // ---- this CTA's partial row: warp w reads lanes 32w.. (rows) of each M-tile, N columns (o)
  float* out = A.partial + (size_t)blockIdx.x * SEG;
  if (!s_abort) {
    for (int m = 0; m < MT; ++m) {
      const int row = m * 128 + 32 * warp + lane;
      float v[32];
      if (any) {
        const uint32_t t = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(m * N);
        float v0[16];
        c_tmem_ld16(t, v0);
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = v0[k];
        if (N == 32) {
          c_tmem_ld16(t + 16, v0);
#pragma unroll
          for (int k = 0; k < 16; ++k) v[16 + k] = v0[k];
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = 0.f;
      }
      if (row == ONES) {
        for (int o = 0; o < COUT; ++o) out[SEG - COUT + o] = v[o];
      } else if (MODE == 1 && row < 27) {  // row = tap * 3 + c -> W1[o][c][tap]
        for (int o = 0; o < COUT; ++o) out[o * 27 + (row % 3) * 9 + row / 3] = v[o];
      } else if (MODE != 1 && row < 288) {  // row = tap * 32 + c -> W[o][c][tap]
        for (int o = 0; o < COUT; ++o) out[(o * 32 + (row & 31)) * 9 + (row >> 5)] = v[o];
      }
    }
  }

  // A wait that gave up may leave MMAs running: wait for them before the tensor memory is freed.
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && issued && s_abort && c_wait(bar, phase, kCDrainNs) != 0) atomicOr(A.error, 512);
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCTmemCols));
  }
}

namespace {

template <int MODE>
cudaError_t launch_wgrad_tc_t(const RefineWgradArgs& a, cudaStream_t s) {
  constexpr int MR = MODE == 1 ? 128 : 384, N = MODE == 3 ? 16 : 32;
  constexpr int used = 8 * MR * 16 + 8 * N * 16 + kWHW * kWHH * kWRowB + kWPx * kWRowB + 16;
  constexpr int smem = used < 54 * 1024 ? 54 * 1024 : used;  // at most four CTAs (their TMEM) per SM
  cudaError_t e = ensure_dynamic_smem(reinterpret_cast<const void*>(wgrad_tc_kernel<MODE>), smem);
  if (e != cudaSuccess) return e;
  wgrad_tc_kernel<MODE><<<a.n_ctas, kWThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_refine_wgrad(int mode, const RefineWgradArgs& a, cudaStream_t s) {
  if (mode == 1) return launch_wgrad_tc_t<1>(a, s);
  if (mode == 2) return launch_wgrad_tc_t<2>(a, s);
  if (mode == 3) return launch_wgrad_tc_t<3>(a, s);
  return cudaErrorInvalidValue;
}

}  // namespace lfk
