// lf_raster.cu - the fragment stage: rasterise, depth test within each view,
// fetch, weight, accumulate and normalise (Eq. 2, Sec. 4.2 and 4.2.2).
//
// One CTA owns one TW x TH screen tile and one thread owns one pixel, so the
// FP32 accumulators of Eq. 2's numerator and denominator stay in registers for
// the whole tile (the paper's accumulation framebuffer becomes registers, and
// its second pass becomes the epilogue).  For each view whose disk footprint
// overlaps the tile (bits of the tile's view mask, visited in view order):
//   1. each pixel evaluates its disk weight at its sphere crossing; views no
//      pixel of the tile sees are skipped;
//   2. the view's triangle segment is streamed in chunks of blockDim: each
//      thread tests one triangle's bounding box against the tile, and the
//      overlapping ones are compacted in id order (warp ballots + a block
//      prefix sum) into shared memory with their edge functions re-based to
//      the tile origin;
//   3. every pixel tests every listed triangle with three int32 multiply-adds
//      (the int64 edge function divided by 256, exact because pixel centres
//      step by 256 subpixels) and keeps the nearest fragment by FP32 1/z,
//      ties to the lower id;
//   4. the winner is projected into the source view and sampled bilinearly,
//      weighted, and accumulated.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <type_traits>

#include "lf_internal.h"
#include "lf_launch.h"

namespace lfk {

// 80-byte stride: eight consecutive 16-byte stores hit distinct bank groups.
struct __align__(16) TileTri {
  int32_t q0, q1, q2, id;   // id bit 31: edge deltas too large for the int32 path
  int32_t a0, b0, a1, b1;
  int32_t a2, b2;
  float ia, ib;
  float ic;
  int32_t pad[7];           // pad[0]: view slot within the round
};
static_assert(sizeof(TileTri) == 80, "TileTri layout");

__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0, float b1, float b2) {
  return __fmaf_rn(a0, b0, __fmaf_rn(a1, b1, __fmul_rn(a2, b2)));
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16; x *= 0x85EBCA6Bu;
  x ^= x >> 13; x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

template <int FMT>
__device__ __forceinline__ float3 texel(const void* tex, int idx, float scale) {
  if constexpr (FMT == LF_TEX_F32) {
    float4 c = __ldg(reinterpret_cast<const float4*>(tex) + idx);
    return make_float3(c.x, c.y, c.z);
  } else if constexpr (FMT == LF_TEX_U8) {
    uchar4 c = __ldg(reinterpret_cast<const uchar4*>(tex) + idx);
    const float k = 1.0f / 255.0f;
    return make_float3(__fmul_rn(c.x, k), __fmul_rn(c.y, k), __fmul_rn(c.z, k));
  } else if constexpr (FMT == LF_TEX_BF16) {
    uint2 p = __ldg(reinterpret_cast<const uint2*>(tex) + idx);
    return make_float3(__uint_as_float(p.x << 16), __uint_as_float(p.x & 0xffff0000u), __uint_as_float(p.y << 16));
  } else {
    uint32_t p = __ldg(reinterpret_cast<const uint32_t*>(tex) + idx);
    __nv_fp8x2_e4m3 lo, hi;
    lo.__x = (__nv_fp8x2_storage_t)(p & 0xffffu);
    hi.__x = (__nv_fp8x2_storage_t)(p >> 16);
    float2 a = static_cast<float2>(lo);
    float2 b = static_cast<float2>(hi);
    return make_float3(__fmul_rn(a.x, scale), __fmul_rn(a.y, scale), __fmul_rn(b.x, scale));
  }
}

// Bilinear sample of one view (tex points at its first texel) at bilinear
// coordinates (u, v) = (s - 1/2, t - 1/2), clamp to edge.  The float clamp only
// keeps the integer conversion in range; it does not change the result.
template <int FMT>
__device__ __forceinline__ float3 bilinear(const void* tex, int W, int H, float u, float v, float scale,
                                           uint32_t* bits, int64_t bit_base) {
  u = fminf(fmaxf(u, -1.0f), (float)W);
  v = fminf(fmaxf(v, -1.0f), (float)H);
  const float fu = floorf(u), fv = floorf(v);
  const float al = __fsub_rn(u, fu), be = __fsub_rn(v, fv);
  const int iu = (int)fu, jv = (int)fv;
  const int i0 = min(max(iu, 0), W - 1), i1 = min(max(iu + 1, 0), W - 1);
  const int j0 = min(max(jv, 0), H - 1), j1 = min(max(jv + 1, 0), H - 1);
  const int t00 = j0 * W + i0, t10 = j0 * W + i1, t01 = j1 * W + i0, t11 = j1 * W + i1;
  const float3 c00 = texel<FMT>(tex, t00, scale), c10 = texel<FMT>(tex, t10, scale);
  const float3 c01 = texel<FMT>(tex, t01, scale), c11 = texel<FMT>(tex, t11, scale);
  if (bits) {
    const int64_t t[4] = {bit_base + t00, bit_base + t10, bit_base + t01, bit_base + t11};
    for (int k = 0; k < 4; ++k) atomicOr(&bits[t[k] >> 5], 1u << (t[k] & 31));
  }
  // explicit roundings: the same image whatever code the caller is compiled into
  const float nal = __fsub_rn(1.0f, al), nbe = __fsub_rn(1.0f, be);
  const float w00 = __fmul_rn(nal, nbe), w10 = __fmul_rn(al, nbe), w01 = __fmul_rn(nal, be), w11 = __fmul_rn(al, be);
  return make_float3(__fmaf_rn(w11, c11.x, __fmaf_rn(w01, c01.x, __fmaf_rn(w10, c10.x, __fmul_rn(w00, c00.x)))),
                     __fmaf_rn(w11, c11.y, __fmaf_rn(w01, c01.y, __fmaf_rn(w10, c10.y, __fmul_rn(w00, c00.y)))),
                     __fmaf_rn(w11, c11.z, __fmaf_rn(w01, c01.z, __fmaf_rn(w10, c10.z, __fmul_rn(w00, c00.z)))));
}


constexpr int kViewsPerRound = 32;  // views a warp handles per round (one per lane)
constexpr int kWinnerBuf = 8;       // buffered depth-test winners per pixel before shading
constexpr int kPx = 2;              // vertically adjacent pixels per lane

// A warp's private shared memory: its view table, its compacted triangles and
// its pixels' buffered depth winners.
struct WarpSmem {
  TileTri tri[32];
  long long q64[32 * 3];
  float wiz[kWinnerBuf][kPx][32];
  uint8_t wslot[kWinnerBuf][kPx][32];
  float4 cc[kViewsPerRound];
  float Hm[kViewsPerRound][12];
  const void* tex[kViewsPerRound];
  float inv_r[kViewsPerRound];
  int bstart[kViewsPerRound], bcount[kViewsPerRound], gbase[kViewsPerRound], gcount[kViewsPerRound];
  int views[kViewsPerRound];
  int off[kViewsPerRound + 1];
};

// With oval disks (Sec. 4.4) a warp also holds each view's oval constants:
// n (3), x (3), y (3), k, u0, v0, 1/e_u+, 1/e_u-, 1/e_v+, 1/e_v-.
struct WarpSmemOval : WarpSmem {
  float ov[kViewsPerRound][16];
};

// Oval membership, the FP32 decision (fixed order, as the oracle takes it):
// the ray (ex, ey, 1) meets the disk plane at t = k / (n.e) >= 0; inside where
// (u / e_u)^2 + (v / e_v)^2 < 1, the extents chosen by the signs of u and v.
// Returns rho^2 (the weight is 1 - sqrt(rho^2)), or 2 when outside.
__device__ __forceinline__ float oval_rho2(const float* o, float ex, float ey) {
  const float den = __fmaf_rn(o[0], ex, __fmaf_rn(o[1], ey, o[2]));
  if (den == 0.0f) return 2.0f;
  const float t = __fdiv_rn(o[9], den);
  if (!(t >= 0.0f)) return 2.0f;
  const float ue = __fmaf_rn(o[3], ex, __fmaf_rn(o[4], ey, o[5]));
  const float ve = __fmaf_rn(o[6], ex, __fmaf_rn(o[7], ey, o[8]));
  const float u = __fmaf_rn(t, ue, -o[10]), v = __fmaf_rn(t, ve, -o[11]);
  const float a = __fmul_rn(u, u >= 0.0f ? o[12] : o[13]);
  const float b = __fmul_rn(v, v >= 0.0f ? o[14] : o[15]);
  const float r2 = __fmaf_rn(a, a, __fmul_rn(b, b));
  return r2 < 1.0f ? r2 : 2.0f;
}

// The next (up to 32) views of the tile's mask in increasing order, resuming
// at (cur_word, cur_bits) when the previous round stopped inside a word.
__device__ __forceinline__ int collect_views(const uint32_t* mask, int mask_words, int* views, int& cur_word,
                                             bool& partial, uint32_t& pbits) {
  const int lane = threadIdx.x & 31;
  int n = 0;
  while (cur_word < mask_words) {
    const int wl = cur_word + lane;
    uint32_t b = 0;
    if (wl < mask_words) b = (lane == 0 && partial) ? pbits : __ldg(mask + wl);
    const int c = __popc(b);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - c;
    const int room = kViewsPerRound - n;
    const int take = min(max(room - excl, 0), c);
    uint32_t bb = b;
    for (int k = 0; k < take; ++k) {
      const int bp = __ffs(bb) - 1;
      bb &= bb - 1;
      views[n + excl + k] = wl * 32 + bp;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total <= room) {
      n += total;
      cur_word += 32;
      partial = false;
      continue;
    }
    const unsigned over = __ballot_sync(0xffffffffu, incl > room);
    const int L = __ffs(over) - 1;
    pbits = __shfl_sync(0xffffffffu, bb, L);
    n = kViewsPerRound;
    cur_word += L;
    partial = true;
    break;
  }
  __syncwarp();
  return n;
}

// One warp's strip of a tile: TW x (2 * 32/TW) pixels, two vertically adjacent
// pixels per lane.  The warp works alone (no block barrier): per round of up
// to 32 views from the tile mask it (a) loads their per-eye records and this
// tile's bin range for each, (b) tests every pixel's sphere crossing against
// each disk (one bit per view), (c) gathers the bin entries of the views some
// pixel of the strip sees, keeps the triangles whose box and edge functions
// reach the strip, compacts them with a ballot and tests each against both
// pixels, keeping the nearest fragment per view; (d) when the view changes, a
// pixel's winner is buffered, and buffered winners are shaded (bilinear
// fetch, weight, accumulate) with both pixels' texel loads in flight.
// SELECT: only the disk tests - every view some pixel of the strip sees is
// marked in A.visible, and nothing is drawn (the first pass of a two-level frame).
template <int TW, int TH, int FMT, bool INSPECT, bool MANY_EYES, bool OVAL, bool SELECT>
__device__ void raster_strip(const FrameArgs& A, const int item, const int strip, WarpSmem& S) {
  constexpr int ROWS = (32 / TW) * kPx;
  const int lane = threadIdx.x & 31;
  const uint32_t* mask = A.tile_masks + (int64_t)item * A.mask_words;
  // the eye holding this tile: the last one whose first tile is <= item (a
  // binary search in the batch kernel, whose calls hold up to 128 eyes; a scan
  // in the per-call kernel, which keeps its registers for the pixels)
  int e = 0;
  if constexpr (MANY_EYES) {
    for (int lo = 0, hi = A.n_eyes; hi - lo > 1;) {
      const int mid = (lo + hi) >> 1;
      if (A.eyes[mid].tile_base <= item) lo = mid;
      else hi = mid;
      e = lo;
    }
  } else {
    while (e + 1 < A.n_eyes && A.eyes[e + 1].tile_base <= item) ++e;
  }
  const EyeParams& E = A.eyes[e];
  const int tile = item - E.tile_base;
  const int tx = tile % E.tiles_x, ty = tile / E.tiles_x;
  const int i0 = tx * TW, j0 = ty * TH;
  const int di = lane % TW;
  const int dj0 = strip * ROWS;                      // strip rows, tile-relative
  const int dj = dj0 + (lane / TW) * kPx;            // this lane's first row, tile-relative
  const int wrow0 = j0 + dj0, wrow1 = wrow0 + ROWS - 1;
  const int pi = i0 + di;
  const EyeFloat& EF = A.eyes_f[e];
  const float ex = __fdiv_rn(__fsub_rn(__fadd_rn((float)pi, 0.5f), EF.cx), EF.fx);
  const float px = (float)pi + 0.5f;
  const int64_t P0x = 256 * (int64_t)i0 + 128, P0y = 256 * (int64_t)j0 + 128;
  const int64_t tex_per_view = (int64_t)A.src_w * A.src_h;

  bool valid[kPx], has_p[kPx];
  float ey[kPx], py[kPx], p[kPx][3];
  float acc_r[kPx], acc_g[kPx], acc_b[kPx], acc_w[kPx];
  int n_rec[kPx];
#pragma unroll
  for (int q = 0; q < kPx; ++q) {
    const int pj = j0 + dj + q;
    valid[q] = pi < E.W && pj < E.H;
    // Eye ray (Eq. 1) and its crossing of the capture sphere, FP32, fixed order.
    ey[q] = __fdiv_rn(__fsub_rn(__fadd_rn((float)pj, 0.5f), EF.cy), EF.fy);
    py[q] = (float)pj + 0.5f;
    float d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = __fmaf_rn(EF.R[k * 3 + 0], ex, __fmaf_rn(EF.R[k * 3 + 1], ey[q], EF.R[k * 3 + 2]));
    const float qa = dot3_rn(d[0], d[1], d[2], d[0], d[1], d[2]);
    const float qb = dot3_rn(EF.o[0], EF.o[1], EF.o[2], d[0], d[1], d[2]);
    const float qc = __fsub_rn(dot3_rn(EF.o[0], EF.o[1], EF.o[2], EF.o[0], EF.o[1], EF.o[2]), EF.R2);
    const float disc = __fsub_rn(__fmul_rn(qb, qb), __fmul_rn(qa, qc));
    has_p[q] = OVAL && valid[q];  // ovals are met in their own planes, not at the sphere
    p[q][0] = p[q][1] = p[q][2] = 0.0f;
    if (!OVAL && valid[q] && disc >= 0.0f) {
      const float t = __fdiv_rn(__fsub_rn(__fsqrt_rn(disc), qb), qa);
      if (t >= 0.0f) {
        has_p[q] = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) p[q][k] = __fmaf_rn(t, d[k], EF.o[k]);
      }
    }
    acc_r[q] = acc_g[q] = acc_b[q] = acc_w[q] = 0.0f;
    n_rec[q] = 0;
  }

  int cur_word = 0;
  bool partial = false;
  uint32_t pbits = 0;
  for (;;) {
    // ---- the next round of views, and their records
    const int nv = collect_views(mask, A.mask_words, S.views, cur_word, partial, pbits);
    if (nv == 0) break;
    if (lane < nv) {
      const ViewRec& VR = A.vrecs[(int64_t)e * A.n_views + S.views[lane]];
      if constexpr (OVAL) {
        float* o = static_cast<WarpSmemOval&>(S).ov[lane];
#pragma unroll
        for (int k = 0; k < 3; ++k) { o[k] = VR.ov_n[k]; o[3 + k] = VR.ov_x[k]; o[6 + k] = VR.ov_y[k]; }
        o[9] = VR.ov_k; o[10] = VR.ov_u0; o[11] = VR.ov_v0;
        o[12] = VR.ov_ru[0]; o[13] = VR.ov_ru[1]; o[14] = VR.ov_rv[0]; o[15] = VR.ov_rv[1];
      } else {
        S.cc[lane] = *reinterpret_cast<const float4*>(VR.cc);
        S.inv_r[lane] = VR.inv_r;
      }
      if constexpr (!SELECT) {  // the disk tests alone need only the disk
        S.tex[lane] = VR.tex;
        int b0 = 0, bn = 0, g0 = 0, gn = 0;
        if (VR.bin_off >= 0) {
          const int lx = tx - VR.btx0, ly = ty - VR.bty0;
          if (lx >= 0 && lx < VR.bntx && ly >= 0 && ly < VR.bnty) {
            const int* offs = A.bin_offsets + VR.bin_off + ly * VR.bntx + lx;
            b0 = offs[0];
            bn = offs[1] - b0;
          }
          g0 = VR.big_base;
          gn = VR.big_count;
        }
        S.bstart[lane] = b0;
        S.bcount[lane] = bn;
        S.gbase[lane] = g0;
        S.gcount[lane] = gn;
#pragma unroll
        for (int k = 0; k < 12; ++k) S.Hm[lane][k] = VR.Hm[k];
      }
    }
    __syncwarp();
    // ---- disk membership of each pixel's sphere crossing, one bit per view
    uint32_t inmask[kPx];
#pragma unroll
    for (int q = 0; q < kPx; ++q) {
      inmask[q] = 0u;
      if (has_p[q]) {
        for (int sl = 0; sl < nv; ++sl) {
          if constexpr (OVAL) {
            if (oval_rho2(static_cast<WarpSmemOval&>(S).ov[sl], ex, ey[q]) < 1.0f) inmask[q] |= 1u << sl;
          } else {
            const float4 cc = S.cc[sl];
            const float dx = __fsub_rn(p[q][0], cc.x), dy = __fsub_rn(p[q][1], cc.y), dz = __fsub_rn(p[q][2], cc.z);
            if (dot3_rn(dx, dy, dz, dx, dy, dz) < cc.w) inmask[q] |= 1u << sl;
          }
        }
      }
    }
    uint32_t wmask = inmask[0];
#pragma unroll
    for (int q = 1; q < kPx; ++q) wmask |= inmask[q];
    wmask = __reduce_or_sync(0xffffffffu, wmask);  // views some pixel of the strip sees
    if constexpr (SELECT) {
      if (lane < nv && ((wmask >> lane) & 1u)) A.visible[(int64_t)e * A.n_views + S.views[lane]] = 1;
      __syncwarp();  // the view table is rewritten by the next round
      continue;
    }
    if (lane < nv && ((wmask >> lane) & 1u)) A.active[(int64_t)e * A.n_views + S.views[lane]] = 1;
    {
      // exclusive prefix of the seen views' entry counts
      const int c = (lane < nv && ((wmask >> lane) & 1u)) ? S.bcount[lane] + S.gcount[lane] : 0;
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      S.off[lane] = incl - c;
      if (lane == 31) S.off[32] = incl;
    }
    __syncwarp();
    const int T = S.off[32];

    int cur = -1;
    // Depth winner per pixel as one key: the bits of 1/z (> 0, so they order as
    // unsigned integers) above 0x7fffffff - id, so the largest key is the
    // nearest fragment and equal depths go to the lower id.  0: none yet.
    uint64_t best_key[kPx];
    int wcount[kPx], next_emit[kPx];
    int n_cover[kPx], min_id[kPx], max_id[kPx];
    uint32_t hash[kPx];
#pragma unroll
    for (int q = 0; q < kPx; ++q) {
      best_key[q] = 0; wcount[q] = 0; next_emit[q] = 0;
      n_cover[q] = 0; min_id[q] = 0x7fffffff; max_id[q] = -1; hash[q] = 0u;
    }
    auto shade_flush = [&]() {
      const int kmax = max(wcount[0], wcount[kPx - 1]);
      for (int k = 0; k < kmax; ++k) {
#pragma unroll
        for (int q = 0; q < kPx; ++q) {
          if (k >= wcount[q]) continue;
          const int sl = S.wslot[k][q][lane];
          const float iz = S.wiz[k][q][lane];
          float w;
          if constexpr (OVAL) {
            // rho^2 < 1 here (the view was kept for this pixel); the weight 1 - rho is a value
            const float r2 = oval_rho2(static_cast<WarpSmemOval&>(S).ov[sl], ex, ey[q]);
            w = fmaxf(0.0f, 1.0f - (r2 > 0.0f ? __fmul_rn(r2, rsqrtf(r2)) : 0.0f));
          } else {
            const float4 cc = S.cc[sl];
            const float dx = __fsub_rn(p[q][0], cc.x), dy = __fsub_rn(p[q][1], cc.y), dz = __fsub_rn(p[q][2], cc.z);
            const float d2 = dot3_rn(dx, dy, dz, dx, dy, dz);
            // the weight is a value, not a decision: fast square root
            const float dist = d2 > 0.0f ? __fmul_rn(d2, rsqrtf(d2)) : 0.0f;
            w = fmaxf(0.0f, __fmaf_rn(-dist, S.inv_r[sl], 1.0f));
          }
          const float* Hm = S.Hm[sl];
          const float hx = fmaf(Hm[0], px, fmaf(Hm[1], py[q], fmaf(Hm[9], iz, Hm[2])));
          const float hy = fmaf(Hm[3], px, fmaf(Hm[4], py[q], fmaf(Hm[10], iz, Hm[5])));
          const float hz = fmaf(Hm[6], px, fmaf(Hm[7], py[q], fmaf(Hm[11], iz, Hm[8])));
          if (hz > 0.0f) {
            const int v = S.views[sl];
            const float rz = __fdividef(1.0f, hz);
            const float scale = (FMT == LF_TEX_FP8E4M3) ? A.views[v].tex_scale : 1.0f;
            const float3 c = bilinear<FMT>(S.tex[sl], A.src_w, A.src_h, __fmul_rn(hx, rz), __fmul_rn(hy, rz),
                                           scale, INSPECT ? A.texel_bits : nullptr, (int64_t)v * tex_per_view);
            acc_r[q] = __fmaf_rn(w, c.x, acc_r[q]);
            acc_g[q] = __fmaf_rn(w, c.y, acc_g[q]);
            acc_b[q] = __fmaf_rn(w, c.z, acc_b[q]);
            acc_w[q] = __fadd_rn(acc_w[q], w);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kPx; ++q) wcount[q] = 0;
    };
    auto emit = [&](int q, int sl, int nc, int win, int mn, int mx, uint32_t h) {
      if (n_rec[q] < A.max_records) {
        lf_frag_record r;
        r.view = S.views[sl];
        r.n_cover = nc;
        r.winner = win;
        r.min_id = nc ? mn : -1;
        r.max_id = nc ? mx : -1;
        r.id_hash = h;
        const int64_t pix = (int64_t)(j0 + dj + q) * E.W + pi;
        A.records[pix * A.max_records + n_rec[q]] = r;
      }
      ++n_rec[q];
    };
    // Close the running view: buffer each pixel's winner; in the inspection
    // form, emit records for it and for seen views before `upto` without triangles.
    auto finalize = [&](int upto) {
      bool full = false;
#pragma unroll
      for (int q = 0; q < kPx; ++q) {
        if (cur >= 0 && ((inmask[q] >> cur) & 1u)) {
          if constexpr (INSPECT) {
            for (int sl = next_emit[q]; sl < cur; ++sl)
              if ((inmask[q] >> sl) & 1u) emit(q, sl, 0, -1, 0, 0, 0u);
            emit(q, cur, n_cover[q], best_key[q] ? 0x7fffffff - (int)(uint32_t)best_key[q] : -1, min_id[q], max_id[q],
                 hash[q]);
            next_emit[q] = cur + 1;
          }
          if (best_key[q]) {
            S.wslot[wcount[q]][q][lane] = (uint8_t)cur;
            S.wiz[wcount[q]][q][lane] = __uint_as_float((uint32_t)(best_key[q] >> 32));
            full |= (++wcount[q] == kWinnerBuf);
          }
        }
        if constexpr (INSPECT) {
          for (int sl = next_emit[q]; sl < upto; ++sl)
            if ((inmask[q] >> sl) & 1u) emit(q, sl, 0, -1, 0, 0, 0u);
          if (upto > next_emit[q]) next_emit[q] = upto;
        }
      }
      if (full) shade_flush();
    };

    // ---- triangles of the seen views from this tile's bins, in view order
    for (int f0 = 0; f0 < T; f0 += 32) {
      const int f = f0 + lane;
      bool pred = false;
      int sl = 0;
      int4 ra, rb, rc;
      int64_t q64[3];
      bool big = false;
      if (f < T) {
        int lo = 0, hi = nv;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (S.off[mid] <= f) lo = mid;
          else hi = mid;
        }
        sl = lo;
        const int k = f - S.off[sl];
        const int idx = k < S.bcount[sl] ? __ldg(A.bin_entries + S.bstart[sl] + k)
                                         : __ldg(A.bin_entries + S.gbase[sl] + (k - S.bcount[sl]));
        const TriRec* tr = A.pool + idx;
        ra = __ldg(reinterpret_cast<const int4*>(tr));       // bbox, x0, x1
        rb = __ldg(reinterpret_cast<const int4*>(tr) + 1);   // x2, y0, y1, y2
        rc = __ldg(reinterpret_cast<const int4*>(tr) + 2);   // ia, ib, ic, id_tl
        const int bx0 = (int16_t)(ra.x & 0xffff), by0 = ra.x >> 16;
        const int bx1 = (int16_t)(ra.y & 0xffff), by1 = ra.y >> 16;
        pred = bx0 <= i0 + TW - 1 && bx1 >= i0 && by0 <= wrow1 && by1 >= wrow0;
        if (pred) {
          const int32_t X[3] = {ra.z, ra.w, rb.x};
          const int32_t Y[3] = {rb.y, rb.z, rb.w};
#pragma unroll
          for (int k2 = 0; k2 < 3; ++k2) {
            const int k1 = (k2 + 1) % 3;
            const int64_t DX = (int64_t)X[k1] - X[k2], DY = (int64_t)Y[k1] - Y[k2];
            const int64_t Ev = DX * (P0y - Y[k2]) - DY * (P0x - X[k2]) + ((rc.w >> k2) & 1) - 1;
            q64[k2] = Ev >> 8;  // floor division by 256
            big |= (DX >= kBigEdge || DX <= -kBigEdge || DY >= kBigEdge || DY <= -kBigEdge);
            // largest value of this edge over the strip's pixel centres; < 0 rejects the strip
            const int64_t emax = q64[k2] + max((int64_t)0, -DY * (TW - 1)) +
                                 max(DX * (int64_t)dj0, DX * (int64_t)(dj0 + ROWS - 1));
            pred &= emax >= 0;
          }
        }
      }
      const uint32_t ballot = __ballot_sync(0xffffffffu, pred);
      const int n_list = __popc(ballot);
      if (pred) {
        const int pos = __popc(ballot & ((1u << lane) - 1u));
        const int32_t X[3] = {ra.z, ra.w, rb.x};
        const int32_t Y[3] = {rb.y, rb.z, rb.w};
        TileTri tt;
        tt.q0 = (int32_t)max(min(q64[0], (int64_t)kQClamp), -(int64_t)kQClamp);
        tt.q1 = (int32_t)max(min(q64[1], (int64_t)kQClamp), -(int64_t)kQClamp);
        tt.q2 = (int32_t)max(min(q64[2], (int64_t)kQClamp), -(int64_t)kQClamp);
        tt.id = (rc.w >> 3) | (big ? (int32_t)0x80000000 : 0);
        tt.a0 = Y[0] - Y[1]; tt.b0 = X[1] - X[0];
        tt.a1 = Y[1] - Y[2]; tt.b1 = X[2] - X[1];
        tt.a2 = Y[2] - Y[0]; tt.b2 = X[0] - X[2];
        tt.ia = __int_as_float(rc.x); tt.ib = __int_as_float(rc.y); tt.ic = __int_as_float(rc.z);
        tt.pad[0] = sl;
        S.tri[pos] = tt;
        if (big) {
          S.q64[pos * 3 + 0] = q64[0];
          S.q64[pos * 3 + 1] = q64[1];
          S.q64[pos * 3 + 2] = q64[2];
        }
      }
      __syncwarp();
      for (int t = 0; t < n_list; ++t) {
        const int4 w0 = *reinterpret_cast<const int4*>(&S.tri[t]);           // q0 q1 q2 id
        const int4 w3 = *(reinterpret_cast<const int4*>(&S.tri[t]) + 3);     // ic, slot, -, -
        const int tsl = w3.y;
        if (tsl != cur) {
          finalize(tsl);
          cur = tsl;
#pragma unroll
          for (int q = 0; q < kPx; ++q) {
            best_key[q] = 0;
            if constexpr (INSPECT) {
              n_cover[q] = 0; min_id[q] = 0x7fffffff; max_id[q] = -1; hash[q] = 0u;
            }
          }
        }
        const int4 w1 = *(reinterpret_cast<const int4*>(&S.tri[t]) + 1);     // a0 b0 a1 b1
        const int4 w2 = *(reinterpret_cast<const int4*>(&S.tri[t]) + 2);     // a2 b2 ia ib
        const int id = w0.w & 0x7fffffff;
        const float ia = __int_as_float(w2.z), ib = __int_as_float(w2.w), ic = __int_as_float(w3.x);
        bool cov[kPx];
        if (w0.w >= 0) {
          int k0 = w0.x + w1.x * di + w1.y * dj;
          int k1 = w0.y + w1.z * di + w1.w * dj;
          int k2 = w0.z + w2.x * di + w2.y * dj;
#pragma unroll
          for (int q = 0; q < kPx; ++q) {
            cov[q] = (k0 | k1 | k2) >= 0;
            k0 += w1.y; k1 += w1.w; k2 += w2.y;
          }
        } else {
          int64_t k0 = S.q64[t * 3 + 0] + (int64_t)w1.x * di + (int64_t)w1.y * dj;
          int64_t k1 = S.q64[t * 3 + 1] + (int64_t)w1.z * di + (int64_t)w1.w * dj;
          int64_t k2 = S.q64[t * 3 + 2] + (int64_t)w2.x * di + (int64_t)w2.y * dj;
#pragma unroll
          for (int q = 0; q < kPx; ++q) {
            cov[q] = (k0 | k1 | k2) >= 0;
            k0 += w1.y; k1 += w1.w; k2 += w2.y;
          }
        }
#pragma unroll
        for (int q = 0; q < kPx; ++q) {
          if (!cov[q] || !((inmask[q] >> tsl) & 1u)) continue;
          if constexpr (INSPECT) {
            ++n_cover[q];
            min_id[q] = min(min_id[q], id);
            max_id[q] = max(max_id[q], id);
            hash[q] ^= mix32((uint32_t)id);
          }
          const float iz = __fmaf_rn(ia, ex, __fmaf_rn(ib, ey[q], ic));
          // nearest wins; equal depths go to the lower id, whatever the visiting order
          if (iz > 0.0f) {
            const uint64_t key = ((uint64_t)__float_as_uint(iz) << 32) | (uint32_t)(0x7fffffff - id);
            if (key > best_key[q]) best_key[q] = key;
          }
        }
      }
      __syncwarp();
    }
    finalize(nv);
    shade_flush();
    __syncwarp();  // the view table is rewritten by the next round
  }
  if constexpr (SELECT) return;
#pragma unroll
  for (int q = 0; q < kPx; ++q) {
    if (!valid[q]) continue;
    const int64_t pix = (int64_t)(j0 + dj + q) * E.W + pi;
    float4 out;
    if (acc_w[q] > 0.0f) {
      const float inv = __frcp_rn(acc_w[q]);
      out = make_float4(__fmul_rn(acc_r[q], inv), __fmul_rn(acc_g[q], inv), __fmul_rn(acc_b[q], inv), 1.0f);
    } else {
      out = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    reinterpret_cast<float4*>(E.out)[pix] = out;
    if constexpr (INSPECT) {
      A.counts[pix] = n_rec[q];
      if (n_rec[q] > A.max_records) atomicOr(A.error_word, kErrRecordOverflow);
    }
  }
}

// Non-persistent: one CTA per tile, warp w takes strip w.  Persistent: every
// warp takes (tile, strip) work items from the device counter by itself.
template <int TW, int TH, int FMT, bool INSPECT, bool PERSISTENT, bool OVAL, bool SELECT = false>
__global__ void __launch_bounds__(TW * TH / kPx, 6) raster_kernel(FrameArgs A) {
  constexpr int WARPS = TW * TH / kPx / 32;
  using Smem = typename std::conditional<OVAL, WarpSmemOval, WarpSmem>::type;
  __shared__ Smem S[WARPS];
  const int warp = threadIdx.x >> 5;
  // Launched early (programmatic dependent launch), the blocks wait here until
  // the set-up grid before this one has completed: everything read below (eye
  // constants, tile masks, view records, bins, the work counter) is written by
  // the kernels of the frame before this one.
  griddep_wait();
  if constexpr (!PERSISTENT) {
    raster_strip<TW, TH, FMT, INSPECT, false, OVAL, SELECT>(A, blockIdx.x, warp, S[warp]);
  } else {
    const int n_items = A.total_tiles * WARPS;
    for (;;) {
      int item = 0;
      if ((threadIdx.x & 31) == 0) item = atomicAdd(A.work_counter, 1);
      item = __shfl_sync(0xffffffffu, item, 0);
      if (item >= n_items) break;
      raster_strip<TW, TH, FMT, INSPECT, true, OVAL, SELECT>(A, item / WARPS, item % WARPS, S[warp]);
    }
  }
}

template <int TW, int TH, int FMT, bool OVAL>
static cudaError_t launch_disk(const FrameArgs& a, bool inspect, bool persistent, int pblocks, cudaStream_t s,
                               bool pdl) {
  const dim3 block(TW * TH / kPx);
  if (inspect) return launch_kernel(raster_kernel<TW, TH, FMT, true, false, OVAL>, dim3(a.total_tiles), block, 0, s, pdl, a);
  if (persistent) return launch_kernel(raster_kernel<TW, TH, FMT, false, true, OVAL>, dim3(pblocks), block, 0, s, pdl, a);
  return launch_kernel(raster_kernel<TW, TH, FMT, false, false, OVAL>, dim3(a.total_tiles), block, 0, s, pdl, a);
}

template <int TW, int TH, int FMT>
static cudaError_t launch_fmt(const FrameArgs& a, bool inspect, bool persistent, int pblocks, cudaStream_t s,
                              bool pdl) {
  if (a.disk_mode == 1) return launch_disk<TW, TH, FMT, true>(a, inspect, persistent, pblocks, s, pdl);
  return launch_disk<TW, TH, FMT, false>(a, inspect, persistent, pblocks, s, pdl);
}

template <int TW, int TH>
static cudaError_t launch_tile(const FrameArgs& a, bool inspect, bool persistent, int pblocks, cudaStream_t s,
                               bool pdl) {
  switch (a.tex_format) {
    case LF_TEX_F32: return launch_fmt<TW, TH, LF_TEX_F32>(a, inspect, persistent, pblocks, s, pdl);
    case LF_TEX_U8: return launch_fmt<TW, TH, LF_TEX_U8>(a, inspect, persistent, pblocks, s, pdl);
    case LF_TEX_BF16: return launch_fmt<TW, TH, LF_TEX_BF16>(a, inspect, persistent, pblocks, s, pdl);
    case LF_TEX_FP8E4M3: return launch_fmt<TW, TH, LF_TEX_FP8E4M3>(a, inspect, persistent, pblocks, s, pdl);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_raster(const FrameArgs& a, bool inspect, bool persistent, int pblocks, cudaStream_t s, bool pdl) {
  if (a.total_tiles <= 0) return cudaSuccess;
  if (a.tile_w == 16 && a.tile_h == 16) return launch_tile<16, 16>(a, inspect, persistent, pblocks, s, pdl);
  if (a.tile_w == 32 && a.tile_h == 8) return launch_tile<32, 8>(a, inspect, persistent, pblocks, s, pdl);
  if (a.tile_w == 8 && a.tile_h == 8) return launch_tile<8, 8>(a, inspect, persistent, pblocks, s, pdl);
  return cudaErrorInvalidValue;
}

template <int TW, int TH, bool OVAL>
static cudaError_t occupancy_disk(int fmt, int* n) {
  switch (fmt) {
    case LF_TEX_F32:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, raster_kernel<TW, TH, LF_TEX_F32, false, true, OVAL>,
                                                           TW * TH / kPx, 0);
    case LF_TEX_U8:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, raster_kernel<TW, TH, LF_TEX_U8, false, true, OVAL>,
                                                           TW * TH / kPx, 0);
    case LF_TEX_BF16:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, raster_kernel<TW, TH, LF_TEX_BF16, false, true, OVAL>,
                                                           TW * TH / kPx, 0);
    default:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          n, raster_kernel<TW, TH, LF_TEX_FP8E4M3, false, true, OVAL>, TW * TH / kPx, 0);
  }
}

template <int TW, int TH>
static cudaError_t occupancy_tile(int fmt, int disk_mode, int* n) {
  return disk_mode == 1 ? occupancy_disk<TW, TH, true>(fmt, n) : occupancy_disk<TW, TH, false>(fmt, n);
}

template <int TW, int TH>
static cudaError_t launch_select_tile(const FrameArgs& a, cudaStream_t s) {
  if (a.disk_mode == 1) raster_kernel<TW, TH, LF_TEX_F32, false, false, true, true><<<a.total_tiles, TW * TH / kPx, 0, s>>>(a);
  else raster_kernel<TW, TH, LF_TEX_F32, false, false, false, true><<<a.total_tiles, TW * TH / kPx, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_select(const FrameArgs& a, cudaStream_t s) {
  if (a.total_tiles <= 0) return cudaSuccess;
  if (a.tile_w == 16 && a.tile_h == 16) return launch_select_tile<16, 16>(a, s);
  if (a.tile_w == 32 && a.tile_h == 8) return launch_select_tile<32, 8>(a, s);
  if (a.tile_w == 8 && a.tile_h == 8) return launch_select_tile<8, 8>(a, s);
  return cudaErrorInvalidValue;
}

// The views each eye draws in a two-level frame (Sec. 7.2): a fine view that it
// selects and whose image is resident; a coarse view that it selects and whose
// disk overlaps a selected fine view whose image is missing.
__global__ void drawn_kernel(FrameArgs A) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x, e = blockIdx.y;
  if (v >= A.n_views) return;
  const uint8_t* vis = A.visible + (int64_t)e * A.n_views;
  bool on = false;
  if (v < A.n_fine) {
    on = vis[v] && A.page_of_view[v] >= 0;
  } else if (vis[v]) {
    const int c = v - A.n_fine;
    for (int k = A.overlap_off[c]; k < A.overlap_off[c + 1] && !on; ++k) {
      const int f = A.overlap_ids[k];
      on = vis[f] && A.page_of_view[f] < 0;
    }
  }
  if (on) atomicOr(A.enable_bits + (int64_t)e * A.mask_words + (v >> 5), 1u << (v & 31));
}

// Only the drawn views stay in the tile masks: one thread per (tile, mask word).
__global__ void enable_masks_kernel(FrameArgs A) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)A.total_tiles * A.mask_words) return;
  const int tile = (int)(idx / A.mask_words), w = (int)(idx % A.mask_words);
  int e = 0;
  for (int lo = 0, hi = A.n_eyes; hi - lo > 1;) {  // the last eye whose first tile is <= tile
    const int mid = (lo + hi) >> 1;
    if (A.eyes[mid].tile_base <= tile) lo = mid;
    else hi = mid;
    e = lo;
  }
  A.tile_masks[idx] &= A.enable_bits[(int64_t)e * A.mask_words + w];
}

cudaError_t launch_drawn(const FrameArgs& a, cudaStream_t s) {
  dim3 grid((a.n_views + 127) / 128, a.n_eyes);
  drawn_kernel<<<grid, 128, 0, s>>>(a);
  const int64_t n = (int64_t)a.total_tiles * a.mask_words;
  if (n > 0) enable_masks_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t raster_occupancy(int tile_w, int tile_h, int fmt, int disk_mode, int* n) {
  if (tile_w == 16 && tile_h == 16) return occupancy_tile<16, 16>(fmt, disk_mode, n);
  if (tile_w == 32 && tile_h == 8) return occupancy_tile<32, 8>(fmt, disk_mode, n);
  return occupancy_tile<8, 8>(fmt, disk_mode, n);
}

}  // namespace lfk
