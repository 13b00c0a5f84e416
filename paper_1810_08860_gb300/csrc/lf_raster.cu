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

#include "lf_internal.h"

namespace lfk {

struct __align__(16) TileTri {
  int32_t q0, q1, q2, id;   // id bit 31: edge deltas too large for the int32 path
  int32_t a0, b0, a1, b1;
  int32_t a2, b2;
  float ia, ib;
  float ic;
  int32_t pad[3];
};
static_assert(sizeof(TileTri) == 64, "TileTri layout");

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
__device__ __forceinline__ float3 texel(const void* tex, int64_t idx, float scale) {
  if constexpr (FMT == LF_TEX_F32) {
    float4 c = __ldg(reinterpret_cast<const float4*>(tex) + idx);
    return make_float3(c.x, c.y, c.z);
  } else if constexpr (FMT == LF_TEX_U8) {
    uchar4 c = __ldg(reinterpret_cast<const uchar4*>(tex) + idx);
    const float k = 1.0f / 255.0f;
    return make_float3(c.x * k, c.y * k, c.z * k);
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
    return make_float3(a.x * scale, a.y * scale, b.x * scale);
  }
}

template <int FMT>
__device__ __forceinline__ float3 bilinear(const void* tex, int64_t base, int W, int H, float u, float v,
                                           float scale, uint32_t* bits) {
  u = fminf(fmaxf(u, -1.0f), (float)W);
  v = fminf(fmaxf(v, -1.0f), (float)H);
  float fu = floorf(u), fv = floorf(v);
  float al = u - fu, be = v - fv;
  int i0 = (int)fu, j0 = (int)fv;
  int i1 = min(i0 + 1, W - 1), j1 = min(j0 + 1, H - 1);
  i0 = max(i0, 0);
  j0 = max(j0, 0);
  i1 = max(i1, 0);
  j1 = max(j1, 0);
  i0 = min(i0, W - 1);
  j0 = min(j0, H - 1);
  int64_t r0 = base + (int64_t)j0 * W, r1 = base + (int64_t)j1 * W;
  float3 c00 = texel<FMT>(tex, r0 + i0, scale), c10 = texel<FMT>(tex, r0 + i1, scale);
  float3 c01 = texel<FMT>(tex, r1 + i0, scale), c11 = texel<FMT>(tex, r1 + i1, scale);
  if (bits) {
    int64_t t[4] = {r0 + i0, r0 + i1, r1 + i0, r1 + i1};
    for (int k = 0; k < 4; ++k) atomicOr(&bits[t[k] >> 5], 1u << (t[k] & 31));
  }
  float w00 = (1.0f - al) * (1.0f - be), w10 = al * (1.0f - be), w01 = (1.0f - al) * be, w11 = al * be;
  return make_float3(w00 * c00.x + w10 * c10.x + w01 * c01.x + w11 * c11.x,
                     w00 * c00.y + w10 * c10.y + w01 * c01.y + w11 * c11.y,
                     w00 * c00.z + w10 * c10.z + w01 * c01.z + w11 * c11.z);
}

template <int TW, int TH, int FMT, bool INSPECT>
__device__ void raster_tile(const FrameArgs& A, int item, TileTri* s_tri, int64_t* s_q64, int* s_warp) {
  constexpr int BLOCK = TW * TH;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int e = 0;
  while (e + 1 < A.n_eyes && A.eyes[e + 1].tile_base <= item) ++e;
  const EyeParams& E = A.eyes[e];
  const int tile = item - E.tile_base;
  const int tx = tile % E.tiles_x, ty = tile / E.tiles_x;
  const int i0 = tx * TW, j0 = ty * TH;
  const int di = tid % TW, dj = tid / TW;
  const int pi = i0 + di, pj = j0 + dj;
  const bool valid = pi < E.W && pj < E.H;

  // Eye ray (Eq. 1) and its crossing of the capture sphere, FP32, fixed order.
  const float fx = __double2float_rn(E.fx), fy = __double2float_rn(E.fy);
  const float cx = __double2float_rn(E.cx), cy = __double2float_rn(E.cy);
  const float ex = __fdiv_rn(__fsub_rn(__fadd_rn((float)pi, 0.5f), cx), fx);
  const float ey = __fdiv_rn(__fsub_rn(__fadd_rn((float)pj, 0.5f), cy), fy);
  float d[3], o[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d[k] = __fmaf_rn(__double2float_rn(E.R[k * 3 + 0]), ex,
                     __fmaf_rn(__double2float_rn(E.R[k * 3 + 1]), ey, __double2float_rn(E.R[k * 3 + 2])));
    o[k] = __double2float_rn(__dsub_rn(E.t[k], A.sphere_c[k]));
  }
  const float R2 = __double2float_rn(__dmul_rn(A.sphere_r, A.sphere_r));
  const float qa = dot3_rn(d[0], d[1], d[2], d[0], d[1], d[2]);
  const float qb = dot3_rn(o[0], o[1], o[2], d[0], d[1], d[2]);
  const float qc = __fsub_rn(dot3_rn(o[0], o[1], o[2], o[0], o[1], o[2]), R2);
  const float disc = __fsub_rn(__fmul_rn(qb, qb), __fmul_rn(qa, qc));
  bool has_p = false;
  float p[3] = {0.f, 0.f, 0.f};
  if (disc >= 0.0f) {
    float t = __fdiv_rn(__fsub_rn(__fsqrt_rn(disc), qb), qa);
    if (t >= 0.0f) {
      has_p = true;
#pragma unroll
      for (int k = 0; k < 3; ++k) p[k] = __fmaf_rn(t, d[k], o[k]);
    }
  }
  const float px = (float)pi + 0.5f, py = (float)pj + 0.5f;
  float acc_r = 0.f, acc_g = 0.f, acc_b = 0.f, acc_w = 0.f;
  int n_rec = 0;
  const int64_t pix = (int64_t)pj * E.W + pi;
  const int64_t P0x = 256 * (int64_t)i0 + 128, P0y = 256 * (int64_t)j0 + 128;
  const int64_t tex_per_view = (int64_t)A.src_w * A.src_h;

  const uint32_t* mask = A.tile_masks + (int64_t)item * A.mask_words;
  for (int wd = 0; wd < A.mask_words; ++wd) {
    uint32_t bits = mask[wd];
    while (bits) {
      const int v = wd * 32 + __ffs(bits) - 1;
      bits &= bits - 1;
      const ViewRec& VR = A.vrecs[(int64_t)e * A.n_views + v];
      const float4 cc = *reinterpret_cast<const float4*>(VR.cc);
      bool inside = false;
      float w = 0.0f;
      if (valid && has_p) {
        float dx = __fsub_rn(p[0], cc.x), dy = __fsub_rn(p[1], cc.y), dz = __fsub_rn(p[2], cc.z);
        float d2 = dot3_rn(dx, dy, dz, dx, dy, dz);
        inside = d2 < cc.w;
        w = fmaxf(0.0f, 1.0f - sqrtf(d2) * VR.inv_r);
      }
      if (!__syncthreads_or(inside)) continue;
      if (tid == 0) A.active[(int64_t)e * A.n_views + v] = 1;

      float best_iz = 0.0f;
      int best_id = -1;
      int n_cover = 0, min_id = 0x7fffffff, max_id = -1;
      uint32_t hash = 0;
      const int seg_base = VR.seg_base, seg_count = VR.seg_count;
      for (int c0 = 0; c0 < seg_count; c0 += BLOCK) {
        const int c = c0 + tid;
        bool pred = false;
        const TriRec* tr = A.pool + seg_base + c;
        if (c < seg_count) {
          const int2 bb = *reinterpret_cast<const int2*>(tr);
          const int bx0 = (int16_t)(bb.x & 0xffff), by0 = bb.x >> 16;
          const int bx1 = (int16_t)(bb.y & 0xffff), by1 = bb.y >> 16;
          pred = bx0 <= i0 + TW - 1 && bx1 >= i0 && by0 <= j0 + TH - 1 && by1 >= j0;
        }
        const uint32_t ballot = __ballot_sync(0xffffffffu, pred);
        if (lane == 0) s_warp[warp] = __popc(ballot);
        __syncthreads();
        int off = 0, n_list = 0;
#pragma unroll
        for (int w2 = 0; w2 < BLOCK / 32; ++w2) {
          int cw = s_warp[w2];
          off += (w2 < warp) ? cw : 0;
          n_list += cw;
        }
        if (pred) {
          const int pos = off + __popc(ballot & ((1u << lane) - 1u));
          const int32_t X[3] = {tr->x[0], tr->x[1], tr->x[2]};
          const int32_t Y[3] = {tr->y[0], tr->y[1], tr->y[2]};
          const int32_t idtl = tr->id_tl;
          TileTri tt;
          bool big = false;
          int64_t q64[3];
          int32_t a[3], b[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int k1 = (k + 1) % 3;
            const int64_t DX = (int64_t)X[k1] - X[k], DY = (int64_t)Y[k1] - Y[k];
            const int64_t Ev = DX * (P0y - Y[k]) - DY * (P0x - X[k]) + ((idtl >> k) & 1) - 1;
            q64[k] = Ev >> 8;  // floor division by 256
            a[k] = (int32_t)(-DY);
            b[k] = (int32_t)DX;
            big |= (DX >= kBigEdge || DX <= -kBigEdge || DY >= kBigEdge || DY <= -kBigEdge);
          }
          tt.q0 = (int32_t)max(min(q64[0], (int64_t)kQClamp), -(int64_t)kQClamp);
          tt.q1 = (int32_t)max(min(q64[1], (int64_t)kQClamp), -(int64_t)kQClamp);
          tt.q2 = (int32_t)max(min(q64[2], (int64_t)kQClamp), -(int64_t)kQClamp);
          tt.id = (idtl >> 3) | (big ? (int32_t)0x80000000 : 0);
          tt.a0 = a[0]; tt.b0 = b[0]; tt.a1 = a[1]; tt.b1 = b[1]; tt.a2 = a[2]; tt.b2 = b[2];
          tt.ia = tr->ia; tt.ib = tr->ib; tt.ic = tr->ic;
          tt.pad[0] = tt.pad[1] = tt.pad[2] = 0;
          s_tri[pos] = tt;
          if (big) {
            s_q64[pos * 3 + 0] = q64[0];
            s_q64[pos * 3 + 1] = q64[1];
            s_q64[pos * 3 + 2] = q64[2];
          }
        }
        __syncthreads();
        for (int t = 0; t < n_list; ++t) {
          const TileTri& T = s_tri[t];
          bool cov;
          if (T.id >= 0) {
            const int k0 = T.q0 + T.a0 * di + T.b0 * dj;
            const int k1 = T.q1 + T.a1 * di + T.b1 * dj;
            const int k2 = T.q2 + T.a2 * di + T.b2 * dj;
            cov = (k0 | k1 | k2) >= 0;
          } else {
            const int64_t k0 = s_q64[t * 3 + 0] + (int64_t)T.a0 * di + (int64_t)T.b0 * dj;
            const int64_t k1 = s_q64[t * 3 + 1] + (int64_t)T.a1 * di + (int64_t)T.b1 * dj;
            const int64_t k2 = s_q64[t * 3 + 2] + (int64_t)T.a2 * di + (int64_t)T.b2 * dj;
            cov = (k0 | k1 | k2) >= 0;
          }
          if (cov) {
            const int id = T.id & 0x7fffffff;
            if constexpr (INSPECT) {
              ++n_cover;
              min_id = min(min_id, id);
              max_id = max(max_id, id);
              hash ^= mix32((uint32_t)id);
            }
            const float iz = __fmaf_rn(T.ia, ex, __fmaf_rn(T.ib, ey, T.ic));
            if (iz > 0.0f && (best_id < 0 || iz > best_iz)) {
              best_iz = iz;
              best_id = id;
            }
          }
        }
        __syncthreads();
      }
      if (inside) {
        if (best_id >= 0) {
          const float* Hm = VR.Hm;
          const float hx = fmaf(Hm[0], px, fmaf(Hm[1], py, fmaf(Hm[9], best_iz, Hm[2])));
          const float hy = fmaf(Hm[3], px, fmaf(Hm[4], py, fmaf(Hm[10], best_iz, Hm[5])));
          const float hz = fmaf(Hm[6], px, fmaf(Hm[7], py, fmaf(Hm[11], best_iz, Hm[8])));
          if (hz > 0.0f) {
            const float rz = 1.0f / hz;
            const float scale = (FMT == LF_TEX_FP8E4M3) ? A.views[v].tex_scale : 1.0f;
            const float3 c = bilinear<FMT>(A.textures, (int64_t)v * tex_per_view, A.src_w, A.src_h, hx * rz,
                                           hy * rz, scale, INSPECT ? A.texel_bits : nullptr);
            acc_r = fmaf(w, c.x, acc_r);
            acc_g = fmaf(w, c.y, acc_g);
            acc_b = fmaf(w, c.z, acc_b);
            acc_w += w;
          }
        }
        if constexpr (INSPECT) {
          if (n_rec < A.max_records) {
            lf_frag_record r;
            r.view = v;
            r.n_cover = n_cover;
            r.winner = best_id;
            r.min_id = n_cover ? min_id : -1;
            r.max_id = max_id;
            r.id_hash = hash;
            A.records[pix * A.max_records + n_rec] = r;
          }
          ++n_rec;
        }
      }
    }
  }
  if (valid) {
    float4 out;
    if (acc_w > 0.0f) {
      const float inv = 1.0f / acc_w;
      out = make_float4(acc_r * inv, acc_g * inv, acc_b * inv, 1.0f);
    } else {
      out = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    reinterpret_cast<float4*>(E.out)[pix] = out;
    if constexpr (INSPECT) {
      A.counts[pix] = n_rec;
      if (n_rec > A.max_records) atomicOr(A.error_word, kErrRecordOverflow);
    }
  }
}

template <int TW, int TH, int FMT, bool INSPECT, bool PERSISTENT>
__global__ void __launch_bounds__(TW * TH) raster_kernel(FrameArgs A) {
  __shared__ TileTri s_tri[TW * TH];
  __shared__ int64_t s_q64[TW * TH * 3];
  __shared__ int s_warp[TW * TH / 32];
  if constexpr (!PERSISTENT) {
    raster_tile<TW, TH, FMT, INSPECT>(A, blockIdx.x, s_tri, s_q64, s_warp);
  } else {
    __shared__ int s_item;
    for (;;) {
      if (threadIdx.x == 0) s_item = atomicAdd(A.work_counter, 1);
      __syncthreads();
      const int item = s_item;
      __syncthreads();
      if (item >= A.total_tiles) break;
      raster_tile<TW, TH, FMT, INSPECT>(A, item, s_tri, s_q64, s_warp);
    }
  }
}

template <int TW, int TH, int FMT>
static cudaError_t launch_fmt(const FrameArgs& a, bool inspect, bool persistent, int pblocks, cudaStream_t s) {
  if (inspect) {
    raster_kernel<TW, TH, FMT, true, false><<<a.total_tiles, TW * TH, 0, s>>>(a);
  } else if (persistent) {
    raster_kernel<TW, TH, FMT, false, true><<<pblocks, TW * TH, 0, s>>>(a);
  } else {
    raster_kernel<TW, TH, FMT, false, false><<<a.total_tiles, TW * TH, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <int TW, int TH>
static cudaError_t launch_tile(const FrameArgs& a, bool inspect, bool persistent, int pblocks, cudaStream_t s) {
  switch (a.tex_format) {
    case LF_TEX_F32: return launch_fmt<TW, TH, LF_TEX_F32>(a, inspect, persistent, pblocks, s);
    case LF_TEX_U8: return launch_fmt<TW, TH, LF_TEX_U8>(a, inspect, persistent, pblocks, s);
    case LF_TEX_BF16: return launch_fmt<TW, TH, LF_TEX_BF16>(a, inspect, persistent, pblocks, s);
    case LF_TEX_FP8E4M3: return launch_fmt<TW, TH, LF_TEX_FP8E4M3>(a, inspect, persistent, pblocks, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_raster(const FrameArgs& a, bool inspect, bool persistent, int pblocks, cudaStream_t s) {
  if (a.total_tiles <= 0) return cudaSuccess;
  if (a.tile_w == 16 && a.tile_h == 16) return launch_tile<16, 16>(a, inspect, persistent, pblocks, s);
  if (a.tile_w == 32 && a.tile_h == 8) return launch_tile<32, 8>(a, inspect, persistent, pblocks, s);
  if (a.tile_w == 8 && a.tile_h == 8) return launch_tile<8, 8>(a, inspect, persistent, pblocks, s);
  return cudaErrorInvalidValue;
}

template <int TW, int TH>
static cudaError_t occupancy_tile(int fmt, int* n) {
  switch (fmt) {
    case LF_TEX_F32:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, raster_kernel<TW, TH, LF_TEX_F32, false, true>, TW * TH, 0);
    case LF_TEX_U8:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, raster_kernel<TW, TH, LF_TEX_U8, false, true>, TW * TH, 0);
    case LF_TEX_BF16:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, raster_kernel<TW, TH, LF_TEX_BF16, false, true>, TW * TH, 0);
    default:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, raster_kernel<TW, TH, LF_TEX_FP8E4M3, false, true>, TW * TH, 0);
  }
}

cudaError_t raster_occupancy(int tile_w, int tile_h, int fmt, int* n) {
  if (tile_w == 16 && tile_h == 16) return occupancy_tile<16, 16>(fmt, n);
  if (tile_w == 32 && tile_h == 8) return occupancy_tile<32, 8>(fmt, n);
  return occupancy_tile<8, 8>(fmt, n);
}

}  // namespace lfk
