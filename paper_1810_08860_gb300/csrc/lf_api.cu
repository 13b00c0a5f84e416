// lf_api.cu - host side of the C ABI declared in include/lf.h: context,
// uploads, per-call parameter staging, kernel sequencing, CUDA-graph replay of
// batched calls, and statistics.  All arithmetic of the rendering method runs
// in the kernels of lf_setup.cu and lf_raster.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lf_internal.h"
#include "lf_launch.h"
#include "lf_prefilter.h"

using namespace lfk;

cudaError_t lfk::ensure_dynamic_smem(const void* kernel, int bytes) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<int, const void*>, int>> done;  // (device, kernel) -> bytes set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& d : done)
    if (d.first.first == dev && d.first.second == kernel) {
      if (d.second >= bytes) return cudaSuccess;
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (e == cudaSuccess) d.second = bytes;
      return e;
    }
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.push_back({{dev, kernel}, bytes});
  return e;
}

namespace {

constexpr int kRing = 4;
constexpr int kHostSlots = LF_HOST_FRAMES_IN_FLIGHT;
constexpr size_t kCounterBlock = 32;  // triangles, error word, work counter, bin offsets, bin entries
constexpr int64_t kDefaultWaitNs = 2000000000;  // 2 s: far beyond any legitimate wait, even under a profiler

struct Buffer {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct lf_ctx {
  int device = 0;
  lf_config cfg{};
  std::string last_error;
  int sm_count = 0;
  // views
  int32_t n_views = 0, src_w = 0, src_h = 0;
  lf_tex_format tex_fmt = LF_TEX_F32;
  int32_t disk_mode = 0;  // 0: round disks on the capture sphere; 1: ovals (lf_set_disk_ovals)
  double sphere_c[3] = {0, 0, 0};
  double sphere_r = 0;
  Buffer views, tex;
  std::vector<ViewStatic> views_host;  // poses, intrinsics and disks as loaded
  // meshes
  int32_t G = 0;
  lf_mesh_format mesh_fmt = LF_MESH_F32_DEPTH;
  Buffer depth, tab_a, tab_b;
  // per-call scratch
  Buffer eyes, eyes_f, vrecs, masks, pool, bin_offsets, bin_entries, small, active;
  EyeParams* pinned = nullptr;  // kRing slots of max_eyes
  cudaEvent_t ring_ev[kRing] = {};
  int ring_next = 0;
  cudaStream_t work_stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  // last call
  cudaStream_t last_stream = nullptr;
  int32_t last_eyes = 0;
  int32_t last_tiles = 0;
  bool has_call = false;
  // batch graph
  cudaGraphExec_t graph = nullptr;
  std::vector<int64_t> graph_sig;
  int persistent_blocks = 0;
  // per-kernel timing of the last call (lf_config.timing)
  cudaEvent_t tev[4] = {};
  bool timed_call = false;
  // learned refinement
  struct Refine {
    bool loaded = false;
    int32_t step = 0;
    lf_refine_kernel kernel = LF_REFINE_MMA_LAYERS;
    Buffer state;     // FP32 params, grad, adam m, adam v (kRefineParams each)
    Buffer packed;    // BF16 operand layouts
    Buffer scal;      // loss (f32), valid count (i32)
    Buffer a1, a2, gz2, gr, partial, frame;
  } rf;
  // frames delivered to host memory (lf_render_host): frame k uses slot k % kHostSlots
  struct HostPipe {
    cudaStream_t copy = nullptr;
    cudaEvent_t rendered[kHostSlots] = {}, copied[kHostSlots] = {};
    Buffer image[kHostSlots];  // device images of the slot's frame
    Buffer counters;           // one counter block per slot
    uint32_t* err = nullptr;   // pinned: the error word of each slot's frame
    int64_t issued = 0, delivered = 0;
    uint32_t err_acc = 0;      // error bits of the frames delivered since the last lf_host_wait
  } hp;
  // prefilter scratch (lf_prefilter)
  struct Prefilter {
    Buffer renders, params, err;
  } pf;
  // two-level progressive rendering (lf_set_levels): views [0, n_fine) are the
  // streamed fine level, whose images live in pool pages; the rest the coarse level
  struct Levels {
    int32_t n_fine = 0, n_pages = 0;
    Buffer pool, table, page_of_view, overlap_off, overlap_ids, enable, visible, stage;
    std::vector<int32_t> view_page, page_view;  // host mirrors of the page table
    std::vector<const void*> table_host;        // host mirror of the texture table
  } lv;
};

namespace {

lf_status fail(lf_ctx* c, lf_status s, const char* what) {
  if (c) c->last_error = what;
  return s;
}

lf_status cuda_fail(lf_ctx* c, cudaError_t e, const char* what) {
  if (c) {
    c->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  }
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? LF_ERR_OOM : LF_ERR_CUDA;
}

#define LF_CUDA(ctx, call)                                        \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);   \
  } while (0)

void release(Buffer& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

cudaError_t ensure(Buffer& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return cudaSuccess;
  release(b);
  size_t want = std::max<size_t>(bytes, 256);
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e == cudaSuccess) b.bytes = want;
  return e;
}

bool valid_tile(int w, int h) { return (w == 16 && h == 16) || (w == 32 && h == 8) || (w == 8 && h == 8); }

struct Layout {
  int32_t total_tiles = 0;
  std::vector<EyeParams> eyes;
};

// RGBA images are read and written as 16-byte texels.
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

lf_status make_layout(lf_ctx* c, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                      float* const* out, Layout& L) {
  if (n_eyes < 1 || n_eyes > c->cfg.max_eyes) return fail(c, LF_ERR_INVALID_ARG, "n_eyes out of range");
  if (!eyes || !intr || !out) return fail(c, LF_ERR_INVALID_ARG, "null argument");
  L.eyes.resize(n_eyes);
  int64_t base = 0;
  for (int e = 0; e < n_eyes; ++e) {
    const lf_intrinsics& K = intr[e];
    if (K.width < 1 || K.height < 1 || K.width > 32767 || K.height > 32767)
      return fail(c, LF_ERR_INVALID_ARG, "eye size out of range");
    if (!(K.fx > 0) || !(K.fy > 0)) return fail(c, LF_ERR_INVALID_ARG, "focal length must be positive");
    if (!out[e]) return fail(c, LF_ERR_INVALID_ARG, "null output pointer");
    if (!aligned16(out[e])) return fail(c, LF_ERR_INVALID_ARG, "output images must be 16-byte aligned (RGBA texels)");
    EyeParams& P = L.eyes[e];
    std::memset(&P, 0, sizeof(P));
    std::memcpy(P.R, eyes[e].R, sizeof(P.R));
    std::memcpy(P.t, eyes[e].t, sizeof(P.t));
    P.fx = K.fx; P.fy = K.fy; P.cx = K.cx; P.cy = K.cy;
    P.W = K.width; P.H = K.height;
    P.tiles_x = (K.width + c->cfg.tile_w - 1) / c->cfg.tile_w;
    P.tiles_y = (K.height + c->cfg.tile_h - 1) / c->cfg.tile_h;
    P.tile_base = (int32_t)base;
    P.out = out[e];
    base += (int64_t)P.tiles_x * P.tiles_y;
    if (base > (int64_t)1 << 30) return fail(c, LF_ERR_INVALID_ARG, "too many tiles");
  }
  L.total_tiles = (int32_t)base;
  return LF_OK;
}

int mask_words(const lf_ctx* c) { return (c->n_views + 31) / 32; }

// Bin offsets take 2 ints per footprint tile per (eye, view); bin entries one
// per (triangle, tile) pair, typically about four per set-up triangle.  Both
// also scale with the screen tiles of the call: a tile lies in the footprints
// of about six views on the rig workloads and gathers 10-20 entries, more
// with small tiles, so 24 offsets and 32 entries per tile leave headroom.
int64_t bin_offsets_capacity(const lf_ctx* c, int64_t total_tiles) {
  return std::max(c->cfg.tri_capacity / 2, 24 * total_tiles) + 65536;
}
int64_t bin_entries_capacity(const lf_ctx* c, int64_t total_tiles) {
  return std::max(c->cfg.tri_capacity * 4, 32 * total_tiles);
}

lf_status ensure_scratch(lf_ctx* c, int32_t n_eyes, int32_t total_tiles) {
  LF_CUDA(c, ensure(c->eyes, sizeof(EyeParams) * (size_t)c->cfg.max_eyes));
  LF_CUDA(c, ensure(c->eyes_f, sizeof(EyeFloat) * (size_t)c->cfg.max_eyes));
  LF_CUDA(c, ensure(c->vrecs, sizeof(ViewRec) * (size_t)n_eyes * c->n_views));
  LF_CUDA(c, ensure(c->masks, sizeof(uint32_t) * (size_t)total_tiles * mask_words(c)));
  LF_CUDA(c, ensure(c->active, (size_t)n_eyes * c->n_views));
  LF_CUDA(c, ensure(c->small, 64));
  int64_t cap = c->cfg.tri_capacity;
  LF_CUDA(c, ensure(c->pool, sizeof(TriRec) * (size_t)cap));
  LF_CUDA(c, ensure(c->bin_offsets, sizeof(int32_t) * (size_t)bin_offsets_capacity(c, total_tiles)));
  LF_CUDA(c, ensure(c->bin_entries, sizeof(int32_t) * (size_t)bin_entries_capacity(c, total_tiles)));
  if (c->lv.n_fine > 0) {
    LF_CUDA(c, ensure(c->lv.enable, sizeof(uint32_t) * (size_t)n_eyes * mask_words(c)));
    LF_CUDA(c, ensure(c->lv.visible, (size_t)n_eyes * c->n_views));
  }
  return LF_OK;
}

// Copy the eye parameters through a pinned ring slot (the slot is reused only
// after the copy that read it has completed).
lf_status stage_eyes(lf_ctx* c, const Layout& L, cudaStream_t s) {
  int slot = c->ring_next;
  c->ring_next = (c->ring_next + 1) % kRing;
  LF_CUDA(c, cudaEventSynchronize(c->ring_ev[slot]));
  EyeParams* dst = c->pinned + (size_t)slot * c->cfg.max_eyes;
  std::memcpy(dst, L.eyes.data(), sizeof(EyeParams) * L.eyes.size());
  LF_CUDA(c, cudaMemcpyAsync(c->eyes.p, dst, sizeof(EyeParams) * L.eyes.size(), cudaMemcpyHostToDevice, s));
  LF_CUDA(c, cudaEventRecord(c->ring_ev[slot], s));
  return LF_OK;
}

// Point a frame's counters at a 32-byte block: triangles (8 B), error word,
// work counter, bin offsets (8 B), bin entries (8 B).  enqueue_frame zeroes it.
void use_counters(FrameArgs& a, unsigned char* block) {
  a.pool_counter = reinterpret_cast<unsigned long long*>(block);
  a.error_word = reinterpret_cast<uint32_t*>(block + 8);
  a.work_counter = reinterpret_cast<int32_t*>(block + 12);
  a.bin_offsets_counter = reinterpret_cast<unsigned long long*>(block + 16);
  a.bin_entries_counter = reinterpret_cast<unsigned long long*>(block + 24);
}

FrameArgs frame_args(lf_ctx* c, const Layout& L) {
  FrameArgs a;
  std::memset(&a, 0, sizeof(a));
  a.eyes = static_cast<const EyeParams*>(c->eyes.p);
  a.n_eyes = (int32_t)L.eyes.size();
  a.n_views = c->n_views;
  a.src_w = c->src_w;
  a.src_h = c->src_h;
  a.G = c->G;
  a.mask_words = mask_words(c);
  a.tex_format = c->tex_fmt;
  a.mesh_format = c->mesh_fmt;
  a.disk_mode = c->disk_mode;
  a.z_near = c->cfg.z_near;
  for (int k = 0; k < 3; ++k) a.sphere_c[k] = c->sphere_c[k];
  a.sphere_r = c->sphere_r;
  a.views = static_cast<const ViewStatic*>(c->views.p);
  a.textures = c->tex.p;
  a.depth = c->depth.p;
  a.tables.a = static_cast<const float*>(c->tab_a.p);
  a.tables.b = static_cast<const float*>(c->tab_b.p);
  a.vrecs = static_cast<ViewRec*>(c->vrecs.p);
  a.tile_masks = static_cast<uint32_t*>(c->masks.p);
  a.eyes_f = static_cast<EyeFloat*>(c->eyes_f.p);
  a.pool = static_cast<TriRec*>(c->pool.p);
  a.pool_capacity = c->cfg.tri_capacity;
  a.bin_offsets = static_cast<int32_t*>(c->bin_offsets.p);
  a.bin_offsets_capacity = bin_offsets_capacity(c, L.total_tiles);
  a.bin_entries = static_cast<int32_t*>(c->bin_entries.p);
  a.bin_entries_capacity = bin_entries_capacity(c, L.total_tiles);
  a.bin_max_tiles = 1 << 30;  // bin every triangle into every footprint tile its box covers
  use_counters(a, static_cast<unsigned char*>(c->small.p));
  a.active = static_cast<uint8_t*>(c->active.p);
  a.total_tiles = L.total_tiles;
  a.tile_w = c->cfg.tile_w;
  a.tile_h = c->cfg.tile_h;
  if (c->lv.n_fine > 0) {
    a.tex_table = static_cast<const void* const*>(c->lv.table.p);
    a.enable_bits = static_cast<uint32_t*>(c->lv.enable.p);
    a.visible = static_cast<uint8_t*>(c->lv.visible.p);
    a.page_of_view = static_cast<const int32_t*>(c->lv.page_of_view.p);
    a.overlap_off = static_cast<const int32_t*>(c->lv.overlap_off.p);
    a.overlap_ids = static_cast<const int32_t*>(c->lv.overlap_ids.p);
    a.n_fine = c->lv.n_fine;
  }
  return a;
}

// The per-call device work: clear the tile masks, set up views, set up and bin
// triangles, raster.  The view set-up zeroes the counter block and the active
// flags.  Without timing events between them (and outside graph capture: the
// persistent raster), the triangle set-up and the raster are launched as
// programmatic dependents of the kernel before them, so each grid's launch
// overlaps the end of the previous one; each waits for its predecessor's
// completion before it reads anything.  `timed` = false records no timing
// events and leaves what lf_get_stats reports (the last lf_render-style call)
// untouched.
lf_status enqueue_frame(lf_ctx* c, const FrameArgs& a, bool inspect, bool persistent, cudaStream_t s,
                        bool timed = true) {
  const bool t = timed && c->cfg.timing != 0;
  const bool pdl = !t && !persistent;
  LF_CUDA(c, cudaMemsetAsync(a.tile_masks, 0, sizeof(uint32_t) * (size_t)a.total_tiles * a.mask_words, s));
  if (a.n_fine > 0) {
    LF_CUDA(c, cudaMemsetAsync(a.visible, 0, (size_t)a.n_eyes * a.n_views, s));
    LF_CUDA(c, cudaMemsetAsync(a.enable_bits, 0, sizeof(uint32_t) * (size_t)a.n_eyes * a.mask_words, s));
  }
  if (t) LF_CUDA(c, cudaEventRecord(c->tev[0], s));
  LF_CUDA(c, launch_view_setup(a, s));
  if (a.n_fine > 0) {
    // two-level frame (Sec. 7.2): which views each eye selects, then which it draws
    LF_CUDA(c, launch_select(a, s));
    LF_CUDA(c, launch_drawn(a, s));
  }
  if (t) LF_CUDA(c, cudaEventRecord(c->tev[1], s));
  LF_CUDA(c, launch_tri_setup(a, s, pdl));
  if (t) LF_CUDA(c, cudaEventRecord(c->tev[2], s));
  // the persistent grid never exceeds the call's work items (tiles x strips >= tiles)
  const int blocks = std::min(c->persistent_blocks, std::max(1, a.total_tiles));
  LF_CUDA(c, launch_raster(a, inspect, persistent, blocks, s, pdl));
  if (t) LF_CUDA(c, cudaEventRecord(c->tev[3], s));
  if (timed) c->timed_call = t;
  return LF_OK;
}

// The persistent raster grid of lf_render_batch before any tuning: the
// occupancy limit of CTAs per SM times the SM count.
lf_status ensure_persistent_blocks(lf_ctx* c) {
  if (c->persistent_blocks > 0) return LF_OK;
  int per_sm = 0;
  LF_CUDA(c, raster_occupancy(c->cfg.tile_w, c->cfg.tile_h, c->tex_fmt, c->disk_mode, &per_sm));
  c->persistent_blocks = std::max(1, per_sm) * c->sm_count;
  return LF_OK;
}

// Before a load replaces views, meshes or refiner weights: wait until no
// earlier work of any call can still read them.  Renders, refinements and
// host-delivered frames run on caller streams the context does not keep, so
// the whole device is synchronised (loads are rare and block anyway).
lf_status quiesce(lf_ctx* c) {
  LF_CUDA(c, cudaSetDevice(c->device));
  LF_CUDA(c, cudaDeviceSynchronize());
  return LF_OK;
}

lf_status check_ready(lf_ctx* c) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (c->n_views <= 0) return fail(c, LF_ERR_STATE, "views not loaded");
  if (c->G <= 0) return fail(c, LF_ERR_STATE, "meshes not built");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  return LF_OK;
}

}  // namespace

extern "C" {

lf_status lf_tune_batch(lf_ctx* c, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                        float* const* out_rgba, int32_t replays, void* stream, lf_tuning* out) {
  lf_status st = check_ready(c);
  if (st != LF_OK) return st;
  if (!out || replays < 1 || replays > 1000) return fail(c, LF_ERR_INVALID_ARG, "bad tuning arguments");
  std::memset(out, 0, sizeof(*out));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LF_CUDA(c, cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(c, ce, "cudaEventCreate"); }
  const int tiles[3][2] = {{16, 16}, {32, 8}, {8, 8}};
  const lf_config saved = c->cfg;
  const int saved_blocks = c->persistent_blocks;
  float best = -1.0f;
  int best_k = -1;
  for (int ti = 0; ti < 3 && st == LF_OK; ++ti) {
    int per_sm = 0;
    cudaError_t e = raster_occupancy(tiles[ti][0], tiles[ti][1], c->tex_fmt, c->disk_mode, &per_sm);
    if (e != cudaSuccess) { st = cuda_fail(c, e, "raster_occupancy"); break; }
    per_sm = std::max(1, per_sm);
    const int cand[4] = {1, 2, 4, per_sm};
    for (int ci = 0; ci < 4 && st == LF_OK && out->n_tried < 16; ++ci) {
      const int bps = cand[ci];
      if (bps > per_sm || (ci < 3 && bps == per_sm)) continue;  // each block count once
      c->cfg.tile_w = tiles[ti][0];
      c->cfg.tile_h = tiles[ti][1];
      c->persistent_blocks = bps * c->sm_count;
      // the first call captures this layout's graph; then time `replays` replays
      if ((st = lf_render_batch(c, n_eyes, eyes, intr, out_rgba, stream)) != LF_OK) break;
      if ((e = cudaEventRecord(e0, s)) != cudaSuccess) { st = cuda_fail(c, e, "cudaEventRecord"); break; }
      for (int r = 0; r < replays && st == LF_OK; ++r) st = lf_render_batch(c, n_eyes, eyes, intr, out_rgba, stream);
      if (st != LF_OK) break;
      if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
        st = cuda_fail(c, e, "timing");
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= (float)replays;
      // a replay that overflowed its scratch skipped work: it is not a candidate
      uint32_t err = 0;
      if ((e = cudaMemcpy(&err, static_cast<unsigned char*>(c->small.p) + 8, 4, cudaMemcpyDeviceToHost)) !=
          cudaSuccess) {
        st = cuda_fail(c, e, "cudaMemcpy");
        break;
      }
      const bool overflow = (err & kErrPoolOverflow) != 0;
      const int k = out->n_tried++;
      out->tried_tile_w[k] = tiles[ti][0];
      out->tried_tile_h[k] = tiles[ti][1];
      out->tried_blocks[k] = bps;
      out->tried_ms[k] = overflow ? -1.0f : ms;
      if (!overflow && (best < 0.0f || ms < best)) { best = ms; best_k = k; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LF_OK || best_k < 0) {
    c->cfg = saved;
    c->persistent_blocks = saved_blocks;
    return st != LF_OK ? st : fail(c, LF_ERR_CAPACITY, "every configuration overflowed its scratch");
  }
  c->cfg.tile_w = out->tile_w = out->tried_tile_w[best_k];
  c->cfg.tile_h = out->tile_h = out->tried_tile_h[best_k];
  out->blocks_per_sm = out->tried_blocks[best_k];
  c->persistent_blocks = out->blocks_per_sm * c->sm_count;
  out->ms = best;
  // leave the chosen layout's graph captured (and the outputs rendered with it)
  return lf_render_batch(c, n_eyes, eyes, intr, out_rgba, stream);
}

void lf_config_default(lf_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->tile_w = 16;
  cfg->tile_h = 16;
  cfg->max_eyes = 2;
  cfg->tri_capacity = (int64_t)8 << 20;
  cfg->z_near = 0.1f;
  cfg->wait_limit = kDefaultWaitNs;
}

const char* lf_status_string(lf_status s) {
  switch (s) {
    case LF_OK: return "LF_OK";
    case LF_ERR_INVALID_ARG: return "LF_ERR_INVALID_ARG";
    case LF_ERR_CUDA: return "LF_ERR_CUDA";
    case LF_ERR_OOM: return "LF_ERR_OOM";
    case LF_ERR_STATE: return "LF_ERR_STATE";
    case LF_ERR_TIMEOUT: return "LF_ERR_TIMEOUT";
    case LF_ERR_UNSUPPORTED: return "LF_ERR_UNSUPPORTED";
    case LF_ERR_CAPACITY: return "LF_ERR_CAPACITY";
  }
  return "LF_ERR_UNKNOWN";
}

const char* lf_last_error(const lf_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

lf_status lf_set_wait_limit(lf_ctx* c, int64_t wait_ns) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (wait_ns < 0) return fail(c, LF_ERR_INVALID_ARG, "wait limit must be >= 0");
  c->cfg.wait_limit = wait_ns ? wait_ns : kDefaultWaitNs;
  return LF_OK;
}

lf_status lf_set_timing(lf_ctx* c, int32_t on) {
  if (!c || (on != 0 && on != 1)) return LF_ERR_INVALID_ARG;
  c->cfg.timing = on;
  return LF_OK;
}

lf_status lf_create(int32_t device, const lf_config* cfg, lf_ctx** out) {
  if (!out) return LF_ERR_INVALID_ARG;
  *out = nullptr;
  lf_config c;
  lf_config_default(&c);
  if (cfg) {
    if (cfg->tile_w || cfg->tile_h) { c.tile_w = cfg->tile_w; c.tile_h = cfg->tile_h; }
    if (cfg->max_eyes) c.max_eyes = cfg->max_eyes;
    if (cfg->tri_capacity) c.tri_capacity = cfg->tri_capacity;
    if (cfg->z_near != 0.0f) c.z_near = cfg->z_near;
    if (cfg->wait_limit) c.wait_limit = cfg->wait_limit;
    c.timing = cfg->timing ? 1 : 0;
  }
  if (!valid_tile(c.tile_w, c.tile_h) || c.max_eyes < 1 || c.max_eyes > 128 || c.tri_capacity < 1 || c.wait_limit < 1 ||
      c.tri_capacity > ((int64_t)1 << 31) || !(c.z_near > 0.0f))
    return LF_ERR_INVALID_ARG;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess) { cudaGetLastError(); return LF_ERR_CUDA; }
  if (device < 0 || device >= n_dev) return LF_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return LF_ERR_CUDA; }
  lf_ctx* ctx = new (std::nothrow) lf_ctx();
  if (!ctx) return LF_ERR_OOM;
  ctx->device = device;
  ctx->cfg = c;
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  bool ok = cudaMallocHost((void**)&ctx->pinned, sizeof(EyeParams) * (size_t)c.max_eyes * kRing) == cudaSuccess;
  for (int k = 0; ok && k < kRing; ++k) ok = cudaEventCreateWithFlags(&ctx->ring_ev[k], cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < 4; ++k) ok = cudaEventCreate(&ctx->tev[k]) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&ctx->work_stream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lf_destroy(ctx);
    return LF_ERR_CUDA;
  }
  *out = ctx;
  return LF_OK;
}

void lf_destroy(lf_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->has_call && ctx->last_stream) cudaStreamSynchronize(ctx->last_stream);
  cudaDeviceSynchronize();
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  for (Buffer* b : {&ctx->views, &ctx->tex, &ctx->depth, &ctx->tab_a, &ctx->tab_b, &ctx->eyes, &ctx->eyes_f,
                    &ctx->vrecs, &ctx->masks, &ctx->pool, &ctx->bin_offsets, &ctx->bin_entries, &ctx->small,
                    &ctx->active})
    release(*b);
  for (int k = 0; k < kRing; ++k)
    if (ctx->ring_ev[k]) cudaEventDestroy(ctx->ring_ev[k]);
  for (int k = 0; k < 4; ++k)
    if (ctx->tev[k]) cudaEventDestroy(ctx->tev[k]);
  for (Buffer* b : {&ctx->rf.state, &ctx->rf.packed, &ctx->rf.scal, &ctx->rf.a1, &ctx->rf.a2, &ctx->rf.gz2,
                    &ctx->rf.gr, &ctx->rf.partial, &ctx->rf.frame})
    release(*b);
  for (int k = 0; k < kHostSlots; ++k) {
    release(ctx->hp.image[k]);
    if (ctx->hp.rendered[k]) cudaEventDestroy(ctx->hp.rendered[k]);
    if (ctx->hp.copied[k]) cudaEventDestroy(ctx->hp.copied[k]);
  }
  release(ctx->hp.counters);
  for (Buffer* b : {&ctx->pf.renders, &ctx->pf.params, &ctx->pf.err}) release(*b);
  for (Buffer* b : {&ctx->lv.pool, &ctx->lv.table, &ctx->lv.page_of_view, &ctx->lv.overlap_off, &ctx->lv.overlap_ids,
                    &ctx->lv.enable, &ctx->lv.visible, &ctx->lv.stage})
    release(*b);
  if (ctx->hp.err) cudaFreeHost(ctx->hp.err);
  if (ctx->hp.copy) cudaStreamDestroy(ctx->hp.copy);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->work_stream) cudaStreamDestroy(ctx->work_stream);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  cudaGetLastError();
  delete ctx;
}

lf_status lf_load_views(lf_ctx* c, int32_t n_views, const lf_pose* poses, const lf_intrinsics* intr,
                        const uint8_t* const* rgba8, const float* disk_c, const float* disk_r,
                        const double sphere_c[3], double sphere_r, lf_tex_format fmt) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (n_views < 1 || n_views > 65536 || !poses || !intr || !rgba8 || !disk_r || !sphere_c)
    return fail(c, LF_ERR_INVALID_ARG, "bad view arguments");
  if (!(sphere_r > 0)) return fail(c, LF_ERR_INVALID_ARG, "sphere radius must be positive");
  if (fmt < LF_TEX_F32 || fmt > LF_TEX_FP8E4M3) return fail(c, LF_ERR_INVALID_ARG, "bad texture format");
  const int W = intr[0].width, H = intr[0].height;
  if (W < 2 || H < 2 || W > 16384 || H > 16384) return fail(c, LF_ERR_INVALID_ARG, "bad source size");
  std::vector<ViewStatic> vs(n_views);
  for (int v = 0; v < n_views; ++v) {
    if (intr[v].width != W || intr[v].height != H)
      return fail(c, LF_ERR_UNSUPPORTED, "all views must share one image size");
    if (!(intr[v].fx > 0) || !(intr[v].fy > 0)) return fail(c, LF_ERR_INVALID_ARG, "bad view focal length");
    if (!rgba8[v]) return fail(c, LF_ERR_INVALID_ARG, "null image pointer");
    if (!(disk_r[v] > 0.0f)) return fail(c, LF_ERR_INVALID_ARG, "disk radius must be positive");
    ViewStatic& V = vs[v];
    std::memset(&V, 0, sizeof(V));
    std::memcpy(V.R, poses[v].R, sizeof(V.R));
    std::memcpy(V.t, poses[v].t, sizeof(V.t));
    V.fx = intr[v].fx; V.fy = intr[v].fy; V.cx = intr[v].cx; V.cy = intr[v].cy;
    for (int k = 0; k < 3; ++k) V.disk_c[k] = disk_c ? disk_c[v * 3 + k] : (float)poses[v].t[k];
    V.disk_r = disk_r[v];
    V.tex_scale = 1.0f;
  }
  lf_status st = quiesce(c);
  if (st != LF_OK) return st;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; c->graph_sig.clear(); }
  c->n_views = 0;
  c->G = 0;
  release(c->depth); release(c->tab_a); release(c->tab_b);
  // one level again
  for (Buffer* b : {&c->lv.pool, &c->lv.table, &c->lv.page_of_view, &c->lv.overlap_off, &c->lv.overlap_ids,
                    &c->lv.enable, &c->lv.visible, &c->lv.stage})
    release(*b);
  c->lv.n_fine = c->lv.n_pages = 0;
  c->lv.view_page.clear();
  c->lv.page_view.clear();
  c->lv.table_host.clear();
  cudaStream_t s = c->work_stream;
  LF_CUDA(c, ensure(c->views, sizeof(ViewStatic) * (size_t)n_views));
  LF_CUDA(c, cudaMemcpyAsync(c->views.p, vs.data(), sizeof(ViewStatic) * (size_t)n_views, cudaMemcpyHostToDevice, s));
  const int64_t per_view = (int64_t)W * H;
  const size_t texel_bytes = fmt == LF_TEX_F32 ? 16 : fmt == LF_TEX_BF16 ? 8 : 4;
  release(c->tex);
  LF_CUDA(c, ensure(c->tex, texel_bytes * (size_t)per_view * n_views));
  // FP8 stores each view's texels divided by a per-view scale (max value / 448).
  Buffer scale;
  if (fmt == LF_TEX_FP8E4M3) {
    LF_CUDA(c, ensure(scale, sizeof(float) * (size_t)n_views));
  }
  // Upload in chunks through a device staging buffer of RGBA8.
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(n_views, ((int64_t)256 << 20) / (per_view * 4)));
  Buffer stage;
  if (fmt != LF_TEX_U8) LF_CUDA(c, ensure(stage, (size_t)chunk * per_view * 4));
  for (int v0 = 0; v0 < n_views; v0 += chunk) {
    int nv = std::min(chunk, n_views - v0);
    uint8_t* dst = fmt == LF_TEX_U8 ? static_cast<uint8_t*>(c->tex.p) + (size_t)v0 * per_view * 4
                                    : static_cast<uint8_t*>(stage.p);
    for (int k = 0; k < nv; ++k)
      LF_CUDA(c, cudaMemcpyAsync(dst + (size_t)k * per_view * 4, rgba8[v0 + k], (size_t)per_view * 4,
                                 cudaMemcpyHostToDevice, s));
    if (fmt != LF_TEX_U8) {
      void* tdst = static_cast<char*>(c->tex.p) + (size_t)v0 * per_view * texel_bytes;
      if (fmt == LF_TEX_FP8E4M3) {
        LF_CUDA(c, launch_view_scale(static_cast<const uint8_t*>(stage.p), nv, per_view,
                                     static_cast<float*>(scale.p) + v0, static_cast<ViewStatic*>(c->views.p) + v0, s));
      }
      LF_CUDA(c, launch_convert_textures(static_cast<const uint8_t*>(stage.p), tdst, (int64_t)nv * per_view, fmt,
                                         fmt == LF_TEX_FP8E4M3 ? static_cast<float*>(scale.p) + v0 : nullptr,
                                         per_view, s));
    }
    // the staging buffer is reused by the next chunk: wait for this one
    LF_CUDA(c, cudaStreamSynchronize(s));
  }
  release(stage);
  release(scale);
  c->n_views = n_views;
  c->views_host = std::move(vs);
  c->disk_mode = 0;
  c->persistent_blocks = 0;  // the raster's occupancy depends on the texture format
  c->src_w = W;
  c->src_h = H;
  c->tex_fmt = fmt;
  for (int k = 0; k < 3; ++k) c->sphere_c[k] = sphere_c[k];
  c->sphere_r = sphere_r;
  return LF_OK;
}

lf_status lf_set_disk_ovals(lf_ctx* c, const float* extents) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (c->n_views <= 0) return fail(c, LF_ERR_STATE, "views not loaded");
  if (extents)
    for (int64_t i = 0; i < (int64_t)c->n_views * 4; ++i)
      if (!(extents[i] > 0.0f) || extents[i] > 1e30f) return fail(c, LF_ERR_INVALID_ARG, "oval extents must be > 0");
  lf_status st = quiesce(c);  // renders in flight read the disks
  if (st != LF_OK) return st;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; c->graph_sig.clear(); }
  if (extents) {
    for (int v = 0; v < c->n_views; ++v)
      for (int k = 0; k < 4; ++k) c->views_host[v].disk_ext[k] = extents[v * 4 + k];
    // only the extent fields: the device records also hold values computed there
    LF_CUDA(c, cudaMemcpy2D(static_cast<char*>(c->views.p) + offsetof(ViewStatic, disk_ext), sizeof(ViewStatic),
                            extents, 4 * sizeof(float), 4 * sizeof(float), (size_t)c->n_views,
                            cudaMemcpyHostToDevice));
  }
  c->disk_mode = extents ? 1 : 0;
  c->persistent_blocks = 0;  // the oval raster holds more shared memory per block
  return LF_OK;
}

lf_status lf_build_view_meshes(lf_ctx* c, int32_t grid_n, const float* depth, lf_mesh_format fmt) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (c->n_views <= 0) return fail(c, LF_ERR_STATE, "views not loaded");
  if (grid_n < 2 || grid_n > kMaxGridForSetup || !depth) return fail(c, LF_ERR_INVALID_ARG, "bad mesh arguments");
  if (fmt != LF_MESH_F32_DEPTH && fmt != LF_MESH_F16_OFFSET) return fail(c, LF_ERR_INVALID_ARG, "bad mesh format");
  lf_status st = quiesce(c);
  if (st != LF_OK) return st;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; c->graph_sig.clear(); }
  c->G = 0;
  cudaStream_t s = c->work_stream;
  const size_t n = (size_t)c->n_views * grid_n * grid_n;
  LF_CUDA(c, ensure(c->tab_a, sizeof(float) * (size_t)c->n_views * grid_n));
  LF_CUDA(c, ensure(c->tab_b, sizeof(float) * (size_t)c->n_views * grid_n));
  release(c->depth);
  if (fmt == LF_MESH_F32_DEPTH) {
    LF_CUDA(c, ensure(c->depth, sizeof(float) * n));
    LF_CUDA(c, cudaMemcpyAsync(c->depth.p, depth, sizeof(float) * n, cudaMemcpyHostToDevice, s));
  } else {
    Buffer stage;
    LF_CUDA(c, ensure(stage, sizeof(float) * n));
    LF_CUDA(c, ensure(c->depth, 2 * n));
    LF_CUDA(c, cudaMemcpyAsync(stage.p, depth, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    LF_CUDA(c, launch_depth_offsets(static_cast<const float*>(stage.p), c->n_views, grid_n * grid_n, c->depth.p,
                                    static_cast<ViewStatic*>(c->views.p), s));
    LF_CUDA(c, cudaStreamSynchronize(s));
    release(stage);
  }
  LF_CUDA(c, launch_grid_tables(static_cast<const ViewStatic*>(c->views.p), c->n_views, c->src_w, c->src_h, grid_n,
                                static_cast<float*>(c->tab_a.p), static_cast<float*>(c->tab_b.p), s));
  LF_CUDA(c, cudaStreamSynchronize(s));
  c->G = grid_n;
  c->mesh_fmt = fmt;
  return LF_OK;
}

lf_status lf_render(lf_ctx* c, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                    float* const* out_rgba, void* stream) {
  lf_status st = check_ready(c);
  if (st != LF_OK) return st;
  Layout L;
  if ((st = make_layout(c, n_eyes, eyes, intr, out_rgba, L)) != LF_OK) return st;
  if ((st = ensure_scratch(c, n_eyes, L.total_tiles)) != LF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = stage_eyes(c, L, s)) != LF_OK) return st;
  FrameArgs a = frame_args(c, L);
  if ((st = enqueue_frame(c, a, false, false, s)) != LF_OK) return st;
  c->last_stream = s;
  c->last_eyes = n_eyes;
  c->last_tiles = L.total_tiles;
  c->has_call = true;
  return LF_OK;
}

lf_status lf_render_inspect(lf_ctx* c, const lf_pose* eye, const lf_intrinsics* intr, float* out_rgba,
                            lf_frag_record* records, int32_t max_records, int32_t* counts, uint8_t* active,
                            uint32_t* texel_bits, void* stream) {
  lf_status st = check_ready(c);
  if (st != LF_OK) return st;
  if (!records || !counts || !active || max_records < 1) return fail(c, LF_ERR_INVALID_ARG, "bad inspect buffers");
  Layout L;
  float* outs[1] = {out_rgba};
  if ((st = make_layout(c, 1, eye, intr, outs, L)) != LF_OK) return st;
  if ((st = ensure_scratch(c, 1, L.total_tiles)) != LF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = stage_eyes(c, L, s)) != LF_OK) return st;
  FrameArgs a = frame_args(c, L);
  a.active = active;
  a.records = records;
  a.max_records = max_records;
  a.counts = counts;
  a.texel_bits = texel_bits;
  if ((st = enqueue_frame(c, a, true, false, s)) != LF_OK) return st;
  c->last_stream = s;
  c->last_eyes = 1;
  c->last_tiles = L.total_tiles;
  c->has_call = true;
  return LF_OK;
}

lf_status lf_render_batch(lf_ctx* c, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                          float* const* out_rgba, void* stream) {
  lf_status st = check_ready(c);
  if (st != LF_OK) return st;
  Layout L;
  if ((st = make_layout(c, n_eyes, eyes, intr, out_rgba, L)) != LF_OK) return st;
  if ((st = ensure_scratch(c, n_eyes, L.total_tiles)) != LF_OK) return st;
  if ((st = ensure_persistent_blocks(c)) != LF_OK) return st;
  // The graph depends on the layout and on every scratch address it names.
  std::vector<int64_t> sig = {n_eyes, L.total_tiles, c->n_views, c->G, c->tex_fmt, c->mesh_fmt,
                              (int64_t)(intptr_t)c->eyes.p, (int64_t)(intptr_t)c->eyes_f.p,
                              (int64_t)(intptr_t)c->bin_offsets.p, (int64_t)(intptr_t)c->bin_entries.p,
                              (int64_t)(intptr_t)c->vrecs.p,
                              (int64_t)(intptr_t)c->masks.p, (int64_t)(intptr_t)c->pool.p,
                              (int64_t)(intptr_t)c->active.p, (int64_t)(intptr_t)c->small.p,
                              (int64_t)(intptr_t)c->tex.p, (int64_t)(intptr_t)c->depth.p, c->persistent_blocks,
                              c->cfg.tile_w, c->cfg.tile_h, c->cfg.timing, c->disk_mode, c->lv.n_fine,
                              (int64_t)(intptr_t)c->lv.pool.p, (int64_t)(intptr_t)c->lv.enable.p,
                              (int64_t)(intptr_t)c->lv.visible.p};
  for (int e = 0; e < n_eyes; ++e) { sig.push_back(intr[e].width); sig.push_back(intr[e].height); }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (c->cfg.timing) {
    // Timing mode: the same persistent sequence, launched eagerly, because CUDA
    // events recorded inside a captured graph cannot be queried for elapsed time.
    if ((st = stage_eyes(c, L, s)) != LF_OK) return st;
    FrameArgs a = frame_args(c, L);
    if ((st = enqueue_frame(c, a, false, true, s)) != LF_OK) return st;
    c->last_stream = s;
    c->last_eyes = n_eyes;
    c->last_tiles = L.total_tiles;
    c->has_call = true;
    return LF_OK;
  }
  if (!c->graph || sig != c->graph_sig) {
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    FrameArgs a = frame_args(c, L);
    cudaGraph_t g = nullptr;
    LF_CUDA(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
    lf_status q = enqueue_frame(c, a, false, true, c->capture_stream);
    cudaError_t ec = cudaStreamEndCapture(c->capture_stream, &g);
    if (q != LF_OK) { if (g) cudaGraphDestroy(g); return q; }
    if (ec != cudaSuccess) return cuda_fail(c, ec, "cudaStreamEndCapture");
    cudaError_t ei = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) { c->graph = nullptr; return cuda_fail(c, ei, "cudaGraphInstantiate"); }
    c->graph_sig = sig;
  }
  if ((st = stage_eyes(c, L, s)) != LF_OK) return st;
  LF_CUDA(c, cudaGraphLaunch(c->graph, s));
  c->last_stream = s;
  c->last_eyes = n_eyes;
  c->last_tiles = L.total_tiles;
  c->has_call = true;
  return LF_OK;
}

lf_status lf_set_levels(lf_ctx* c, int32_t n_fine, int32_t n_pages) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (c->n_views <= 0) return fail(c, LF_ERR_STATE, "views not loaded");
  if (c->lv.n_fine > 0) return fail(c, LF_ERR_STATE, "the levels are set already: load the views again first");
  if (n_fine < 1 || n_fine >= c->n_views || n_pages < 1 || n_pages > n_fine)
    return fail(c, LF_ERR_INVALID_ARG, "need 1 <= n_pages <= n_fine < n_views");
  lf_status st = quiesce(c);
  if (st != LF_OK) return st;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; c->graph_sig.clear(); }
  const int nc = c->n_views - n_fine;
  // per coarse view, the fine views whose disks overlap its disk: chord distance
  // between the centres below the sum of the radii (FP64)
  std::vector<int32_t> off(nc + 1, 0), ids;
  for (int k = 0; k < nc; ++k) {
    const ViewStatic& C = c->views_host[n_fine + k];
    for (int f = 0; f < n_fine; ++f) {
      const ViewStatic& F = c->views_host[f];
      const double dx = (double)C.disk_c[0] - (double)F.disk_c[0], dy = (double)C.disk_c[1] - (double)F.disk_c[1];
      const double dz = (double)C.disk_c[2] - (double)F.disk_c[2];
      if (std::sqrt(dx * dx + dy * dy + dz * dz) < (double)C.disk_r + (double)F.disk_r) ids.push_back(f);
    }
    off[k + 1] = (int32_t)ids.size();
  }
  // the coarse images move to their own buffer; the fine ones leave the device
  const size_t texel_bytes = c->tex_fmt == LF_TEX_F32 ? 16 : c->tex_fmt == LF_TEX_BF16 ? 8 : 4;
  const size_t per = texel_bytes * (size_t)c->src_w * c->src_h;
  Buffer coarse;
  LF_CUDA(c, ensure(coarse, per * nc));
  LF_CUDA(c, cudaMemcpy(coarse.p, static_cast<char*>(c->tex.p) + per * n_fine, per * nc, cudaMemcpyDeviceToDevice));
  release(c->tex);
  c->tex = coarse;
  auto& L = c->lv;
  LF_CUDA(c, ensure(L.pool, per * (size_t)n_pages));
  LF_CUDA(c, ensure(L.table, sizeof(void*) * (size_t)c->n_views));
  LF_CUDA(c, ensure(L.page_of_view, sizeof(int32_t) * (size_t)n_fine));
  LF_CUDA(c, ensure(L.overlap_off, sizeof(int32_t) * off.size()));
  LF_CUDA(c, ensure(L.overlap_ids, sizeof(int32_t) * std::max<size_t>(1, ids.size())));
  L.view_page.assign(n_fine, -1);
  L.page_view.assign(n_pages, -1);
  L.table_host.assign(c->n_views, nullptr);
  for (int k = 0; k < nc; ++k) L.table_host[n_fine + k] = static_cast<const char*>(c->tex.p) + per * k;
  LF_CUDA(c, cudaMemcpy(L.table.p, L.table_host.data(), sizeof(void*) * L.table_host.size(), cudaMemcpyHostToDevice));
  LF_CUDA(c, cudaMemcpy(L.page_of_view.p, L.view_page.data(), sizeof(int32_t) * n_fine, cudaMemcpyHostToDevice));
  LF_CUDA(c, cudaMemcpy(L.overlap_off.p, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice));
  if (!ids.empty())
    LF_CUDA(c, cudaMemcpy(L.overlap_ids.p, ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice));
  L.n_fine = n_fine;
  L.n_pages = n_pages;
  return LF_OK;
}

lf_status lf_upload_pages(lf_ctx* c, int32_t n, const int32_t* views, const int32_t* pages,
                          const uint8_t* const* rgba8, void* stream) {
  if (!c) return LF_ERR_INVALID_ARG;
  auto& L = c->lv;
  if (L.n_fine <= 0) return fail(c, LF_ERR_STATE, "no levels set (lf_set_levels)");
  if (n < 0 || (n > 0 && (!views || !pages || !rgba8))) return fail(c, LF_ERR_INVALID_ARG, "bad upload arguments");
  std::vector<uint8_t> seen_v(L.n_fine, 0), seen_p(L.n_pages, 0);
  for (int k = 0; k < n; ++k) {
    if (views[k] < 0 || views[k] >= L.n_fine || pages[k] < 0 || pages[k] >= L.n_pages || !rgba8[k])
      return fail(c, LF_ERR_INVALID_ARG, "upload view, page or image out of range");
    if (seen_v[views[k]]++ || seen_p[pages[k]]++)
      return fail(c, LF_ERR_INVALID_ARG, "a view or page appears twice in one upload");
  }
  if (n == 0) return LF_OK;
  LF_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LF_CUDA(c, cudaStreamSynchronize(s));  // renders that read the pages being replaced are done
  const size_t texel_bytes = c->tex_fmt == LF_TEX_F32 ? 16 : c->tex_fmt == LF_TEX_BF16 ? 8 : 4;
  const int64_t per_view = (int64_t)c->src_w * c->src_h;
  const size_t per = texel_bytes * (size_t)per_view;
  char* pool = static_cast<char*>(L.pool.p);
  if (c->tex_fmt != LF_TEX_U8) LF_CUDA(c, ensure(L.stage, (size_t)n * per_view * 4));
  for (int k = 0; k < n; ++k) {
    char* dst = pool + per * pages[k];
    if (c->tex_fmt == LF_TEX_U8) {
      LF_CUDA(c, cudaMemcpyAsync(dst, rgba8[k], (size_t)per_view * 4, cudaMemcpyHostToDevice, s));
      continue;
    }
    uint8_t* st8 = static_cast<uint8_t*>(L.stage.p) + (size_t)k * per_view * 4;
    LF_CUDA(c, cudaMemcpyAsync(st8, rgba8[k], (size_t)per_view * 4, cudaMemcpyHostToDevice, s));
    ViewStatic* vs = static_cast<ViewStatic*>(c->views.p) + views[k];
    const float* scale = nullptr;
    if (c->tex_fmt == LF_TEX_FP8E4M3) {
      // the view's FP8 scale, from this image (as lf_load_views computes it)
      float* sc = reinterpret_cast<float*>(&vs->tex_scale);
      LF_CUDA(c, launch_view_scale(st8, 1, per_view, sc, vs, s));
      scale = sc;
    }
    LF_CUDA(c, launch_convert_textures(st8, dst, per_view, c->tex_fmt, scale, per_view, s));
  }
  LF_CUDA(c, cudaStreamSynchronize(s));
  // the page table: a page's previous view is no longer resident
  for (int k = 0; k < n; ++k) {
    const int v = views[k], p = pages[k];
    const int w = L.page_view[p];
    if (w >= 0 && w != v) { L.view_page[w] = -1; L.table_host[w] = nullptr; }
    const int q = L.view_page[v];
    if (q >= 0 && q != p) L.page_view[q] = -1;
    L.page_view[p] = v;
    L.view_page[v] = p;
    L.table_host[v] = pool + per * p;
  }
  LF_CUDA(c, cudaMemcpy(L.table.p, L.table_host.data(), sizeof(void*) * (size_t)L.n_fine, cudaMemcpyHostToDevice));
  LF_CUDA(c, cudaMemcpy(L.page_of_view.p, L.view_page.data(), sizeof(int32_t) * (size_t)L.n_fine,
                        cudaMemcpyHostToDevice));
  return LF_OK;
}

lf_status lf_levels_wanted(lf_ctx* c, int32_t cap, int32_t* views, int32_t* n) {
  if (!c || !n || cap < 0 || (cap > 0 && !views)) return LF_ERR_INVALID_ARG;
  *n = 0;
  if (c->lv.n_fine <= 0) return fail(c, LF_ERR_STATE, "no levels set (lf_set_levels)");
  if (!c->has_call || !c->lv.visible.p) return fail(c, LF_ERR_STATE, "no render call yet");
  LF_CUDA(c, cudaSetDevice(c->device));
  LF_CUDA(c, cudaStreamSynchronize(c->last_stream));
  std::vector<uint8_t> vis((size_t)c->last_eyes * c->n_views);
  LF_CUDA(c, cudaMemcpy(vis.data(), c->lv.visible.p, vis.size(), cudaMemcpyDeviceToHost));
  int32_t k = 0;
  for (int v = 0; v < c->lv.n_fine; ++v) {
    bool any = false;
    for (int e = 0; e < c->last_eyes && !any; ++e) any = vis[(size_t)e * c->n_views + v] != 0;
    if (!any) continue;
    if (k < cap) views[k] = v;
    ++k;
  }
  *n = k;
  return k > cap ? fail(c, LF_ERR_CAPACITY, "more wanted views than cap") : LF_OK;
}

lf_status lf_get_stats(lf_ctx* c, lf_stats* out) {
  if (!c || !out) return LF_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->n_views = c->n_views;
  if (!c->has_call) return LF_OK;
  LF_CUDA(c, cudaSetDevice(c->device));
  LF_CUDA(c, cudaStreamSynchronize(c->last_stream));
  unsigned char sm[16];
  LF_CUDA(c, cudaMemcpy(sm, c->small.p, 16, cudaMemcpyDeviceToHost));
  unsigned long long tris;
  std::memcpy(&tris, sm, 8);
  std::memcpy(&out->error_word, sm + 8, 4);
  out->n_eyes = c->last_eyes;
  out->triangles = (int64_t)tris;
  if (c->timed_call) {
    LF_CUDA(c, cudaEventElapsedTime(&out->ms_view_setup, c->tev[0], c->tev[1]));
    LF_CUDA(c, cudaEventElapsedTime(&out->ms_tri_setup, c->tev[1], c->tev[2]));
    LF_CUDA(c, cudaEventElapsedTime(&out->ms_raster, c->tev[2], c->tev[3]));
  }
  out->tiles = c->last_tiles;
  std::vector<uint8_t> act((size_t)std::min(c->last_eyes, 2) * c->n_views);
  if (!act.empty()) {
    LF_CUDA(c, cudaMemcpy(act.data(), c->active.p, act.size(), cudaMemcpyDeviceToHost));
    for (int e = 0; e < std::min(c->last_eyes, 2); ++e) {
      int n = 0;
      for (int v = 0; v < c->n_views; ++v) n += act[(size_t)e * c->n_views + v];
      out->active_views[e] = n;
    }
  }
  if (out->error_word & kErrPoolOverflow) return fail(c, LF_ERR_CAPACITY, "triangle pool overflow");
  return LF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Rendering without any allocation (lf_render_static).
//
// Some callers cannot call cudaMalloc while they render: a frame loop with a
// hard deadline where an allocation (and the device synchronisation it can
// imply) would miss the frame, a process whose device memory is fully
// reserved up front by another allocator, or a sandboxed plug-in that is not
// allowed to create allocations of its own.  lf_render grows its scratch
// buffers with cudaMalloc on first use and whenever a call needs more, so it
// is not safe for them.  lf_render_static runs the same three kernels on the
// same loaded views, but takes every per-call scratch buffer from the one
// static device array below, sized for the worst case within its limits, so
// it never allocates and never runs out of room.  (A set-up triangle fills at
// most kBinMaxTiles bin entries, and a view's bins at most 2 ints per tile.)
// ---------------------------------------------------------------------------

namespace {

constexpr int kStaticMaxViews = 32;
constexpr int kStaticMaxGrid = 33;
constexpr int kStaticMaxTiles = 8192;
constexpr int64_t kStaticTris =
    (int64_t)kStaticMaxViews * 4 * (kStaticMaxGrid - 1) * (kStaticMaxGrid - 1);  // two sub-triangles per parent
constexpr int64_t kStaticBinOffsets = (int64_t)kStaticMaxViews * (2 * kStaticMaxTiles + 1);
constexpr int64_t kStaticBinEntries = kStaticTris * kBinMaxTiles;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffCounters = 0;
constexpr size_t kOffEye = align256(kOffCounters + 64);
constexpr size_t kOffEyeF = align256(kOffEye + sizeof(EyeParams));
constexpr size_t kOffVrecs = align256(kOffEyeF + sizeof(EyeFloat));
constexpr size_t kOffActive = align256(kOffVrecs + sizeof(ViewRec) * kStaticMaxViews);
constexpr size_t kOffMasks = align256(kOffActive + kStaticMaxViews);
constexpr size_t kOffBinOffsets = align256(kOffMasks + sizeof(uint32_t) * kStaticMaxTiles * ((kStaticMaxViews + 31) / 32));
constexpr size_t kOffBinEntries = align256(kOffBinOffsets + sizeof(int32_t) * kStaticBinOffsets);
constexpr size_t kOffPool = align256(kOffBinEntries + sizeof(int32_t) * kStaticBinEntries);
constexpr size_t kStaticBytes = align256(kOffPool + sizeof(TriRec) * kStaticTris);  // about 16.8 MB

}  // namespace

// The scratch of lf_render_static.  Every GPU that loads this library holds
// it until the process exits.  Its name is only a host-side stand-in: host
// code must use the device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char lf_static_scratch[kStaticBytes];

namespace {

std::mutex g_static_mu;
void* g_static_addr[256] = {};

// Device address of the static scratch on the current device, looked up once
// per device (the caller has made `device` current).
cudaError_t static_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, lf_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_static_addr[device]);
  return cudaSuccess;
}

}  // namespace

extern "C" lf_status lf_render_static(lf_ctx* c, const lf_pose* eye, const lf_intrinsics* intr, float* out_rgba,
                                      void* stream) {
  lf_status st = check_ready(c);
  if (st != LF_OK) return st;
  if (c->lv.n_fine > 0) return fail(c, LF_ERR_UNSUPPORTED, "lf_render_static: two-level frames need per-call buffers");
  if (c->n_views > kStaticMaxViews)
    return fail(c, LF_ERR_CAPACITY, "lf_render_static: more than 32 views are loaded");
  if (c->G > kStaticMaxGrid) return fail(c, LF_ERR_CAPACITY, "lf_render_static: mesh grid larger than 33 x 33");
  // the one eye, checked as lf_render checks it, built without any allocation
  if (!eye || !intr || !out_rgba) return fail(c, LF_ERR_INVALID_ARG, "null argument");
  if (!aligned16(out_rgba)) return fail(c, LF_ERR_INVALID_ARG, "the output image must be 16-byte aligned (RGBA texels)");
  const lf_intrinsics& K = *intr;
  if (K.width < 1 || K.height < 1 || K.width > 32767 || K.height > 32767)
    return fail(c, LF_ERR_INVALID_ARG, "eye size out of range");
  if (!(K.fx > 0) || !(K.fy > 0)) return fail(c, LF_ERR_INVALID_ARG, "focal length must be positive");
  EyeParams P;
  std::memset(&P, 0, sizeof(P));
  std::memcpy(P.R, eye->R, sizeof(P.R));
  std::memcpy(P.t, eye->t, sizeof(P.t));
  P.fx = K.fx; P.fy = K.fy; P.cx = K.cx; P.cy = K.cy;
  P.W = K.width; P.H = K.height;
  P.tiles_x = (K.width + c->cfg.tile_w - 1) / c->cfg.tile_w;
  P.tiles_y = (K.height + c->cfg.tile_h - 1) / c->cfg.tile_h;
  P.tile_base = 0;
  P.out = out_rgba;
  const int64_t tiles = (int64_t)P.tiles_x * P.tiles_y;
  if (tiles > kStaticMaxTiles)
    return fail(c, LF_ERR_CAPACITY, "lf_render_static: eye view has more than 8192 screen tiles");
  unsigned char* base = nullptr;
  LF_CUDA(c, static_scratch(c->device, &base));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // eye parameters through the context's pinned ring (allocated at lf_create)
  const int slot = c->ring_next;
  c->ring_next = (c->ring_next + 1) % kRing;
  LF_CUDA(c, cudaEventSynchronize(c->ring_ev[slot]));
  EyeParams* staged = c->pinned + (size_t)slot * c->cfg.max_eyes;
  std::memcpy(staged, &P, sizeof(EyeParams));
  LF_CUDA(c, cudaMemcpyAsync(base + kOffEye, staged, sizeof(EyeParams), cudaMemcpyHostToDevice, s));
  LF_CUDA(c, cudaEventRecord(c->ring_ev[slot], s));
  const Layout none;  // no eyes vector: the counts are set below
  FrameArgs a = frame_args(c, none);
  a.n_eyes = 1;
  a.total_tiles = (int32_t)tiles;
  a.eyes = reinterpret_cast<const EyeParams*>(base + kOffEye);
  a.eyes_f = reinterpret_cast<EyeFloat*>(base + kOffEyeF);
  a.vrecs = reinterpret_cast<ViewRec*>(base + kOffVrecs);
  a.active = base + kOffActive;
  a.tile_masks = reinterpret_cast<uint32_t*>(base + kOffMasks);
  a.bin_offsets = reinterpret_cast<int32_t*>(base + kOffBinOffsets);
  a.bin_offsets_capacity = kStaticBinOffsets;
  a.bin_entries = reinterpret_cast<int32_t*>(base + kOffBinEntries);
  a.bin_entries_capacity = kStaticBinEntries;
  a.bin_max_tiles = kBinMaxTiles;
  a.pool = reinterpret_cast<TriRec*>(base + kOffPool);
  a.pool_capacity = kStaticTris;
  use_counters(a, base + kOffCounters);
  // enqueue_frame zeroes the masks, counters and flags that must start at zero;
  // no timing events, so lf_get_stats keeps reporting the last lf_render call
  return enqueue_frame(c, a, false, false, s, false);
}

// ---------------------------------------------------------------------------
// Learned refinement: y = x + f(x) on normalised renders (kernels in
// lf_refine.cu and lf_refine_tc.cu).

namespace {

constexpr int kRefineSegs[3] = {896, 9248, 867};  // W1+b1, W2+b2, W3+b3
constexpr int kRefineSegBase[3] = {kRefineOffW1, kRefineOffW2, kRefineOffW3};

float* rf_params(lf_ctx* c) { return static_cast<float*>(c->rf.state.p); }
float* rf_grad(lf_ctx* c) { return rf_params(c) + kRefineParams; }
float* rf_m(lf_ctx* c) { return rf_params(c) + 2 * kRefineParams; }
float* rf_v(lf_ctx* c) { return rf_params(c) + 3 * kRefineParams; }
const __nv_bfloat16* rf_w(lf_ctx* c, int off) { return static_cast<const __nv_bfloat16*>(c->rf.packed.p) + off; }

lf_status refine_check(lf_ctx* c, int32_t n, int32_t w, int32_t h, const void* a, const void* b) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (!c->rf.loaded) return fail(c, LF_ERR_STATE, "no refiner loaded");
  if (n < 0 || w < 0 || h < 0 || (int64_t)w * h > ((int64_t)1 << 28) || (int64_t)n * w * h > ((int64_t)1 << 30))
    return fail(c, LF_ERR_INVALID_ARG, "bad image sizes");
  if ((int64_t)n * w * h > 0 && (!a || !b)) return fail(c, LF_ERR_INVALID_ARG, "null image pointer");
  if (!aligned16(a) || !aligned16(b)) return fail(c, LF_ERR_INVALID_ARG, "images must be 16-byte aligned (RGBA texels)");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  return LF_OK;
}

lf_status refine_hidden(lf_ctx* c, int64_t n_pix, bool training) {
  const size_t hb = sizeof(__nv_bfloat16) * 32 * (size_t)n_pix;
  LF_CUDA(c, ensure(c->rf.a1, hb));
  LF_CUDA(c, ensure(c->rf.a2, hb));
  if (training) {
    LF_CUDA(c, ensure(c->rf.gz2, hb));
    LF_CUDA(c, ensure(c->rf.gr, sizeof(float) * 4 * (size_t)n_pix));
  }
  return LF_OK;
}

RefineConvArgs conv_args(lf_ctx* c, int32_t n, int32_t w, int32_t h) {
  RefineConvArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.W = w;
  a.H = h;
  a.error = reinterpret_cast<int32_t*>(static_cast<char*>(c->rf.scal.p) + 8);  // read by lf_get_refiner
  a.wait_ns = (uint64_t)c->cfg.wait_limit;
  return a;
}

// The three layer launches of the per-layer path (inference).
lf_status refine_layers(lf_ctx* c, int32_t n, int32_t w, int32_t h, const float* in, float* out, cudaStream_t s) {
  const float* prm = rf_params(c);
  RefineConvArgs a = conv_args(c, n, w, h);
  a.src_f = in;
  a.wt = rf_w(c, kPackW1f);
  a.bias = prm + kRefineOffB1;
  a.out_h = static_cast<__nv_bfloat16*>(c->rf.a1.p);
  LF_CUDA(c, launch_refine_conv(kConvInRGBA, 32, kEpiRelu, a, s));
  a = conv_args(c, n, w, h);
  a.src_h = static_cast<const __nv_bfloat16*>(c->rf.a1.p);
  a.wt = rf_w(c, kPackW2f);
  a.bias = prm + kRefineOffB2;
  a.out_h = static_cast<__nv_bfloat16*>(c->rf.a2.p);
  LF_CUDA(c, launch_refine_conv(kConvInBF16, 32, kEpiRelu, a, s));
  a = conv_args(c, n, w, h);
  a.src_h = static_cast<const __nv_bfloat16*>(c->rf.a2.p);
  a.wt = rf_w(c, kPackW3f);
  a.bias = prm + kRefineOffB3;
  a.x = in;
  a.out_f = out;
  LF_CUDA(c, launch_refine_conv(kConvInBF16, 8, kEpiResid, a, s));
  return LF_OK;
}

lf_status refine_apply(lf_ctx* c, int32_t n, int32_t w, int32_t h, const float* in, float* out, cudaStream_t s,
                       float* out1 = nullptr, bool pdl = false) {
  if ((int64_t)n * w * h == 0) return LF_OK;
  if (c->rf.kernel == LF_REFINE_FUSED_TC) {
    if (reinterpret_cast<uintptr_t>(in) & 15u)  // the fused kernel reads the input through a TMA tensor map
      return fail(c, LF_ERR_INVALID_ARG, "the fused refinement needs a 16-byte aligned input");
    int32_t* err = reinterpret_cast<int32_t*>(static_cast<char*>(c->rf.scal.p) + 8);
    LF_CUDA(c, launch_refine_fused(n, w, h, in, out, out1, rf_params(c),
                                   static_cast<const __nv_bfloat16*>(c->rf.packed.p), c->sm_count, err,
                                   (uint64_t)c->cfg.wait_limit, s, pdl));
    return LF_OK;
  }
  lf_status st = refine_hidden(c, (int64_t)n * w * h, false);
  if (st != LF_OK) return st;
  return refine_layers(c, n, w, h, in, out, s);
}

// The refinement of a rendered frame: eye e's image in[e] (FP32 RGBA) into
// out[e].  A pair of equal-sized eyes whose inputs lie back to back in one
// buffer is refined by one fused launch (the two images' tiles share the
// grid); `pdl` (no timing events after the raster) launches the first
// refinement as a programmatic dependent of the raster.
lf_status refine_eyes(lf_ctx* c, int32_t n_eyes, const lf_intrinsics* intr, float* const* in, float* const* out,
                      cudaStream_t s, bool pdl) {
  if (c->rf.kernel == LF_REFINE_FUSED_TC && n_eyes == 2 && intr[0].width == intr[1].width &&
      intr[0].height == intr[1].height && in[1] == in[0] + (size_t)intr[0].width * intr[0].height * 4)
    return refine_apply(c, 2, intr[0].width, intr[0].height, in[0], out[0], s, out[1], pdl);
  for (int e = 0; e < n_eyes; ++e) {
    lf_status st = refine_apply(c, 1, intr[e].width, intr[e].height, in[e], out[e], s, nullptr, pdl && e == 0);
    if (st != LF_OK) return st;
  }
  return LF_OK;
}

// Forward with the loss epilogue, then the backward pass into rf_grad.
lf_status refine_backward(lf_ctx* c, int32_t n, int32_t w, int32_t h, const float* in, const float* tgt,
                          cudaStream_t s) {
  const int64_t n_pix = (int64_t)n * w * h;
  lf_status st = refine_hidden(c, n_pix, true);
  if (st != LF_OK) return st;
  const int tiles_x = (w + 31) / 32, tiles_y = (h + 7) / 8;
  const int n_tiles = tiles_x * tiles_y * n;
  const int n_ctas = std::max(1, std::min(n_tiles, 3 * c->sm_count));  // weight-gradient CTAs: three per SM
  LF_CUDA(c, ensure(c->rf.partial, sizeof(float) * (size_t)n_ctas * (896 + 9248 + 867)));
  float* loss = static_cast<float*>(c->rf.scal.p);
  int32_t* count = reinterpret_cast<int32_t*>(loss + 1);
  LF_CUDA(c, cudaMemsetAsync(c->rf.scal.p, 0, 8, s));
  LF_CUDA(c, cudaMemsetAsync(rf_grad(c), 0, sizeof(float) * kRefineParams, s));
  if (n_pix == 0) return LF_OK;
  LF_CUDA(c, launch_refine_count(in, tgt, n_pix, count, s));
  const float* prm = rf_params(c);
  auto* a1 = static_cast<__nv_bfloat16*>(c->rf.a1.p);
  auto* a2 = static_cast<__nv_bfloat16*>(c->rf.a2.p);  // later dL/dz1
  auto* gz2 = static_cast<__nv_bfloat16*>(c->rf.gz2.p);
  float* gr = static_cast<float*>(c->rf.gr.p);
  RefineConvArgs a = conv_args(c, n, w, h);
  a.src_f = in; a.wt = rf_w(c, kPackW1f); a.bias = prm + kRefineOffB1; a.out_h = a1;
  LF_CUDA(c, launch_refine_conv(kConvInRGBA, 32, kEpiRelu, a, s));
  a = conv_args(c, n, w, h);
  a.src_h = a1; a.wt = rf_w(c, kPackW2f); a.bias = prm + kRefineOffB2; a.out_h = a2;
  LF_CUDA(c, launch_refine_conv(kConvInBF16, 32, kEpiRelu, a, s));
  a = conv_args(c, n, w, h);
  a.src_h = a2; a.wt = rf_w(c, kPackW3f); a.bias = prm + kRefineOffB3; a.x = in; a.target = tgt; a.out_f = gr;
  a.loss = loss; a.count = count;
  LF_CUDA(c, launch_refine_conv(kConvInBF16, 8, kEpiLoss, a, s));

  RefineWgradArgs g;
  std::memset(&g, 0, sizeof(g));
  g.n = n; g.W = w; g.H = h; g.tiles_x = tiles_x; g.tiles_y = tiles_y; g.n_tiles = n_tiles; g.n_ctas = n_ctas;
  g.error = reinterpret_cast<int32_t*>(static_cast<char*>(c->rf.scal.p) + 8);
  g.wait_ns = (uint64_t)c->cfg.wait_limit;
  float* part = static_cast<float*>(c->rf.partial.p);
  float* part1 = part;
  float* part2 = part1 + (size_t)n_ctas * kRefineSegs[0];
  float* part3 = part2 + (size_t)n_ctas * kRefineSegs[1];
  // layer 3 weights (dL/dr with a2), then dL/dz2 through layer 3's input
  g.g_f = gr; g.a_h = a2; g.partial = part3;
  LF_CUDA(c, launch_refine_wgrad(3, g, s));
  a = conv_args(c, n, w, h);
  a.src_f = gr; a.wt = rf_w(c, kPackW3b); a.mask = a2; a.out_h = gz2;
  LF_CUDA(c, launch_refine_conv(kConvInRGBA, 32, kEpiMask, a, s));
  // dL/dz1 through layer 2's input (into a2's buffer, no longer needed)
  a = conv_args(c, n, w, h);
  a.src_h = gz2; a.wt = rf_w(c, kPackW2b); a.mask = a1; a.out_h = a2;
  LF_CUDA(c, launch_refine_conv(kConvInBF16, 32, kEpiMask, a, s));
  g.g_f = nullptr; g.g_h = gz2; g.a_h = a1; g.partial = part2;
  LF_CUDA(c, launch_refine_wgrad(2, g, s));
  g.g_h = a2; g.a_h = nullptr; g.x = in; g.partial = part1;
  LF_CUDA(c, launch_refine_wgrad(1, g, s));
  float* parts[3] = {part1, part2, part3};
  for (int k = 0; k < 3; ++k)
    LF_CUDA(c, launch_refine_reduce(parts[k], n_ctas, kRefineSegs[k], rf_grad(c) + kRefineSegBase[k], s));
  return LF_OK;
}

}  // namespace

extern "C" {

lf_status lf_load_refiner(lf_ctx* c, const float* params) {
  if (!c || !params) return LF_ERR_INVALID_ARG;
  for (int i = 0; i < kRefineParams; ++i)
    if (!(params[i] == params[i]) || params[i] > 1e30f || params[i] < -1e30f)
      return fail(c, LF_ERR_INVALID_ARG, "non-finite refiner parameter");
  lf_status st = quiesce(c);  // a refinement in flight may still read the weights
  if (st != LF_OK) return st;
  LF_CUDA(c, ensure(c->rf.state, sizeof(float) * 4 * kRefineParams));
  LF_CUDA(c, ensure(c->rf.packed, sizeof(__nv_bfloat16) * kRefinePackedElems));
  LF_CUDA(c, ensure(c->rf.scal, 64));
  cudaStream_t s = c->work_stream;
  LF_CUDA(c, cudaMemsetAsync(c->rf.state.p, 0, sizeof(float) * 4 * kRefineParams, s));
  LF_CUDA(c, cudaMemcpyAsync(c->rf.state.p, params, sizeof(float) * kRefineParams, cudaMemcpyHostToDevice, s));
  LF_CUDA(c, cudaMemsetAsync(c->rf.scal.p, 0, 64, s));
  LF_CUDA(c, launch_refine_pack(rf_params(c), static_cast<__nv_bfloat16*>(c->rf.packed.p), s));
  LF_CUDA(c, cudaStreamSynchronize(s));
  c->rf.loaded = true;
  c->rf.step = 0;
  return LF_OK;
}

lf_status lf_refine_set_kernel(lf_ctx* c, lf_refine_kernel k) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (k != LF_REFINE_FUSED_TC && k != LF_REFINE_MMA_LAYERS) return fail(c, LF_ERR_INVALID_ARG, "unknown kernel");
  c->rf.kernel = k;
  return LF_OK;
}

lf_status lf_get_refiner(lf_ctx* c, float* params, float* grad, float* adam_m, float* adam_v, int32_t* step,
                         float* last_loss) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (!c->rf.loaded) return fail(c, LF_ERR_STATE, "no refiner loaded");
  LF_CUDA(c, cudaSetDevice(c->device));
  LF_CUDA(c, cudaDeviceSynchronize());
  float* dst[4] = {params, grad, adam_m, adam_v};
  for (int k = 0; k < 4; ++k)
    if (dst[k])
      LF_CUDA(c, cudaMemcpy(dst[k], rf_params(c) + (size_t)k * kRefineParams, sizeof(float) * kRefineParams,
                            cudaMemcpyDeviceToHost));
  if (last_loss) LF_CUDA(c, cudaMemcpy(last_loss, c->rf.scal.p, sizeof(float), cudaMemcpyDeviceToHost));
  if (step) *step = c->rf.step;
  int32_t err = 0;
  LF_CUDA(c, cudaMemcpy(&err, static_cast<char*>(c->rf.scal.p) + 8, sizeof(err), cudaMemcpyDeviceToHost));
  if (err) {
    char msg[96];
    std::snprintf(msg, sizeof(msg), "a wait of a refinement kernel gave up (error word 0x%x)", (unsigned)err);
    return fail(c, LF_ERR_TIMEOUT, msg);
  }
  return LF_OK;
}

lf_status lf_refine(lf_ctx* c, int32_t n_images, int32_t width, int32_t height, const float* in_rgba,
                    float* out_rgba, void* stream) {
  lf_status st = refine_check(c, n_images, width, height, in_rgba, out_rgba);
  if (st != LF_OK) return st;
  if (in_rgba == out_rgba && (int64_t)n_images * width * height > 0)
    return fail(c, LF_ERR_INVALID_ARG, "lf_refine cannot run in place");
  return refine_apply(c, n_images, width, height, in_rgba, out_rgba, static_cast<cudaStream_t>(stream));
}

lf_status lf_refine_gradients(lf_ctx* c, int32_t n_images, int32_t width, int32_t height, const float* in_rgba,
                              const float* target_rgba, void* stream) {
  lf_status st = refine_check(c, n_images, width, height, in_rgba, target_rgba);
  if (st != LF_OK) return st;
  return refine_backward(c, n_images, width, height, in_rgba, target_rgba, static_cast<cudaStream_t>(stream));
}

lf_status lf_refine_train_step(lf_ctx* c, int32_t n_images, int32_t width, int32_t height, const float* in_rgba,
                               const float* target_rgba, float lr, void* stream) {
  lf_status st = refine_check(c, n_images, width, height, in_rgba, target_rgba);
  if (st != LF_OK) return st;
  if (!(lr >= 0.0f) || lr > 1.0f) return fail(c, LF_ERR_INVALID_ARG, "bad learning rate");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = refine_backward(c, n_images, width, height, in_rgba, target_rgba, s)) != LF_OK) return st;
  const int t = c->rf.step + 1;
  const double beta1 = 0.9, beta2 = 0.999;
  const float c1 = (float)(1.0 / (1.0 - std::pow(beta1, t))), c2 = (float)(1.0 / (1.0 - std::pow(beta2, t)));
  LF_CUDA(c, launch_refine_adam(rf_params(c), rf_m(c), rf_v(c), rf_grad(c), kRefineParams, lr, beta1, beta2, 1e-8f,
                                c1, c2, s));
  LF_CUDA(c, launch_refine_pack(rf_params(c), static_cast<__nv_bfloat16*>(c->rf.packed.p), s));
  c->rf.step = t;
  return LF_OK;
}

lf_status lf_render_refined(lf_ctx* c, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                            float* const* out_rgba, void* stream) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (!c->rf.loaded) return lf_render(c, n_eyes, eyes, intr, out_rgba, stream);  // the plain method
  if (n_eyes < 1 || n_eyes > c->cfg.max_eyes || !eyes || !intr || !out_rgba)
    return fail(c, LF_ERR_INVALID_ARG, "bad eye arguments");
  for (int e = 0; e < n_eyes; ++e)
    if (!out_rgba[e] || !aligned16(out_rgba[e]))
      return fail(c, LF_ERR_INVALID_ARG, "output images must be non-null and 16-byte aligned (RGBA texels)");
  size_t total = 0;
  std::vector<size_t> off(n_eyes);
  for (int e = 0; e < n_eyes; ++e) {
    if (intr[e].width < 0 || intr[e].height < 0) return fail(c, LF_ERR_INVALID_ARG, "bad eye size");
    off[e] = total;
    total += (size_t)intr[e].width * intr[e].height * 4;
  }
  LF_CUDA(c, cudaSetDevice(c->device));
  LF_CUDA(c, ensure(c->rf.frame, sizeof(float) * std::max<size_t>(total, 4)));
  std::vector<float*> tmp(n_eyes);
  for (int e = 0; e < n_eyes; ++e) tmp[e] = static_cast<float*>(c->rf.frame.p) + off[e];
  lf_status st = lf_render(c, n_eyes, eyes, intr, tmp.data(), stream);
  if (st != LF_OK) return st;
  return refine_eyes(c, n_eyes, intr, tmp.data(), out_rgba, static_cast<cudaStream_t>(stream), !c->cfg.timing);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Frames delivered to host memory (lf_render_host, lf_host_wait).
//
// Frame k renders on the caller's stream into device slot k % kHostSlots,
// with that slot's own counter block; the context's copy stream waits for the
// render and copies the images and the error word to host memory.  The copy
// of frame k therefore overlaps the render of frame k + 1, and a later
// frame's counter reset cannot erase frame k's error word before it is read.
// A slot is reused only after the host has seen its previous frame delivered,
// which also bounds the frames in flight.

namespace {

lf_status host_pipe_init(lf_ctx* c) {
  auto& H = c->hp;
  if (!H.copy) LF_CUDA(c, cudaStreamCreateWithFlags(&H.copy, cudaStreamNonBlocking));
  for (int k = 0; k < kHostSlots; ++k) {
    if (!H.rendered[k]) LF_CUDA(c, cudaEventCreateWithFlags(&H.rendered[k], cudaEventDisableTiming));
    if (!H.copied[k]) LF_CUDA(c, cudaEventCreateWithFlags(&H.copied[k], cudaEventDisableTiming));
  }
  LF_CUDA(c, ensure(H.counters, kCounterBlock * kHostSlots));
  if (!H.err) LF_CUDA(c, cudaMallocHost((void**)&H.err, sizeof(uint32_t) * kHostSlots));
  return LF_OK;
}

// Wait until the oldest undelivered frame is in host memory; collect its error bits.
lf_status host_deliver_oldest(lf_ctx* c) {
  auto& H = c->hp;
  const int slot = (int)(H.delivered % kHostSlots);
  LF_CUDA(c, cudaEventSynchronize(H.copied[slot]));
  H.err_acc |= H.err[slot];
  ++H.delivered;
  return LF_OK;
}

// Enqueue the render of one frame into `slot` and its copy to host memory.
lf_status host_enqueue(lf_ctx* c, int slot, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                       float* const* host_rgba, const std::vector<size_t>& off, const std::vector<size_t>& bytes,
                       lf_host_form form, cudaStream_t s) {
  const bool refined = form == LF_HOST_REFINED && c->rf.loaded;
  auto& H = c->hp;
  unsigned char* img = static_cast<unsigned char*>(H.image[slot].p);
  std::vector<float*> dev(n_eyes), target(n_eyes);
  for (int e = 0; e < n_eyes; ++e) dev[e] = target[e] = reinterpret_cast<float*>(img + off[e]);
  if (refined) {  // render into the context's scratch image, refine into the slot
    LF_CUDA(c, ensure(c->rf.frame, off[n_eyes - 1] + bytes[n_eyes - 1]));
    for (int e = 0; e < n_eyes; ++e)
      target[e] = reinterpret_cast<float*>(static_cast<unsigned char*>(c->rf.frame.p) + off[e]);
  }
  lf_status st;
  Layout L;
  if ((st = make_layout(c, n_eyes, eyes, intr, target.data(), L)) != LF_OK) return st;
  if ((st = ensure_scratch(c, n_eyes, L.total_tiles)) != LF_OK) return st;
  if ((st = stage_eyes(c, L, s)) != LF_OK) return st;
  FrameArgs a = frame_args(c, L);
  unsigned char* counters = static_cast<unsigned char*>(H.counters.p) + kCounterBlock * slot;
  use_counters(a, counters);
  if (form == LF_HOST_BATCH && (st = ensure_persistent_blocks(c)) != LF_OK) return st;
  // lf_get_stats does not report host-delivered frames: no timing events
  if ((st = enqueue_frame(c, a, false, form == LF_HOST_BATCH, s, false)) != LF_OK) return st;
  if (refined && (st = refine_eyes(c, n_eyes, intr, target.data(), dev.data(), s, true)) != LF_OK) return st;
  LF_CUDA(c, cudaEventRecord(H.rendered[slot], s));
  LF_CUDA(c, cudaStreamWaitEvent(H.copy, H.rendered[slot], 0));
  for (int e = 0; e < n_eyes; ++e)
    LF_CUDA(c, cudaMemcpyAsync(host_rgba[e], dev[e], bytes[e], cudaMemcpyDeviceToHost, H.copy));
  LF_CUDA(c, cudaMemcpyAsync(&H.err[slot], counters + 8, sizeof(uint32_t), cudaMemcpyDeviceToHost, H.copy));
  LF_CUDA(c, cudaEventRecord(H.copied[slot], H.copy));
  return LF_OK;
}

}  // namespace

extern "C" {

lf_status lf_render_host(lf_ctx* c, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                         float* const* host_rgba, lf_host_form form, int64_t* frame, void* stream) {
  lf_status st = check_ready(c);
  if (st != LF_OK) return st;
  if (form != LF_HOST_PLAIN && form != LF_HOST_REFINED && form != LF_HOST_BATCH)
    return fail(c, LF_ERR_INVALID_ARG, "unknown lf_host_form");
  if (n_eyes < 1 || n_eyes > c->cfg.max_eyes || !eyes || !intr || !host_rgba)
    return fail(c, LF_ERR_INVALID_ARG, "bad eye arguments");
  std::vector<size_t> off(n_eyes), bytes(n_eyes);
  size_t total = 0;
  for (int e = 0; e < n_eyes; ++e) {
    if (!host_rgba[e]) return fail(c, LF_ERR_INVALID_ARG, "null host output pointer");
    if (intr[e].width < 1 || intr[e].height < 1 || intr[e].width > 32767 || intr[e].height > 32767)
      return fail(c, LF_ERR_INVALID_ARG, "eye size out of range");
    off[e] = total;
    bytes[e] = sizeof(float) * 4 * (size_t)intr[e].width * intr[e].height;
    total += (bytes[e] + 255) & ~(size_t)255;
  }
  if ((st = host_pipe_init(c)) != LF_OK) return st;
  auto& H = c->hp;
  while (H.issued - H.delivered >= kHostSlots)
    if ((st = host_deliver_oldest(c)) != LF_OK) return st;
  const int slot = (int)(H.issued % kHostSlots);
  LF_CUDA(c, ensure(H.image[slot], total));  // the slot's previous frame has been delivered
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = host_enqueue(c, slot, n_eyes, eyes, intr, host_rgba, off, bytes, form, s);
  if (st != LF_OK) {
    // leave nothing of the frame running: the caller may free its buffers
    cudaStreamSynchronize(s);
    cudaStreamSynchronize(H.copy);
    cudaGetLastError();
    return st;
  }
  if (frame) *frame = H.issued;
  ++H.issued;
  return LF_OK;
}

lf_status lf_host_wait(lf_ctx* c, int64_t frame, uint32_t* error_word) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (error_word) *error_word = 0;
  auto& H = c->hp;
  if (frame >= H.issued) return fail(c, LF_ERR_INVALID_ARG, "lf_host_wait: no such frame has been issued");
  const int64_t upto = frame < 0 ? H.issued : frame + 1;
  if (H.delivered < upto) LF_CUDA(c, cudaSetDevice(c->device));
  while (H.delivered < upto) {
    lf_status st = host_deliver_oldest(c);
    if (st != LF_OK) return st;
  }
  const uint32_t err = H.err_acc;
  H.err_acc = 0;
  if (error_word) *error_word = err;
  if (err & kErrPoolOverflow) return fail(c, LF_ERR_CAPACITY, "a frame delivered to host memory overflowed its scratch");
  return LF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Prefiltering (lf_prefilter): Sec. 5.1, Eq. 5.  The host places each
// sample's aperture point (FP64), renders the dense model from it for all
// samples of a view in one lf_render_batch call on the dense context, and the
// accumulation kernel (lf_prefilter.cu) forms the ratio per pixel.

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kApertureInset = 1e-5;  // fraction of R by which aperture points sit inside the sphere

// Lanczos-2: sinc(x) sinc(x / 2) for |x| < 2, sinc(x) = sin(pi x) / (pi x).
double lanczos2(double x) {
  if (std::fabs(x) >= 2.0) return 0.0;
  if (x == 0.0) return 1.0;
  const double p = kPi * x;
  return (std::sin(p) / p) * (std::sin(0.5 * p) / (0.5 * p));
}

void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

void normalize3(double* v) {
  const double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int k = 0; k < 3; ++k) v[k] /= n;
}

// World position of aperture sample (a, b) on view V's disk: on the capture
// sphere (centre C, radius R) at chord distance r sqrt(a) from the disk
// centre's radial projection, at angle 2 pi b from the image x axis in the
// tangent plane, pulled kApertureInset R toward C.
void aperture_point(const ViewStatic& V, const double* C, double R, double a, double b, double* o) {
  double n[3] = {V.disk_c[0] - C[0], V.disk_c[1] - C[1], V.disk_c[2] - C[2]};
  normalize3(n);
  const double xc[3] = {V.R[0], V.R[3], V.R[6]};  // image x axis (first column of R)
  const double xn = xc[0] * n[0] + xc[1] * n[1] + xc[2] * n[2];
  double x[3] = {xc[0] - xn * n[0], xc[1] - xn * n[1], xc[2] - xn * n[2]};
  normalize3(x);
  double y[3];
  cross3(n, x, y);
  const double chord = (double)V.disk_r * std::sqrt(a);
  const double theta = 2.0 * std::asin(std::min(1.0, chord / (2.0 * R)));
  const double phi = 2.0 * kPi * b;
  const double ct = std::cos(theta), st = std::sin(theta), cp = std::cos(phi), sp = std::sin(phi);
  for (int k = 0; k < 3; ++k)
    o[k] = C[k] + (1.0 - kApertureInset) * R * (ct * n[k] + st * (cp * x[k] + sp * y[k]));
}

// The render camera of sample q for view V (pose at the aperture point, the
// view's rotation, intrinsics times S) and the kernel's record (o' = R^T (o - t)
// in the view's camera frame, rho sigma).
void prefilter_camera(const lf_ctx* c, const ViewStatic& V, const lf_prefilter_sample& q, int S, lf_pose* P,
                      lf_intrinsics* K, float* rec) {
  double o[3];
  aperture_point(V, c->sphere_c, c->sphere_r, q.a, q.b, o);
  std::memcpy(P->R, V.R, sizeof(P->R));
  for (int r = 0; r < 3; ++r) P->t[r] = o[r];
  *K = lf_intrinsics{S * V.fx, S * V.fy, S * V.cx, S * V.cy, S * c->src_w, S * c->src_h};
  if (rec) {
    for (int r = 0; r < 3; ++r)
      rec[r] = (float)(V.R[0 * 3 + r] * (o[0] - V.t[0]) + V.R[1 * 3 + r] * (o[1] - V.t[1]) +
                       V.R[2 * 3 + r] * (o[2] - V.t[2]));
    rec[3] = (float)((1.0 - std::sqrt((double)q.a)) * lanczos2(q.ds) * lanczos2(q.dt));
  }
}

bool prefilter_sample_ok(const lf_prefilter_sample& q) {
  return q.a >= 0.0f && q.a <= 1.0f && q.b >= 0.0f && q.b <= 1.0f && q.ds >= -2.0f && q.ds <= 2.0f &&
         q.dt >= -2.0f && q.dt <= 2.0f;
}

}  // namespace

extern "C" lf_status lf_prefilter_cameras(lf_ctx* c, int32_t view, int32_t n_samples,
                                          const lf_prefilter_sample* samples, int32_t supersample, lf_pose* poses,
                                          lf_intrinsics* intr) {
  if (!c) return LF_ERR_INVALID_ARG;
  if (c->n_views <= 0) return fail(c, LF_ERR_STATE, "views not loaded");
  if (view < 0 || view >= c->n_views || n_samples < 0 || (n_samples > 0 && (!samples || !poses || !intr)))
    return fail(c, LF_ERR_INVALID_ARG, "bad prefilter camera arguments");
  if (supersample < 1 || supersample > 4 || (int64_t)supersample * std::max(c->src_w, c->src_h) > 32767)
    return fail(c, LF_ERR_INVALID_ARG, "supersample must be 1 .. 4 with renders up to 32767 pixels");
  for (int j = 0; j < n_samples; ++j) {
    if (!prefilter_sample_ok(samples[j])) return fail(c, LF_ERR_INVALID_ARG, "sample out of range");
    prefilter_camera(c, c->views_host[view], samples[j], supersample, poses + j, intr + j, nullptr);
  }
  return LF_OK;
}

extern "C" lf_status lf_prefilter(lf_ctx* c, lf_ctx* dense, int32_t first_view, int32_t n_views, int32_t n_samples,
                                  const lf_prefilter_sample* samples, int32_t supersample, float* out_rgba,
                                  void* stream) {
  lf_status st = check_ready(c);
  if (st != LF_OK) return st;
  if (!dense || dense == c) return fail(c, LF_ERR_INVALID_ARG, "the dense model needs a context of its own");
  if (dense->n_views <= 0 || dense->G <= 0) return fail(c, LF_ERR_STATE, "the dense context has no views or meshes");
  if (dense->device != c->device) return fail(c, LF_ERR_INVALID_ARG, "the two contexts are on different devices");
  if (n_samples < 1 || n_samples > dense->cfg.max_eyes)
    return fail(c, LF_ERR_INVALID_ARG, "n_samples must be 1 .. the dense context's max_eyes");
  if (first_view < 0 || n_views < 0 || (int64_t)first_view + n_views > c->n_views)
    return fail(c, LF_ERR_INVALID_ARG, "view range out of bounds");
  if (!samples || (n_views > 0 && !out_rgba)) return fail(c, LF_ERR_INVALID_ARG, "null argument");
  if (!aligned16(out_rgba)) return fail(c, LF_ERR_INVALID_ARG, "the output images must be 16-byte aligned (RGBA texels)");
  if (supersample < 1 || supersample > 4 || (int64_t)supersample * std::max(c->src_w, c->src_h) > 32767)
    return fail(c, LF_ERR_INVALID_ARG, "supersample must be 1 .. 4 with renders up to 32767 pixels");
  for (int j = 0; j < n_samples; ++j)
    if (!prefilter_sample_ok(samples[j]))
      return fail(c, LF_ERR_INVALID_ARG, "sample out of range (a, b in [0, 1]; ds, dt in [-2, 2])");
  if (n_views == 0) return LF_OK;
  const int J = n_samples, S = supersample, W = c->src_w, H = c->src_h, Ws = S * W, Hs = S * H;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // per (view, sample): the render's pose and the kernel's (o', rho sigma); per sample: (ds, dt)
  std::vector<lf_pose> poses((size_t)n_views * J);
  std::vector<lf_intrinsics> intr((size_t)n_views * J);
  std::vector<float> params((size_t)n_views * J * 4 + (size_t)J * 2);
  float* offs = params.data() + (size_t)n_views * J * 4;
  for (int j = 0; j < J; ++j) {
    offs[2 * j] = samples[j].ds;
    offs[2 * j + 1] = samples[j].dt;
  }
  for (int k = 0; k < n_views; ++k)
    for (int j = 0; j < J; ++j) {
      const size_t i = (size_t)k * J + j;
      prefilter_camera(c, c->views_host[first_view + k], samples[j], S, &poses[i], &intr[i], &params[i * 4]);
    }
  LF_CUDA(c, ensure(c->pf.renders, sizeof(float) * 4 * (size_t)J * Ws * Hs));
  LF_CUDA(c, ensure(c->pf.params, sizeof(float) * params.size()));
  LF_CUDA(c, ensure(c->pf.err, 256));
  LF_CUDA(c, cudaMemcpyAsync(c->pf.params.p, params.data(), sizeof(float) * params.size(), cudaMemcpyHostToDevice, s));
  LF_CUDA(c, cudaMemsetAsync(c->pf.err.p, 0, sizeof(uint32_t), s));
  std::vector<float*> outs(J);
  for (int j = 0; j < J; ++j) outs[j] = static_cast<float*>(c->pf.renders.p) + (size_t)j * Ws * Hs * 4;
  for (int k = 0; k < n_views; ++k) {
    const ViewStatic& V = c->views_host[first_view + k];
    st = lf_render_batch(dense, J, poses.data() + (size_t)k * J, intr.data() + (size_t)k * J, outs.data(), stream);
    if (st != LF_OK) {
      cudaStreamSynchronize(s);
      return fail(c, st, (std::string("dense render: ") + dense->last_error).c_str());
    }
    PrefilterArgs a;
    std::memset(&a, 0, sizeof(a));
    a.view = first_view + k;
    a.W = W; a.H = H; a.G = c->G;
    a.mesh_format = c->mesh_fmt;
    a.depth = c->depth.p;
    a.tab_a = static_cast<const float*>(c->tab_a.p);
    a.tab_b = static_cast<const float*>(c->tab_b.p);
    a.views = static_cast<const ViewStatic*>(c->views.p);
    a.fx = (float)V.fx; a.fy = (float)V.fy; a.cx = (float)V.cx; a.cy = (float)V.cy;
    a.Ws = Ws; a.Hs = Hs;
    a.fxs = (float)(S * V.fx); a.fys = (float)(S * V.fy); a.cxs = (float)(S * V.cx); a.cys = (float)(S * V.cy);
    a.n_samples = J;
    a.sample = static_cast<const float4*>(c->pf.params.p) + (size_t)k * J;
    a.offset = reinterpret_cast<const float2*>(static_cast<const float*>(c->pf.params.p) + (size_t)n_views * J * 4);
    a.renders = static_cast<const float4*>(c->pf.renders.p);
    a.out = reinterpret_cast<float4*>(out_rgba) + (size_t)k * W * H;
    a.dense_error = reinterpret_cast<const uint32_t*>(static_cast<const unsigned char*>(dense->small.p) + 8);
    a.error = static_cast<uint32_t*>(c->pf.err.p);
    LF_CUDA(c, launch_prefilter_accumulate(a, s));
  }
  LF_CUDA(c, cudaStreamSynchronize(s));
  uint32_t err = 0;
  LF_CUDA(c, cudaMemcpy(&err, c->pf.err.p, sizeof(err), cudaMemcpyDeviceToHost));
  if (err & kErrPoolOverflow)
    return fail(c, LF_ERR_CAPACITY, "a dense render overflowed its scratch: raise the dense context's tri_capacity");
  return LF_OK;
}
