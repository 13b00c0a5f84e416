// lf_internal.h - device data layout shared by the library's kernels and host code.
//
// HBM layout (all resident for the context's lifetime):
//   ViewStatic[n_views]           pose, intrinsics, disk, storage scales
//   textures                      n_views x H x W texels, row-major, one of
//                                 float4 / uchar4 / 4 x bf16 / 4 x e4m3
//   depth grids                   n_views x G x G (float, or half + per-view origin)
//   grid ray tables a_j, b_k      n_views x G floats each
// Per call (scratch, reused in stream order):
//   EyeParams[n_eyes]             eye pose, intrinsics, tile range, output pointer
//   ViewRec[n_eyes x n_views]     composed transforms, footprint, triangle segment
//   tile masks                    per eye tile, one bit per view whose disk footprint
//                                 overlaps the tile (ceil(n_views/32) words)
//   EyeFloat[n_eyes]              the eye's FP32 constants (rounded once, on the device)
//   TriRec pool                   set-up (sub-)triangles, one contiguous segment per
//                                 (eye, view), grouped by 4x4-cell clusters
//   bin offsets / bin entries     per (eye, view): its triangles binned into the screen
//                                 tiles of its footprint (pool indices), plus a list of
//                                 triangles spanning more than bin_max_tiles tiles
// Two-level progressive rendering (lf_set_levels): the coarse views' textures,
// a pool of pages holding fine views' textures, a per-view texture table and
// page table, per coarse view the fine views whose disks overlap it (CSR), and
// per call the exact view selection and the drawn-view bits of each eye.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/lf.h"

namespace lfk {

constexpr int kMaxTileThreads = 256;
constexpr int kSnapLimit = 1 << 29;     // |snapped| must stay below 2^29 subpixels
constexpr int kBigEdge = 1 << 22;       // edge deltas from 2^22 subpixels use the int64 path
constexpr int kQClamp = 1 << 28;        // clamp of the per-tile edge offset in the int32 path
constexpr int kBinSmemTiles = 8192;     // footprint tiles a binning CTA counts in shared memory (at least)

#ifdef __CUDACC__
// Programmatic dependent launch (sm_90 and later).  A kernel launched with the
// programmatic stream serialization attribute may start before the previous
// kernel of its stream has completed; griddep_wait() returns once that kernel
// has completed and its memory is visible (at once when the launch had no such
// attribute).  griddep_release() lets the next kernel of the stream launch as
// soon as every block of this one has executed it (or exited).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif

// device error bits
constexpr uint32_t kErrPoolOverflow = 1u << 0;
constexpr uint32_t kErrRecordOverflow = 1u << 1;

struct ViewStatic {
  double R[9];
  double t[3];
  double fx, fy, cx, cy;
  float disk_c[3];
  float disk_r;
  float depth_origin;   // z0 for the FP16-offset mesh format
  float tex_scale;      // decode scale for FP8 textures
  int32_t pad[2];
  float disk_ext[4];    // oval extents (+u, -u, +v, -v) in metres when ovals are set
};

struct EyeParams {
  double R[9];
  double t[3];
  double fx, fy, cx, cy;
  int32_t W, H;
  int32_t tiles_x, tiles_y;
  int32_t tile_base;    // first tile index of this eye in the call's flattened tile range
  int32_t pad;
  float* out;           // H x W float4
};

// FP32 copies of an eye's parameters feeding the integer decisions, each the
// round-to-nearest of the FP64 value (of t - C and R^2 for the sphere terms).
struct __align__(16) EyeFloat {
  float R[9];
  float o[3];           // eye centre minus capture-sphere centre
  float fx, fy, cx, cy;
  float R2;             // capture-sphere radius squared
  float pad[3];
};

struct __align__(16) ViewRec {
  float Hm[12];         // eye pixel (x, y, 1) and 1/z -> source (u, v) homogeneous; Hm 3x3 then hv
  float cc[4];          // disk centre relative to the capture sphere centre, then r^2
  float inv_r;
  int32_t tri_base;     // first set-up triangle of this (eye, view) in the pool
  int32_t tri_count;    // its set-up triangles
  int32_t bin_off;      // its tile bins in the offset pool (-1: none): bntx*bnty+1 entry offsets
  int32_t bb[4];        // conservative footprint in pixels, inclusive; bb[0] > bb[2] when empty
  int16_t btx0, bty0, bntx, bnty;  // the tiles of the footprint box
  int32_t big_base;     // entries of the triangles spanning more than kBinMaxTiles tiles
  int32_t big_count;
  float Mf[12];         // camera -> eye rotation (3x3) then translation, FP32
  // oval disk (Sec. 4.4) in the eye frame, each the FP32 rounding of an FP64
  // value: plane normal n, u and v axes x, y (columns of M = R_eye^T R_i),
  // k = n.c', u0 = x.c', v0 = y.c' (c' the disk centre), reciprocal extents
  float ov_n[3], ov_x[3], ov_y[3], ov_k, ov_u0, ov_v0;
  float ov_ru[2], ov_rv[2];   // 1 / e_u+, 1 / e_u-, 1 / e_v+, 1 / e_v-
  const void* tex;            // the view's first texel (a pool page for a fine view of a two-level frame)
};

struct __align__(16) TriRec {
  int16_t bx0, by0, bx1, by1;   // pixel-centre bounding box clipped to screen and footprint
  int32_t x[3], y[3];           // snapped vertices (1/256 px), positively oriented
  float ia, ib, ic;             // 1/z = ia ex + ib ey + ic
  int32_t id_tl;                // parent id << 3 | top-left flags of edges 0..2
};
static_assert(sizeof(TriRec) == 48, "TriRec layout");

constexpr int kClusterCells = 4;         // cells per cluster side (set-up works cluster by cluster)
constexpr int kBinMaxTiles = 16;         // the static-scratch render's cap on tiles binned per triangle
constexpr int kMaxGridForSetup = 257;    // (G-1)/4 squared clusters must fit the set-up kernel's table

struct GridTables {
  const float* a;   // n_views x G
  const float* b;   // n_views x G
};

struct FrameArgs {
  const EyeParams* eyes;
  int32_t n_eyes;
  int32_t n_views;
  int32_t src_w, src_h;
  int32_t G;
  int32_t mask_words;
  int32_t tex_format;
  int32_t mesh_format;
  int32_t disk_mode;       // 0: round disks on the capture sphere; 1: ovals (Sec. 4.4)
  float z_near;
  double sphere_c[3];
  double sphere_r;
  const ViewStatic* views;
  const void* textures;
  const void* depth;
  GridTables tables;
  ViewRec* vrecs;
  uint32_t* tile_masks;
  EyeFloat* eyes_f;
  TriRec* pool;
  int64_t pool_capacity;
  unsigned long long* pool_counter;
  int32_t* bin_offsets;
  int64_t bin_offsets_capacity;
  unsigned long long* bin_offsets_counter;
  int32_t* bin_entries;
  int64_t bin_entries_capacity;
  int32_t bin_max_tiles;   // triangles spanning more tiles go to their view's list of big ones
  unsigned long long* bin_entries_counter;
  uint32_t* error_word;
  uint8_t* active;         // n_eyes x n_views view-selection flags
  int32_t total_tiles;
  int32_t tile_w, tile_h;
  // inspection outputs (one eye)
  lf_frag_record* records;
  int32_t max_records;
  int32_t* counts;
  uint32_t* texel_bits;
  // persistent batch raster
  int32_t* work_counter;
  // two-level progressive rendering (all null / 0 with one level)
  const void* const* tex_table;  // per view: its texels (a pool page for fine views; null when not resident)
  uint32_t* enable_bits;         // n_eyes x mask_words: the views each eye draws
  uint8_t* visible;              // n_eyes x n_views: exact view selection of every view
  const int32_t* page_of_view;   // per fine view: its page, -1 when not resident
  const int32_t* overlap_off;    // per coarse view: its range in overlap_ids (n_views - n_fine + 1 entries)
  const int32_t* overlap_ids;    // fine views whose disks overlap the coarse view's
  int32_t n_fine;                // views [0, n_fine) are the streamed fine level
};

// launchers (return cudaGetLastError())
cudaError_t launch_grid_tables(const ViewStatic* views, int n_views, int src_w, int src_h, int G,
                               float* a, float* b, cudaStream_t s);
cudaError_t launch_convert_textures(const uint8_t* src, void* dst, int64_t n_texels, int fmt,
                                    const float* scale_per_texel_view, int64_t texels_per_view,
                                    cudaStream_t s);
cudaError_t launch_view_setup(const FrameArgs& a, cudaStream_t s);
cudaError_t launch_tri_setup(const FrameArgs& a, cudaStream_t s, bool pdl);
cudaError_t launch_raster(const FrameArgs& a, bool inspect, bool persistent, int persistent_blocks,
                          cudaStream_t s, bool pdl = false);
cudaError_t raster_occupancy(int tile_w, int tile_h, int tex_format, int disk_mode, int* blocks_per_sm);
// Two-level frames: the exact view selection of every view into a.visible (the
// raster's disk tests alone), then the drawn views into a.enable_bits, which
// are then ANDed into the tile masks.
cudaError_t launch_select(const FrameArgs& a, cudaStream_t s);
cudaError_t launch_drawn(const FrameArgs& a, cudaStream_t s);
// FP8 textures: per-view scale = max(RGB) / 255 / 448, also stored in views[v].tex_scale.
cudaError_t launch_view_scale(const uint8_t* rgba8, int n_views, int64_t texels_per_view, float* scale,
                              ViewStatic* views, cudaStream_t s);
// FP16-offset meshes: per-view origin z0 = min depth (views[v].depth_origin), half(z - z0) per vertex.
cudaError_t launch_depth_offsets(const float* depth, int n_views, int per_view, void* dst_half, ViewStatic* views,
                                 cudaStream_t s);

// ---------------------------------------------------------------- refinement
// y = x + f(x), f = conv3x3(3->32) . ReLU . conv3x3(32->32) . ReLU . conv3x3(32->3).

constexpr int kRefineParams = 11011;  // W1 864, b1 32, W2 9216, b2 32, W3 864, b3 3
constexpr int kRefineOffW1 = 0, kRefineOffB1 = 864, kRefineOffW2 = 896, kRefineOffB2 = 10112;
constexpr int kRefineOffW3 = 10144, kRefineOffB3 = 11008;
// packed BF16 operands: w1f [32][32], w2f [9][32][32], w3f [9][8][32], w3b [32][32], w2b [9][32][32]
// (the per-layer convolutions, rearranged by them into core-matrix blocks), then the fused kernel's B operands: L1 [3 dy][2 g][32][8] (pair-packed
// taps), L2 [3 dy][2 kc][2 g][96][8], L3 [3 dy][2 kc][2 g][16][8] (kernel columns along N)
constexpr int kPackW1f = 0, kPackW2f = 1024, kPackW3f = 10240, kPackW3b = 12544, kPackW2b = 13568;
constexpr int kPackTc = 22784;
constexpr int kRefinePackedElems = 22784 + 1536 + 9216 + 1536;

enum : int { kConvInRGBA = 0, kConvInBF16 = 1 };
enum : int { kEpiRelu = 0, kEpiMask = 1, kEpiResid = 2, kEpiLoss = 3 };

struct RefineConvArgs {
  int32_t n, H, W;
  const float* src_f;          // kConvInRGBA: n*H*W RGBA (channels 0..2 used)
  const __nv_bfloat16* src_h;  // kConvInBF16: n*H*W*32
  const __nv_bfloat16* wt;     // packed weights of this layer
  const float* bias;           // kEpiRelu: 32; kEpiResid / kEpiLoss: 3
  __nv_bfloat16* out_h;        // kEpiRelu / kEpiMask: n*H*W*32
  const __nv_bfloat16* mask;   // kEpiMask: the ReLU output whose sign gates the gradient
  const float* x;              // kEpiResid / kEpiLoss: the network input (RGBA)
  const float* target;         // kEpiLoss: target RGBA
  float* out_f;                // kEpiResid: refined RGBA; kEpiLoss: dL/dr (RGB, a = 0)
  float* loss;                 // kEpiLoss: += sum of squared errors / (3 N)
  const int32_t* count;        // kEpiLoss: N, pixels valid in input and target
  int32_t* error;              // set (bit 6) if the wait for a tile's MMAs gave up
  uint64_t wait_ns;            // bound on that wait
};

struct RefineWgradArgs {
  int32_t n, H, W;
  int32_t tiles_x, tiles_y, n_tiles, n_ctas;
  const float* g_f;            // mode 3: dL/dr RGBA
  const __nv_bfloat16* g_h;    // modes 1, 2: dL/dz (32 channels)
  const __nv_bfloat16* a_h;    // modes 2, 3: the layer input (32 channels)
  const float* x;              // mode 1: the network input RGBA
  float* partial;              // [n_ctas][segment]
  int32_t* error;              // set (bit 8) if a wait for a chunk's MMAs gave up
  uint64_t wait_ns;            // bound on that wait
};

cudaError_t launch_refine_conv(int in_mode, int cout, int epi, const RefineConvArgs& a, cudaStream_t s);
cudaError_t launch_refine_wgrad(int mode, const RefineWgradArgs& a, cudaStream_t s);
cudaError_t launch_refine_reduce(const float* partial, int n_rows, int seg, float* grad, cudaStream_t s);
cudaError_t launch_refine_count(const float* x, const float* t, int64_t n_pix, int32_t* count, cudaStream_t s);
cudaError_t launch_refine_adam(float* p, float* m, float* v, const float* g, int n, float lr, double beta1,
                               double beta2, float eps, float c1, float c2, cudaStream_t s);
cudaError_t launch_refine_pack(const float* params, __nv_bfloat16* w, cudaStream_t s);
// Fused inference (lf_refine_tc.cu): all three layers per tile, tcgen05 MMAs.
// Image i goes to out + i*h*w*4, except image 1 to out1 when out1 is set; with
// pdl the launch is a programmatic dependent of the kernel before it.
cudaError_t launch_refine_fused(int32_t n, int32_t w, int32_t h, const float* in, float* out, float* out1,
                                const float* params, const __nv_bfloat16* packed, int sm_count, int32_t* error,
                                uint64_t wait_ns, cudaStream_t s, bool pdl);

}  // namespace lfk
