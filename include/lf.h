/*
 * lf.h - C ABI of a GB300 (sm_103a) renderer for panoramic light fields
 * stored as disk-blended source views with per-view geometry, after
 * Overbeck et al., "A System for Acquiring, Processing, and Rendering
 * Panoramic Light Field Stills for Virtual Reality", TOG 37(6), 2018.
 *
 * The library answers the ray queries of Eq. 1 for every pixel of one or
 * more eye views with the disk-based reconstruction of Eq. 2:
 *
 *     L(o, e) = sum_i I_i(s_i, t_i) rho_i(u_i, v_i) / sum_i rho_i(u_i, v_i)
 *
 * where I_i is a bilinear sample of source view i at the point where the eye
 * ray meets view i's own depth-displaced triangle mesh (Sec. 4.1, 4.5), and
 * rho_i is the linear disk kernel of Sec. 4.1 evaluated at the ray's crossing
 * p of the capture sphere: w_i = max(0, 1 - |p - c_i| / r_i), with disk
 * centre c_i (by default view i's centre of projection) and radius r_i.
 * Each mesh is depth tested against itself only (intra-image occlusion,
 * Sec. 4.2.2); the sums are accumulated in FP32 and normalised (the two
 * passes of Sec. 4.2).
 *
 * Conventions shared by every call:
 *  - A pose is a camera->world rigid transform: R is a row-major 3x3 rotation
 *    whose columns are the camera axes in world coordinates, t is the centre
 *    of projection.  Camera x points right, y down, z forward.
 *  - Intrinsics are pinhole (fx, fy, cx, cy) in pixel units.  Pixel (i, j)
 *    covers [i, i+1) x [j, j+1); its centre is (i + 1/2, j + 1/2).
 *  - Images are row-major, top row first, RGBA with 4 bytes (or 4 floats) per
 *    pixel.  Source alpha is ignored.
 *  - Every entry point returns an lf_status; none throws or aborts.  Calls
 *    that take a stream are asynchronous on it; launch errors are returned at
 *    once, and conditions found on the device (scratch overflow) are returned
 *    by lf_get_stats, which waits for the last call.
 *  - A context is not thread safe; use one context per host thread, and one
 *    stream at a time per context (the library's scratch buffers are reused
 *    in stream order).
 *
 * Ownership: the library copies host inputs before returning (the caller may
 * free them).  Device output buffers belong to the caller.  The library owns
 * its textures, meshes and scratch, which are freed by lf_destroy.
 */
#ifndef LF_H_
#define LF_H_

#include <stdint.h>

#if defined(__GNUC__)
#define LF_API __attribute__((visibility("default")))
#else
#define LF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lf_ctx lf_ctx;

typedef enum {
  LF_OK = 0,
  LF_ERR_INVALID_ARG = 1,  /* a pointer, size or enum value is out of range */
  LF_ERR_CUDA = 2,         /* a CUDA runtime call failed (see lf_last_error) */
  LF_ERR_OOM = 3,          /* a device or pinned allocation failed */
  LF_ERR_STATE = 4,        /* views or meshes not loaded, or loaded with other sizes */
  LF_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  LF_ERR_UNSUPPORTED = 6,  /* a valid request the library does not implement */
  LF_ERR_CAPACITY = 7      /* per-frame scratch too small; raise lf_config.tri_capacity */
} lf_status;

/* Storage of the source textures on the device (accumulation is always FP32). */
typedef enum {
  LF_TEX_F32 = 0,      /* 4 x float per texel, value k/255 (the plain form) */
  LF_TEX_U8 = 1,       /* 4 x uint8 per texel */
  LF_TEX_BF16 = 2,     /* 4 x bfloat16 per texel */
  LF_TEX_FP8E4M3 = 3   /* 4 x FP8 E4M3 per texel times a per-view FP32 scale */
} lf_tex_format;

/* Storage of the per-view depth grids on the device. */
typedef enum {
  LF_MESH_F32_DEPTH = 0,   /* FP32 z-depth per vertex */
  LF_MESH_F16_OFFSET = 1   /* FP16 (z - z0_i) per vertex plus an FP32 origin z0_i per view */
} lf_mesh_format;

typedef struct {
  double R[9];   /* camera->world rotation, row-major */
  double t[3];   /* centre of projection, world */
} lf_pose;

typedef struct {
  double fx, fy, cx, cy;
  int32_t width, height;
} lf_intrinsics;

/* Creation-time configuration.  Zeroed fields take the default in brackets. */
typedef struct {
  int32_t tile_w, tile_h;   /* screen tile in pixels: 16x16, 32x8 or 8x8 [16x16] */
  int32_t max_eyes;         /* eyes per lf_render / lf_render_batch call [2] */
  int32_t timing;           /* 1: bracket each kernel with CUDA events on the call's stream [0] */
  int64_t tri_capacity;     /* set-up triangle records per call [8 Mi]; the triangle
                               bins get max(4 x this, 32 per screen tile) entries */
  float z_near;             /* eye-space near clip plane in metres [0.1] */
  int32_t pad1;
  int64_t wait_limit;       /* bound in nanoseconds (%globaltimer) on each device wait - the
                               fused refinement's mbarrier waits - after which the kernel
                               gives up, reports LF_ERR_TIMEOUT and returns [2e9 = 2 s] */
} lf_config;

/* Counters of the last completed render call on the context. */
typedef struct {
  int32_t n_eyes;
  int32_t n_views;
  int32_t active_views[2];  /* views with a nonzero disk weight at some pixel, eyes 0 and 1 */
  int64_t triangles;        /* triangle pool records the call took: per view its set-up
                               (sub-)triangles, or an upper bound of them (one per candidate
                               triangle, two where two vertices lie in front of z_near) */
  int64_t tiles;            /* screen tiles rasterised */
  uint32_t error_word;      /* device error bits, 0 when clean */
  float ms_view_setup;      /* kernel durations of the last call when lf_config.timing = 1, else 0 */
  float ms_tri_setup;
  float ms_raster;
} lf_stats;

/* One (pixel, view) record of the inspection call: a view whose disk holds
 * the pixel's sphere crossing, its mesh coverage and its depth-test winner. */
typedef struct {
  int32_t view;
  int32_t n_cover;    /* (sub-)triangles whose snapped edges cover the pixel centre */
  int32_t winner;     /* parent triangle id of the depth-test winner, -1 if none */
  int32_t min_id;     /* smallest covering parent id, -1 if none */
  int32_t max_id;     /* largest covering parent id, -1 if none */
  uint32_t id_hash;   /* xor over covering ids of the murmur3 32-bit finaliser of the id */
} lf_frag_record;

/* Defaults for lf_config (fills every field). */
LF_API void lf_config_default(lf_config* cfg);

/* Create a context on CUDA device `device`.  cfg may be NULL for defaults.
 * Errors: LF_ERR_INVALID_ARG (bad device or config), LF_ERR_CUDA. */
LF_API lf_status lf_create(int32_t device, const lf_config* cfg, lf_ctx** out);

/* Free the context and all its device memory.  NULL-safe. */
LF_API void lf_destroy(lf_ctx* ctx);

/*
 * Load the source views (the light field images of Sec. 4.1) and their disks.
 *   n_views     number of views (1 .. 65536)
 *   poses       n_views camera->world poses (host)
 *   intr        n_views intrinsics (host); every view must have the same
 *               width and height (else LF_ERR_UNSUPPORTED)
 *   rgba8       n_views host pointers, each width*height*4 bytes
 *   disk_c      n_views*3 floats, disk centres in world (host), or NULL for
 *               the views' centres of projection (Sec. 4.1 places each disk
 *               at its image's centre of projection)
 *   disk_r      n_views floats, disk radii in metres (host), all > 0
 *   sphere_c    centre of the capture sphere (3 doubles, world)
 *   sphere_r    its radius in metres (> 0); p is the larger-root crossing of
 *               each eye ray with this sphere
 *   fmt         device storage of the textures
 * Replaces any views loaded before (meshes must then be rebuilt); first waits
 * for all work on the device, since renders in flight may read the old views.
 * Blocks until the upload is complete.  Errors: LF_ERR_INVALID_ARG, LF_ERR_OOM,
 * LF_ERR_UNSUPPORTED, LF_ERR_CUDA.
 */
LF_API lf_status lf_load_views(lf_ctx* ctx, int32_t n_views, const lf_pose* poses, const lf_intrinsics* intr,
                        const uint8_t* const* rgba8, const float* disk_c, const float* disk_r,
                        const double sphere_c[3], double sphere_r, lf_tex_format fmt);

/*
 * Switch the loaded views to asymmetric oval disks (Sec. 4.4), or back to
 * round ones (extents NULL).  Disk i then lies in the plane through its
 * centre normal to view i's optical axis, with u and v along the view's image
 * x and y axes; (u, v) is where the eye ray meets that plane (t >= 0), and the
 * oval is the union of four quarter ellipses with semi-axes e_u+ (u >= 0),
 * e_u- (u < 0), e_v+, e_v-:  rho^2 = (u / e_u)^2 + (v / e_v)^2, inside where
 * rho^2 < 1 (decided in FP32), weight w = 1 - rho.  The capture sphere plays no
 * part in this mode.  Sec. 4.4 sizes the extents to reach the farthest
 * Delaunay 1-ring neighbour along each axis (the Python helper oval_extents).
 *   extents  host, n_views x 4 floats (+u, -u, +v, -v) in metres, all > 0
 * Waits for all work on the device first; later renders of every form use
 * the ovals.  lf_load_views resets to round disks.  Errors: LF_ERR_STATE (no
 * views), LF_ERR_INVALID_ARG, LF_ERR_CUDA.
 */
LF_API lf_status lf_set_disk_ovals(lf_ctx* ctx, const float* extents);

/*
 * Build each view's mesh (Sec. 4.5): a grid_n x grid_n grid of vertices (j, k)
 * at source pixel-edge coordinates (j W/(grid_n-1), k H/(grid_n-1)), displaced
 * along the view's pixel rays to the given z-depths, split into two triangles
 * per cell, (j,k)(j+1,k)(j,k+1) and (j+1,k)(j+1,k+1)(j,k+1), with ids
 * 2 (k (grid_n-1) + j) and that plus one.
 *   grid_n   2 .. 257
 *   depth    host, n_views*grid_n*grid_n floats, row k then column j, z-depth
 *            in the view's camera frame (> 0)
 *   fmt      device storage of the depth grids
 * Requires lf_load_views first (else LF_ERR_STATE).  Waits for all work on the
 * device first (renders in flight may read the old meshes); blocks until done.
 */
LF_API lf_status lf_build_view_meshes(lf_ctx* ctx, int32_t grid_n, const float* depth, lf_mesh_format fmt);

/*
 * Render n_eyes eye views (Eq. 1-2) into caller-owned device buffers.
 *   n_eyes    1 .. lf_config.max_eyes (typically 2, a stereo pair)
 *   eyes      n_eyes eye poses (host)
 *   intr      n_eyes eye intrinsics (host); width, height 1 .. 32767
 *   out_rgba  n_eyes device pointers (host array), each height*width*4 floats:
 *             (sum w rgb / sum w, 1) where sum w > 0, else (0, 0, 0, 0)
 *   stream    cudaStream_t to run on (NULL = legacy default stream)
 * Asynchronous.  Errors: LF_ERR_INVALID_ARG, LF_ERR_STATE, LF_ERR_CAPACITY,
 * LF_ERR_CUDA (including a device error left by an earlier call).
 */
LF_API lf_status lf_render(lf_ctx* ctx, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                    float* const* out_rgba, void* stream);

/*
 * Render many eyes of mixed sizes in one launch sequence: a persistent
 * raster kernel takes (eye, tile) work items from a device queue, and the
 * whole sequence is replayed as a CUDA graph captured once per batch layout.
 * Same arguments and output as lf_render; n_eyes up to lf_config.max_eyes.
 * The graph is re-captured when the number or sizes of the eyes change.  With
 * lf_config.timing set, the sequence is launched without the graph (events
 * inside a captured graph cannot be timed) so lf_get_stats can report it.
 */
LF_API lf_status lf_render_batch(lf_ctx* ctx, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                          float* const* out_rgba, void* stream);

/*
 * Inspection form of lf_render for one eye, for testing coverage and view
 * selection: besides the image it writes, per pixel, up to max_records
 * lf_frag_record entries in increasing view order (records[(j*W+i)*max_records
 * + k]) and their count in counts[j*W+i] (which may exceed max_records; the
 * excess is dropped), the per-view selection flags active[v] (1 if view v's
 * disk holds some pixel's sphere crossing), and optionally a bitset over all
 * views' texels (bit v*W*H + y*W + x) marking the texels read by winners'
 * bilinear footprints (caller zeroes it; NULL to skip).  All buffers are
 * device memory owned by the caller.
 */
LF_API lf_status lf_render_inspect(lf_ctx* ctx, const lf_pose* eye, const lf_intrinsics* intr, float* out_rgba,
                            lf_frag_record* records, int32_t max_records, int32_t* counts,
                            uint8_t* active, uint32_t* texel_bits, void* stream);

/*
 * Render one eye like lf_render, without allocating anything.  The paper has
 * no counterpart: this is for callers that cannot call cudaMalloc while they
 * render - a frame loop with a hard deadline, a process whose device memory
 * is reserved up front by another allocator, a plug-in that may not allocate.
 * lf_render grows its scratch with cudaMalloc on first use; this entry point
 * instead takes all per-call scratch from one static device array of about
 * 16.8 MB that every GPU loading the library holds until the process exits.
 *   Limits (else LF_ERR_CAPACITY and a message in lf_last_error): at most 32
 *   loaded views, a mesh grid of at most 33 x 33, at most 8192 screen tiles
 *   (1024 x 512 pixels with 8 x 8 tiles, 1024 x 2048 with 16 x 16).  Within
 *   them the scratch cannot overflow.
 *   eye, intr   host, as for lf_render (one eye)
 *   out_rgba    caller-owned device buffer, height*width*4 floats
 *   stream      cudaStream_t to run on
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  All calls share the array and it
 * keeps the last call's contents (each call clears what must start at zero),
 * so calls whose work overlaps on the GPU - on different streams, or from
 * different contexts on one device - race and must be serialised by the
 * caller.  lf_get_stats does not report these calls.
 */
LF_API lf_status lf_render_static(lf_ctx* ctx, const lf_pose* eye, const lf_intrinsics* intr, float* out_rgba,
                                  void* stream);

/* What lf_render_host renders. */
typedef enum {
  LF_HOST_PLAIN = 0,    /* lf_render */
  LF_HOST_REFINED = 1,  /* lf_render_refined (the plain method if no refiner is loaded) */
  LF_HOST_BATCH = 2     /* lf_render_batch's persistent raster over all eyes, launched without a graph */
} lf_host_form;

/*
 * Frames delivered to host memory: a render (see lf_host_form) followed by
 * the device-to-host copy of its images, pipelined so that the copy of one
 * frame overlaps the rendering of the next - a client that reads its pixels back (an encoder, a
 * compositor on another device, a file writer) pays max(render, copy) per
 * frame instead of their sum.  The paper has no counterpart: its renderer
 * displays from the GPU (Sec. 4.2).
 * The frame renders on `stream` into one of LF_HOST_FRAMES_IN_FLIGHT device
 * image slots the context owns; a copy stream of the context then copies the
 * images, and the frame's device error word, to host memory.
 *   n_eyes, eyes, intr  as for lf_render (1 .. lf_config.max_eyes eyes, mixed sizes allowed)
 *   host_rgba  n_eyes host pointers, each height*width*4 floats (the output
 *              of lf_render).  Pinned memory (cudaHostAlloc, cudaHostRegister)
 *              lets the copy run asynchronously; with pageable memory the call
 *              returns only after its own copy has finished (no overlap).
 *   form       LF_HOST_PLAIN, LF_HOST_REFINED or LF_HOST_BATCH
 *   frame      out (may be NULL): the frame's number, counting from 0 per context
 *   stream     cudaStream_t the render runs on, in order with the caller's work
 * The images of a frame are complete, and its host buffers may be read or
 * reused, once lf_host_wait has returned for that frame or a later one.  When
 * LF_HOST_FRAMES_IN_FLIGHT frames are undelivered, the call first waits for
 * the oldest.  lf_get_stats does not report these frames; lf_host_wait
 * returns their error bits.  Errors: as lf_render, plus LF_ERR_INVALID_ARG for
 * a NULL host pointer or an unknown form.  On an error nothing of the frame is
 * left running.
 */
#define LF_HOST_FRAMES_IN_FLIGHT 3
LF_API lf_status lf_render_host(lf_ctx* ctx, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                                float* const* host_rgba, lf_host_form form, int64_t* frame, void* stream);

/*
 * Wait until frame `frame` of lf_render_host, and every earlier frame, is in
 * host memory (frame < 0: every frame issued so far).  *error_word (may be
 * NULL) receives the OR of the device error bits of the frames delivered since
 * the previous lf_host_wait, including those lf_render_host waited for.
 * Errors: LF_ERR_INVALID_ARG for a frame not yet issued, LF_ERR_CAPACITY if one
 * of those frames overflowed its per-call scratch (raise
 * lf_config.tri_capacity), LF_ERR_CUDA.
 */
LF_API lf_status lf_host_wait(lf_ctx* ctx, int64_t frame, uint32_t* error_word);

/* Outcome of lf_tune_batch. */
typedef struct {
  int32_t tile_w, tile_h;     /* the chosen screen tile (also the size of the per-view bins) */
  int32_t blocks_per_sm;      /* the chosen persistent raster CTAs per SM */
  int32_t n_tried;
  float ms;                   /* mean replay time of the chosen configuration */
  int32_t tried_tile_w[16];
  int32_t tried_tile_h[16];
  int32_t tried_blocks[16];
  float tried_ms[16];         /* mean replay time of each candidate; -1 if it overflowed */
} lf_tuning;

/*
 * Autotune lf_render_batch for one batch layout (the number and sizes of the
 * eyes): for each screen tile shape (16x16, 32x8, 8x8), which also sets the
 * size of the per-view triangle bins, and each persistent raster grid (1, 2,
 * 4 or the occupancy limit of CTAs per SM), capture the batch graph and time
 * `replays` replays with CUDA events on `stream`; keep the fastest on the
 * context (later lf_render, lf_render_batch and lf_render_inspect calls use
 * its tile shape).  A candidate whose replay overflowed the per-call scratch
 * (error word set) is recorded with time -1 and never chosen; if every one
 * overflowed, returns LF_ERR_CAPACITY.  Arguments as for lf_render_batch; the
 * outputs hold the last render.  Blocks until done.  No counterpart in the paper, whose tile
 * size (64x64 image tiles, Sec. 4.2.1) is a fixed streaming unit.
 */
LF_API lf_status lf_tune_batch(lf_ctx* ctx, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                               float* const* out_rgba, int32_t replays, void* stream, lf_tuning* out);

/* ------------------------------------------------------------------------
 * Learned refinement.  Sec. 5 (Eq. 4-5) improves the real-time reconstruction
 * by projecting a higher-quality offline reconstruction (denser light field
 * images, depth maps before simplification) onto it.  A small network learns
 * that projection in image space: for a normalised render x (RGB of an RGBA
 * image from lf_render),
 *     y = x + f(x),  f = conv3x3(3->32) . ReLU . conv3x3(32->32) . ReLU . conv3x3(32->3),
 * zero padding at the image border; pixels with alpha 0 stay (0,0,0,0) and
 * refined pixels get alpha 1.  Weights are used as BF16 on the tensor cores
 * with FP32 accumulation; the context keeps FP32 master weights and Adam
 * moments (Kingma & Ba 2015: beta1 0.9, beta2 0.999, eps 1e-8).
 *
 * Parameter vector (host FP32, LF_REFINE_N_PARAMS entries, in this order):
 *   W1[32][3][3][3], b1[32], W2[32][32][3][3], b2[32], W3[3][32][3][3], b3[3],
 * where W[o][c][ky][kx] multiplies input channel c at pixel offset (ky-1, kx-1).
 * Images are device pointers to n_images x height x width x 4 FP32 (RGBA,
 * row-major, images back to back), owned by the caller.  All calls run on
 * `stream` (NULL = legacy default stream) in order with the caller's work.
 * ------------------------------------------------------------------------ */
#define LF_REFINE_N_PARAMS 11011

typedef enum {
  LF_REFINE_FUSED_TC = 0,    /* one kernel, all three layers per tile, tcgen05 MMAs into TMEM */
  LF_REFINE_MMA_LAYERS = 1   /* three launches (one per layer), tcgen05, hidden maps in HBM */
} lf_refine_kernel;

/* Load refinement weights (copied; the caller keeps `params`).  Resets the
 * Adam moments and step to 0.  Waits for all work on the device first (a
 * refinement in flight may read the old weights).  LF_ERR_INVALID_ARG on a
 * NULL or non-finite parameter. */
LF_API lf_status lf_load_refiner(lf_ctx* ctx, const float* params);

/* Choose the inference kernel of lf_refine and lf_render_refined (default
 * LF_REFINE_MMA_LAYERS).  Training always uses the per-layer kernels.  The
 * fused kernel reads its input through a TMA tensor map: with it, `in_rgba`
 * must be 16-byte aligned (LF_ERR_INVALID_ARG otherwise). */
LF_API lf_status lf_refine_set_kernel(lf_ctx* ctx, lf_refine_kernel kernel);

/* Copy the refiner state to host arrays of LF_REFINE_N_PARAMS floats (any may
 * be NULL): FP32 master weights, the gradient of the last lf_refine_gradients
 * or lf_refine_train_step call, the Adam moments; the Adam step count and the
 * last loss.  Synchronises the device.  LF_ERR_STATE if no refiner is loaded;
 * LF_ERR_TIMEOUT if a wait inside a refinement kernel gave up since the
 * refiner was loaded (its outputs are then incomplete). */
LF_API lf_status lf_get_refiner(lf_ctx* ctx, float* params, float* grad, float* adam_m, float* adam_v,
                                int32_t* step, float* last_loss);

/* out = refined(in) for n_images images of width x height.  `in` and `out`
 * must not overlap (the 3x3 windows read neighbouring tiles).  Sizes up to
 * 2^28 pixels per image and 2^30 in all; 0 images or pixels is a no-op.
 * LF_ERR_STATE if no refiner is loaded. */
LF_API lf_status lf_refine(lf_ctx* ctx, int32_t n_images, int32_t width, int32_t height, const float* in_rgba,
                           float* out_rgba, void* stream);

/* Gradient of the loss with respect to the parameters, left on the context
 * (read it with lf_get_refiner).  The loss is the mean squared error over the
 * RGB channels of the pixels whose alpha is > 0 in both the input and the
 * target, over all n_images pairs.  No pixel valid in both: loss 0, gradient 0. */
LF_API lf_status lf_refine_gradients(lf_ctx* ctx, int32_t n_images, int32_t width, int32_t height,
                                     const float* in_rgba, const float* target_rgba, void* stream);

/* lf_refine_gradients followed by one Adam update with learning rate lr
 * (0 <= lr <= 1) of the master weights and a refresh of their BF16 copies. */
LF_API lf_status lf_refine_train_step(lf_ctx* ctx, int32_t n_images, int32_t width, int32_t height,
                                      const float* in_rgba, const float* target_rgba, float lr, void* stream);

/* lf_render followed by lf_refine of every eye (through a scratch image the
 * context owns; with the fused kernel, two eyes of equal size are refined by
 * one launch).  With no refiner loaded it is lf_render, the plain method. */
LF_API lf_status lf_render_refined(lf_ctx* ctx, int32_t n_eyes, const lf_pose* eyes, const lf_intrinsics* intr,
                                   float* const* out_rgba, void* stream);

/* ------------------------------------------------------------------------
 * Prefiltering the light field images (Sec. 5).  Each image i of the
 * real-time model is replaced by a Monte Carlo estimate (Eq. 5) of the 4D
 * integral of Eq. 4 over the disk D_i (ray origins) and the pixel basis
 * (ray targets on view i's own mesh) of a higher-quality model's ray query:
 *     I'_i(s', t') = sum_j rho_j sigma_j Lbar_j / sum_j rho_j sigma_j.
 * sigma is the separable Lanczos-2 kernel (Sec. 5.1) and rho the linear disk
 * kernel.  The J samples are shared by every pixel of every view.  Sample j
 * puts the ray origin on the capture sphere at chord distance r_i sqrt(a) from
 * the disk centre, at angle 2 pi b from view i's image x axis (uniform in area),
 * 1e-5 R inside the sphere, with weight rho = 1 - sqrt(a); the ray passes
 * through the mesh point of image point (s' + ds, t' + dt), clamped to the
 * image.  Lbar for the rays of one (view, sample), which share their origin,
 * is a render of the dense model (lf_render_batch on `dense`) at that origin
 * with view i's rotation and intrinsics times `supersample`, read by a
 * bilinear filter at each mesh point's projection, on colour premultiplied by
 * the render's alpha.
 * ------------------------------------------------------------------------ */
typedef struct {
  float a, b;    /* aperture: a in [0, 1] (chord r sqrt(a)), b in [0, 1] (angle 2 pi b) */
  float ds, dt;  /* pixel-basis offset in pixels, each in [-2, 2] */
} lf_prefilter_sample;

/*
 * Prefilter views first_view .. first_view + n_views - 1 of the model loaded
 * on `ctx` (views and meshes), with Lbar from the model loaded on `dense` (a
 * second context on the same device, created with max_eyes >= n_samples).
 *   samples     n_samples (1 .. dense max_eyes) samples (host)
 *   supersample render scale, 1 .. 4 (render width and height <= 32767)
 *   out_rgba    device, n_views x H x W x 4 floats, caller-owned: per pixel
 *               (rgb, 1) where the ratio's denominator is > 0, else (0,0,0,0);
 *               not clamped (the Lanczos lobes can overshoot [0, 1])
 *   stream      cudaStream_t to run on
 * The aperture is view i's round disk (radius disk_r) on the capture sphere,
 * also when oval extents are set on `ctx` (uniform samples of a four-quarter
 * oval would need per-quarter area weights in Eq. 5).
 * Uses per-call scratch of n_samples x supersample^2 x W x H x 16 bytes on
 * `ctx`.  Blocks until done.  Errors: LF_ERR_INVALID_ARG, LF_ERR_STATE (either
 * model not loaded), LF_ERR_CAPACITY (a dense render overflowed its scratch:
 * raise the dense context's tri_capacity), LF_ERR_CUDA.
 */
LF_API lf_status lf_prefilter(lf_ctx* ctx, lf_ctx* dense, int32_t first_view, int32_t n_views, int32_t n_samples,
                              const lf_prefilter_sample* samples, int32_t supersample, float* out_rgba, void* stream);

/* The J render cameras lf_prefilter uses for view `view` (host outputs, n_samples
 * each): the pose at each sample's aperture point with the view's rotation, and
 * the view's intrinsics times `supersample`.  Errors: LF_ERR_INVALID_ARG,
 * LF_ERR_STATE. */
LF_API lf_status lf_prefilter_cameras(lf_ctx* ctx, int32_t view, int32_t n_samples, const lf_prefilter_sample* samples,
                                      int32_t supersample, lf_pose* poses, lf_intrinsics* intr);

/* ------------------------------------------------------------------------
 * Page cache for streamed light field images (the tile cache of Sec. 4.2.1
 * with the per-frame decode budget of Sec. 7.2's two-level progressive
 * renderer).  Host-only bookkeeping, no CUDA calls: it decides which of
 * n_items images occupy which of `capacity` device pages; the caller copies
 * each admitted image into its page and renders the coarse level for wanted
 * images left without one.
 * ------------------------------------------------------------------------ */
typedef struct lf_cache lf_cache;

/* n_items >= 1 images, capacity >= 1 pages, all free.  LF_ERR_INVALID_ARG, LF_ERR_OOM. */
LF_API lf_status lf_cache_create(int32_t n_items, int32_t capacity, lf_cache** out);

/* NULL-safe. */
LF_API void lf_cache_destroy(lf_cache* cache);

/*
 * One frame.  `wanted` lists the images the frame needs, most important first
 * (ids in [0, n_items), host).  Resident wanted images stay.  Missing ones are
 * admitted in list order, at most `budget` of them.  Each goes into a free page
 * or else into the page of the earliest admitted image the frame does not want
 * (first in, first out).  Wanted images that find no page stay missing.
 * Outputs (host, caller-owned, room for `budget` entries): the admitted images
 * and their pages, and their count in *n_uploads.  LF_ERR_INVALID_ARG on a bad
 * id or pointer.
 */
LF_API lf_status lf_cache_frame(lf_cache* cache, int32_t n_wanted, const int32_t* wanted, int32_t budget,
                                int32_t* n_uploads, int32_t* upload_items, int32_t* upload_pages);

/* The page of every image after the last frame (-1: not resident), n_items entries (host). */
LF_API lf_status lf_cache_pages(const lf_cache* cache, int32_t* page_of_item);

/* ------------------------------------------------------------------------
 * Two-level progressive rendering (Sec. 7.2), with the image cache of Sec.
 * 4.2.1 on the device.  The loaded views are split into two light fields of
 * the same scene: views [0, n_fine) the fine level, whose images are streamed
 * into a fixed pool of device pages, and views [n_fine, n_views) the coarse
 * level, resident.  Every render call then draws, per eye:
 *   - each fine view the eye selects (its disk holds some pixel's crossing)
 *     whose image is resident in a page;
 *   - each coarse view the eye selects whose disk overlaps (centre distance
 *     below the sum of the radii, FP64) a fine disk the eye selects whose
 *     image is missing - the coarse level "in that region";
 * and Eq. 2 blends whatever mix results.  Residency is per view (the paper
 * streams 64 x 64 tiles).  lf_cache_* decides which images enter which pages.
 * ------------------------------------------------------------------------ */

/* Split the loaded views into the two levels (see above) and give the fine
 * level a pool of n_pages device pages (1 <= n_pages <= n_fine < n_views).
 * The fine images leave the device; every fine view starts not resident.  The
 * coarse level keeps its images.  The split holds until lf_load_views.  Waits
 * for all work on the device.  Errors: LF_ERR_STATE (no views, or levels set
 * already), LF_ERR_INVALID_ARG, LF_ERR_OOM, LF_ERR_CUDA. */
LF_API lf_status lf_set_levels(lf_ctx* ctx, int32_t n_fine, int32_t n_pages);

/* Copy n fine images into pages (the admissions of lf_cache_frame): view
 * views[k] (a fine view) into page pages[k], from host RGBA8 rgba8[k]
 * (width*height*4 bytes, converted to the context's texture format).  The
 * previous image of each page is no longer resident.  No view or page twice
 * in one call.  Waits for `stream` first (renders that read the replaced pages
 * must run on it or be complete) and returns once the pages and the page table
 * are on the device.  Errors: LF_ERR_STATE (no levels), LF_ERR_INVALID_ARG,
 * LF_ERR_CUDA. */
LF_API lf_status lf_upload_pages(lf_ctx* ctx, int32_t n, const int32_t* views, const int32_t* pages,
                                 const uint8_t* const* rgba8, void* stream);

/* The fine views that any eye of the last render call selected, in
 * increasing order - what the next frames want resident (progressive: a frame
 * draws what is resident and asks for what it missed).  Writes up to cap ids
 * to views (host) and their number to *n; LF_ERR_CAPACITY when there are more
 * than cap.  Waits for the last call.  Errors: LF_ERR_STATE (no levels, or no
 * render yet), LF_ERR_INVALID_ARG. */
LF_API lf_status lf_levels_wanted(lf_ctx* ctx, int32_t cap, int32_t* views, int32_t* n);

/* Set lf_config.wait_limit of a live context: each later device wait gives
 * up after wait_ns nanoseconds (0: the default, 2 s).  A wait that gives up
 * leaves that call's output incomplete and makes lf_get_refiner return
 * LF_ERR_TIMEOUT; the context stays usable.  No counterpart in the paper: it
 * bounds the library's own waits (failure detection without hanging a GPU).
 * Errors: LF_ERR_INVALID_ARG for a negative value. */
LF_API lf_status lf_set_wait_limit(lf_ctx* ctx, int64_t wait_ns);

/* Set lf_config.timing of a live context (0 or 1) for the calls that follow.
 * With timing off, lf_render launches the triangle set-up and the raster as
 * programmatic dependents of the kernel before each (a grid's launch overlaps
 * the end of the previous one), which the timing events between the kernels
 * rule out.  No counterpart in the paper.  Errors: LF_ERR_INVALID_ARG for a
 * null context or another value. */
LF_API lf_status lf_set_timing(lf_ctx* ctx, int32_t on);

/* Counters of the last render call; synchronises with its stream. */
LF_API lf_status lf_get_stats(lf_ctx* ctx, lf_stats* out);

/* Human-readable name of a status. */
LF_API const char* lf_status_string(lf_status s);

/* Message of the last error on the context ("" if none). */
LF_API const char* lf_last_error(const lf_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LF_H_ */
