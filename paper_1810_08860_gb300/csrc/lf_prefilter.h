// lf_prefilter.h - the accumulation step of the light field prefilter (Sec. 5.1,
// Eq. 5), shared by lf_prefilter.cu (kernel) and lf_api.cu (host sequencing).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lf_internal.h"

namespace lfk {

struct PrefilterArgs {
  int32_t view;                 // the target view whose pixels are written
  int32_t W, H, G;              // target image size and mesh grid
  int32_t mesh_format;          // lf_mesh_format of the target's depth grids
  const void* depth;            // target depth grids (n_views x G x G)
  const float* tab_a;           // target grid tables: (s_j - cx) / fx per (view, j)
  const float* tab_b;           //                     (t_k - cy) / fy per (view, k)
  const ViewStatic* views;      // target views (FP16-offset origin)
  float fx, fy, cx, cy;         // the view's intrinsics
  int32_t Ws, Hs;               // render size (supersample x W, H)
  float fxs, fys, cxs, cys;     // render intrinsics
  int32_t n_samples;
  const float4* sample;         // per sample: (o'x, o'y, o'z, rho sigma), o' in the view's camera frame
  const float2* offset;         // per sample: (ds, dt)
  const float4* renders;        // n_samples x Hs x Ws RGBA: Lbar from each aperture point
  float4* out;                  // H x W RGBA
  const uint32_t* dense_error;  // error word of the dense renders of this view
  uint32_t* error;              // OR of the dense renders' error words
};

cudaError_t launch_prefilter_accumulate(const PrefilterArgs& a, cudaStream_t s);

}  // namespace lfk
