// lf_launch.h - host-side launch helpers shared by the kernel files.
#pragma once

#include <cuda.h>  // CUtensorMap and its enums (the encoder is reached through the runtime)
#include <cuda_runtime.h>

#include <utility>

namespace lfk {

// Launch `kernel` on stream `s`.  With `pdl` the launch carries the
// programmatic stream serialization attribute: it may begin before the
// previous kernel of the stream has completed, so the kernel must execute
// griddep_wait() before it reads anything that kernel (or an earlier
// operation of the stream) wrote.
template <typename... P, typename... Args>
cudaError_t launch_kernel(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                          Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Raise a kernel's dynamic shared memory limit to `bytes` on the current
// device, once per (device, kernel): the attribute belongs to the device's
// context, so a flag kept per process would leave a second device unset.
// Thread safe.  Defined in lf_api.cu.
cudaError_t ensure_dynamic_smem(const void* kernel, int bytes);

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, reached through the runtime (no link
// against libcuda); null when the driver does not provide it.
inline EncodeTiled encode_tiled() {
  static const EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

}  // namespace lfk
