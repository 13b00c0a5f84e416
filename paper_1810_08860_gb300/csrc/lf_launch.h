// lf_launch.h - host-side launch helpers shared by the kernel files.
#pragma once

#include <cuda_runtime.h>

namespace lfk {

// Raise a kernel's dynamic shared memory limit to `bytes` on the current
// device, once per (device, kernel): the attribute belongs to the device's
// context, so a flag kept per process would leave a second device unset.
// Thread safe.  Defined in lf_api.cu.
cudaError_t ensure_dynamic_smem(const void* kernel, int bytes);

}  // namespace lfk
