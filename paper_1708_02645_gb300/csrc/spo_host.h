// Host-side helpers shared by the C-ABI translation units.  Not part of the
// C ABI.
#pragma once

#include <cuda_runtime.h>

#include "spo.h"

namespace spo_detail {

spo_status fail(spo_status status, const char *fmt, ...);

// Makes `device` current for the scope and restores the caller's device.
class DeviceGuard {
  public:
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
        if (prev_ != device) ok_ = cudaSetDevice(device) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev_ >= 0) cudaSetDevice(prev_);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
    bool ok() const { return ok_; }

  private:
    int prev_ = -1;
    bool ok_ = true;
};

// SPO_ECUDA with the CUDA error's name and text.
inline spo_status cuda_fail(cudaError_t e, const char *what) {
    return fail(SPO_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

}  // namespace spo_detail
