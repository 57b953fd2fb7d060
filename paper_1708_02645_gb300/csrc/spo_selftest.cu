// spo_selftest_wait: exercises the failure path of the bounded device-side
// waits without faulting anything.  A probe kernel initialises an mbarrier
// that nothing will ever arrive on (no copy or MMA is issued), waits on it
// with the given limit through the same wait routine the kernels use, and on
// giving up sets bit 0 of the device status word and exits; the host reads
// and clears the word.
#include <cuda_runtime.h>

#include "spo.h"
#include "spo_batch.h"
#include "spo_internal.h"
#include "spo_tma.cuh"

namespace {

using spo_detail::fail;

__global__ void wait_probe_kernel(unsigned long long limit_ns, unsigned int *status) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = spo_dev::smem_addr(&bar);
    if (threadIdx.x == 0) spo_dev::mbar_init(b, 1);
    __syncthreads();
    if (!spo_dev::mbar_wait_limit(b, 0, limit_ns) && threadIdx.x == 0) atomicOr(status, 1u);
}

}  // namespace

extern "C" spo_status spo_selftest_wait(uint64_t limit_ns, void *stream, int *timed_out) {
    fail(SPO_OK, "");
    if (!timed_out) return fail(SPO_EINVAL, "timed_out is NULL");
    if (limit_ns > 1000000000ull) return fail(SPO_EINVAL, "limit above one second");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int *status = nullptr;
    cudaError_t e = spo_detail::device_status_address(&status);
    unsigned int flags = 0;
    // start from a clear word
    if (e == cudaSuccess) e = spo_detail::read_device_status(&flags, true, st);
    if (e == cudaSuccess) {
        wait_probe_kernel<<<1, 32, 0, st>>>(limit_ns, status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = spo_detail::read_device_status(&flags, true, st);
    if (e != cudaSuccess) return fail(SPO_ECUDA, "probe: %s", cudaGetErrorString(e));
    *timed_out = (flags & 1u) ? 1 : 0;
    return SPO_OK;
}
