// Binning of positions by brick (a counting sort), so that the brick kernel
// can evaluate all positions whose windows lie in one staged block of the
// table, and the gather kernel can visit positions in spatial order.
//
//   1. bin_count_kernel:  key = brick of the position's cell; slot = rank of
//                         the position within its brick (atomic counter);
//                         the last block to finish (a ticket counter after a
//                         fence) turns the counts into offsets = their
//                         exclusive prefix sum and zeroes the counts (and
//                         the ticket) for the next call, so no block waits
//                         on another and no memset is needed
//   2. bin_scatter_kernel: perm[offsets[key] + slot] = position index, and
//                         the position with its index in the same sorted slot
//   3. bin_records_kernel: when the workspace has room for them, the weight
//                         record of every sorted slot (its position's 36
//                         basis weights, cells and index: the brick kernel's
//                         slot), formed once here instead of once per orbital
//                         tile; one thread per sorted slot, so that a warp's
//                         32 records (5.6 KB) leave as contiguous stores
//                         (written from the scatter, at scattered slots,
//                         they ran at about a fifth of the DRAM rate)
// (bin_scan_kernel is the stand-alone scan, used by the crowd binning.)
//
// The order inside a brick depends on atomic arrival order; every output of
// a position depends only on that position, so results are unaffected.
#include "spo_batch.h"
#include "spo_device.cuh"
#include "spo_internal.h"
#include "spo_tma.cuh"

namespace {

using namespace spo_dev;
using spo_detail::kBrick;

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kCountThreads = 1024;
static_assert(kSlotF4 == spo_detail::kWeightRecordF4, "a weight record is one brick-kernel slot");

// Exclusive scan of counts[0..n) into offsets[0..n] by one block of THREADS
// threads, in chunks of THREADS * kScanItems with a running carry; with
// CLEAR the counts are zeroed once read.  Reads go to L2 (counts were
// updated by other blocks' atomics).
template <int THREADS, bool CLEAR>
__device__ void block_scan_counts(int *counts, int *offsets, int n) {
    __shared__ int warp_sums[THREADS / 32];
    __shared__ int carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < n; base += THREADS * kScanItems) {
        int v[kScanItems];
        int sum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int i = base + tid * kScanItems + k;
            v[k] = i < n ? __ldcg(counts + i) : 0;
            if (CLEAR && i < n) counts[i] = 0;
            sum += v[k];
        }
        int incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int w = lane < THREADS / 32 ? warp_sums[lane] : 0;
            int wi = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, d);
                if (lane >= d) wi += y;
            }
            if (lane < THREADS / 32) warp_sums[lane] = wi - w;   // exclusive prefix of warp totals
        }
        __syncthreads();
        int run = carry_s + warp_sums[warp] + incl - sum;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int i = base + tid * kScanItems + k;
            if (i < n) offsets[i] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == THREADS - 1) carry_s = run;   // last thread holds the chunk total
        __syncthreads();
    }
    if (tid == 0) offsets[n] = carry_s;
}

// Exclusive scan of counts[0..n) into offsets[0..n], one block (the crowd
// binning's counts are cleared by its own memset).
__global__ void __launch_bounds__(kScanThreads)
bin_scan_kernel(int *__restrict__ counts, int *__restrict__ offsets, int n) {
    block_scan_counts<kScanThreads, false>(counts, offsets, n);
}

// counts[0..nbins) must be zero and counts[nbins] (the ticket) zero on entry;
// both are zero again on exit, with offsets[0..nbins] written.
__global__ void __launch_bounds__(kCountThreads)
bin_count_kernel(const float *__restrict__ pos, int64_t P, GridAxis gx, GridAxis gy, GridAxis gz, int nby,
                 int nbz, int nbins, int *__restrict__ counts, int *__restrict__ offsets,
                 int *__restrict__ keys, int *__restrict__ slots, unsigned int *__restrict__ status) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        int cx, cy, cz;
        float t;
        reduce_axis(__ldg(pos + 3 * p + 0), gx, cx, t);
        reduce_axis(__ldg(pos + 3 * p + 1), gy, cy, t);
        reduce_axis(__ldg(pos + 3 * p + 2), gz, cz, t);
        int key = ((cx / kBrick) * nby + cy / kBrick) * nbz + cz / kBrick;
        if (!bounds_ok(key >= 0 && key < nbins, status)) key = 0;   // debug builds
        keys[p] = key;
        slots[p] = atomicAdd(counts + key, 1);
    }
    // the last block to finish scans (no block waits for another)
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();   // this block's counts before its ticket
        last = atomicAdd(counts + nbins, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) {
        grid_dependents_launch();   // after this block's writes (see the scatter)
        return;
    }
    __threadfence();   // every block's counts are visible to this one
    block_scan_counts<kCountThreads, true>(counts, offsets, nbins);
    if (threadIdx.x == 0) counts[nbins] = 0;
    __syncthreads();
    grid_dependents_launch();
}

__global__ void bin_scatter_kernel(const float *__restrict__ pos, const int *__restrict__ keys,
                                   const int *__restrict__ slots, const int *__restrict__ offsets,
                                   int *__restrict__ perm, float4 *__restrict__ sorted, int64_t P,
                                   unsigned int *__restrict__ status) {
    grid_dependency_wait();     // the counts, keys, slots and offsets are complete
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = offsets[keys[p]] + slots[p];
        if (!bounds_ok(i >= 0 && i < P, status)) continue;   // debug builds: a sorted slot in range
        perm[i] = (int)p;
        sorted[i] = make_float4(__ldg(pos + 3 * p), __ldg(pos + 3 * p + 1), __ldg(pos + 3 * p + 2),
                                __int_as_float((int)p));
    }
    // the next grid's CTAs may be scheduled (the brick kernel's issue their
    // table copies) and wait for this grid; the CTA triggers after all its
    // threads' writes, so the wait covers them where a dependency ends at
    // the trigger
    __syncthreads();
    grid_dependents_launch();
}

constexpr int kRecThreads = 256;

// The weight record of every sorted slot, a warp's 32 records formed in
// shared memory and copied out as contiguous 16-byte stores.
__global__ void __launch_bounds__(kRecThreads)
bin_records_kernel(const float4 *__restrict__ sorted, int64_t P, GridAxis gx, GridAxis gy, GridAxis gz,
                   float4 *__restrict__ wrec) {
    __shared__ float4 stage[kRecThreads * kSlotF4];
    grid_dependency_wait();     // the sorted positions are complete
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *ws = stage + warp * 32 * kSlotF4;
    for (int64_t base = (int64_t)blockIdx.x * kRecThreads; base < P; base += (int64_t)gridDim.x * kRecThreads) {
        const int64_t i = base + threadIdx.x, w0 = base + warp * 32;
        if (i < P) {
            const float4 r = sorted[i];
            make_weight_record(r, __float_as_int(r.w), gx, gy, gz, ws + lane * kSlotF4);
        }
        __syncwarp();
        const int64_t n = P - w0 < 32 ? P - w0 : 32;   // records of this warp (none past the end)
        for (int64_t c = lane; c < n * kSlotF4; c += 32) wrec[w0 * kSlotF4 + c] = ws[c];
        __syncwarp();
    }
    __syncthreads();
    grid_dependents_launch();
}

}  // namespace

namespace spo_detail {

cudaError_t launch_scan(const int *counts, int *offsets, int n, cudaStream_t stream) {
    // the stand-alone scan only reads the counts
    bin_scan_kernel<<<1, kScanThreads, 0, stream>>>(const_cast<int *>(counts), offsets, n);
    return cudaGetLastError();
}

cudaError_t launch_bin(const float *pos, int64_t P, int nx, int ny, int nz, int nbx, int nby,
                       int nbz, Workspace &w, cudaStream_t stream) {
    // w.counts holds nbins + 1 zeroed ints (the counts and the ticket); the
    // count kernel leaves them zeroed
    const int nbins = nbx * nby * nbz;
    const int threads = kCountThreads;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((P + threads - 1) / threads, 152 * 16));
    unsigned int *status = nullptr;   // the index checks' flag word (SPO_CHECK_BOUNDS builds)
#ifdef SPO_CHECK_BOUNDS
    if (cudaError_t es = device_status_address(&status); es != cudaSuccess) return es;
#endif
    bin_count_kernel<<<blocks, threads, 0, stream>>>(pos, P, grid_axis(nx), grid_axis(ny), grid_axis(nz), nby,
                                                     nbz, nbins, w.counts, w.offsets, w.keys, w.slots, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // programmatic dependent launch: the scatter is scheduled while the
    // count kernel runs and waits for it in the kernel
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, bin_scatter_kernel, pos, (const int *)w.keys, (const int *)w.slots,
                           (const int *)w.offsets, w.perm, w.sorted, P, status);
    if (e != cudaSuccess || !w.wrec) return e;
    // the records, a programmatic dependent of the scatter as well
    cfg.gridDim = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((P + kRecThreads - 1) / kRecThreads,
                                                                        152 * 8)));
    cfg.blockDim = dim3((unsigned)kRecThreads);
    return cudaLaunchKernelEx(&cfg, bin_records_kernel, (const float4 *)w.sorted, P, grid_axis(nx),
                              grid_axis(ny), grid_axis(nz), w.wrec);
}

}  // namespace spo_detail
