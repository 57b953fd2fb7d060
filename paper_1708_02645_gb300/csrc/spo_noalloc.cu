// spo_eval_noalloc: the binned evaluation with its scratch in a fixed,
// file-scope device array instead of memory the library allocates.
//
// Some callers must not have the library allocate device memory: a host
// application that hands every byte of the GPU to its own pool allocator
// and forbids other allocations, or a time-stepping loop that cannot afford
// the device-wide synchronisation that cudaMalloc and cudaFree may cause in
// the middle of its stream pipeline.  This entry point serves them: it
// allocates nothing on any call, and its scratch (brick counts and offsets,
// one key, slot, permutation entry and sorted position per position) is the
// array below (7.9 MB),
// which exists once per device from the time the library's device code is
// loaded on that device until the process exits.
//
// Limits: at most SPO_NOALLOC_MAX_POSITIONS positions per call and at most
// SPO_NOALLOC_MAX_BRICKS bricks of 4x4x4 cells in the set's grid.
//
// The array is shared by every call on a device and keeps the contents of
// the last call.  Each call first clears the brick counts and the binning's
// ticket (a cudaMemsetAsync on the call's stream, which allocates nothing);
// everything else is overwritten before it is read.  Calls whose work
// overlaps on the GPU (on different streams, or from several host threads)
// race on the array and give wrong results, and may write outside `out`
// (a count raised by the other call moves this call's sorted slots past P);
// the clear confines the damage to the overlapping calls.  Order them, for
// example on one stream.
//
// The strategy is the one spo_eval's AUTO takes for the same set, kind and
// batch size (the gather kernel, in input order or in binned order, or the
// brick kernel), so the outputs are those of spo_eval bit for bit.
//
// The array's device address is looked up once per device and kept for the
// life of the process; after cudaDeviceReset the old address is stale and
// this entry point must not be called again in that process.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>

#include "spo.h"
#include "spo_internal.h"

namespace {

constexpr size_t kMaxPositions = SPO_NOALLOC_MAX_POSITIONS;
constexpr size_t kMaxBricks = SPO_NOALLOC_MAX_BRICKS;

// [counts: kMaxBricks][offsets: kMaxBricks + 1][keys][slots][perm: kMaxPositions ints each]
// [sorted: kMaxPositions float4], every part starting on a 256-byte boundary
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kCountsOff = 0;
constexpr size_t kOffsetsOff = kCountsOff + align256((kMaxBricks + 1) * sizeof(int));   // + ticket
constexpr size_t kKeysOff = kOffsetsOff + align256((kMaxBricks + 1) * sizeof(int));
constexpr size_t kSlotsOff = kKeysOff + align256(kMaxPositions * sizeof(int));
constexpr size_t kPermOff = kSlotsOff + align256(kMaxPositions * sizeof(int));
constexpr size_t kSortedOff = kPermOff + align256(kMaxPositions * sizeof(int));
constexpr size_t kScratchBytes = kSortedOff + align256(kMaxPositions * sizeof(float4));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
spo_status scratch_address(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices)
        return spo_detail::fail(SPO_EUNSUPPORTED, "device %d beyond the %d supported", device,
                                kMaxDevices);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return spo_detail::fail(SPO_ECUDA, "cudaGetSymbolAddress of the scratch array: %s",
                                    cudaGetErrorString(e));
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[device]);
    return SPO_OK;
}

spo_status device_pointer(const void *ptr, int device, const char *name) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
        cudaGetLastError();
        return spo_detail::fail(SPO_EINVAL, "%s is not a CUDA pointer", name);
    }
    if (attr.type == cudaMemoryTypeManaged) return SPO_OK;
    if (attr.type != cudaMemoryTypeDevice || attr.device != device)
        return spo_detail::fail(SPO_EINVAL, "%s must be device memory of device %d", name, device);
    return SPO_OK;
}

}  // namespace

extern "C" spo_status spo_eval_noalloc(const spo_set *set, spo_kind kind, const float *pos,
                                       int64_t P, float *out, void *stream) {
    using spo_detail::fail;
    fail(SPO_OK, "");   // clear the thread's last error message
    if (!set) return fail(SPO_EINVAL, "set is NULL");
    if (kind != SPO_KIND_V && kind != SPO_KIND_VGL && kind != SPO_KIND_VGH)
        return fail(SPO_EINVAL, "invalid kind %d", (int)kind);
    if (P < 0) return fail(SPO_EINVAL, "P = %lld is negative", (long long)P);
    if (P == 0) return SPO_OK;
    if (P > (int64_t)kMaxPositions)
        return fail(SPO_EINVAL, "P = %lld exceeds SPO_NOALLOC_MAX_POSITIONS = %lld", (long long)P,
                    (long long)kMaxPositions);
    const int64_t bricks = (int64_t)set->nbx * set->nby * set->nbz;
    if (bricks > (int64_t)kMaxBricks)
        return fail(SPO_EINVAL, "the grid has %lld bricks, above SPO_NOALLOC_MAX_BRICKS = %lld",
                    (long long)bricks, (long long)kMaxBricks);
    if (!pos || !out) return fail(SPO_EINVAL, "pos or out is NULL");
    if ((reinterpret_cast<uintptr_t>(pos) & 3) || (reinterpret_cast<uintptr_t>(out) & 3))
        return fail(SPO_EINVAL, "pos and out must be 4-byte aligned");

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return fail(SPO_ECUDA, "cudaGetDevice failed");
    if (prev != set->device && cudaSetDevice(set->device) != cudaSuccess)
        return fail(SPO_ECUDA, "cannot select device %d", set->device);
    spo_status st = device_pointer(pos, set->device, "pos");
    if (st == SPO_OK) st = device_pointer(out, set->device, "out");
    unsigned char *base = nullptr;
    if (st == SPO_OK) st = scratch_address(set->device, &base);
    const spo_algo algo = spo_detail::auto_algo(set, kind, P);
    if (st == SPO_OK && algo == SPO_ALGO_GATHER) {
        // input order: no binning, the scratch is not touched
        cudaError_t e = spo_detail::launch_gather(set->storage, kind, spo_detail::view_of(set), pos,
                                                  nullptr, P, out, static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess)
            st = fail(SPO_ECUDA, "spo_eval_noalloc launch: %s", cudaGetErrorString(e));
    } else if (st == SPO_OK) {
        spo_detail::Workspace w;
        w.stream = static_cast<cudaStream_t>(stream);
        w.counts = reinterpret_cast<int *>(base + kCountsOff);
        w.offsets = reinterpret_cast<int *>(base + kOffsetsOff);
        w.keys = reinterpret_cast<int *>(base + kKeysOff);
        w.slots = reinterpret_cast<int *>(base + kSlotsOff);
        w.perm = reinterpret_cast<int *>(base + kPermOff);
        w.sorted = reinterpret_cast<float4 *>(base + kSortedOff);
        w.cap_positions = (int64_t)kMaxPositions;
        w.cap_bins = (int64_t)kMaxBricks;
        // the binning needs counts[0..bricks) and the ticket counts[bricks] at zero
        cudaError_t e = cudaMemsetAsync(w.counts, 0, (size_t)(bricks + 1) * sizeof(int), w.stream);
        if (e == cudaSuccess)
            e = spo_detail::launch_bin(pos, P, set->nx, set->ny, set->nz, set->nbx, set->nby,
                                       set->nbz, w, w.stream);
        if (e == cudaSuccess) {
            if (algo == SPO_ALGO_BRICK)
                e = spo_detail::launch_brick(set->storage, kind, set, pos, w, P, out, w.stream);
            else
                e = spo_detail::launch_gather(set->storage, kind, spo_detail::view_of(set), pos,
                                              w.perm, P, out, w.stream);
        }
        if (e != cudaSuccess)
            st = fail(SPO_ECUDA, "spo_eval_noalloc launch: %s", cudaGetErrorString(e));
    }
    if (prev >= 0 && prev != set->device) cudaSetDevice(prev);
    return st;
}
