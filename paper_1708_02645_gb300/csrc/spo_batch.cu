// Batched crowds: a plan over several orbital sets that evaluates many
// walkers (each with its own positions, count and output buffer) with one
// binning over all sets' bricks and one launch of the batched brick kernel.
// The plan owns every scratch buffer, so an evaluation allocates nothing and
// the whole sequence can be recorded into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <new>

#include "spo.h"
#include "spo_batch.h"
#include "spo_device.cuh"
#include "spo_host.h"
#include "spo_internal.h"

struct spo_batch {
    int device = 0;
    int nsets = 0;
    const spo_set *sets[spo_detail::kMaxBatchSets] = {};
    spo_dtype storage = SPO_F32;
    int64_t max_positions = 0;
    int max_items = 0;
    int total_bricks = 0;
    int tile = 32;                   // orbital tile of the batched brick kernel
    bool tile_tuned = false;         // tile picked by timing (spo_batch_graph)
    unsigned int *status = nullptr;  // device status word

    // device scratch
    spo_work *d_items = nullptr;     // [max_items]
    int64_t *d_start = nullptr;      // [max_items + 1]
    int *d_item_of = nullptr;        // [max_positions]
    int *counts = nullptr, *offsets = nullptr;    // [total_bricks], [total_bricks + 1]
    int *keys = nullptr, *slots = nullptr;        // [max_positions]
    float4 *sorted = nullptr;                     // [max_positions]
    float4 *wrec = nullptr;                       // [max_positions][11] weight records
    float **dst = nullptr;                        // [max_positions]

    // pinned staging of the item table, and the event after its last copy
    spo_work *h_items = nullptr;
    int64_t *h_start = nullptr;
    cudaEvent_t staged = nullptr;

    // recorded graph
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

using spo_detail::BatchParams;
using spo_detail::BatchSetDesc;
using spo_detail::cuda_fail;
using spo_detail::DeviceGuard;
using spo_detail::fail;
using spo_detail::kBrick;

__global__ void batch_item_of_kernel(const int64_t *__restrict__ start, int nitems,
                                     int *__restrict__ item_of) {
    for (int i = blockIdx.x; i < nitems; i += gridDim.x)
        for (int64_t g = start[i] + threadIdx.x; g < start[i + 1]; g += blockDim.x) item_of[g] = i;
}

__global__ void batch_bin_count_kernel(const spo_work *__restrict__ items,
                                       const int64_t *__restrict__ start,
                                       const int *__restrict__ item_of, int64_t Ptot,
                                       const __grid_constant__ BatchParams bp, int *__restrict__ counts,
                                       int *__restrict__ keys, int *__restrict__ slots) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < Ptot;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int i = item_of[g];
        const int64_t l = g - start[i];
        const spo_work it = items[i];
        const BatchSetDesc &d = bp.sets[it.set];
        int cx, cy, cz;
        float t;
        spo_dev::reduce_axis(__ldg(it.pos + 3 * l + 0), d.gx, cx, t);
        spo_dev::reduce_axis(__ldg(it.pos + 3 * l + 1), d.gy, cy, t);
        spo_dev::reduce_axis(__ldg(it.pos + 3 * l + 2), d.gz, cz, t);
        const int key = d.brick_base + ((cx / kBrick) * d.nby + cy / kBrick) * d.nbz + cz / kBrick;
        keys[g] = key;
        slots[g] = atomicAdd(counts + key, 1);
    }
}

__global__ void batch_scatter_kernel(const spo_work *__restrict__ items,
                                     const int64_t *__restrict__ start,
                                     const int *__restrict__ item_of, int64_t Ptot,
                                     const __grid_constant__ BatchParams bp,
                                     const int *__restrict__ keys, const int *__restrict__ slots,
                                     const int *__restrict__ offsets, float4 *__restrict__ sorted,
                                     float **__restrict__ dst) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < Ptot;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int i = item_of[g];
        const int64_t l = g - start[i];
        const spo_work it = items[i];
        const BatchSetDesc &d = bp.sets[it.set];
        const int idx = offsets[keys[g]] + slots[g];
        sorted[idx] = make_float4(__ldg(it.pos + 3 * l), __ldg(it.pos + 3 * l + 1), __ldg(it.pos + 3 * l + 2),
                                  __int_as_float((int)g));
        dst[idx] = it.out + l * d.rows * d.N;
    }
}

constexpr int kRecThreads = 256;

// The weight record of every sorted slot (the position's basis weights,
// formed once for every orbital tile), one thread per slot: a warp's 32
// records are formed in shared memory and copied out as contiguous 16-byte
// stores (formed in the scatter, at scattered slots, the records were
// written at about a fifth of the DRAM rate).
__global__ void __launch_bounds__(kRecThreads)
batch_records_kernel(const spo_work *__restrict__ items, const int *__restrict__ item_of, int64_t Ptot,
                     const __grid_constant__ BatchParams bp, const float4 *__restrict__ sorted,
                     float4 *__restrict__ wrec) {
    constexpr int R = spo_detail::kWeightRecordF4;
    __shared__ float4 stage[kRecThreads * R];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *ws = stage + warp * 32 * R;
    for (int64_t base = (int64_t)blockIdx.x * kRecThreads; base < Ptot; base += (int64_t)gridDim.x * kRecThreads) {
        const int64_t idx = base + threadIdx.x, w0 = base + warp * 32;
        if (idx < Ptot) {
            const float4 r = sorted[idx];
            const int g = __float_as_int(r.w);
            const BatchSetDesc &d = bp.sets[items[item_of[g]].set];
            spo_dev::make_weight_record(r, g, d.gx, d.gy, d.gz, ws + lane * R);
        }
        __syncwarp();
        const int64_t n = Ptot - w0 < 32 ? Ptot - w0 : 32;   // records of this warp (none past the end)
        for (int64_t c = lane; c < n * R; c += 32) wrec[w0 * R + c] = ws[c];
        __syncwarp();
    }
}

void free_plan(spo_batch *b) {
    cudaFree(b->d_items);
    cudaFree(b->d_start);
    cudaFree(b->d_item_of);
    cudaFree(b->counts);
    cudaFree(b->offsets);
    cudaFree(b->keys);
    cudaFree(b->slots);
    cudaFree(b->sorted);
    cudaFree(b->wrec);
    cudaFree(b->dst);
    if (b->h_items) cudaFreeHost(b->h_items);
    if (b->h_start) cudaFreeHost(b->h_start);
    if (b->staged) cudaEventDestroy(b->staged);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
}


BatchParams make_params(const spo_batch *b, spo_kind kind, int tile, int64_t Ptot) {
    BatchParams bp;
    memset(&bp, 0, sizeof(bp));
    bp.nsets = b->nsets;
    // 32-orbital tiles run on z-adjacent pairs of bricks when every set has
    // the pair map (as the single-set kernel does)
    bp.pair = tile == 32 ? 1 : 0;
    for (int k = 0; k < b->nsets; ++k)
        if (!b->sets[k]->has_pair_map) bp.pair = 0;
    int brick = 0, unit = 0;
    for (int k = 0; k < b->nsets; ++k) {
        const spo_set *s = b->sets[k];
        bp.maps[k] = s->block_map[bp.pair ? 2 : (tile == 64 ? 1 : 0)];
        BatchSetDesc &d = bp.sets[k];
        d.gx = spo_dev::grid_axis(s->nx);
        d.gy = spo_dev::grid_axis(s->ny);
        d.gz = spo_dev::grid_axis(s->nz);
        d.nby = s->nby;
        d.nbz = s->nbz;
        d.nbins = s->nbx * s->nby * s->nbz;
        d.brick_base = brick;
        d.ntiles = (int)((s->N + tile - 1) / tile);
        d.unit_base = unit;
        d.rows = spo_rows(kind);
        d.N = s->N;
        brick += d.nbins;
        unit += (bp.pair ? s->nbx * s->nby * ((s->nbz + 1) / 2) : d.nbins) * d.ntiles;
    }
    bp.total_bricks = brick;
    bp.total_units = unit;
    bp.eager = Ptot >= 4 * (int64_t)brick;
    return bp;
}

// Host checks of an item table; fills start[0..nitems] (prefix sums).
spo_status check_items(const spo_batch *b, const spo_work *items, int nitems, int64_t *start,
                       bool *vec_out) {
    if (nitems < 0 || nitems > b->max_items)
        return fail(SPO_EINVAL, "nitems = %d outside [0, %d]", nitems, b->max_items);
    if (nitems > 0 && !items) return fail(SPO_EINVAL, "items is NULL");
    start[0] = 0;
    *vec_out = true;
    for (int i = 0; i < nitems; ++i) {
        const spo_work &w = items[i];
        if (w.set < 0 || w.set >= b->nsets) return fail(SPO_EINVAL, "item %d: set %d invalid", i, w.set);
        if (w.P < 0) return fail(SPO_EINVAL, "item %d: P < 0", i);
        if (w.P > 0 && (!w.pos || !w.out)) return fail(SPO_EINVAL, "item %d: pos or out is NULL", i);
        if ((reinterpret_cast<uintptr_t>(w.pos) | reinterpret_cast<uintptr_t>(w.out)) & 3)
            return fail(SPO_EINVAL, "item %d: pos and out must be 4-byte aligned", i);
        if ((reinterpret_cast<uintptr_t>(w.out) & 15) || (b->sets[w.set]->N % 4)) *vec_out = false;
        start[i + 1] = start[i] + w.P;
    }
    if (start[nitems] > b->max_positions)
        return fail(SPO_EINVAL, "%lld positions exceed the plan's %lld", (long long)start[nitems],
                    (long long)b->max_positions);
    return SPO_OK;
}

// Queue the evaluation of the item table already on the device.
spo_status queue_work(spo_batch *b, spo_kind kind, int nitems, int64_t Ptot, bool vec_out,
                      cudaStream_t stream) {
    if (Ptot == 0) return SPO_OK;
    const BatchParams bp = make_params(b, kind, b->tile, Ptot);
    cudaError_t e;
    batch_item_of_kernel<<<std::min(nitems, 152 * 8), 256, 0, stream>>>(b->d_start, nitems, b->d_item_of);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->counts, 0, sizeof(int) * (size_t)bp.total_bricks, stream);
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((Ptot + threads - 1) / threads, 152 * 16);
    if (e == cudaSuccess) {
        batch_bin_count_kernel<<<blocks, threads, 0, stream>>>(b->d_items, b->d_start, b->d_item_of,
                                                               Ptot, bp, b->counts, b->keys, b->slots);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = spo_detail::launch_scan(b->counts, b->offsets, bp.total_bricks, stream);
    if (e == cudaSuccess) {
        batch_scatter_kernel<<<blocks, threads, 0, stream>>>(b->d_items, b->d_start, b->d_item_of, Ptot,
                                                             bp, b->keys, b->slots, b->offsets,
                                                             b->sorted, b->dst);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int rb = (int)std::min<int64_t>((Ptot + kRecThreads - 1) / kRecThreads, 152 * 8);
        batch_records_kernel<<<rb, kRecThreads, 0, stream>>>(b->d_items, b->d_item_of, Ptot, bp, b->sorted,
                                                              b->wrec);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = spo_detail::launch_brick_batch(b->storage, kind, b->tile, bp, b->offsets, b->wrec,
                                           b->dst, vec_out, b->status, stream);
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "batched evaluation launch");
}

// Copy the item table to the device through the plan's pinned staging.
spo_status stage_items(spo_batch *b, const spo_work *items, int nitems, const int64_t *start,
                       cudaStream_t stream, bool synchronous) {
    cudaError_t e = cudaEventSynchronize(b->staged);   // the previous copy has left the staging
    if (e != cudaSuccess) return cuda_fail(e, "staging wait");
    if (nitems > 0) memcpy(b->h_items, items, sizeof(spo_work) * (size_t)nitems);
    memcpy(b->h_start, start, sizeof(int64_t) * ((size_t)nitems + 1));
    if (nitems > 0)
        e = cudaMemcpyAsync(b->d_items, b->h_items, sizeof(spo_work) * (size_t)nitems,
                            cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_start, b->h_start, sizeof(int64_t) * ((size_t)nitems + 1),
                            cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->staged, stream);
    if (e == cudaSuccess && synchronous) e = cudaStreamSynchronize(stream);
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "item table upload");
}


}  // namespace

extern "C" {

spo_status spo_batch_create(const spo_set *const *sets, int nsets, int64_t max_positions,
                            int max_items, spo_batch **out) {
    fail(SPO_OK, "");
    if (!out) return fail(SPO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!sets || nsets < 1 || nsets > spo_detail::kMaxBatchSets)
        return fail(SPO_EINVAL, "need 1..%d sets", spo_detail::kMaxBatchSets);
    if (max_positions < 1 || max_positions >= INT_MAX || max_items < 1)
        return fail(SPO_EINVAL, "need 1 <= max_positions < 2^31 and max_items >= 1");
    int64_t bricks = 0;
    for (int k = 0; k < nsets; ++k) {
        if (!sets[k]) return fail(SPO_EINVAL, "set %d is NULL", k);
        if (!sets[k]->has_block_map)
            return fail(SPO_EUNSUPPORTED, "set %d has fewer than 32 padded orbitals", k);
        if (sets[k]->storage != sets[0]->storage || sets[k]->device != sets[0]->device)
            return fail(SPO_EINVAL, "all sets of a plan need one storage type and one device");
        bricks += (int64_t)sets[k]->nbx * sets[k]->nby * sets[k]->nbz;
    }
    if (bricks >= INT_MAX) return fail(SPO_EINVAL, "too many bricks");
    DeviceGuard guard(sets[0]->device);
    if (!guard.ok()) return fail(SPO_ECUDA, "cannot select device %d", sets[0]->device);

    spo_batch *b = new (std::nothrow) spo_batch();
    if (!b) return fail(SPO_ENOMEM, "host allocation of the plan failed");
    b->device = sets[0]->device;
    b->nsets = nsets;
    for (int k = 0; k < nsets; ++k) b->sets[k] = sets[k];
    b->storage = sets[0]->storage;
    b->max_positions = max_positions;
    b->max_items = max_items;
    b->total_bricks = (int)bricks;
    const size_t P = (size_t)max_positions, I = (size_t)max_items, B = (size_t)bricks;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(spo_work) * I);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_start, sizeof(int64_t) * (I + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_item_of, sizeof(int) * P);
    if (e == cudaSuccess) e = cudaMalloc(&b->counts, sizeof(int) * B);
    if (e == cudaSuccess) e = cudaMalloc(&b->offsets, sizeof(int) * (B + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->keys, sizeof(int) * P);
    if (e == cudaSuccess) e = cudaMalloc(&b->slots, sizeof(int) * P);
    if (e == cudaSuccess) e = cudaMalloc(&b->sorted, sizeof(float4) * P);
    if (e == cudaSuccess) e = cudaMalloc(&b->wrec, sizeof(float4) * spo_detail::kWeightRecordF4 * P);
    if (e == cudaSuccess) e = cudaMalloc(&b->dst, sizeof(float *) * P);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_items, sizeof(spo_work) * I);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_start, sizeof(int64_t) * (I + 1));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = spo_detail::device_status_address(&b->status);
    if (e == cudaSuccess) e = spo_detail::prepare_brick_batch();
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan(b);
        delete b;
        return fail(SPO_ENOMEM, "plan allocation failed: %s", cudaGetErrorString(e));
    }
    *out = b;
    return SPO_OK;
}

spo_status spo_batch_eval(spo_batch *b, spo_kind kind, const spo_work *items, int nitems,
                          void *stream) {
    fail(SPO_OK, "");
    if (!b) return fail(SPO_EINVAL, "plan is NULL");
    if (kind != SPO_KIND_V && kind != SPO_KIND_VGL && kind != SPO_KIND_VGH)
        return fail(SPO_EINVAL, "invalid kind %d", (int)kind);
    DeviceGuard guard(b->device);
    if (!guard.ok()) return fail(SPO_ECUDA, "cannot select device %d", b->device);
    int64_t *start = new (std::nothrow) int64_t[(size_t)std::max(nitems, 0) + 1];
    if (!start) return fail(SPO_ENOMEM, "host allocation failed");
    bool vec_out = true;
    spo_status st = check_items(b, items, nitems, start, &vec_out);
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (st == SPO_OK) st = stage_items(b, items, nitems, start, cs, false);
    if (st == SPO_OK) st = queue_work(b, kind, nitems, start[nitems], vec_out, cs);
    delete[] start;
    return st;
}

spo_status spo_eval_batch(const spo_set *const *sets, int nsets, const spo_work *items, int nitems,
                          spo_kind kind, void *stream) {
    fail(SPO_OK, "");
    if (!sets || nsets < 1 || (nitems > 0 && !items) || nitems < 0)
        return fail(SPO_EINVAL, "need sets, nsets >= 1 and an item table");
    if (kind != SPO_KIND_V && kind != SPO_KIND_VGL && kind != SPO_KIND_VGH)
        return fail(SPO_EINVAL, "invalid kind %d", (int)kind);
    if (nitems == 0) return SPO_OK;
    bool planned = nsets <= SPO_BATCH_MAX_SETS;
    int64_t total = 0;
    for (int i = 0; i < nsets; ++i) {
        if (!sets[i]) return fail(SPO_EINVAL, "set %d is NULL", i);
        planned = planned && sets[i]->has_block_map && sets[i]->storage == sets[0]->storage &&
                  sets[i]->device == sets[0]->device;
    }
    for (int k = 0; k < nitems; ++k) {
        if (items[k].set < 0 || items[k].set >= nsets) return fail(SPO_EINVAL, "item %d: bad set", k);
        if (items[k].P < 0) return fail(SPO_EINVAL, "item %d: P < 0", k);
        total += items[k].P;
    }
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (!planned) {
        // sets the one-launch plan cannot take: one evaluation per walker
        for (int k = 0; k < nitems; ++k) {
            if (items[k].P == 0) continue;
            const spo_status st = spo_eval_ex(sets[items[k].set], kind, items[k].pos, items[k].P,
                                              items[k].out, stream, SPO_ALGO_AUTO);
            if (st != SPO_OK) return st;
        }
        return SPO_OK;
    }
    spo_batch *plan = nullptr;
    spo_status st = spo_batch_create(sets, nsets, std::max<int64_t>(total, 1), nitems, &plan);
    if (st != SPO_OK) return st;
    st = spo_batch_eval(plan, kind, items, nitems, stream);
    if (st == SPO_OK && cudaStreamSynchronize(cs) != cudaSuccess)
        st = fail(SPO_ECUDA, "stream synchronisation failed");
    const spo_status ds = spo_batch_destroy(plan);
    return st != SPO_OK ? st : ds;
}

spo_status spo_batch_graph(spo_batch *b, spo_kind kind, const spo_work *items, int nitems,
                           void *stream) {
    fail(SPO_OK, "");
    if (!b) return fail(SPO_EINVAL, "plan is NULL");
    if (kind != SPO_KIND_V && kind != SPO_KIND_VGL && kind != SPO_KIND_VGH)
        return fail(SPO_EINVAL, "invalid kind %d", (int)kind);
    DeviceGuard guard(b->device);
    if (!guard.ok()) return fail(SPO_ECUDA, "cannot select device %d", b->device);
    int64_t *start = new (std::nothrow) int64_t[(size_t)std::max(nitems, 0) + 1];
    if (!start) return fail(SPO_ENOMEM, "host allocation failed");
    bool vec_out = true;
    spo_status st = check_items(b, items, nitems, start, &vec_out);
    const int64_t Ptot = st == SPO_OK ? start[nitems] : 0;
    // the item table is fixed for the graph: copy it now, outside the capture
    if (st == SPO_OK) st = stage_items(b, items, nitems, start, b->capture_stream, true);
    delete[] start;
    if (st != SPO_OK) return st;
    (void)stream;
    // pick the orbital tile once (the faster of the two widths, timed on the
    // plan's own stream) before recording
    if (!b->tile_tuned) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        float best = 1e30f;
        int best_tile = 32;
        cudaError_t te = cudaEventCreate(&e0);
        if (te == cudaSuccess) te = cudaEventCreate(&e1);
        const int tiles[2] = {32, 64};
        for (int ti = 0; ti < 2 && te == cudaSuccess; ++ti) {
            bool ok = true;
            for (int k = 0; k < b->nsets; ++k)
                if (b->sets[k]->Np < tiles[ti]) ok = false;
            if (!ok) continue;
            b->tile = tiles[ti];
            st = queue_work(b, kind, nitems, Ptot, vec_out, b->capture_stream);   // warm-up
            cudaEventRecord(e0, b->capture_stream);
            for (int r = 0; r < 3 && st == SPO_OK; ++r)
                st = queue_work(b, kind, nitems, Ptot, vec_out, b->capture_stream);
            cudaEventRecord(e1, b->capture_stream);
            te = cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (st != SPO_OK) break;
            if (ms < best) {
                best = ms;
                best_tile = tiles[ti];
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st != SPO_OK) return st;
        if (te != cudaSuccess) return cuda_fail(te, "tile timing");
        b->tile = best_tile;
        b->tile_tuned = true;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    st = queue_work(b, kind, nitems, Ptot, vec_out, b->capture_stream);
    e = cudaStreamEndCapture(b->capture_stream, &graph);
    if (st != SPO_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = exec;
    return SPO_OK;
}

spo_status spo_batch_launch(spo_batch *b, void *stream) {
    fail(SPO_OK, "");
    if (!b) return fail(SPO_EINVAL, "plan is NULL");
    if (!b->exec) return fail(SPO_EINVAL, "no graph recorded: call spo_batch_graph first");
    DeviceGuard guard(b->device);
    if (!guard.ok()) return fail(SPO_ECUDA, "cannot select device %d", b->device);
    cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "cudaGraphLaunch");
}

spo_status spo_batch_destroy(spo_batch *b) {
    if (!b) return SPO_OK;
    DeviceGuard guard(b->device);
    cudaDeviceSynchronize();
    free_plan(b);
    delete b;
    return SPO_OK;
}

}  // extern "C"
