// Host side of the libspo C ABI: argument checks, table upload and
// conversion, strategy dispatch, per-stream scratch, the host-buffer
// pipeline and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "spo.h"
#include "spo_host.h"
#include "spo_internal.h"

namespace {

using spo_detail::cuda_fail;
using spo_detail::DeviceGuard;
using spo_detail::fail;

thread_local char g_last_error[512] = "";


size_t dtype_size(spo_dtype t) {
    switch (t) {
        case SPO_F64: return 8;
        case SPO_F32: return 4;
        case SPO_BF16: return 2;
        case SPO_F16: return 2;
    }
    return 0;
}

bool valid_kind(spo_kind k) { return k == SPO_KIND_V || k == SPO_KIND_VGL || k == SPO_KIND_VGH; }


// pointer must be device or managed memory on `device`
spo_status check_device_pointer(const void *ptr, int device, const char *name) {
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();   // clear the error of this query
        return fail(SPO_EINVAL, "%s is not a CUDA pointer", name);
    }
    if (attr.type == cudaMemoryTypeManaged) return SPO_OK;
    if (attr.type != cudaMemoryTypeDevice) return fail(SPO_EINVAL, "%s must be device memory", name);
    if (attr.device != device)
        return fail(SPO_EINVAL, "%s lives on device %d, the set on device %d", name, attr.device,
                    device);
    return SPO_OK;
}

spo_status check_eval_args(const spo_set *set, spo_kind kind, const float *pos, int64_t P,
                           const float *out) {
    if (!set) return fail(SPO_EINVAL, "set is NULL");
    if (!valid_kind(kind)) return fail(SPO_EINVAL, "invalid kind %d", (int)kind);
    if (P < 0) return fail(SPO_EINVAL, "P = %lld is negative", (long long)P);
    if (P == 0) return SPO_OK;
    if (!pos || !out) return fail(SPO_EINVAL, "pos or out is NULL");
    const int64_t rows = spo_rows(kind);
    if (P > (INT64_C(1) << 40) / (rows * set->N))
        return fail(SPO_EINVAL, "P = %lld too large for N = %lld", (long long)P, (long long)set->N);
    return SPO_OK;
}

void free_workspace(spo_detail::Workspace &w) {
    cudaFree(w.counts);
    cudaFree(w.offsets);
    cudaFree(w.keys);
    cudaFree(w.slots);
    cudaFree(w.perm);
    cudaFree(w.sorted);
    cudaFree(w.wrec);
    cudaFree(w.partials);
    cudaFree(w.vscratch);
    w.counts = w.offsets = w.keys = w.slots = w.perm = nullptr;
    w.sorted = w.wrec = nullptr;
    w.partials = w.vscratch = nullptr;
    w.cap_partials = w.cap_vscratch = 0;
    w.cap_positions = w.cap_bins = 0;
}

// The scratch of `stream`, grown to hold P positions.  Caller holds set->mu.
spo_status workspace_for(spo_set *s, cudaStream_t stream, int64_t P, spo_detail::Workspace **out) {
    spo_detail::Workspace *w = nullptr;
    for (auto &x : s->ws)
        if (x.stream == stream) w = &x;
    if (!w) {
        s->ws.emplace_back();
        w = &s->ws.back();
        w->stream = stream;
    }
    const int64_t nbins = (int64_t)s->nbx * s->nby * s->nbz;
    if (w->cap_positions < P || w->cap_bins < nbins) {
        const int64_t cp = std::max<int64_t>(P, w->cap_positions);
        const int64_t cb = std::max<int64_t>(nbins, w->cap_bins);
        // cudaFree waits for queued work that uses the old buffers
        cudaFree(w->counts);
        cudaFree(w->offsets);
        cudaFree(w->keys);
        cudaFree(w->slots);
        cudaFree(w->perm);
        cudaFree(w->sorted);
        cudaFree(w->wrec);
        w->counts = w->offsets = w->keys = w->slots = w->perm = nullptr;
        w->sorted = w->wrec = nullptr;
        w->cap_positions = w->cap_bins = 0;
        // counts: nbins + 1 ints (the last one the count kernel's ticket),
        // zero between calls (the count kernel clears what it used)
        if (cudaMalloc(&w->counts, sizeof(int) * (cb + 1)) != cudaSuccess ||
            cudaMemset(w->counts, 0, sizeof(int) * (cb + 1)) != cudaSuccess ||
            cudaMalloc(&w->offsets, sizeof(int) * (cb + 1)) != cudaSuccess ||
            cudaMalloc(&w->keys, sizeof(int) * cp) != cudaSuccess ||
            cudaMalloc(&w->slots, sizeof(int) * cp) != cudaSuccess ||
            cudaMalloc(&w->perm, sizeof(int) * cp) != cudaSuccess ||
            cudaMalloc(&w->sorted, sizeof(float4) * cp) != cudaSuccess ||
            cudaMalloc(&w->wrec, sizeof(float4) * spo_detail::kWeightRecordF4 * cp) != cudaSuccess) {
            cudaGetLastError();
            free_workspace(*w);
            return fail(SPO_ENOMEM, "cudaMalloc of binning scratch for %lld positions failed",
                        (long long)P);
        }
        w->cap_positions = cp;
        w->cap_bins = cb;
    }
    *out = w;
    return SPO_OK;
}

// Grow a float scratch buffer to `need` elements (cudaFree waits for queued
// work that still uses the old one).
spo_status ensure_floats(float **buf, size_t *cap, size_t need) {
    if (*cap >= need) return SPO_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    if (cudaMalloc(buf, need * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return fail(SPO_ENOMEM, "cudaMalloc of %zu scratch floats failed", need);
    }
    *cap = need;
    return SPO_OK;
}

// The strategy AUTO takes (without a tuned choice), by the mean number of
// positions per brick r = P / bricks.  Measured crossovers (NiO-64 shape,
// FP32, per call with the binning): below r = 1.5 the gather kernel in
// input order wins (no binning, little reuse to gain); a staged block pays
// for itself once a brick holds enough positions to amortise it: r = 5 for
// VGH, 7 for VGL, 8 for V; in between, the gather kernel in binned order
// (L2 reuse without staging) is fastest.
spo_algo choose_algo(const spo_set *s, spo_kind kind, int64_t P) {
    const int64_t nbins = (int64_t)s->nbx * s->nby * s->nbz;
    if (P >= INT_MAX || P < 1024 || 2 * P < 3 * nbins) return SPO_ALGO_GATHER;
    const int64_t brick_from = kind == SPO_KIND_VGH ? 5 : (kind == SPO_KIND_VGL ? 7 : 8);
    if (s->has_block_map && P >= brick_from * nbins) return SPO_ALGO_BRICK;
    return SPO_ALGO_SORTED_GATHER;
}

// Queue the binning of pos into the scratch of `stream`.  Caller holds set->mu.
spo_status bin_queue(spo_set *s, const float *pos, int64_t P, cudaStream_t stream,
                     spo_detail::Workspace **out) {
    if (P >= INT_MAX) return fail(SPO_EINVAL, "binned strategies need P < 2^31");
    spo_detail::Workspace *w = nullptr;
    spo_status st = workspace_for(s, stream, P, &w);
    if (st != SPO_OK) return st;
    cudaError_t e = spo_detail::launch_bin(pos, P, s->nx, s->ny, s->nz, s->nbx, s->nby, s->nbz, *w,
                                           stream);
    if (e != cudaSuccess) {
        w->binned_pos = nullptr;
        w->binned_P = -1;
        return cuda_fail(e, "binning launch");
    }
    w->binned_pos = pos;
    w->binned_P = P;
    *out = w;
    return SPO_OK;
}

// Queue the evaluation stage of a binned strategy.  Caller holds set->mu.
spo_status binned_eval_queue(const spo_set *s, spo_kind kind, const float *pos, int64_t P,
                             float *out, cudaStream_t stream, spo_algo algo,
                             const spo_detail::Workspace &w) {
    cudaError_t e;
    if (algo == SPO_ALGO_BRICK)
        e = spo_detail::launch_brick(s->storage, kind, s, pos, w, P, out, stream);
    else
        e = spo_detail::launch_gather(s->storage, kind, spo_detail::view_of(s), pos, w.perm, P, out,
                                      stream);
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "evaluation launch");
}

spo_status check_binned_algo(const spo_set *set, spo_algo algo) {
    if (algo != SPO_ALGO_SORTED_GATHER && algo != SPO_ALGO_BRICK)
        return fail(SPO_EINVAL, "invalid algo %d for a binned evaluation", (int)algo);
    if (algo == SPO_ALGO_BRICK && !set->has_block_map)
        return fail(SPO_EUNSUPPORTED, "the brick strategy needs at least 32 padded orbitals");
    return SPO_OK;
}

// The strategy AUTO resolves to: the tuned choice for batches within 4x of
// the tuned size, else choose_algo.
spo_algo resolve_auto(const spo_set *set, spo_kind kind, int64_t P) {
    const int k = (int)kind;
    const int64_t tp = set->tuned_P[k];
    return (set->tuned_algo[k] != 0 && P * 4 >= tp && P <= tp * 4) ? static_cast<spo_algo>(set->tuned_algo[k])
                                                                     : choose_algo(set, kind, P);
}

// Queue one evaluation (arguments already checked; device already current).
spo_status eval_queue(const spo_set *set, spo_kind kind, const float *pos, int64_t P, float *out,
                      cudaStream_t stream, spo_algo algo) {
    if (algo == SPO_ALGO_AUTO) algo = resolve_auto(set, kind, P);
    if (algo == SPO_ALGO_GATHER) {
        cudaError_t e = spo_detail::launch_gather(set->storage, kind, spo_detail::view_of(set), pos,
                                                  nullptr, P, out, stream);
        return e == cudaSuccess ? SPO_OK : cuda_fail(e, "gather kernel launch");
    }
    spo_status st = check_binned_algo(set, algo);
    if (st != SPO_OK) return st;
    spo_set *s = const_cast<spo_set *>(set);
    std::lock_guard<std::mutex> lock(s->mu);   // held until the launches are queued
    spo_detail::Workspace *w = nullptr;
    st = bin_queue(s, pos, P, stream, &w);
    if (st != SPO_OK) return st;
    return binned_eval_queue(s, kind, pos, P, out, stream, algo, *w);
}

// Common checks of the device-buffer entry points.
spo_status check_device_eval(const spo_set *set, spo_kind kind, const float *pos, int64_t P,
                             const float *out) {
    spo_status s = check_eval_args(set, kind, pos, P, out);
    if (s != SPO_OK || P == 0) return s;
    if ((s = check_device_pointer(pos, set->device, "pos")) != SPO_OK) return s;
    if ((s = check_device_pointer(out, set->device, "out")) != SPO_OK) return s;
    if ((reinterpret_cast<uintptr_t>(pos) & 3) || (reinterpret_cast<uintptr_t>(out) & 3))
        return fail(SPO_EINVAL, "pos and out must be 4-byte aligned");
    return SPO_OK;
}

}  // namespace

namespace spo_detail {

spo_status eval_queue(const spo_set *set, spo_kind kind, const float *pos, int64_t P, float *out,
                      cudaStream_t stream, spo_algo algo) {
    return ::eval_queue(set, kind, pos, P, out, stream, algo);
}

spo_algo auto_algo(const spo_set *set, spo_kind kind, int64_t P) { return resolve_auto(set, kind, P); }

spo_status fail(spo_status status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return status;
}

}  // namespace spo_detail

extern "C" {

int spo_abi_version(void) { return SPO_ABI_VERSION; }

int spo_rows(spo_kind kind) {
    switch (kind) {
        case SPO_KIND_V: return 1;
        case SPO_KIND_VGL: return 5;
        case SPO_KIND_VGH: return 10;
    }
    return 0;
}

const char *spo_status_str(spo_status s) {
    switch (s) {
        case SPO_OK: return "SPO_OK";
        case SPO_EINVAL: return "SPO_EINVAL: invalid argument";
        case SPO_ENOMEM: return "SPO_ENOMEM: out of memory";
        case SPO_ECUDA: return "SPO_ECUDA: CUDA error";
        case SPO_ETIMEOUT: return "SPO_ETIMEOUT: device-side wait timed out";
        case SPO_EUNSUPPORTED: return "SPO_EUNSUPPORTED: not supported";
    }
    return "unknown spo_status";
}

const char *spo_last_error(void) { return g_last_error; }

spo_status spo_create(const spo_grid *grid, const void *coefs, spo_dtype src_dtype, int64_t N,
                      spo_dtype storage, int coefs_on_device, spo_set **out) {
    g_last_error[0] = '\0';
    if (!out) return fail(SPO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid) return fail(SPO_EINVAL, "grid is NULL");
    if (!coefs) return fail(SPO_EINVAL, "coefs is NULL");
    if (grid->nx < 4 || grid->ny < 4 || grid->nz < 4)
        return fail(SPO_EINVAL, "grid %d x %d x %d: every n_d must be >= 4", grid->nx, grid->ny,
                    grid->nz);
    if (grid->nx > (1 << 20) || grid->ny > (1 << 20) || grid->nz > (1 << 20))
        return fail(SPO_EINVAL, "grid edge above 2^20");
    const int64_t padded_rows = (int64_t)(grid->nx + 3) * (grid->ny + 3) * (grid->nz + 3);
    if (padded_rows > INT32_MAX) return fail(SPO_EINVAL, "grid has more than 2^31-1 padded nodes");
    if (N < 1) return fail(SPO_EINVAL, "N = %lld must be >= 1", (long long)N);
    if (N > (INT64_C(1) << 24)) return fail(SPO_EINVAL, "N = %lld too large", (long long)N);
    if (dtype_size(src_dtype) == 0) return fail(SPO_EINVAL, "invalid src_dtype %d", (int)src_dtype);
    if (storage == SPO_F64)
        return fail(SPO_EUNSUPPORTED, "FP64 is a source type only; store as F32, BF16 or F16");
    if (storage != SPO_F32 && storage != SPO_BF16 && storage != SPO_F16)
        return fail(SPO_EINVAL, "invalid storage dtype %d", (int)storage);

    int device = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    if (coefs_on_device) {
        spo_status s = check_device_pointer(coefs, device, "coefs");
        if (s != SPO_OK) return s;
    }

    spo_set *set = new (std::nothrow) spo_set();
    if (!set) return fail(SPO_ENOMEM, "host allocation of the set failed");
    set->device = device;
    set->num_sms = num_sms;
    set->nx = grid->nx;
    set->ny = grid->ny;
    set->nz = grid->nz;
    set->xp = grid->nx + 3;
    set->yp = grid->ny + 3;
    set->zp = grid->nz + 3;
    set->nbx = (grid->nx + spo_detail::kBrick - 1) / spo_detail::kBrick;
    set->nby = (grid->ny + spo_detail::kBrick - 1) / spo_detail::kBrick;
    set->nbz = (grid->nz + spo_detail::kBrick - 1) / spo_detail::kBrick;
    set->N = N;
    set->Np = (N + 7) / 8 * 8;
    set->storage = storage;
    const size_t es = dtype_size(storage);
    const size_t plane_bytes = (size_t)set->yp * set->zp * set->Np * es;
    set->table_bytes = (size_t)set->xp * plane_bytes;

    e = cudaMalloc(&set->table, set->table_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const size_t bytes = set->table_bytes;
        delete set;
        return fail(SPO_ENOMEM, "cudaMalloc of %zu table bytes failed", bytes);
    }

    // convert slabs of whole x-planes of the source (bounded staging memory)
    const size_t src_plane = (size_t)grid->ny * grid->nz * N * dtype_size(src_dtype);
    const int slab = (int)std::max<int64_t>(
        1, std::min<int64_t>(grid->nx, (int64_t)((size_t)(512u << 20) / src_plane)));
    void *staging = nullptr;
    cudaStream_t stream = nullptr;
    spo_status status = SPO_OK;
    e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) status = cuda_fail(e, "cudaStreamCreate");
    if (status == SPO_OK && !coefs_on_device) {
        e = cudaMalloc(&staging, (size_t)slab * src_plane);
        if (e != cudaSuccess) {
            cudaGetLastError();
            status = fail(SPO_ENOMEM, "cudaMalloc of the upload staging buffer failed");
        }
    }
    for (int x0 = 0; status == SPO_OK && x0 < grid->nx; x0 += slab) {
        const int x1 = std::min(grid->nx, x0 + slab);
        const char *src = static_cast<const char *>(coefs) + (size_t)x0 * src_plane;
        if (!coefs_on_device) {
            e = cudaMemcpyAsync(staging, src, (size_t)(x1 - x0) * src_plane, cudaMemcpyHostToDevice,
                                stream);
            if (e != cudaSuccess) { status = cuda_fail(e, "upload of coefficients"); break; }
            src = static_cast<const char *>(staging);
        }
        e = spo_detail::launch_convert(src, src_dtype, x0, x1, set, stream);
        if (e != cudaSuccess) { status = cuda_fail(e, "conversion kernel"); break; }
        e = cudaStreamSynchronize(stream);   // the staging buffer is reused
        if (e != cudaSuccess) { status = cuda_fail(e, "conversion"); break; }
    }
    // ghost x-planes: padded 0 <- node nx-1 (padded nx), nx+1 <- node 0, nx+2 <- node 1
    const int ghost_src[3] = {grid->nx, 1, 2};
    const int ghost_dst[3] = {0, grid->nx + 1, grid->nx + 2};
    for (int g = 0; status == SPO_OK && g < 3; ++g) {
        char *base = static_cast<char *>(set->table);
        e = cudaMemcpyAsync(base + (size_t)ghost_dst[g] * plane_bytes,
                            base + (size_t)ghost_src[g] * plane_bytes, plane_bytes,
                            cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) status = cuda_fail(e, "ghost plane copy");
    }
    if (status == SPO_OK) {
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) status = cuda_fail(e, "table upload");
    }
    if (staging) cudaFree(staging);
    if (stream) cudaStreamDestroy(stream);
    if (status == SPO_OK) status = spo_detail::make_block_map(set);
    if (status != SPO_OK) {
        cudaFree(set->table);
        delete set;
        return status;
    }
    *out = set;
    return SPO_OK;
}

spo_status spo_destroy(spo_set *set) {
    if (!set) return SPO_OK;
    DeviceGuard guard(set->device);
    cudaDeviceSynchronize();
    for (auto &w : set->ws) free_workspace(w);
    for (int i = 0; i < 2; ++i) {
        if (set->hpos[i]) cudaFree(set->hpos[i]);
        if (set->hout[i]) cudaFree(set->hout[i]);
        if (set->hevent[i]) cudaEventDestroy(set->hevent[i]);
        if (set->hstream[i]) cudaStreamDestroy(set->hstream[i]);
    }
    cudaError_t e = cudaFree(set->table);
    delete set;
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "cudaFree of the table");
}

spo_status spo_eval_ex(const spo_set *set, spo_kind kind, const float *pos, int64_t P, float *out,
                       void *stream, spo_algo algo) {
    g_last_error[0] = '\0';
    if (algo < SPO_ALGO_AUTO || algo > SPO_ALGO_BRICK)
        return fail(SPO_EINVAL, "invalid algo %d", (int)algo);
    if (!set) return fail(SPO_EINVAL, "set is NULL");
    DeviceGuard guard(set->device);
    if (!guard.ok()) return fail(SPO_ECUDA, "cannot select device %d", set->device);
    spo_status s = check_device_eval(set, kind, pos, P, out);
    if (s != SPO_OK || P == 0) return s;
    return eval_queue(set, kind, pos, P, out, static_cast<cudaStream_t>(stream), algo);
}

spo_status spo_eval_ratio(const spo_set *set, const float *pos, int64_t P, const float *rows,
                          int64_t nrows, int64_t ld, const int32_t *row_of, float *ratio,
                          float *v_out, void *stream) {
    g_last_error[0] = '\0';
    if (!set) return fail(SPO_EINVAL, "set is NULL");
    if (P < 0) return fail(SPO_EINVAL, "P = %lld is negative", (long long)P);
    if (P == 0) return SPO_OK;
    if (!pos || !rows || !ratio) return fail(SPO_EINVAL, "pos, rows or ratio is NULL");
    if (nrows < 1 || ld < set->N)
        return fail(SPO_EINVAL, "need nrows >= 1 and ld >= N (nrows = %lld, ld = %lld)",
                    (long long)nrows, (long long)ld);
    if (!row_of && nrows < P) return fail(SPO_EINVAL, "row_of is NULL but nrows < P");
    if (P > (INT64_C(1) << 40) / set->N) return fail(SPO_EINVAL, "P = %lld too large", (long long)P);
    DeviceGuard guard(set->device);
    if (!guard.ok()) return fail(SPO_ECUDA, "cannot select device %d", set->device);
    spo_status st;
    if ((st = check_device_pointer(pos, set->device, "pos")) != SPO_OK) return st;
    if ((st = check_device_pointer(rows, set->device, "rows")) != SPO_OK) return st;
    if ((st = check_device_pointer(ratio, set->device, "ratio")) != SPO_OK) return st;
    if (row_of && (st = check_device_pointer(row_of, set->device, "row_of")) != SPO_OK) return st;
    if (v_out && (st = check_device_pointer(v_out, set->device, "v_out")) != SPO_OK) return st;
    if ((reinterpret_cast<uintptr_t>(pos) | reinterpret_cast<uintptr_t>(rows) |
         reinterpret_cast<uintptr_t>(ratio) | reinterpret_cast<uintptr_t>(row_of) |
         reinterpret_cast<uintptr_t>(v_out)) & 3)
        return fail(SPO_EINVAL, "buffers must be 4-byte aligned");

    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    spo_set *s = const_cast<spo_set *>(set);
    std::lock_guard<std::mutex> lock(s->mu);
    spo_detail::RatioArgs ra{rows, row_of, nrows, ld, nullptr, P};
    cudaError_t e;
    // the fused epilogue once bricks hold a position on average (the other
    // path is the input-order gather and a separate dot product)
    if (s->has_block_map && P >= 1024 && P >= (int64_t)s->nbx * s->nby * s->nbz) {
        spo_detail::Workspace *w = nullptr;
        if ((st = bin_queue(s, pos, P, cs, &w)) != SPO_OK) return st;
        const int ntiles = spo_detail::brick_tiles_of(s);
        if ((st = ensure_floats(&w->partials, &w->cap_partials, (size_t)ntiles * P)) != SPO_OK)
            return st;
        ra.partials = w->partials;
        e = spo_detail::launch_brick_ratio(s, *w, P, v_out, ra, cs);
        if (e == cudaSuccess) e = spo_detail::launch_ratio_reduce(w->partials, ntiles, P, ratio, cs);
    } else {
        spo_detail::Workspace *w = nullptr;
        if ((st = workspace_for(s, cs, P, &w)) != SPO_OK) return st;
        float *v = v_out;
        if (!v) {
            if ((st = ensure_floats(&w->vscratch, &w->cap_vscratch, (size_t)P * s->N)) != SPO_OK)
                return st;
            v = w->vscratch;
        }
        e = spo_detail::launch_gather(s->storage, SPO_KIND_V, spo_detail::view_of(s), pos, nullptr, P,
                                      v, cs);
        if (e == cudaSuccess) e = spo_detail::launch_ratio_dot(v, P, s->N, ra, ratio, cs);
    }
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "ratio launch");
}

spo_status spo_bin(const spo_set *set, const float *pos, int64_t P, void *stream) {
    g_last_error[0] = '\0';
    if (!set) return fail(SPO_EINVAL, "set is NULL");
    if (P < 0) return fail(SPO_EINVAL, "P = %lld is negative", (long long)P);
    if (P > 0 && !pos) return fail(SPO_EINVAL, "pos is NULL");
    DeviceGuard guard(set->device);
    if (!guard.ok()) return fail(SPO_ECUDA, "cannot select device %d", set->device);
    spo_status st;
    if (P > 0 && (st = check_device_pointer(pos, set->device, "pos")) != SPO_OK) return st;
    spo_set *s = const_cast<spo_set *>(set);
    std::lock_guard<std::mutex> lock(s->mu);
    spo_detail::Workspace *w = nullptr;
    return bin_queue(s, pos, P, static_cast<cudaStream_t>(stream), &w);
}

spo_status spo_eval_binned(const spo_set *set, spo_kind kind, const float *pos, int64_t P,
                           float *out, void *stream, spo_algo algo) {
    g_last_error[0] = '\0';
    if (!set) return fail(SPO_EINVAL, "set is NULL");
    DeviceGuard guard(set->device);
    if (!guard.ok()) return fail(SPO_ECUDA, "cannot select device %d", set->device);
    spo_status st = check_device_eval(set, kind, pos, P, out);
    if (st != SPO_OK || P == 0) return st;
    if ((st = check_binned_algo(set, algo)) != SPO_OK) return st;
    spo_set *s = const_cast<spo_set *>(set);
    std::lock_guard<std::mutex> lock(s->mu);
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    for (auto &w : s->ws)
        if (w.stream == cs) {
            if (w.binned_pos != pos || w.binned_P != P)
                return fail(SPO_EINVAL, "pos/P differ from the last spo_bin on this stream");
            return binned_eval_queue(s, kind, pos, P, out, cs, algo, w);
        }
    return fail(SPO_EINVAL, "no spo_bin on this stream for this set");
}

spo_status spo_eval(const spo_set *set, spo_kind kind, const float *pos, int64_t P, float *out,
                    void *stream) {
    return spo_eval_ex(set, kind, pos, P, out, stream, SPO_ALGO_AUTO);
}

spo_status spo_eval_v(const spo_set *set, const float *pos, int64_t P, float *out, void *stream) {
    return spo_eval(set, SPO_KIND_V, pos, P, out, stream);
}

spo_status spo_eval_vgl(const spo_set *set, const float *pos, int64_t P, float *out, void *stream) {
    return spo_eval(set, SPO_KIND_VGL, pos, P, out, stream);
}

spo_status spo_eval_vgh(const spo_set *set, const float *pos, int64_t P, float *out, void *stream) {
    return spo_eval(set, SPO_KIND_VGH, pos, P, out, stream);
}

spo_status spo_reserve(spo_set *set, int64_t P, void *stream) {
    g_last_error[0] = '\0';
    if (!set) return fail(SPO_EINVAL, "set is NULL");
    if (P < 0 || P >= INT_MAX) return fail(SPO_EINVAL, "P = %lld out of range", (long long)P);
    DeviceGuard guard(set->device);
    if (!guard.ok()) return fail(SPO_ECUDA, "cannot select device %d", set->device);
    std::lock_guard<std::mutex> lock(set->mu);
    spo_detail::Workspace *w = nullptr;
    return workspace_for(set, static_cast<cudaStream_t>(stream), std::max<int64_t>(P, 1), &w);
}

spo_status spo_device_status(unsigned int *flags, int clear, void *stream) {
    g_last_error[0] = '\0';
    if (!flags) return fail(SPO_EINVAL, "flags is NULL");
    cudaError_t e = spo_detail::read_device_status(flags, clear != 0, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "device status read");
    if (*flags & 1u) return fail(SPO_ETIMEOUT, "a bounded wait on a TMA copy gave up");
    if (*flags & 2u) return fail(SPO_EINVAL, "an index check failed (SPO_CHECK_BOUNDS build); the access was skipped");
    return SPO_OK;
}

// Device address of pinned, mapped host memory, or nullptr for any other
// kind of pointer (pageable host memory, device memory).
const void *mapped_host_alias(const void *p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (attr.type != cudaMemoryTypeHost || !attr.devicePointer) return nullptr;
    return attr.devicePointer;
}

spo_status spo_eval_host(spo_set *set, spo_kind kind, const float *pos_host, int64_t P,
                         float *out_host, void *stream) {
    g_last_error[0] = '\0';
    spo_status s = check_eval_args(set, kind, pos_host, P, out_host);
    if (s != SPO_OK || P == 0) return s;
    DeviceGuard guard(set->device);
    if (!guard.ok()) return fail(SPO_ECUDA, "cannot select device %d", set->device);

    // Zero-copy: with both buffers pinned and mapped, the kernels read the
    // positions from and write the outputs to host memory directly (over the
    // coherent CPU-GPU link on Grace-Blackwell), with no staging copies.
    const float *pos_dev = static_cast<const float *>(mapped_host_alias(pos_host));
    float *out_dev = static_cast<float *>(const_cast<void *>(mapped_host_alias(out_host)));
    if (pos_dev && out_dev && (reinterpret_cast<uintptr_t>(out_dev) & 3) == 0 &&
        (reinterpret_cast<uintptr_t>(pos_dev) & 3) == 0) {
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        spo_status status = eval_queue(set, kind, pos_dev, P, out_dev, st, SPO_ALGO_AUTO);
        if (status != SPO_OK) return status;
        cudaError_t e = cudaStreamSynchronize(st);
        return e == cudaSuccess ? SPO_OK : cuda_fail(e, "zero-copy evaluation");
    }

    const int64_t rows = spo_rows(kind);
    const size_t out_row = (size_t)rows * (size_t)set->N * sizeof(float);   // per position
    // about four chunks per batch (copies of one overlap the kernel of the
    // next), at most 512 MB of output per chunk, at least 256 positions
    int64_t chunk = std::max<int64_t>((P + 3) / 4, 256);
    chunk = std::min<int64_t>(chunk, std::max<int64_t>(256, (int64_t)((size_t)(512u << 20) / out_row)));
    chunk = std::min<int64_t>(chunk, P);
    const size_t need_pos = (size_t)chunk * 3 * sizeof(float);
    const size_t need_out = (size_t)chunk * out_row;
    cudaError_t e;
    for (int i = 0; i < 2; ++i) {
        if (!set->hstream[i]) {
            e = cudaStreamCreateWithFlags(&set->hstream[i], cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        }
        if (!set->hevent[i]) {
            e = cudaEventCreateWithFlags(&set->hevent[i], cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        }
    }
    if (set->hpos_cap < need_pos || set->hout_cap < need_out) {
        for (int j = 0; j < 2; ++j) {
            cudaStreamSynchronize(set->hstream[j]);
            if (set->hpos[j]) cudaFree(set->hpos[j]);
            if (set->hout[j]) cudaFree(set->hout[j]);
            set->hpos[j] = set->hout[j] = nullptr;
        }
        set->hpos_cap = set->hout_cap = 0;
        for (int j = 0; j < 2; ++j) {
            if (cudaMalloc(&set->hpos[j], need_pos) != cudaSuccess ||
                cudaMalloc(&set->hout[j], need_out) != cudaSuccess) {
                cudaGetLastError();
                return fail(SPO_ENOMEM, "cudaMalloc of %zu staging bytes failed", need_out);
            }
        }
        set->hpos_cap = need_pos;
        set->hout_cap = need_out;
    }
    // order after the caller's stream
    cudaEvent_t start;
    e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    cudaEventRecord(start, static_cast<cudaStream_t>(stream));
    for (int i = 0; i < 2; ++i) cudaStreamWaitEvent(set->hstream[i], start, 0);

    spo_status status = SPO_OK;
    int64_t c = 0;
    for (int64_t p0 = 0; p0 < P; p0 += chunk, ++c) {
        const int i = (int)(c & 1);
        const int64_t np = std::min<int64_t>(chunk, P - p0);
        cudaStream_t st = set->hstream[i];
        e = cudaMemcpyAsync(set->hpos[i], pos_host + 3 * p0, (size_t)np * 3 * sizeof(float),
                            cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { status = cuda_fail(e, "position upload"); break; }
        status = eval_queue(set, kind, set->hpos[i], np, set->hout[i], st, SPO_ALGO_AUTO);
        if (status != SPO_OK) break;
        e = cudaMemcpyAsync(reinterpret_cast<char *>(out_host) + (size_t)p0 * out_row, set->hout[i],
                            (size_t)np * out_row, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) { status = cuda_fail(e, "output download"); break; }
    }
    for (int i = 0; i < 2; ++i) {
        e = cudaStreamSynchronize(set->hstream[i]);
        if (e != cudaSuccess && status == SPO_OK) status = cuda_fail(e, "host-path synchronisation");
    }
    cudaEventDestroy(start);
    return status;
}

spo_status spo_set_param(spo_set *set, spo_param param, int64_t value) {
    g_last_error[0] = '\0';
    if (!set) return fail(SPO_EINVAL, "set is NULL");
    switch (param) {
        case SPO_PARAM_BRICK_VEC:
            if (value != 2 && value != 4)
                return fail(SPO_EINVAL, "SPO_PARAM_BRICK_VEC must be 2 or 4, not %lld", (long long)value);
            set->brick_vec = (int)value;
            return SPO_OK;
        case SPO_PARAM_BRICK_TILE:
            if (value != 32 && value != 64)
                return fail(SPO_EINVAL, "SPO_PARAM_BRICK_TILE must be 32 or 64, not %lld", (long long)value);
            set->brick_tile = (int)value;
            return SPO_OK;
        case SPO_PARAM_BRICK_SCHEDULE:
            if (value != 0 && value != 1)
                return fail(SPO_EINVAL, "SPO_PARAM_BRICK_SCHEDULE must be 0 or 1, not %lld", (long long)value);
            set->brick_schedule = (int)value;
            return SPO_OK;
    }
    return fail(SPO_EINVAL, "unknown parameter %d", (int)param);
}

spo_status spo_get_param(const spo_set *set, spo_param param, int64_t *value) {
    g_last_error[0] = '\0';
    if (!set || !value) return fail(SPO_EINVAL, "set or value is NULL");
    switch (param) {
        case SPO_PARAM_BRICK_VEC: *value = set->brick_vec; return SPO_OK;
        case SPO_PARAM_BRICK_TILE: *value = set->brick_tile; return SPO_OK;
        case SPO_PARAM_BRICK_SCHEDULE: *value = set->brick_schedule; return SPO_OK;
    }
    return fail(SPO_EINVAL, "unknown parameter %d", (int)param);
}

spo_status spo_auto_algo(const spo_set *set, spo_kind kind, int64_t P, spo_algo *algo) {
    g_last_error[0] = '\0';
    if (!set || !algo) return fail(SPO_EINVAL, "set or algo is NULL");
    if (kind != SPO_KIND_V && kind != SPO_KIND_VGL && kind != SPO_KIND_VGH)
        return fail(SPO_EINVAL, "unknown kind %d", (int)kind);
    if (P < 0) return fail(SPO_EINVAL, "P = %lld is negative", (long long)P);
    *algo = resolve_auto(set, kind, P);
    return SPO_OK;
}

spo_status spo_footprint(const spo_set *set, size_t *bytes) {
    if (!set || !bytes) return fail(SPO_EINVAL, "set or bytes is NULL");
    *bytes = set->table_bytes;
    return SPO_OK;
}

spo_status spo_info(const spo_set *set, spo_grid *grid, int64_t *N, int64_t *Np,
                    spo_dtype *storage) {
    if (!set) return fail(SPO_EINVAL, "set is NULL");
    if (grid) *grid = spo_grid{set->nx, set->ny, set->nz};
    if (N) *N = set->N;
    if (Np) *Np = set->Np;
    if (storage) *storage = set->storage;
    return SPO_OK;
}

}  // extern "C"
