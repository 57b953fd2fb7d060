// Host side of the libspo C ABI: argument checks, table upload and
// conversion, launch dispatch, the host-buffer pipeline and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "spo.h"
#include "spo_internal.h"

namespace {

thread_local char g_last_error[512] = "";

// Restores the caller's current device when it goes out of scope.
class DeviceGuard {
  public:
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
        if (prev_ != device) ok_ = cudaSetDevice(device) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev_ >= 0) cudaSetDevice(prev_);
    }
    bool ok() const { return ok_; }

  private:
    int prev_ = -1;
    bool ok_ = true;
};

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

spo_status cuda_fail(cudaError_t e, const char *what) {
    return spo_detail::fail(SPO_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// pointer must be device or managed memory on `device`
spo_status check_device_pointer(const void *ptr, int device, const char *name) {
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();   // clear the sticky-free error of this query
        return spo_detail::fail(SPO_EINVAL, "%s is not a CUDA pointer", name);
    }
    if (attr.type == cudaMemoryTypeManaged) return SPO_OK;
    if (attr.type != cudaMemoryTypeDevice)
        return spo_detail::fail(SPO_EINVAL, "%s must be device memory", name);
    if (attr.device != device)
        return spo_detail::fail(SPO_EINVAL, "%s lives on device %d, the set on device %d", name,
                                attr.device, device);
    return SPO_OK;
}

spo_status check_eval_args(const spo_set *set, spo_kind kind, const float *pos, int64_t P,
                           const float *out) {
    if (!set) return spo_detail::fail(SPO_EINVAL, "set is NULL");
    if (!valid_kind(kind)) return spo_detail::fail(SPO_EINVAL, "invalid kind %d", (int)kind);
    if (P < 0) return spo_detail::fail(SPO_EINVAL, "P = %lld is negative", (long long)P);
    if (P == 0) return SPO_OK;
    if (!pos || !out) return spo_detail::fail(SPO_EINVAL, "pos or out is NULL");
    const int64_t rows = spo_rows(kind);
    // output elements must fit in int64 and the position count in a grid
    if (P > (INT64_C(1) << 40) / (rows * set->N))
        return spo_detail::fail(SPO_EINVAL, "P = %lld too large for N = %lld", (long long)P,
                                (long long)set->N);
    return SPO_OK;
}

}  // namespace

namespace spo_detail {

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
    using spo_detail::fail;
    g_last_error[0] = '\0';
    if (!out) return fail(SPO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid) return fail(SPO_EINVAL, "grid is NULL");
    if (!coefs) return fail(SPO_EINVAL, "coefs is NULL");
    if (grid->nx < 4 || grid->ny < 4 || grid->nz < 4)
        return fail(SPO_EINVAL, "grid %d x %d x %d: every n_d must be >= 4", grid->nx, grid->ny,
                    grid->nz);
    const int64_t cells = (int64_t)grid->nx * grid->ny * grid->nz;
    if (cells > INT32_MAX) return fail(SPO_EINVAL, "grid has more than 2^31-1 nodes");
    if (N < 1) return fail(SPO_EINVAL, "N = %lld must be >= 1", (long long)N);
    if (N > (INT64_C(1) << 24)) return fail(SPO_EINVAL, "N = %lld too large", (long long)N);
    if (dtype_size(src_dtype) == 0) return fail(SPO_EINVAL, "invalid src_dtype %d", (int)src_dtype);
    if (storage == SPO_F64)
        return fail(SPO_EUNSUPPORTED, "FP64 is a source type only; store as F32, BF16 or F16");
    if (storage != SPO_F32 && storage != SPO_BF16 && storage != SPO_F16)
        return fail(SPO_EINVAL, "invalid storage dtype %d", (int)storage);

    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (coefs_on_device) {
        spo_status s = check_device_pointer(coefs, device, "coefs");
        if (s != SPO_OK) return s;
    }

    spo_set *set = new (std::nothrow) spo_set();
    if (!set) return fail(SPO_ENOMEM, "host allocation of the set failed");
    set->device = device;
    set->nx = grid->nx;
    set->ny = grid->ny;
    set->nz = grid->nz;
    set->N = N;
    set->Np = (N + 7) / 8 * 8;
    set->storage = storage;
    set->table_bytes = (size_t)cells * (size_t)set->Np * dtype_size(storage);

    e = cudaMalloc(&set->table, set->table_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const size_t bytes = set->table_bytes;
        delete set;
        return fail(SPO_ENOMEM, "cudaMalloc of %zu table bytes failed", bytes);
    }

    // convert in slabs of rows so that the staging buffer stays bounded
    const size_t src_row_bytes = (size_t)N * dtype_size(src_dtype);
    const int64_t slab_rows =
        std::max<int64_t>(1, std::min<int64_t>(cells, (int64_t)((256u << 20) / src_row_bytes)));
    void *staging = nullptr;
    cudaStream_t stream = nullptr;
    spo_status status = SPO_OK;
    e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) status = cuda_fail(e, "cudaStreamCreate");
    if (status == SPO_OK && !coefs_on_device) {
        e = cudaMalloc(&staging, (size_t)slab_rows * src_row_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            status = fail(SPO_ENOMEM, "cudaMalloc of the upload staging buffer failed");
        }
    }
    for (int64_t r0 = 0; status == SPO_OK && r0 < cells; r0 += slab_rows) {
        const int64_t nrows = std::min<int64_t>(slab_rows, cells - r0);
        const char *src = static_cast<const char *>(coefs) + (size_t)r0 * src_row_bytes;
        if (!coefs_on_device) {
            e = cudaMemcpyAsync(staging, src, (size_t)nrows * src_row_bytes,
                                cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) { status = cuda_fail(e, "upload of coefficients"); break; }
            src = static_cast<const char *>(staging);
        }
        char *dst = static_cast<char *>(set->table) + (size_t)r0 * set->Np * dtype_size(storage);
        e = spo_detail::launch_convert(src, src_dtype, dst, storage, nrows, N, set->Np, stream);
        if (e != cudaSuccess) { status = cuda_fail(e, "conversion kernel"); break; }
        // the staging buffer is reused by the next slab
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) { status = cuda_fail(e, "conversion"); break; }
    }
    if (staging) cudaFree(staging);
    if (stream) cudaStreamDestroy(stream);
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

spo_status spo_eval(const spo_set *set, spo_kind kind, const float *pos, int64_t P, float *out,
                    void *stream) {
    g_last_error[0] = '\0';
    spo_status s = check_eval_args(set, kind, pos, P, out);
    if (s != SPO_OK || P == 0) return s;
    DeviceGuard guard(set->device);
    if (!guard.ok()) return spo_detail::fail(SPO_ECUDA, "cannot select device %d", set->device);
    if ((s = check_device_pointer(pos, set->device, "pos")) != SPO_OK) return s;
    if ((s = check_device_pointer(out, set->device, "out")) != SPO_OK) return s;
    if ((reinterpret_cast<uintptr_t>(pos) & 3) || (reinterpret_cast<uintptr_t>(out) & 3))
        return spo_detail::fail(SPO_EINVAL, "pos and out must be 4-byte aligned");
    spo_detail::EvalArgs a{set->table, set->nx, set->ny, set->nz, set->N, set->Np, pos, P, out};
    cudaError_t e = spo_detail::launch_eval(set->storage, kind, a, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SPO_OK : cuda_fail(e, "evaluation launch");
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

spo_status spo_eval_host(spo_set *set, spo_kind kind, const float *pos_host, int64_t P,
                         float *out_host, void *stream) {
    using spo_detail::fail;
    g_last_error[0] = '\0';
    spo_status s = check_eval_args(set, kind, pos_host, P, out_host);
    if (s != SPO_OK || P == 0) return s;
    DeviceGuard guard(set->device);
    if (!guard.ok()) return fail(SPO_ECUDA, "cannot select device %d", set->device);

    const int64_t rows = spo_rows(kind);
    const size_t out_row = (size_t)rows * (size_t)set->N * sizeof(float);   // per position
    // chunks of about 64 MB of output, at least 256 positions
    const int64_t chunk = std::min<int64_t>(P, std::max<int64_t>(256, (int64_t)((64u << 20) / out_row)));
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
        if (set->hpos_cap < need_pos || set->hout_cap < need_out) {
            // grow both buffers of both streams
            for (int j = 0; j < 2; ++j) {
                if (set->hstream[j]) cudaStreamSynchronize(set->hstream[j]);
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
        spo_detail::EvalArgs a{set->table, set->nx, set->ny, set->nz, set->N, set->Np,
                               set->hpos[i], np, set->hout[i]};
        e = spo_detail::launch_eval(set->storage, kind, a, st);
        if (e != cudaSuccess) { status = cuda_fail(e, "evaluation launch"); break; }
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

spo_status spo_footprint(const spo_set *set, size_t *bytes) {
    if (!set || !bytes) return spo_detail::fail(SPO_EINVAL, "set or bytes is NULL");
    *bytes = set->table_bytes;
    return SPO_OK;
}

spo_status spo_info(const spo_set *set, spo_grid *grid, int64_t *N, int64_t *Np,
                    spo_dtype *storage) {
    if (!set) return spo_detail::fail(SPO_EINVAL, "set is NULL");
    if (grid) *grid = spo_grid{set->nx, set->ny, set->nz};
    if (N) *N = set->N;
    if (Np) *Np = set->Np;
    if (storage) *storage = set->storage;
    return SPO_OK;
}

}  // extern "C"
