// spo_autotune: pick the evaluation strategy and tuning of a set by timing.
//
// Candidates: the gather kernel, the gather kernel in binned order, and the
// brick kernel with 32- or 64-orbital tiles, 2 or 4 orbitals per thread and
// the per-item or persistent schedule.  Each is timed with CUDA events on
// synthetic uniform positions (a few launches after one warm-up); the
// fastest is applied to the set.  Results are cached per key in the process
// and, when SPO_TUNE_CACHE names a file, in that file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "spo.h"
#include "spo_internal.h"

namespace {

using spo_detail::fail;

// uniform positions in the unit cube from a counter-based hash (splitmix64)
__global__ void uniform_positions_kernel(float *pos, int64_t n3, unsigned long long seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        pos[i] = (float)(z >> 40) * (1.0f / 16777216.0f);
    }
}

struct Candidate {
    spo_algo algo;
    int tile, vec, schedule;
};

std::mutex g_cache_mu;
std::map<std::string, spo_tuning> g_cache;
bool g_file_loaded = false;

std::string cache_key(const spo_set *s, spo_kind kind, int64_t P) {
    int bucket = 0;
    while ((INT64_C(1) << (bucket + 1)) <= P) ++bucket;
    char buf[160];
    snprintf(buf, sizeof(buf), "grid=%dx%dx%d,N=%lld,storage=%d,kind=%d,P=2^%d,sms=%d", s->nx, s->ny,
             s->nz, (long long)s->N, (int)s->storage, (int)kind, bucket, s->num_sms);
    return buf;
}

void load_file_cache() {
    if (g_file_loaded) return;
    g_file_loaded = true;
    const char *path = getenv("SPO_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[200];
    spo_tuning t;
    memset(&t, 0, sizeof(t));
    while (fscanf(f, "%199s %d %d %d %d %f", key, &t.algo, &t.brick_tile, &t.brick_vec,
                  &t.brick_schedule, &t.ms) == 6)
        g_cache[key] = t;
    fclose(f);
}

void append_file_cache(const std::string &key, const spo_tuning &t) {
    const char *path = getenv("SPO_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %.6f\n", key.c_str(), t.algo, t.brick_tile, t.brick_vec,
            t.brick_schedule, t.ms);
    fclose(f);
}

void apply(spo_set *s, spo_kind kind, int64_t P, const spo_tuning &t) {
    s->brick_tile = t.brick_tile;
    s->brick_vec = t.brick_vec;
    s->brick_schedule = t.brick_schedule;
    s->tuned_algo[(int)kind] = t.algo;
    s->tuned_P[(int)kind] = P;
}

}  // namespace

extern "C" spo_status spo_autotune(spo_set *set, spo_kind kind, int64_t P, void *stream,
                                   spo_tuning *best) {
    fail(SPO_OK, "");
    if (!set || !best) return fail(SPO_EINVAL, "set or best is NULL");
    if (kind != SPO_KIND_V && kind != SPO_KIND_VGL && kind != SPO_KIND_VGH)
        return fail(SPO_EINVAL, "invalid kind %d", (int)kind);
    if (P < 1 || P >= (INT64_C(1) << 31) || P > (INT64_C(1) << 36) / (spo_rows(kind) * set->N))
        return fail(SPO_EINVAL, "P = %lld out of range", (long long)P);
    const std::string key = cache_key(set, kind, P);
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        load_file_cache();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            *best = it->second;
            best->from_cache = 1;
            apply(set, kind, P, *best);
            return SPO_OK;
        }
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != set->device) cudaSetDevice(set->device);
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    float *pos = nullptr, *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    spo_status st = SPO_OK;
    cudaError_t e = cudaMalloc(&pos, sizeof(float) * 3 * (size_t)P);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * (size_t)P * spo_rows(kind) * set->N);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        st = fail(SPO_ENOMEM, "autotune scratch allocation failed");
    }
    if (st == SPO_OK) {
        uniform_positions_kernel<<<152 * 8, 256, 0, cs>>>(pos, 3 * P, 0x5EEDull + (unsigned long long)P);
        if (cudaGetLastError() != cudaSuccess) st = fail(SPO_ECUDA, "position generation failed");
    }
    Candidate cands[16];
    int nc = 0;
    cands[nc++] = {SPO_ALGO_GATHER, 32, 4, 0};
    if (P < INT_MAX) cands[nc++] = {SPO_ALGO_SORTED_GATHER, 32, 4, 0};
    if (set->has_block_map && P < INT_MAX) {
        const int tiles[2] = {32, 64};
        for (int ti = 0; ti < 2; ++ti) {
            if (tiles[ti] == 64 && set->Np < 64) continue;
            for (int v = 2; v <= 4; v += 2) cands[nc++] = {SPO_ALGO_BRICK, tiles[ti], v, 0};
            cands[nc++] = {SPO_ALGO_BRICK, tiles[ti], 4, 1};
        }
    }
    const int saved_tile = set->brick_tile, saved_vec = set->brick_vec,
              saved_sched = set->brick_schedule;
    spo_tuning winner;
    memset(&winner, 0, sizeof(winner));
    winner.ms = 1e30f;
    for (int c = 0; st == SPO_OK && c < nc; ++c) {
        set->brick_tile = cands[c].tile;
        set->brick_vec = cands[c].vec;
        set->brick_schedule = cands[c].schedule;
        const int reps = 3;
        st = spo_detail::eval_queue(set, kind, pos, P, out, cs, cands[c].algo);   // warm-up
        if (st != SPO_OK) break;
        cudaEventRecord(e0, cs);
        for (int r = 0; r < reps && st == SPO_OK; ++r)
            st = spo_detail::eval_queue(set, kind, pos, P, out, cs, cands[c].algo);
        cudaEventRecord(e1, cs);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(SPO_ECUDA, "autotune timing failed");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (st == SPO_OK && ms < winner.ms) {
            winner.algo = cands[c].algo;
            winner.brick_tile = cands[c].tile;
            winner.brick_vec = cands[c].vec;
            winner.brick_schedule = cands[c].schedule;
            winner.ms = ms;
        }
    }
    set->brick_tile = saved_tile;
    set->brick_vec = saved_vec;
    set->brick_schedule = saved_sched;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(pos);   // cudaFree waits for the timed work
    cudaFree(out);
    if (prev >= 0 && prev != set->device) cudaSetDevice(prev);
    if (st != SPO_OK) return st;
    winner.from_cache = 0;
    apply(set, kind, P, winner);
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        g_cache[key] = winner;
        append_file_cache(key, winner);
    }
    *best = winner;
    return SPO_OK;
}
