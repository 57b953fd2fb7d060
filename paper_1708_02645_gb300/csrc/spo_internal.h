// Internal declarations shared by the host API and the kernels.  Not part of
// the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "spo.h"

namespace spo_detail {

// Edge of a brick in cells: positions are binned by brick, and the brick
// kernel stages the (kBrick + 3)^3 table rows a brick's windows touch.
constexpr int kBrick = 4;
constexpr int kBlockEdge = kBrick + 3;
// float4 per weight record (a position's 36 basis weights, cells and index)
constexpr int kWeightRecordF4 = 11;

// Scratch of the binned path for one stream: brick counts and offsets, one
// key and slot per position, the position permutation sorted by brick, and
// the positions themselves in that order (x, y, z, original index as bits).
struct Workspace {
    cudaStream_t stream = nullptr;
    int *counts = nullptr;    // [nbins + 1], zero between binnings (the last: a ticket)
    int *offsets = nullptr;   // [nbins + 1]
    int *keys = nullptr;      // [P]
    int *slots = nullptr;     // [P]
    int *perm = nullptr;      // [P]
    float4 *sorted = nullptr; // [P]
    float4 *wrec = nullptr;   // [P][11] weight records in sorted order, or nullptr (the
                              // brick kernel then forms the weights itself)
    float *partials = nullptr;   // [ratio tiles][P] partial dot products (ratios)
    float *vscratch = nullptr;   // [P][N] values for the unfused ratio path
    size_t cap_partials = 0, cap_vscratch = 0;   // floats
    int64_t cap_positions = 0;
    int64_t cap_bins = 0;
    const float *binned_pos = nullptr;   // positions of the last binning
    int64_t binned_P = -1;
};

}  // namespace spo_detail

struct spo_set {
    int device = 0;
    int nx = 0, ny = 0, nz = 0;            // grid intervals
    int xp = 0, yp = 0, zp = 0;            // padded node counts, n + 3
    int nbx = 0, nby = 0, nbz = 0;         // bricks per axis
    int64_t N = 0;      // orbitals
    int64_t Np = 0;     // padded orbital stride of the table (multiple of 8)
    spo_dtype storage = SPO_F32;
    void *table = nullptr;   // [xp][yp][zp][Np] of the storage type; padded node
                             // i' holds grid node (i' - 1) mod n
    size_t table_bytes = 0;
    int brick_vec = 4;       // orbitals per thread in the brick kernel (2 or 4)
    int brick_tile = 32;     // orbitals per brick-kernel tile (32 or 64)
    int brick_schedule = 0;  // 0: one CTA per (brick, tile); 1: persistent pipelined CTAs
    int num_sms = 0;         // multiprocessors of the set's device
    // strategy chosen by spo_autotune for each kind, for batches near tuned_P
    int tuned_algo[3] = {0, 0, 0};
    int64_t tuned_P[3] = {0, 0, 0};
    CUtensorMap block_map[3];   // 4-D TMA maps of the table, boxes (32 | 64, 7, 7, 7) and
                                // (32, 11, 7, 7) for z-adjacent brick pairs
    bool has_block_map = false; // Np >= 32: the brick kernel can serve this set
    bool has_pair_map = false;  // block_map[2] exists (nz >= 8): 32-orbital tiles run on brick pairs
    unsigned int *status = nullptr;   // device status word (bit 0: a bounded wait gave up)

    // scratch of the binned path, one per stream (guarded by mu)
    std::mutex mu;
    std::vector<spo_detail::Workspace> ws;

    // staging for spo_eval_host: two streams, each with its own device
    // buffers for one chunk of positions and outputs
    cudaStream_t hstream[2] = {nullptr, nullptr};
    cudaEvent_t hevent[2] = {nullptr, nullptr};
    float *hpos[2] = {nullptr, nullptr};
    float *hout[2] = {nullptr, nullptr};
    size_t hpos_cap = 0, hout_cap = 0;   // bytes per buffer
};

namespace spo_detail {

// Records a formatted message for spo_last_error() and returns `status`.
spo_status fail(spo_status status, const char *fmt, ...);

// Queue one evaluation with explicit strategy (arguments checked, device
// current); SPO_ALGO_AUTO resolves through the set's tuning.
spo_status eval_queue(const spo_set *set, spo_kind kind, const float *pos, int64_t P, float *out,
                      cudaStream_t stream, spo_algo algo);

// The strategy SPO_ALGO_AUTO resolves to for this set, kind and batch size
// (the autotuned choice near the tuned size, else the measured rule).
spo_algo auto_algo(const spo_set *set, spo_kind kind, int64_t P);

// Geometry of one table as the kernels see it.
struct TableView {
    const void *table;
    int nx, ny, nz;      // intervals
    int yp, zp;          // padded node counts (y, z)
    int64_t N, Np;
};

inline TableView view_of(const spo_set *s) {
    return TableView{s->table, s->nx, s->ny, s->nz, s->yp, s->zp, s->N, s->Np};
}

// Gather kernel: one thread = 4 orbitals of one position, corner rows read
// straight from global memory.  perm == nullptr evaluates positions in
// order; otherwise thread-group i evaluates position perm[i].
cudaError_t launch_gather(spo_dtype storage, spo_kind kind, const TableView &t,
                          const float *pos, const int *perm, int64_t P, float *out,
                          cudaStream_t stream);

// Binning: counts/keys/slots, exclusive scan into offsets, permutation.
cudaError_t launch_bin(const float *pos, int64_t P, int nx, int ny, int nz, int nbx, int nby,
                       int nbz, Workspace &w, cudaStream_t stream);

// Brick kernel over all (brick, orbital tile) items of a binned batch.
cudaError_t launch_brick(spo_dtype storage, spo_kind kind, const spo_set *set,
                         const float *pos, const Workspace &w, int64_t P, float *out,
                         cudaStream_t stream);

// Convert the source coefficients of grid x-planes [x0, x1) (src_dtype,
// [x1-x0][ny][nz][N]) into every padded table row that holds one of them.
cudaError_t launch_convert(const void *src, spo_dtype src_dtype, int x0, int x1,
                           const spo_set *set, cudaStream_t stream);

// Arguments of the ratio epilogue of the V kernels.
struct RatioArgs {
    const float *rows;      // [nrows][ld]
    const int *row_of;      // [P] or nullptr
    int64_t nrows, ld;
    float *partials;        // [ntiles][P]
    int64_t P;
};

// The brick kernels of one storage type T (float, __nv_bfloat16, __half),
// instantiated in spo_brick_f32.cu, spo_brick_bf16.cu and spo_brick_f16.cu.
template <typename T>
cudaError_t brick_eval_typed(spo_kind kind, const spo_set *set, const Workspace &w, int64_t P, float *out,
                             cudaStream_t stream);
template <typename T>
cudaError_t brick_ratio_typed(const spo_set *set, const Workspace &w, int64_t P, float *out,
                              const RatioArgs &ra, cudaStream_t stream);

// Brick kernel for V with the ratio epilogue: per (tile, position) partial
// dot products into r.partials; values to out unless out is nullptr.
cudaError_t launch_brick_ratio(const spo_set *set, const Workspace &w, int64_t P, float *out,
                               const RatioArgs &r, cudaStream_t stream);

// ratio[p] = sum over tiles of partials[t][p], tiles in order.
cudaError_t launch_ratio_reduce(const float *partials, int ntiles, int64_t P, float *ratio,
                                cudaStream_t stream);

// ratio[p] = sum_j rows[row_of[p]][j] v[p][j] (one warp per position).
cudaError_t launch_ratio_dot(const float *v, int64_t P, int64_t N, const RatioArgs &r, float *ratio,
                             cudaStream_t stream);

// Number of orbital tiles of the brick kernel for a set.
int brick_tiles_of(const spo_set *set);

// Build the brick kernel's tensor maps for a set (host; driver entry point).
spo_status make_block_map(spo_set *set);

// Orbital tile the brick kernel uses for a set (brick_tile, limited by Np).
int brick_tile_of(const spo_set *set);

// Device-side error word (bounded waits that gave up); read and clear.
cudaError_t read_device_status(unsigned int *flags, bool clear, cudaStream_t stream);

}  // namespace spo_detail
