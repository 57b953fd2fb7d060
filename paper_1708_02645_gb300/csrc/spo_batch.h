// Descriptors of a batched evaluation over several orbital sets (internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "spo.h"
#include "spo_device.cuh"

namespace spo_detail {

constexpr int kMaxBatchSets = SPO_BATCH_MAX_SETS;

// One set as the batched kernels see it.
struct BatchSetDesc {
    spo_dev::GridAxis gx, gy, gz;
    int nby, nbz;
    int nbins;        // bricks of this set
    int brick_base;   // first global brick of this set
    int ntiles;       // orbital tiles of the brick kernel
    int unit_base;    // first (brick or brick pair, tile) unit of this set
    int rows;         // output rows per position (1, 5 or 10)
    int pad;
    int64_t N;
};

// Everything the batched kernels need about the sets, passed by value as a
// __grid_constant__ parameter (the tensor maps must live in parameter space).
struct BatchParams {
    CUtensorMap maps[kMaxBatchSets];
    BatchSetDesc sets[kMaxBatchSets];
    int nsets;
    int total_units;
    int total_bricks;
    int eager;
    int pair;         // units are z-adjacent pairs of bricks (32-orbital tiles, pair maps)
};

// Binning of all walkers' positions into the global brick space: counts,
// keys and slots; then (after the scan) sorted records and the address of
// each position's first output row.
cudaError_t launch_batch_bin(const spo_work *items, const int64_t *item_start, int nitems,
                             int *item_of, int64_t Ptot, const BatchParams &bp, int *counts,
                             int *offsets, int *keys, int *slots, float4 *sorted, float **dst,
                             cudaStream_t stream);

// The brick kernel over every (set, brick, tile) unit of the batch.
cudaError_t launch_brick_batch(spo_dtype storage, spo_kind kind, int tile, const BatchParams &bp,
                               const int *offsets, const float4 *wrec, float *const *dst,
                               bool vec_out, unsigned int *status, cudaStream_t stream);

// Allow the batched brick kernels their dynamic shared memory (host, once).
cudaError_t prepare_brick_batch();

// Device address of the device status word (for kernels in other files).
cudaError_t device_status_address(unsigned int **addr);

// Exclusive scan of n counts into offsets[0..n] (one CTA).
cudaError_t launch_scan(const int *counts, int *offsets, int n, cudaStream_t stream);

}  // namespace spo_detail
