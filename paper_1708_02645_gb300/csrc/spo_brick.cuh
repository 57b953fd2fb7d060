// Brick kernel: one CTA per (brick, orbital tile of 32 or 64 orbitals).
//
// Positions are binned by brick (kBrick^3 cells, spo_bin.cu).  Every window
// of a position in brick (bx, by, bz) lies in the padded table nodes
// [4bx, 4bx+7) x [4by, 4by+7) x [4bz, 4bz+7), so one TMA copy (a 4-D box of
// tile x 7 x 7 x 7 nodes, 88 KB for 64 FP32 orbitals) stages everything the
// brick's positions need for one orbital tile.  The positions of the brick
// are then evaluated from shared memory (2 or 4 orbitals per thread, so a
// corner row is one conflict-free 8- or 16-byte shared load per thread for
// FP32, 4 or 8 bytes for BF16/FP16); positions are read as sorted
// (x, y, z, index) records written by the binning, one round ahead; each
// position's 36 weights, cells and index are formed once per batch by the
// binning (a 176-byte weight record per position, spo_device.cuh
// make_weight_record), and every orbital tile's CTA copies the records of
// its positions into slots in shared memory, one round ahead (without
// records, three lanes of a position's group form its slot); the
// z -> y -> x reduction and its FMA order are
// those of the gather kernel (spo_device.cuh), and outputs are scattered
// back to each position's own rows with streaming stores.  With 32-orbital
// tiles and at least two bricks along z, a CTA takes a z-adjacent pair of
// bricks instead (PAIR: one 7 x 7 x 11-node box).
//
// Against the gather kernel, the table bytes moved from L2 to the SMs drop
// from 64 rows per evaluation to 343 rows per (brick, tile), and the L2 sees
// neighbouring bricks' blocks in launch order, so DRAM reads approach one
// pass over the table per batch.  Two (64-orbital tiles), three (brick
// pairs) or four (32-orbital tiles) CTAs run per SM, so one CTA's copy
// overlaps the others' arithmetic.
//
// The wait on the copy is bounded (2 s of %globaltimer): if it ever gives up,
// the CTA sets bit 0 of the device status word and returns.
//
// The kernel templates and their launchers; spo_brick_f32.cu, spo_brick_bf16.cu
// and spo_brick_f16.cu each instantiate them for one storage type (so the
// three compile in parallel), and spo_brick.cu dispatches on the set's type.
// Included by those three translation units only.
#pragma once

#include <cuda.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "spo_batch.h"
#include "spo_device.cuh"
#include "spo_internal.h"
#include "spo_tma.cuh"

namespace {


using namespace spo_dev;
using spo_detail::kBlockEdge;
using spo_detail::kBrick;

constexpr int kBlockRows = kBlockEdge * kBlockEdge * kBlockEdge;   // 343
// Threads per CTA and CTAs per SM for an orbital tile: a 64-orbital FP32
// block is 88 KB (2 CTAs of 256 threads per SM), a 32-orbital one 44 KB
// (4 CTAs of 128 threads); either way 16 warps and at most 128 registers per
// thread.
template <int TILE>
struct BrickShape {
    static constexpr int threads = TILE >= 64 ? 256 : 128;
    static constexpr int ctas_per_sm = TILE >= 64 ? 2 : 4;
};

// bytes of the weight slots of a CTA: one slot per position of a round
template <int TILE, int V>
constexpr size_t kSlotBytes = (size_t)(BrickShape<TILE>::threads / (TILE / V)) * kSlotF4 * 16;


// RATIO (KIND = V only): each position's values are also multiplied by its
// row of A^-1 and reduced over the position's lanes; one partial dot product
// per (tile, position) goes to ra.partials.  out may then be nullptr.
//
// PAIR: one CTA per (z-adjacent pair of bricks, tile); the pair's block is
// one 7 x 7 x 11-node TMA box (69 KB for 32 FP32 orbitals, 3 CTAs per SM)
// and its positions are the two bricks' contiguous ranges of the sorted
// order, so each CTA evaluates twice as many positions per staged node and
// per start-up.  The arithmetic per position is unchanged (same bits).
// REC: the binning formed every position's weight record (wrec), and each
// orbital tile copies them into its slots; without REC the slots are formed
// here from the sorted position records (the allocation-free entry point,
// whose fixed scratch holds no records).
// The pair form runs 3 CTAs per SM with FP32 blocks (72 KB of shared memory
// each) and 4 with 16-bit blocks (half the bytes; 128 registers, a few
// bytes spilled): BF16 VGH 0.483 -> 0.467 ms, FP16 0.553 -> 0.539 ms.
template <typename T, int KIND, int TILE, int V, bool VEC_OUT, bool RATIO = false, bool PAIR = false,
          bool REC = true>
__global__ void __launch_bounds__(BrickShape<TILE>::threads,
                                  PAIR ? (sizeof(T) == 2 ? 4 : 3) : BrickShape<TILE>::ctas_per_sm)
spo_brick_kernel(const __grid_constant__ CUtensorMap map, GridAxis gx, GridAxis gy, GridAxis gz,
                 int nby, int nbz, int ntiles, int64_t N, const int *__restrict__ offsets,
                 const float4 *__restrict__ sorted, const float4 *__restrict__ wrec,
                 float *__restrict__ out, int eager, spo_detail::RatioArgs ra,
                 unsigned int *__restrict__ status)
{
    static_assert(!RATIO || KIND == SPO_KIND_V, "ratios are formed from values");
    constexpr int NC = Rows<KIND>::value;
    constexpr int kThreads = BrickShape<TILE>::threads;
    constexpr int kVec = V;                   // orbitals per thread
    constexpr int TPP = TILE / kVec;          // threads per position
    constexpr int PPR = kThreads / TPP;       // positions per round
    constexpr int kBZ = PAIR ? 2 * kBrick + 3 : kBlockEdge;   // block nodes along z
    constexpr uint32_t kBytes = kBlockEdge * kBlockEdge * kBZ * TILE * sizeof(T);
    extern __shared__ __align__(1024) unsigned char smem[];
    T *block = reinterpret_cast<T *>(smem);   // [7][7][7][TILE]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kBytes);
    float4 *wslots = reinterpret_cast<float4 *>(smem + kBytes + 16);   // [PPR][kSlotF4]

    const int brick = blockIdx.x / ntiles;
    const int tile = blockIdx.x - brick * ntiles;
    // brick (bx, by, bz) is bin (bx nby + by) nbz + bz of the sorted order
    const int nbzu = PAIR ? (nbz + 1) / 2 : nbz;
    const int bzu = brick % nbzu, by = (brick / nbzu) % nby, bx = brick / (nbzu * nby);
    const int bz = PAIR ? 2 * bzu : bzu;
    const int b0 = (bx * nby + by) * nbz + bz;
    const int b1 = b0 + ((PAIR && bz + 1 < nbz) ? 2 : 1);
    const uint32_t bar_s = smem_addr(bar);

    // With `eager` (bricks hold several positions on average) the copy is
    // issued first and the brick's position range is read while it flies;
    // otherwise empty bricks are skipped before any copy.
    // Launched as a programmatic dependent of the binning: the table block
    // depends only on the table, so its copy is issued before waiting for
    // the binning (offsets, sorted records, weight records).
    int begin = 0, end = 0;
    if (!eager) {
        grid_dependency_wait();
        begin = __ldg(offsets + b0);
        end = __ldg(offsets + b1);
        if (begin == end) return;
    }
    if (threadIdx.x == 0) {
        mbar_init(bar_s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar_s, kBytes);
        tma_load_4d(smem_addr(block), &map, bar_s, tile * TILE, bz * kBrick, by * kBrick, bx * kBrick);
    }
    if (eager) {
        grid_dependency_wait();
        begin = __ldg(offsets + b0);
        end = __ldg(offsets + b1);
    }
    __syncthreads();   // the barrier's initialisation is visible to every thread
    if (begin == end) {   // (eager only) nothing to do, but the copy must land first
        if (threadIdx.x == 0 && !mbar_wait_bounded(bar_s, 0)) atomicOr(status, 1u);
        return;
    }

    const int q = threadIdx.x % TPP;
    // positions are taken in rounds of PPR; the trip count of the loop is
    // uniform over each warp (groups past the end sit the round out), so the
    // warp can share the weight slots
    const int wg0 = (int)(threadIdx.x >> 5) * (32 / TPP);   // first position group of this warp
    float4 *slot = wslots + (threadIdx.x / TPP) * kSlotF4;
    int i = begin + threadIdx.x / TPP;
    // Each round, lane q of a position's group brings parts q, q + TPP, ...
    // of the position's weight slot: copies of the record the binning formed
    // (REC), or else the slot formed here from the position record (x, y,
    // z, index) in part 0.  Both are loaded one round early.
    constexpr int NPART = REC ? (kSlotF4 + TPP - 1) / TPP : 1;
    auto fetch = [&](int ii, float4 (&r)[NPART]) {
        if (ii >= end) return;
        if constexpr (REC) {
#pragma unroll
            for (int k = 0; k < NPART; ++k)
                if (q + k * TPP < kSlotF4) r[k] = __ldg(wrec + (int64_t)ii * kSlotF4 + q + k * TPP);
        } else {
            r[0] = __ldg(sorted + ii);
        }
    };
    float4 cur[NPART];
#pragma unroll
    for (int k = 0; k < NPART; ++k) cur[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    fetch(i, cur);
    bool ready = false;
    for (int ib = begin + wg0; ib < end; ib += PPR, i += PPR) {
        float4 nxt[NPART];
#pragma unroll
        for (int k = 0; k < NPART; ++k) nxt[k] = cur[k];
        fetch(i + PPR, nxt);
        __syncwarp();   // the previous round's reads of the slots are done
        if constexpr (REC) {
#pragma unroll
            for (int k = 0; k < NPART; ++k)
                if (q + k * TPP < kSlotF4) slot[q + k * TPP] = cur[k];
        } else {
            stage_axis_weights(q, cur[0], gx, gy, gz, slot);
        }
        __syncwarp();
        if (!ready) {   // the first round's weights were formed while the copy flew
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar_s, 0))) {
                if ((threadIdx.x & 31) == 0) atomicOr(status, 1u);
                return;
            }
            ready = true;
        }
        // Evaluates the position whose weight slot is sl on KV orbitals from
        // orbital o of the tile (lane kq of the position's TILE / KV lanes).
        auto eval = [&](auto kv, const float4 *sl, int kq) {
            constexpr int KV = decltype(kv)::value;
            Axis Y, Z;
            const int4 cells = *reinterpret_cast<const int4 *>(sl + 10);
            const int p = cells.w;
            unpack4(sl[4], Y.w);
            unpack4(sl[5], Y.d);
            unpack4(sl[6], Y.dd);
            unpack4(sl[7], Z.w);
            unpack4(sl[8], Z.d);
            unpack4(sl[9], Z.dd);
            // the binning put the cell in this brick; the clamp keeps the
            // shared memory index in range even if it had not (debug builds
            // check it, and the record's position index)
            const int ux = cells.x - bx * kBrick, uy = cells.y - by * kBrick, uz = cells.z - bz * kBrick;
            if (!bounds_ok(ux >= 0 && ux < kBrick && uy >= 0 && uy < kBrick && uz >= 0 &&
                               uz < (PAIR ? 2 : 1) * kBrick && p >= 0,
                           status))
                return;
            const int lx = min(max(ux, 0), kBrick - 1);
            const int ly = min(max(uy, 0), kBrick - 1);
            const int lz = min(max(uz, 0), (PAIR ? 2 : 1) * kBrick - 1);
            const T *base = block + ((lx * kBlockEdge + ly) * kBZ + lz) * TILE + kq * KV;
            const int64_t ko0 = (int64_t)tile * TILE + kq * KV;   // first orbital of this lane
            float acc[NC][KV];
            window_reduce_staged<KIND, KV, true>(sl, Y, Z,
                                [&](int a, int b, int g, float *v) {
                                    load_coefs<T, KV, false>(
                                        base + ((a * kBlockEdge + b) * kBZ + g) * TILE, v);
                                },
                                acc);
            if constexpr (RATIO) {
                int r = ra.row_of ? __ldg(ra.row_of + p) : p;
                r = (int)min(max((int64_t)r, (int64_t)0), ra.nrows - 1);
                const float *arow = ra.rows + (int64_t)r * ra.ld + ko0;
                float dot = 0.0f;
#pragma unroll
                for (int k = 0; k < KV; ++k)
                    if (ko0 + k < N) dot = fmaf(acc[0][k], __ldg(arow + k), dot);
                // the TPP lanes of this position form an aligned group of the warp
                const unsigned lane = threadIdx.x & 31u;
                const unsigned gmask = TPP >= 32 ? 0xffffffffu
                                                 : (((1u << TPP) - 1u) << (lane & ~(unsigned)(TPP - 1)));
#pragma unroll
                for (int off = TPP / 2; off > 0; off >>= 1) dot += __shfl_xor_sync(gmask, dot, off);
                if (kq == 0) ra.partials[(int64_t)tile * ra.P + p] = dot;
            }
            if (ko0 < N && (!RATIO || out != nullptr))
                store_rows<NC, KV, VEC_OUT>(out + (int64_t)p * NC * N + ko0, N, N - ko0, acc);
        };
        // A warp whose last round holds 1 or 2 positions gives each of them
        // 16 lanes of 2 orbitals (the same arithmetic per orbital, so the
        // same bits) instead of running with 2 or 3 of its 4 groups idle.
        constexpr bool kRemap = !RATIO && kVec == 4 && TPP == 8;
        if (kRemap && end - ib <= 2) {
            const int half = (int)(threadIdx.x & 31) >> 4;
            if (half < end - ib) eval(std::integral_constant<int, 2>{}, wslots + (wg0 + half) * kSlotF4,
                                      (int)(threadIdx.x & 15));
        } else if (i < end) {
            eval(std::integral_constant<int, kVec>{}, slot, q);
        }
#pragma unroll
        for (int k = 0; k < NPART; ++k) cur[k] = nxt[k];
    }
    if (!ready && threadIdx.x == 0) {
        // a thread with no position still must not leave while the copy
        // writes shared memory that another CTA could reuse
        if (!mbar_wait_bounded(bar_s, 0)) atomicOr(status, 1u);
    }
}

// ---------------------------------------------------------------------------
// persistent, software-pipelined brick kernel
// ---------------------------------------------------------------------------
// One CTA per SM (16 warps).  CTA c owns items c, c + G, c + 2G, ... (G =
// grid size; an item is a (brick, orbital tile) pair; empty bricks are
// skipped), so the CTAs of the GPU sweep the table together and neighbouring
// blocks meet in L2.  NBUF slots rotate through shared memory; filling a
// slot means: write the item's metadata (brick, tile, first sorted position,
// count), then one mbarrier transaction that carries the TMA copy of the
// item's block and a bulk copy of up to kStage of its sorted position
// records.  Consumers therefore read control data and positions from shared
// memory only.  The slot of item k is refilled with item k + NBUF by the last
// warp to finish with item k, so copies run NBUF - 1 items ahead.
//
// Work is cut into tasks of 4 positions (one per 8-lane group, 4 orbitals
// per lane, TILE / 32 passes), items padded to whole tasks.  Warp w takes
// tasks w, w + 16, w + 32, ... of the CTA's task stream, so a warp never
// waits for the other warps of an item.  Every warp waits on every slot
// fill in sequence order (this keeps barrier phases unambiguous) and
// releases every item in order once its next task lies beyond it.  The fill
// after the last item carries an end marker.  The fill for item m is issued
// once every warp released item m - NBUF; the earliest item not yet released
// by all warps always has its fill issued, so the pipeline cannot deadlock.
// Waits are bounded (bit 0 of the device status word on time-out).
constexpr int kStage = 128;   // position records staged per item

struct __align__(16) SlotMeta {
    int j;        // index of the item in the CTA's sequence (-1: end marker)
    int cnt;      // positions in the brick
    int begin;    // first sorted position of the brick
    int tile;     // orbital tile
    int bx, by, bz;   // brick coordinates
    int pad;
};

template <typename T, int TILE>
struct PipeShape {
    static constexpr int threads = 512;
    static constexpr int warps = threads / 32;
    static constexpr uint32_t block_bytes = kBlockRows * TILE * sizeof(T);
    static constexpr uint32_t block_stride = (block_bytes + 1023u) / 1024u * 1024u;
    static constexpr uint32_t stage_bytes = kStage * 16u;
    static constexpr int buffers_fit = (int)((200u * 1024u) / (block_stride + stage_bytes));
    static constexpr int nbuf = buffers_fit >= 4 ? 4 : (buffers_fit >= 3 ? 3 : 2);
    static constexpr size_t stage_off = (size_t)nbuf * block_stride;
    static constexpr size_t meta_off = stage_off + (size_t)nbuf * stage_bytes;
    static constexpr size_t bar_off = meta_off + (size_t)nbuf * sizeof(SlotMeta);
    static constexpr size_t rel_off = bar_off + 8 * (size_t)nbuf;
    static constexpr size_t smem = rel_off + 4 * (size_t)nbuf;
};

template <typename T, int KIND, int TILE, bool VEC_OUT>
__global__ void __launch_bounds__(512, 1)
spo_brick_pipe_kernel(const __grid_constant__ CUtensorMap map, GridAxis gx, GridAxis gy, GridAxis gz,
                      int nby, int nbz, int ntiles, int nitems, int64_t N,
                      const int *__restrict__ offsets, const float4 *__restrict__ sorted,
                      float *__restrict__ out, unsigned int *__restrict__ status)
{
    using Shape = PipeShape<T, TILE>;
    constexpr int NC = Rows<KIND>::value;
    constexpr int NBUF = Shape::nbuf;
    constexpr int NWARPS = Shape::warps;
    constexpr int PASSES = TILE / 32;
    constexpr int kVec = 4;
    extern __shared__ __align__(1024) unsigned char smem[];
    const float4 *stage = reinterpret_cast<const float4 *>(smem + Shape::stage_off);
    SlotMeta *meta = reinterpret_cast<SlotMeta *>(smem + Shape::meta_off);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + Shape::bar_off);
    int *released = reinterpret_cast<int *>(smem + Shape::rel_off);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int group = lane >> 3, gl = lane & 7;
    const int G = gridDim.x;

    // producer helpers (one thread at a time): the smallest j' >= j whose
    // item is non-empty, or -1; and the fill of a slot
    auto next_nonempty = [&](int j) -> int {
        for (;; ++j) {
            const int64_t item = (int64_t)blockIdx.x + (int64_t)j * G;
            if (item >= nitems) return -1;
            const int b = (int)(item / ntiles);
            if (__ldg(offsets + b + 1) > __ldg(offsets + b)) return j;
        }
    };
    auto fill = [&](int j, int slot) {
        const uint32_t bar = smem_addr(full + slot);
        SlotMeta &sm = meta[slot];
        if (j < 0) {   // end marker: no copy, the arrival alone completes the phase
            sm.j = -1;
            sm.cnt = 0;
            mbar_arrive(bar);
            return;
        }
        const int item = blockIdx.x + j * G;
        const int brick = item / ntiles, tile = item - brick * ntiles;
        const int begin = __ldg(offsets + brick), cnt = __ldg(offsets + brick + 1) - begin;
        const int bz = brick % nbz, by = (brick / nbz) % nby, bx = brick / (nbz * nby);
        sm.j = j;
        sm.cnt = cnt;
        sm.begin = begin;
        sm.tile = tile;
        sm.bx = bx;
        sm.by = by;
        sm.bz = bz;
        const int staged = min(cnt, kStage);
        mbar_arrive_expect_tx(bar, Shape::block_bytes + 16u * (uint32_t)staged);
        tma_load_4d(smem_addr(smem + (size_t)slot * Shape::block_stride), &map, bar, tile * TILE,
                    bz * kBrick, by * kBrick, bx * kBrick);
        bulk_load(smem_addr(stage + (size_t)slot * kStage), sorted + begin, 16u * (uint32_t)staged,
                  bar);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < NBUF; ++s) {
            mbar_init(smem_addr(full + s), 1);
            released[s] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // the first NBUF fills (end marker after the last item)
        int j = next_nonempty(0);
        for (int s = 0; s < NBUF; ++s) {
            fill(j, s);
            if (j < 0) break;
            j = next_nonempty(j + 1);
        }
    }

    // warp-uniform cursor: sequence number k of the current item and the
    // task just past it (its metadata stays in the slot, read per task)
    int k = 0, tend = 0;
    auto enter = [&](int kk) -> bool {   // wait for item kk's fill; false at the end
        const int slot = kk % NBUF;
        if (!mbar_wait_bounded(smem_addr(full + slot), (kk / NBUF) & 1)) {
            if (lane == 0) atomicOr(status, 1u);
            return false;
        }
        if (meta[slot].j < 0) return false;
        tend += (meta[slot].cnt + 3) >> 2;
        return true;
    };
    if (!enter(0)) return;

    for (int t = warp;; t += NWARPS) {
        // move past items wholly before task t: release each in order; the
        // last warp to release item k refills its slot with item k + NBUF
        while (t >= tend) {
            const int slot = k % NBUF;
            __syncwarp();
            if (lane == 0 && atomicAdd(released + slot, 1) == NWARPS - 1) {
                int ja = meta[slot].j;
                released[slot] = 0;
                for (int s = 0; s < NBUF && ja >= 0; ++s) ja = next_nonempty(ja + 1);
                fill(ja, slot);
            }
            __syncwarp();
            ++k;
            if (!enter(k)) return;
        }
        const int slot = k % NBUF;
        const SlotMeta sm = meta[slot];
        const int local = (t - (tend - ((sm.cnt + 3) >> 2))) * 4 + group;
        if (local < sm.cnt) {
            const float4 rec = local < kStage ? stage[slot * kStage + local]
                                              : __ldg(sorted + sm.begin + local);
            const int p = __float_as_int(rec.w);
            XAxis X;
            Axis Y, Z;
            make_xaxis(rec.x, gx, X);
            make_axis(rec.y, gy, Y);
            make_axis(rec.z, gz, Z);
            const int ux = X.cell - sm.bx * kBrick, uy = Y.cell - sm.by * kBrick, uz = Z.cell - sm.bz * kBrick;
            const bool inside = bounds_ok(ux >= 0 && ux < kBrick && uy >= 0 && uy < kBrick && uz >= 0 &&
                                              uz < kBrick && p >= 0,
                                          status);
            const int lx = min(max(ux, 0), kBrick - 1);
            const int ly = min(max(uy, 0), kBrick - 1);
            const int lz = min(max(uz, 0), kBrick - 1);
            const T *block = reinterpret_cast<const T *>(smem + (size_t)slot * Shape::block_stride);
            const int64_t tile0 = (int64_t)sm.tile * TILE;
#pragma unroll 1
            for (int pass = 0; pass < PASSES && inside; ++pass) {
                const int o_tile = pass * 32 + gl * kVec;   // orbital within the tile
                const T *base = block + ((lx * kBlockEdge + ly) * kBlockEdge + lz) * TILE + o_tile;
                float acc[NC][kVec];
                window_reduce<KIND, kVec, true>(X, gx, Y, Z,
                                    [&](int a, int b, int g, float *v) {
                                        load_coefs<T, kVec, false>(
                                            base + ((a * kBlockEdge + b) * kBlockEdge + g) * TILE, v);
                                    },
                                    acc);
                const int64_t o0 = tile0 + o_tile;
                if (o0 < N)
                    store_rows<NC, kVec, VEC_OUT>(out + (int64_t)p * NC * N + o0, N, N - o0, acc);
            }
        }
    }
}

// Launch as a programmatic dependent of the previous kernel in the stream
// (the binning's scatter): CTAs may be scheduled while it finishes and wait
// for it in the kernel (grid_dependency_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                             cudaStream_t stream, Args &&...args) {
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename T, int KIND, int TILE, int V, bool REC = true>
cudaError_t brick_launch(const spo_set *s, const spo_detail::Workspace &w, int64_t P, float *out,
                         cudaStream_t stream) {
    const int nbins = s->nbx * s->nby * s->nbz;
    const int ntiles = (int)((s->N + TILE - 1) / TILE);
    const bool vec_out = (s->N % V == 0) && ((reinterpret_cast<uintptr_t>(out) % (4 * V)) == 0);
    const int eager = P >= 4 * (int64_t)nbins;   // about 4+ positions per brick
    if constexpr (TILE == 32) {
      if (s->has_pair_map) {   // 32-orbital tiles on z-adjacent brick pairs
        constexpr size_t kSmemP = (size_t)kBlockEdge * kBlockEdge * (2 * kBrick + 3) * TILE * sizeof(T) + 16 +
                                 kSlotBytes<TILE, V>;
        const int64_t blocks = (int64_t)s->nbx * s->nby * ((s->nbz + 1) / 2) * ntiles;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        auto kernel = vec_out ? spo_brick_kernel<T, KIND, TILE, V, true, false, true, REC>
                              : spo_brick_kernel<T, KIND, TILE, V, false, false, true, REC>;
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemP);
        if (e != cudaSuccess) return e;
        return launch_dependent(kernel, (unsigned)blocks, BrickShape<TILE>::threads, kSmemP, stream,
                                s->block_map[2], grid_axis(s->nx), grid_axis(s->ny), grid_axis(s->nz), s->nby,
                                s->nbz, ntiles, s->N, w.offsets, w.sorted, w.wrec, out, eager,
                                spo_detail::RatioArgs{}, s->status);
      }
    }
    constexpr size_t kSmem = (size_t)kBlockRows * TILE * sizeof(T) + 16 + kSlotBytes<TILE, V>;
    const int64_t blocks = (int64_t)nbins * ntiles;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    auto kernel = vec_out ? spo_brick_kernel<T, KIND, TILE, V, true, false, false, REC>
                          : spo_brick_kernel<T, KIND, TILE, V, false, false, false, REC>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    const CUtensorMap &map = s->block_map[TILE == 64 ? 1 : 0];
    return launch_dependent(kernel, (unsigned)blocks, BrickShape<TILE>::threads, kSmem, stream, map,
                            grid_axis(s->nx), grid_axis(s->ny), grid_axis(s->nz), s->nby, s->nbz, ntiles, s->N,
                            w.offsets, w.sorted, w.wrec, out, eager, spo_detail::RatioArgs{}, s->status);
}

template <typename T, int TILE, int V>
cudaError_t brick_ratio_launch(const spo_set *s, const spo_detail::Workspace &w, int64_t P,
                               float *out, const spo_detail::RatioArgs &ra, cudaStream_t stream) {
    if (!w.wrec) return cudaErrorInvalidValue;   // ratio workspaces always hold weight records
    constexpr size_t kSmem = (size_t)kBlockRows * TILE * sizeof(T) + 16 + kSlotBytes<TILE, V>;
    const int nbins = s->nbx * s->nby * s->nbz;
    const int ntiles = (int)((s->N + TILE - 1) / TILE);
    const int64_t blocks = (int64_t)nbins * ntiles;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const bool vec_out = out && (s->N % V == 0) && ((reinterpret_cast<uintptr_t>(out) % (4 * V)) == 0);
    auto kernel = vec_out ? spo_brick_kernel<T, SPO_KIND_V, TILE, V, true, true>
                          : spo_brick_kernel<T, SPO_KIND_V, TILE, V, false, true>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    const CUtensorMap &map = s->block_map[TILE == 64 ? 1 : 0];
    const int eager = P >= 4 * (int64_t)nbins;
    kernel<<<(unsigned)blocks, BrickShape<TILE>::threads, kSmem, stream>>>(
        map, grid_axis(s->nx), grid_axis(s->ny), grid_axis(s->nz), s->nby, s->nbz, ntiles, s->N,
        w.offsets, w.sorted, w.wrec, out, eager,
        ra, s->status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t brick_ratio_all(const spo_set *s, const spo_detail::Workspace &w, int64_t P,
                              float *out, const spo_detail::RatioArgs &ra, cudaStream_t stream) {
    const bool v4 = s->brick_vec == 4;
    if (spo_detail::brick_tile_of(s) == 64)
        return v4 ? brick_ratio_launch<T, 64, 4>(s, w, P, out, ra, stream)
                  : brick_ratio_launch<T, 64, 2>(s, w, P, out, ra, stream);
    return v4 ? brick_ratio_launch<T, 32, 4>(s, w, P, out, ra, stream)
              : brick_ratio_launch<T, 32, 2>(s, w, P, out, ra, stream);
}

template <typename T, int KIND, int TILE>
cudaError_t brick_pipe_launch(const spo_set *s, const spo_detail::Workspace &w, float *out,
                              cudaStream_t stream) {
    using Shape = PipeShape<T, TILE>;
    const int nbins = s->nbx * s->nby * s->nbz;
    const int ntiles = (int)((s->N + TILE - 1) / TILE);
    const int64_t nitems = (int64_t)nbins * ntiles;
    if (nitems > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const bool vec_out = (s->N % 4 == 0) && ((reinterpret_cast<uintptr_t>(out) % 16) == 0);
    auto kernel = vec_out ? spo_brick_pipe_kernel<T, KIND, TILE, true>
                          : spo_brick_pipe_kernel<T, KIND, TILE, false>;
    cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Shape::smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(nitems, s->num_sms);
    kernel<<<grid, Shape::threads, Shape::smem, stream>>>(
        s->block_map[TILE == 64 ? 1 : 0], grid_axis(s->nx), grid_axis(s->ny), grid_axis(s->nz),
        s->nby, s->nbz, ntiles, (int)nitems, s->N, w.offsets, w.sorted, out, s->status);
    return cudaGetLastError();
}

template <typename T, int KIND>
cudaError_t brick_typed(const spo_set *s, const spo_detail::Workspace &w, int64_t P, float *out,
                        cudaStream_t stream) {
    if (s->brick_schedule == 1)
        return spo_detail::brick_tile_of(s) == 64 ? brick_pipe_launch<T, KIND, 64>(s, w, out, stream)
                                                  : brick_pipe_launch<T, KIND, 32>(s, w, out, stream);
    // without weight records (the allocation-free scratch) one tuning serves:
    // every tuning gives the same bits
    if (!w.wrec) return brick_launch<T, KIND, 32, 4, false>(s, w, P, out, stream);
    const bool v4 = s->brick_vec == 4;
    if (spo_detail::brick_tile_of(s) == 64)
        return v4 ? brick_launch<T, KIND, 64, 4>(s, w, P, out, stream)
                  : brick_launch<T, KIND, 64, 2>(s, w, P, out, stream);
    return v4 ? brick_launch<T, KIND, 32, 4>(s, w, P, out, stream)
              : brick_launch<T, KIND, 32, 2>(s, w, P, out, stream);
}

template <typename T>
cudaError_t brick_kind_all(spo_kind kind, const spo_set *s, const spo_detail::Workspace &w, int64_t P,
                       float *out, cudaStream_t stream) {
    switch (kind) {
        case SPO_KIND_V: return brick_typed<T, SPO_KIND_V>(s, w, P, out, stream);
        case SPO_KIND_VGL: return brick_typed<T, SPO_KIND_VGL>(s, w, P, out, stream);
        case SPO_KIND_VGH: return brick_typed<T, SPO_KIND_VGH>(s, w, P, out, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

namespace spo_detail {

template <typename T>
cudaError_t brick_eval_typed(spo_kind kind, const spo_set *s, const Workspace &w, int64_t P, float *out,
                             cudaStream_t stream) {
    return brick_kind_all<T>(kind, s, w, P, out, stream);
}

template <typename T>
cudaError_t brick_ratio_typed(const spo_set *s, const Workspace &w, int64_t P, float *out,
                              const RatioArgs &ra, cudaStream_t stream) {
    return brick_ratio_all<T>(s, w, P, out, ra, stream);
}

}  // namespace spo_detail
