/*
 * spo.h — C ABI of libspo, GB300 (sm_103a) evaluation of periodic tricubic
 * B-spline single-particle orbitals (SPOs).
 *
 * The operation (arXiv 1708.02645): the Slater matrix of Sec. 3, eq. (sj),
 * has entries A(i,j) = phi_i(r_j); Alg. 1 needs, for each proposed electron
 * position, the values phi_i(r) of all orbitals ("ratio", through the
 * determinant lemma, eq. md_lemma) and their gradients and Laplacians
 * ("derivatives").  Sec. 6.1 names the B-spline routines Bspline-v,
 * Bspline-vgh and SPO-vgl; by Sec. 6.2 their data is a read-only table with
 * four indices (three grid axes and the orbital), shared by all threads,
 * read at random and bound by memory bandwidth; Sec. 5.2 keeps that table and its evaluation in
 * single precision.  The B-spline itself is cited, not printed, in Sec. 3;
 * this library uses the uniform cubic B-spline on the periodic unit cube:
 *
 *   phi_n(r) = sum_{m in Z^3} c[m mod n][n] prod_d B3(r_d n_d - m_d)
 *
 * with basis function m centred on grid node (m_x/n_x, m_y/n_y, m_z/n_z).
 *
 * Conventions shared by every call:
 *   - grid: n_x x n_y x n_z intervals on the unit cube, each n_d >= 4;
 *   - coefficient table: C order [nx][ny][nz][N], orbital index fastest;
 *   - positions: FP32, [P][3] (x, y, z per position), any finite value,
 *     wrapped periodically; NaN or Inf give unspecified values for that
 *     position but never an out-of-range access;
 *   - outputs: FP32, one row of N orbitals per component, rows contiguous
 *     per position (structure of arrays across orbitals):
 *       V   : [P][N]
 *       VGL : [P][5][N]    v, gx, gy, gz, lap
 *       VGH : [P][10][N]   v, gx, gy, gz, hxx, hxy, hxz, hyy, hyz, hzz
 *     Gradients and Hessians are Cartesian (d/dr, not d/du).
 *   - arithmetic: FP32 accumulation for every storage type.
 *
 * Errors: every call returns a status.  Argument errors are detected on the
 * host, before anything is launched, and return SPO_EINVAL (or
 * SPO_EUNSUPPORTED); spo_last_error() then describes the problem.  CUDA
 * errors map to SPO_ECUDA.  Evaluation calls are asynchronous on the given
 * stream unless stated otherwise.  No C++ exception crosses this interface.
 *
 * Streams are passed as void* holding a cudaStream_t (NULL = the legacy
 * default stream), so that this header needs no CUDA include.
 */
#ifndef SPO_H
#define SPO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPO_ABI_VERSION 1

typedef enum {
    SPO_OK = 0,
    SPO_EINVAL = 1,        /* bad argument: null pointer, bad size, wrong memory kind */
    SPO_ENOMEM = 2,        /* device or host allocation failed */
    SPO_ECUDA = 3,         /* a CUDA runtime call or launch failed */
    SPO_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    SPO_EUNSUPPORTED = 5   /* a valid request the library does not support */
} spo_status;

typedef enum {
    SPO_F64 = 0,   /* source coefficients only; never a storage type */
    SPO_F32 = 1,
    SPO_BF16 = 2,
    SPO_F16 = 3
} spo_dtype;

typedef enum {
    SPO_KIND_V = 0,     /* values only (Bspline-v)               1 row  */
    SPO_KIND_VGL = 1,   /* value, gradient, Laplacian (SPO-vgl)  5 rows */
    SPO_KIND_VGH = 2    /* value, gradient, Hessian (Bspline-vgh) 10 rows */
} spo_kind;

typedef struct {
    int32_t nx, ny, nz;
} spo_grid;

/* Evaluation strategy (all give the same values; see spo_eval_ex). */
typedef enum {
    SPO_ALGO_AUTO = 0,           /* library's choice from the batch shape */
    SPO_ALGO_GATHER = 1,         /* positions in given order, corner rows from global memory */
    SPO_ALGO_SORTED_GATHER = 2,  /* positions binned by brick first, then gathered */
    SPO_ALGO_BRICK = 3           /* binned; each brick's table block staged in shared memory */
} spo_algo;

/* Tuning parameters of a set (see spo_set_param). */
typedef enum {
    SPO_PARAM_BRICK_VEC = 0,  /* orbitals per thread in the brick kernel: 4 (default) or 2 */
    SPO_PARAM_BRICK_TILE = 1, /* orbitals per staged block: 32 (default) or 64 (32 when Np < 64) */
    SPO_PARAM_BRICK_SCHEDULE = 2 /* 0: one CTA per (brick, tile) (default); 1: one persistent
                                    CTA per SM with a pipeline of TMA-staged blocks (4 orbitals
                                    per thread; SPO_PARAM_BRICK_VEC then has no effect) */
} spo_param;

/* Opaque orbital set: one converted coefficient table resident on one GPU. */
typedef struct spo_set spo_set;

/*
 * spo_create — upload one orbital set (Sec. 6.2: the read-only table).
 *
 *   grid            n_x, n_y, n_z >= 4.
 *   coefs           [nx][ny][nz][N] coefficients of type src_dtype, on the
 *                   host (coefs_on_device == 0, pageable or pinned) or on the
 *                   current device (coefs_on_device != 0).  Read only; the
 *                   caller keeps ownership and may free it after return.
 *   src_dtype       SPO_F64, SPO_F32, SPO_BF16 or SPO_F16.
 *   N               number of orbitals, >= 1.
 *   storage         SPO_F32, SPO_BF16 or SPO_F16: type of the device table.
 *                   Conversion rounds to nearest even, once, from src_dtype;
 *                   FP16 subnormals are kept.
 *   out             receives the new set.
 *
 * The table is stored orbital-contiguous as [nx+3][ny+3][nz+3][Np] on the
 * device that is current at the call: padded node i' holds grid node
 * (i' - 1) mod n (3 ghost nodes per axis, so that every 4x4x4 window is a
 * contiguous box), Np = N rounded up to a multiple of 8, padding orbitals
 * zero.  (nx+3)(ny+3)(nz+3) must fit in int32.  The call is synchronous: on return the
 * table is ready and every temporary buffer is freed.  The library owns the
 * table until spo_destroy.
 */
spo_status spo_create(const spo_grid *grid, const void *coefs, spo_dtype src_dtype,
                      int64_t N, spo_dtype storage, int coefs_on_device, spo_set **out);

/* Free the set's device memory (synchronises the device first so that no
 * queued evaluation still reads it).  NULL is accepted and ignored. */
spo_status spo_destroy(spo_set *set);

/*
 * spo_eval_v / spo_eval_vgl / spo_eval_vgh — evaluate all N orbitals of the
 * set at P positions (Alg. 1 "ratio" needs V; "derivatives" need VGL; the
 * Hessian form is Bspline-vgh of Sec. 6.1).
 *
 *   pos     device pointer, FP32 [P][3].
 *   P       number of positions, >= 0 (0 launches nothing).
 *   out     device pointer, FP32, [P][N], [P][5][N] or [P][10][N].
 *   stream  cudaStream_t to launch on.
 *
 * pos and out must be device (or managed) memory of the set's device, must
 * not overlap, and must stay alive until the stream work completes.  The
 * call returns once the kernel is queued.
 */
spo_status spo_eval_v(const spo_set *set, const float *pos, int64_t P, float *out, void *stream);
spo_status spo_eval_vgl(const spo_set *set, const float *pos, int64_t P, float *out, void *stream);
spo_status spo_eval_vgh(const spo_set *set, const float *pos, int64_t P, float *out, void *stream);

/* The same three evaluations selected by kind (strategy SPO_ALGO_AUTO). */
spo_status spo_eval(const spo_set *set, spo_kind kind, const float *pos, int64_t P,
                    float *out, void *stream);

/*
 * spo_eval_ex — spo_eval with an explicit strategy.  The binned strategies
 * first sort the positions by brick of 4x4x4 cells (a counting sort in
 * device scratch memory owned by the set, one scratch area per stream,
 * allocated on first use of a stream or by spo_reserve, freed by
 * spo_destroy); SPO_ALGO_BRICK then stages each brick's 7x7x7-node block of
 * the table in shared memory with one TMA copy per orbital tile.  Every
 * strategy evaluates the same sums in the same order: outputs are
 * bit-identical across strategies.  SPO_ALGO_BRICK needs at least 32
 * padded orbitals and returns SPO_EUNSUPPORTED otherwise; binned strategies need P < 2^31.  Calls with the same set and
 * stream are ordered by the stream; calls on different streams use
 * different scratch areas.  A call that allocates scratch synchronises the
 * device and cannot be captured in a CUDA graph: call spo_reserve first.
 * SPO_ALGO_AUTO takes the set's tuned strategy (spo_autotune) for batches
 * within 4x of the tuned size, else decides by the mean number of positions
 * per brick r = P / bricks: GATHER for P < 1024 or r < 1.5, BRICK from r = 3
 * (VGH), 8 (VGL) or 12 (V) when the set has 32+ padded orbitals, and
 * SORTED_GATHER in between (crossovers measured on GB300).
 */
spo_status spo_eval_ex(const spo_set *set, spo_kind kind, const float *pos, int64_t P,
                       float *out, void *stream, spo_algo algo);

/*
 * spo_auto_algo — the strategy SPO_ALGO_AUTO takes for this set, kind and
 * batch size P (the rule above, or the tuned choice), written to *algo:
 * SPO_ALGO_GATHER, SPO_ALGO_SORTED_GATHER or SPO_ALGO_BRICK.  Host only;
 * SPO_EINVAL for a NULL argument, an unknown kind or P < 0.
 */
spo_status spo_auto_algo(const spo_set *set, spo_kind kind, int64_t P, spo_algo *algo);

/*
 * spo_eval_ratio — determinant ratios of proposed moves, fused with the
 * value evaluation (Sec. 3, Alg. 1 "ratio", eq. md_lemma: moving electron k
 * to r' gives det(A')/det(A) = row k of A^-1 dotted with (phi_1(r'), ...,
 * phi_N(r')); the non-local pseudopotential quadrature of the local energy
 * needs the same ratio at several points per electron).
 *
 *   pos      device, FP32 [P][3]: the proposed positions.
 *   rows     device, FP32 [nrows][ld]: rows of A^-1 (orbital index fastest,
 *            ld >= N).
 *   row_of   device, int32 [P]: the row of each position (NULL: row p, which
 *            needs nrows >= P).  Indices outside [0, nrows) are clamped.
 *   ratio    device, FP32 [P]: rho_p = sum_j rows[row_of[p]][j] phi_j(pos_p).
 *   v_out    device, FP32 [P][N] or NULL: the values themselves, if wanted.
 *
 * The values never go to memory unless v_out asks for them: each thread
 * multiplies its orbitals' values by the matching row entries and the
 * partial sums are reduced in a fixed order (deterministic; FP32
 * accumulation).  Uses the set's per-stream scratch like spo_eval_ex.
 */
spo_status spo_eval_ratio(const spo_set *set, const float *pos, int64_t P, const float *rows,
                          int64_t nrows, int64_t ld, const int32_t *row_of, float *ratio,
                          float *v_out, void *stream);

/*
 * spo_bin / spo_eval_binned — the two stages of the binned strategies, for
 * callers that evaluate several kinds at the same positions (for example V
 * for the ratio and then VGL for the derivatives of an accepted move, Alg. 1).
 * spo_bin sorts pos (device, [P][3]) by brick into the scratch of `stream`;
 * spo_eval_binned then evaluates with algo SPO_ALGO_SORTED_GATHER or
 * SPO_ALGO_BRICK from that binning, and must receive the same pos and P as
 * the last spo_bin on the same set and stream (else SPO_EINVAL).  pos must
 * not change in between.
 */
spo_status spo_bin(const spo_set *set, const float *pos, int64_t P, void *stream);
spo_status spo_eval_binned(const spo_set *set, spo_kind kind, const float *pos, int64_t P,
                           float *out, void *stream, spo_algo algo);

/*
 * spo_eval_noalloc — the same evaluation as spo_eval, for callers that must
 * not have the library allocate device memory: for example an application
 * whose own pool allocator owns the whole GPU budget, or a loop that cannot
 * take the device-wide synchronisation cudaMalloc and cudaFree may cause
 * while its streams are busy.  The paper has no counterpart to this call;
 * it exists for such callers only.
 *
 * It never allocates: its scratch (the position binning) is a fixed array
 * of about 7.9 MB in the library's device code, present on every device
 * that loads the library until the process exits.  The caller passes pos
 * and out exactly as for spo_eval.  Limits: P <= SPO_NOALLOC_MAX_POSITIONS
 * and a grid of at most SPO_NOALLOC_MAX_BRICKS bricks of 4x4x4 cells; larger
 * requests return SPO_EINVAL without launching anything.
 *
 * It takes the strategy spo_eval's SPO_ALGO_AUTO takes for the same set,
 * kind and P, so its outputs equal spo_eval's bit for bit.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with the set's device current, kept until the process exits:
 * after cudaDeviceReset do not call it again); make that first call before
 * any stream capture.  All calls on a device share the one array and it
 * keeps the last call's contents; each call first clears, on its stream,
 * what must start at zero (the brick counts).  Calls whose GPU work
 * overlaps, on different streams or from several host threads, race: they
 * give wrong results and may write outside their `out`, so order them (one
 * stream does).
 */
#define SPO_NOALLOC_MAX_POSITIONS 262144
#define SPO_NOALLOC_MAX_BRICKS 65536
spo_status spo_eval_noalloc(const spo_set *set, spo_kind kind, const float *pos, int64_t P,
                            float *out, void *stream);

/*
 * Batched crowds — many walkers, each with its own positions and output,
 * against several orbital sets, in one binning and one evaluation launch
 * (Sec. 4.1 and Alg. 1: a population of walkers is advanced together; the
 * paper's outlook, Sec. 6.5, proposes running over table tiles in parallel).
 *
 * spo_work describes one walker: `set` indexes the plan's sets, pos is device
 * FP32 [P][3], out device FP32 [P][rows][N of that set].
 *
 * spo_batch_create(sets, nsets, max_positions, max_items, &plan): a plan over
 *   up to SPO_BATCH_MAX_SETS sets of one storage type (the sets must outlive
 *   the plan; each needs >= 32 padded orbitals).  The plan allocates all
 *   scratch for up to max_positions positions in up to max_items walkers, so
 *   evaluations allocate nothing.
 * spo_batch_eval(plan, kind, items, nitems, stream): copies the item table
 *   to the device and queues the evaluation of every walker on `stream`
 *   (one binning over all sets' bricks, one launch of the brick kernel over
 *   every (set, brick, orbital tile)).  Asynchronous; items may be reused or
 *   freed on return.
 * spo_batch_graph(plan, kind, items, nitems, stream): records the same work
 *   for these items into a CUDA graph held by the plan (the item table is
 *   copied first, synchronously); spo_batch_launch(plan, stream) replays it.
 *   Between replays the caller may change the contents of the pos buffers
 *   (new moves), not the items themselves.
 * Calls on one plan must be ordered (one stream): they share its scratch.
 *
 * spo_eval_batch(sets, nsets, items, nitems, kind, stream): one-call form.
 *   When the sets can share a plan (at most SPO_BATCH_MAX_SETS sets of one
 *   storage type on one device, each with >= 32 padded orbitals) it builds
 *   a temporary plan, queues the batched evaluation and waits for the
 *   stream before freeing the plan (synchronous); otherwise it queues one
 *   spo_eval_ex per walker (asynchronous).  Keep a plan (spo_batch_*) to
 *   avoid the allocation and the wait.
 */
#define SPO_BATCH_MAX_SETS 8

typedef struct {
    int32_t set;
    int32_t reserved;   /* 0 */
    int64_t P;
    const float *pos;
    float *out;
} spo_work;

typedef struct spo_batch spo_batch;

spo_status spo_batch_create(const spo_set *const *sets, int nsets, int64_t max_positions,
                            int max_items, spo_batch **out);
spo_status spo_batch_eval(spo_batch *plan, spo_kind kind, const spo_work *items, int nitems,
                          void *stream);
spo_status spo_batch_graph(spo_batch *plan, spo_kind kind, const spo_work *items, int nitems,
                           void *stream);
spo_status spo_batch_launch(spo_batch *plan, void *stream);
spo_status spo_batch_destroy(spo_batch *plan);
spo_status spo_eval_batch(const spo_set *const *sets, int nsets, const spo_work *items, int nitems,
                          spo_kind kind, void *stream);

/*
 * Failure-path self-test.  Every device-side wait in the kernels (TMA and
 * bulk copies, tensor-core MMAs) is bounded (2 s of %globaltimer); on giving
 * up a kernel sets bit 0 of the device status word, drains what it issued
 * and returns, and spo_device_status reports it.  spo_selftest_wait(limit_ns,
 * stream, &timed_out) runs that path on purpose and harmlessly: a one-warp
 * probe waits, through the same routine, on an mbarrier nothing arrives on,
 * for limit_ns (at most 1 s), then the word is read and cleared; timed_out
 * = 1 means the time-out was detected and reported.  Synchronous.
 */
spo_status spo_selftest_wait(uint64_t limit_ns, void *stream, int *timed_out);

/*
 * Interpolating coefficients.  The table spo_create takes holds B-spline
 * coefficients; grid samples f(m / n) used as coefficients give a smoothed
 * f that does not pass through the samples.  spo_prefilter turns samples
 * into the coefficients of the interpolating spline, in place: along each
 * axis (c[m-1] + 4 c[m] + c[m+1]) / 6 = f[m], periodic (B3 at offsets -1, 0,
 * 1; the prefilter of the uniform cubic B-spline, done as a causal and an
 * anticausal recursion with pole sqrt(3) - 2 per axis, in FP64).
 *
 * spo_prefilter(grid, N, data, dtype, stream): data is a device array
 *   [nx][ny][nz][N] of dtype SPO_F64 or SPO_F32 (C order, orbital fastest),
 *   owned by the caller; queued on stream.  Feed the result to spo_create
 *   with coefs_on_device = 1.
 */
spo_status spo_prefilter(const spo_grid *grid, int64_t N, void *data, spo_dtype dtype, void *stream);

/*
 * Learned surrogate — a small learned function of the position standing in
 * for the B-spline table, aimed at the memory footprint the paper attacks
 * (Sec. 6.3-6.4: memory per walker and up to 3.8x smaller runs); the
 * B-spline stays its teacher and the arbiter of its error.  The paper has no
 * such surrogate; this is one of the patterns built on the path.
 *
 * Function: a periodic multiresolution hashed grid (levels l with
 * resolutions R_l geometric from r_min to r_max; 2^log2_table entries of
 * `features` features per level; corners indexed densely when R_l^3 fits
 * the table, else by the spatial hash (i ^ 2654435761 j ^ 805459861 k);
 * C2 quintic interpolation weights) feeding `layers` softplus layers of
 * width `hidden` and a linear layer of N outputs.  Values, gradients and
 * Laplacians are carried through the network as five channels, so the
 * outputs have the VGL layout [P][5][N] (V: [P][N]).
 *
 * spo_surrogate_create(spec, seed, &s): FP32 master parameters initialised
 *   from splitmix64 streams (grid U(-1e-4, 1e-4), weights U(+-1/sqrt(in)),
 *   biases 0), Adam moments, and inference copies (grid FP16, weights BF16).
 * spo_surrogate_train(s, teacher, steps, batch, lr, channel_weights, seed,
 *   stream, &last_loss): each step draws `batch` uniform positions
 *   (coordinate i of step t: the top 24 bits of splitmix64(seed + (3 batch t
 *   + i + 1) 0x9E3779B97F4A7C15) over 2^24), evaluates the teacher's VGL
 *   for them (the spline kernels), and takes one Adam step on sum_c w_c
 *   mean((out_c - target_c)^2): dense for the perceptron, sparse for the
 *   grid (an entry with no gradient in the step keeps its value and both
 *   moments).  channel_weights = 5 floats (V, Gx, Gy, Gz,
 *   L) or NULL for 1 / mean(target_c^2) of the first batch.  The teacher must
 *   have the same N.  The samples of several consecutive steps (enough for
 *   about 32 positions per brick of the teacher, at most 1 GiB of teacher
 *   values) are drawn and evaluated in one launch and held on the device
 *   until used; the results equal step-by-step draws.  The steps after a
 *   call's first replay a CUDA graph of one step, captured when the sizes,
 *   buffers or settings change.  Synchronous; refreshes the inference
 *   copies.
 * spo_surrogate_eval(s, kind, pos, P, out, precision, stream): kind V or
 *   VGL; precision 0 evaluates the FP32 master parameters (CUDA cores),
 *   precision 1 the inference copies (FP16 grid, BF16 weights and
 *   activations, FP32 accumulation on the tcgen05 tensor cores; out must
 *   be 32-byte aligned, else SPO_EINVAL).
 * spo_surrogate_grad(s, pos, target, P, channel_weights, precision, &loss,
 *   grid, W, b, stream): loss and its gradient with respect to every FP32
 *   master parameter for P device positions [P][3] and device targets
 *   [P][5][N] (same channel weights rule), written to host arrays laid out
 *   as in spo_surrogate_params; precision 0 computes every product in FP32
 *   on the CUDA cores, 1 as training does on the tensor cores (the operands
 *   of the forward, weight-gradient and data-gradient products rounded to
 *   BF16, FP32 accumulation).  Leaves the parameters unchanged; synchronous.
 * spo_surrogate_set_train_precision(s, precision): 1 (default) trains with
 *   the layers' products on the tcgen05 tensor cores as above, 0 in FP32 on
 *   the CUDA cores.
 * spo_surrogate_set_optimizer(s, beta1, beta2, eps, grid_lr_mult): Adam's
 *   moment decay rates and denominator guard (defaults 0.9, 0.99, 1e-15),
 *   and the grid's learning rate as a multiple of `lr` (default 1).
 * spo_surrogate_set_level_lr(s, power): the grid's rate of level l is
 *   further multiplied by (R_0 / R_l)^power (0 <= power <= 4; default 0:
 *   every level at lr * grid_lr_mult).  A feature of level l moves the
 *   Laplacian channel R_l^2 times as much as the value channel, so with
 *   power 2 every level's step changes the Laplacian alike.
 * spo_surrogate_nparams(s, &n) / spo_surrogate_state(s, params, m, v, &step,
 *   restore): the training state for checkpoints: all FP32 master parameters
 *   laid out [grid | W0 | b0 | W1 | b1 | ...] (n floats), Adam's first and
 *   second moments (same layout) and the step count, copied to (restore = 0)
 *   or from (restore != 0) host arrays.  Restoring refreshes the inference
 *   copies.  Synchronous.
 * spo_surrogate_footprint(s, &bytes): device bytes of the inference copies.
 * Calls on one surrogate must be ordered (one stream): they share its
 * scratch (the encoded-feature images of precision 1 grow with P and stay
 * allocated until spo_surrogate_destroy).
 * spo_surrogate_params(s, grid, W, b, to_device): copy all FP32 master
 *   parameters from (to_device != 0) or to host arrays: grid
 *   [levels][2^log2_table][features]; W[l] [out][in]; b[l] [out]
 *   (layers + 1 entries each).  Setting them refreshes the inference copies.
 */
typedef struct {
    int32_t levels, log2_table, features, r_min, r_max, hidden, layers, reserved;
    int64_t N;
} spo_surrogate_spec;

typedef struct spo_surrogate spo_surrogate;

spo_status spo_surrogate_create(const spo_surrogate_spec *spec, uint64_t seed, spo_surrogate **out);
spo_status spo_surrogate_train(spo_surrogate *s, const spo_set *teacher, int64_t steps, int64_t batch,
                               float lr, const float *channel_weights, uint64_t seed, void *stream,
                               float *last_loss);
spo_status spo_surrogate_eval(spo_surrogate *s, spo_kind kind, const float *pos, int64_t P,
                              float *out, int precision, void *stream);
spo_status spo_surrogate_grad(spo_surrogate *s, const float *pos, const float *target, int64_t P,
                              const float *channel_weights, int precision, float *loss, float *grid,
                              float *const *W, float *const *b, void *stream);
spo_status spo_surrogate_set_train_precision(spo_surrogate *s, int precision);
spo_status spo_surrogate_set_level_lr(spo_surrogate *s, float power);
spo_status spo_surrogate_set_optimizer(spo_surrogate *s, float beta1, float beta2, float eps,
                                       float grid_lr_mult);
spo_status spo_surrogate_nparams(const spo_surrogate *s, int64_t *n);
spo_status spo_surrogate_state(spo_surrogate *s, float *params, float *m, float *v, int64_t *step,
                               int restore);
spo_status spo_surrogate_footprint(const spo_surrogate *s, size_t *bytes);
spo_status spo_surrogate_params(spo_surrogate *s, float *grid, float *const *W, float *const *b,
                                int to_device);
spo_status spo_surrogate_destroy(spo_surrogate *s);

/* Allocate (or grow) the set's scratch for `stream` to hold batches of up to
 * P positions, so that later evaluations on that stream allocate nothing.
 * Synchronous. */
spo_status spo_reserve(spo_set *set, int64_t P, void *stream);

/* Device-side status word of the current device: bit 0 = a bounded wait on a
 * TMA copy gave up (the affected outputs are incomplete); bit 1 = in a
 * library built with -DSPO_CHECK_BOUNDS (a debug build: the kernels check
 * the indices they are about to use, such as a position's cell against its
 * brick, a sorted slot, a permutation entry or a window's table rows), a
 * check failed and that access was skipped.  Synchronises `stream`; with
 * clear != 0 the word is reset to zero afterwards.  Returns SPO_ETIMEOUT if
 * bit 0 was set, SPO_EINVAL if bit 1 was, SPO_OK otherwise. */
spo_status spo_device_status(unsigned int *flags, int clear, void *stream);

/*
 * spo_eval_host — the same evaluation with HOST buffers: pos_host [P][3] and
 * out_host ([P][rows][N]) in host memory.  If both buffers are pinned and
 * mapped (cudaHostAlloc / cudaHostRegister, or torch's pin_memory), the
 * kernels read the positions from and write the outputs to host memory
 * directly over the CPU-GPU link (no staging, no copy engines), ordered on
 * `stream`.  Otherwise the positions are copied to the device, evaluated
 * and copied back in chunks on two internal streams, so that copies overlap
 * the kernels (pageable memory works but copies synchronously); that work is
 * ordered after the work already queued on `stream`.  Synchronous: out_host is complete on
 * return.  Device staging buffers are owned by the set, allocated on first
 * use and reused; they are freed by spo_destroy.  Calls on the same set must
 * not run concurrently from several host threads.
 */
spo_status spo_eval_host(spo_set *set, spo_kind kind, const float *pos_host, int64_t P,
                         float *out_host, void *stream);

/*
 * spo_autotune — time the evaluation strategies and tunings for this set,
 * kind and batch size on the set's device (synthetic uniform positions, CUDA
 * events on `stream`), apply the fastest (its tile, orbitals per thread and
 * schedule become the set's parameters, and SPO_ALGO_AUTO uses its strategy
 * for batches within a factor 4 of P) and report it in *best.  Results are
 * cached per (grid, N, storage, kind, power-of-two bucket of P, SM count)
 * for the process and, if the environment variable SPO_TUNE_CACHE names a
 * file, in that file (one line per key), so that later processes skip the
 * timing.  Allocates temporary device memory; synchronous.
 */
typedef struct {
    int32_t algo;            /* spo_algo */
    int32_t brick_tile;
    int32_t brick_vec;
    int32_t brick_schedule;
    float ms;                /* time of one evaluation with this choice */
    int32_t from_cache;      /* 1 if no timing was needed */
} spo_tuning;

spo_status spo_autotune(spo_set *set, spo_kind kind, int64_t P, void *stream, spo_tuning *best);

/* Set or read a tuning parameter.  Tuning changes speed only: every value
 * gives bit-identical outputs.  Invalid parameters or values: SPO_EINVAL.
 * Not thread-safe against evaluations of the same set in flight on the host. */
spo_status spo_set_param(spo_set *set, spo_param param, int64_t value);
spo_status spo_get_param(const spo_set *set, spo_param param, int64_t *value);

/* Device bytes held by the set's table (scratch and the staging buffers of
 * spo_eval_host excluded). */
spo_status spo_footprint(const spo_set *set, size_t *bytes);

/* Shape of a set: grid, N, padded orbital stride Np and storage type.  Any
 * output pointer may be NULL. */
spo_status spo_info(const spo_set *set, spo_grid *grid, int64_t *N, int64_t *Np,
                    spo_dtype *storage);

/* Number of output rows per position for a kind (1, 5 or 10; 0 if invalid). */
int spo_rows(spo_kind kind);

/* Static description of a status code. */
const char *spo_status_str(spo_status status);

/* Description of the last error raised on the calling host thread ("" if
 * none).  The string stays valid until the next call on this thread. */
const char *spo_last_error(void);

/* SPO_ABI_VERSION of the loaded library. */
int spo_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPO_H */
