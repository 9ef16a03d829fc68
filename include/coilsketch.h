/*
 * coilsketch.h - C ABI of libcoilsketch.so: the GPU hot path of coil-sketched iterative MR
 * reconstruction (Oscanoa et al., "Coil Sketching for computationally-efficient MR iterative
 * reconstruction").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Array arguments are DEVICE pointers owned by the caller (allocated e.g. by PyTorch) unless
 *   a comment says "host".  The library never frees them.  Handles (cs_plan) own their internal
 *   workspace and release it in cs_plan_destroy.
 * - complex64 values are interleaved float2 {re, im}.  Images are row-major with x fastest:
 *   [nz][ny][nx] (3D) or [ny][nx] (2D).  Coil-stacked arrays are coil-major: maps [C][image],
 *   k-space [C][N] with samples in the caller's order.
 * - Non-Cartesian trajectories are float [N][ndim] in cycles/pixel, axis order (z, y, x) for 3D
 *   and (y, x) for 2D, each coordinate in [-0.5, 0.5].  Density compensation is float [N].
 * - Every call that takes a cudaStream_t (passed as void*) is asynchronous on that stream
 *   unless stated otherwise.  A null stream means the legacy default stream.
 * - Every function returns a cs_status.  On failure cs_last_error() returns a thread-local
 *   message.  No C++ exception and no abort crosses this boundary.  Argument errors are
 *   detected on the host before anything is launched.
 */
#ifndef COILSKETCH_H
#define COILSKETCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int cs_status;
enum {
    CS_OK = 0,
    CS_ERR_INVALID_ARG = 1,      /* null pointer, negative size, V+S > C, ...              */
    CS_ERR_UNSUPPORTED_SIZE = 2, /* an FFT length with a prime factor outside {2,3,5,7,11},
                                    odd sizes, a dimension above the supported maximum      */
    CS_ERR_CUDA = 3,             /* a CUDA runtime call failed                              */
    CS_ERR_OOM = 4,              /* device allocation failed                                */
    CS_ERR_NONFINITE = 5,        /* a solver reduction produced NaN or Inf                  */
    CS_ERR_TIMEOUT = 6,          /* a bounded device-side wait gave up; the outputs of the
                                    calls since the last status check are invalid            */
    CS_ERR_BOUNDS = 7            /* a device-side index check failed (checked builds)       */
};

enum { CS_CARTESIAN = 0, CS_NONCARTESIAN = 1 };
enum { CS_GAUSSIAN = 0, CS_RADEMACHER = 1 };
enum { CS_NORM_UNIT_VAR = 0, CS_NORM_PAPER_LITERAL = 1 };
enum { CS_PREC_FP32 = 0, CS_PREC_BF16_SPLIT = 1 };
enum { CS_REG_L2 = 0, CS_REG_L1_WAVELET = 1, CS_REG_L1_TV = 2 };

/* Thread-local description of the last error on this thread ("" if none). */
const char* cs_last_error(void);

/* Library version string. */
const char* cs_version(void);

/* Number of kernels this library has launched in the process so far (all devices). */
long long cs_launch_count(void);

/* Optional per-stage timing: while enabled, CUDA events are recorded on the launching stream
 * around every launch of the stages below; cs_profile_read synchronises on those events and
 * returns the summed device time and the launch count of one stage.  cs_profile resets the
 * totals (and turns recording on or off). */
enum { CS_STAGE_SPREAD = 0, CS_STAGE_INTERP = 1, CS_STAGE_FFT_PLAIN = 2, CS_STAGE_EXPAND = 3,
       CS_STAGE_REDUCE = 4 };
cs_status cs_profile(int enable);
cs_status cs_profile_read(int stage, double* total_ms, long long* launches);

/* ------------------------------------------------------------------------------------------
 * Plans.  A plan fixes the image geometry and the sampling operator (Sec. 2.1):
 *   Cartesian:      F~ = U F~_u  - centred orthonormal DFT then the undersampling U, given as
 *                   the ascending row-major list of sampled flat indices;
 *   non-Cartesian:  F~ = F~_n    - Kaiser-Bessel gridding NUFFT (width 4) on an oversampled
 *                   grid, with A = W^1/2 F C (density compensation w).
 * Plan creation copies/derives everything it needs (the caller's trajectory, dcf and mask
 * buffers may be freed afterwards), bins the samples to tiles (integer-exact, stable), and
 * synchronises `stream` before returning.
 * ---------------------------------------------------------------------------------------- */
typedef struct cs_plan cs_plan;

typedef struct {
    int kind;            /* CS_CARTESIAN or CS_NONCARTESIAN                                   */
    int ndim;            /* 2 or 3                                                            */
    int img[3];          /* image size, slow to fast: (nz, ny, nx) or (ny, nx)                */
    int max_coils;       /* largest coil count any later call passes (sizes the workspace)    */
    /* Cartesian */
    const int32_t* mask_idx; /* device, [nsamples] ascending flat indices into the image grid */
    int64_t nsamples;        /* samples per coil N                                           */
    /* non-Cartesian */
    int grid[3];         /* oversampled grid, same order as img (e.g. 1.25 x img), all even   */
    float alpha;         /* oversampling ratio used for the Kaiser-Bessel beta (1.25)         */
    const float* traj;   /* device, [N][ndim] cycles/pixel                                    */
    const float* dcf;    /* device, [N] density compensation w (the operator applies sqrt w)  */
    int tile[3];         /* tile size per axis for binning (>= 4); 0 = library default (16)  */
} cs_geom;
/* Size limits: image sizes even, nx <= 512; grid sizes even, >= the image and <= 800 (the FFT
 * length limit) with prime factors in {2, 3, 5, 7, 11}; non-Cartesian plans need grid points x
 * max_coils < 2^31 and at most 49152 tiles.  Violations return CS_ERR_UNSUPPORTED_SIZE.
 * Samples are ordered by tile and, inside a tile, by halo class (the set of upper neighbour tiles
 * their kernel box reaches), each run in acquisition order. */

cs_status cs_plan_create(const cs_geom* g, void* stream, cs_plan** out);
cs_status cs_plan_destroy(cs_plan* plan);

/* Read back the binning of a non-Cartesian plan (device outputs; tests compare them bit-exactly
 * with the CPU restatement): perm[N] sorted position -> sample index (stable by tile, then halo
 * class), tile_off[ntiles+1], j0[N][ndim] first kernel-box index per axis (unwrapped), ntiles_out[3]
 * tiles per axis (a remainder narrower than 4 widens the last tile). */
cs_status cs_plan_binning(const cs_plan* plan, int32_t* perm, int32_t* tile_off, int32_t* j0,
                          int* ntiles_out, void* stream);

/* Gridding launch parameters of a non-Cartesian plan: coils per warp of the interpolation (1..32)
 * and of the spreading (1..16), consecutive sorted samples per warp of each (1..4096).  Plans
 * start at 16 / 64 / 16 / 64.  Any values give results equal up to rounding order; only the speed
 * changes.
 * cs_plan_autotune: times the interpolation and the spreading of `ncoils` coils (reps timed
 * launches after one untimed, CUDA events on `stream`) for coils per warp in {8, 16, 32} (interp)
 * or {8, 16} (spread) and samples per warp in {32, 64, 128}, on the plan's own scratch buffers
 * (their contents are overwritten), and keeps the fastest of each in the plan.  choice[4]
 * (nullable) receives (interp coils, interp chunk, spread coils, spread chunk); ms[4] (nullable)
 * the best interp and spread ms per launch and those of the configuration before tuning.
 * Synchronous.  Cartesian plans have nothing to tune (returns CS_OK, ms zero). */
cs_status cs_plan_set_gridding(cs_plan* plan, int interp_coils, int interp_chunk, int spread_coils,
                               int spread_chunk);
cs_status cs_plan_autotune(cs_plan* plan, int ncoils, int reps, int* choice, float* ms, void* stream);

/* Tile sizes of a non-Cartesian plan's binning (Sec. 2.1 gridding; the sort order of the samples,
 * not the operator).  cs_plan_set_tile: tile[ndim] (z, y, x order; each >= 4, or the grid size;
 * larger values are clipped to the grid) re-bins the plan exactly as cs_plan_create would with that
 * `tile`: same keys, same stable order.  The per-sample records are rewritten in place, the
 * deterministic-spreading work items rebuilt if the plan has them.  Results of every operator are
 * equal up to rounding order; cs_plan_binning returns the new order.  Synchronous (waits for
 * `stream`); CS_ERR_UNSUPPORTED_SIZE for more than 49152 tiles (the plan is unchanged); after
 * any other error the plan must be destroyed.
 * cs_plan_autotune_tile: re-bins the plan with every cubic candidate cand[ncand] (each >= 4,
 * ncand <= 16), times the interpolation plus the spreading of `ncoils` coils (reps timed rounds
 * after one untimed, CUDA events on `stream`, the plan's scratch buffers overwritten) and leaves
 * the plan binned with the fastest; *best (nullable) receives it and ms[ncand] (nullable) each
 * candidate's ms per round.  Synchronous.
 * Changing the tiles, the gridding parameters or the spreading mode invalidates the CUDA graphs
 * that recon_solve / recon_solve_batched cached for the plan (they are captured again). */
cs_status cs_plan_set_tile(cs_plan* plan, const int* tile, void* stream);
cs_status cs_plan_autotune_tile(cs_plan* plan, int ncoils, int reps, const int* cand, int ncand, int* best,
                                float* ms, void* stream);

/* Spreading mode of a non-Cartesian plan (the adjoint's first step, Sec. 2.1 gridding).
 * on = 0 (default): producer-computes - one warp per run of sorted samples, rows, columns and
 *   planes leaving its sliding window added to the grid with atomic adds; fastest, results equal
 *   up to the rounding order of those additions, which depends on scheduling.
 * on = 1: owner-computes - atomics-free and bit-reproducible: every tile of the grid is
 *   accumulated by one warp at a time from its own samples and the samples of its lower
 *   neighbour tiles whose kernel box reaches it (the halo classes of the binning), in a fixed
 *   order; a tile with more than item_visits sample visits (64..2^20; 0 = keep the current value,
 *   initially 4096) is split into work items whose sums go to private partial slots that a
 *   second kernel adds to the grid in slot order.  Slower (every sample is visited by the owners
 *   of all tiles its box touches).  Building the work items is synchronous and allocates the
 *   partial slots on the device.  Cartesian plans ignore the call (their sampling adjoint has no
 *   accumulation). */
cs_status cs_plan_set_deterministic(cs_plan* plan, int on, int item_visits);

/* ------------------------------------------------------------------------------------------
 * sense_fwd: y = A x for `ncoils` maps (Eq. 1, Eq. 5): y_c = w^1/2 (.) F{c_c (.) x}.
 *   x [image] complex64, maps [ncoils][image] complex64, y [ncoils][N] complex64.
 * sense_adj: x (+)= A^H y = sum_c conj(c_c) (.) F^H{w^1/2 (.) y_c}; with accumulate != 0 the
 *   result is added to x, else x is overwritten.
 * ncoils must not exceed the plan's max_coils.
 * ---------------------------------------------------------------------------------------- */
cs_status sense_fwd(const cs_plan* plan, const float* x, const float* maps, int ncoils,
                    float* y, void* stream);
cs_status sense_adj(const cs_plan* plan, const float* y, const float* maps, int ncoils,
                    float* x, int accumulate, void* stream);

/* Full gradient of the data term (Algorithm 1, "compute true gradient"):
 *   d = A^H (A x - y) with all ncoils coils, the residual formed in k-space without a
 *   separate pass.  x [image], maps [ncoils][image], y [ncoils][N], d [image]. */
cs_status sense_grad(const cs_plan* plan, const float* x, const float* maps, int ncoils,
                     const float* y, float* d, void* stream);

/* ------------------------------------------------------------------------------------------
 * sketched_normal_apply: z = A_S^H A_S v + lambda v for the sketched model with m = V + S
 * coils (Sec. 2.3, Eq. 7-8).  The sketched maps are given as two row blocks so that the V
 * high-energy virtual coils are used in place (no copy): maps_v [V][image] (typically the first
 * V rows of the PCA-rotated maps) and maps_s [S][image] (the sketched combinations).  Either
 * block may be empty (count 0, pointer ignored).
 * ---------------------------------------------------------------------------------------- */
cs_status sketched_normal_apply(const cs_plan* plan, const float* v, const float* maps_v, int V,
                                const float* maps_s, int S, float lambda, float* z, void* stream);

/* ------------------------------------------------------------------------------------------
 * coil_pca: SVD-based coil compression of the k-space data (Sec. 3.1, Algorithm 1 "perform
 * coil compression").  R = Y Y^H over all N samples of y [C][N] (complex64 data, FP32 blocked
 * accumulation, FP64 block sums added in a fixed order, so R and U are bit-reproducible), then
 * a FP64 cyclic Jacobi eigendecomposition on the GPU.  recon_solve's PCA is the same.
 *   U    [C][C] complex64 (column k = eigenvector k; row-major U[c*C + k]), eigenvalues
 *        descending, each column's largest-magnitude entry made real positive;
 *   eig  [C] float64 eigenvalues, descending.
 * Ties between equal eigenvalues admit any orthonormal basis of their eigenspace.
 * ---------------------------------------------------------------------------------------- */
cs_status coil_pca(const float* y, int C, int64_t N, float* U, double* eig, void* stream);

/* coil_pca_noalloc: the same computation as coil_pca for callers that cannot allocate device
 * memory while they run - for example code whose device memory is entirely reserved up front
 * by another allocator, or a service that must not grow its footprint after start-up.  It calls
 * no cudaMalloc/cudaFree and no allocating library routine: its covariance scratch is a static
 * device array of 64 KiB (complex128, at most 64 coils) that every GPU loading the library holds
 * until the process exits.  The paper has no counterpart; this is a deployment variant.
 *   y [C][N] complex64, U [C][C] complex64, eig [C] float64 - device buffers owned by the caller.
 *   C > 64 is rejected with CS_ERR_UNSUPPORTED_SIZE before anything is launched.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All calls share the
 * one array and clear it on their stream before use, so calls that overlap on the GPU (other
 * streams, other threads) race: serialise them. */
cs_status coil_pca_noalloc(const float* y, int C, int64_t N, float* U, double* eig, void* stream);

/* coil_rotate: out[k][l] = sum_c conj(U[c][k]) in[c][l] for k < C_out (c' = U^H c, y' = U^H y),
 * in [C][L], out [C_out][L] complex64 (out must not alias in). */
cs_status coil_rotate(const float* U, const float* in, int C, int C_out, int64_t L, float* out,
                      void* stream);

/* ------------------------------------------------------------------------------------------
 * sketch_draw: the random blocks S~_S^t in R^{S x (C-V)} of the structured sketch
 * S~^t = [[I_V, 0], [0, S~_S^t]] (Sec. 2.3) for t = t0 .. t0+T-1, written to `out`
 * (device, float [T][S][C-V]).  Entries come from Philox4x32-10 (Salmon et al. 2011) with key
 * (seed mod 2^32, seed >> 32) and counter (entry index, t, 0, 0); Gaussian by Box-Muller or
 * Rademacher (Sec. 3.2); scale 1/sqrt(S) (CS_NORM_UNIT_VAR: unbiased, E[S~^T S~] = I) or the
 * paper's literal sigma = 1/S, +-1 (CS_NORM_PAPER_LITERAL); finally rounded to the nearest
 * bfloat16 value so every entry is an exact tensor-core operand.
 * ---------------------------------------------------------------------------------------- */
cs_status sketch_draw(uint64_t seed, int t0, int T, int C, int V, int S, int dist, int norm,
                      float* out, void* stream);

/* ------------------------------------------------------------------------------------------
 * The two element-wise steps of PDHG for l1-TV (Sec. 2.1, Chambolle & Pock 2011) around its
 * data step, as run inside recon_solve; T = forward differences with periodic wrap along every
 * axis of the image dims (slow to fast, ndim 2 or 3).  All arrays device complex64.
 * tv_dual_update: z_a <- proj(z_a + sigma (T xbar)_a), xbar = 2 x - x_prev (x_prev NULL: x),
 *   proj scaling every entry of modulus above lambda down to lambda; z [ndim][image], in place.
 * tv_rhs: rhs = b0 + inv_tau x - T^H z, (T^H z)[r] = sum_a z_a[r - e_a] - z_a[r]; b0 may be NULL
 *   (zero); x_prev_out (may be NULL) receives a copy of x.
 * ---------------------------------------------------------------------------------------- */
cs_status tv_dual_update(const float* x, const float* x_prev, float* z, int ndim, const int* dims, float sigma,
                         float lambda, void* stream);
cs_status tv_rhs(const float* b0, const float* x, const float* z, int ndim, const int* dims, float inv_tau,
                 float* rhs, float* x_prev_out, void* stream);

/* Synchronise `stream` and report (then clear) a device-side timeout of a bounded wait. */
cs_status cs_device_status(void* stream);

/* One Philox4x32-10 block on the host (known-answer testing of the generator). */
cs_status cs_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ------------------------------------------------------------------------------------------
 * sketched_maps: the sketched sensitivity maps of Eq. 8 for the random block only:
 *   maps_s[s][d] = sum_j S[s][j] maps_rot[V + j][d], s < S, j < C - V
 * (rows 0..V-1 of the sketched maps are maps_rot[0..V-1] themselves and are not copied).
 * precision CS_PREC_FP32: FP32 CUDA-core contraction; CS_PREC_BF16_SPLIT: tensor-core BF16
 * contraction (tcgen05, accumulator in tensor memory) of the BF16-exact sketch with a two-term
 * BF16 split of the maps (hi + lo), FP32 accumulation, relative error about 2^-17 per term;
 * limited to S <= 16 and C - V <= 64.  Its waits on the tensor cores are bounded: a wait that
 * gives up is reported as CS_ERR_TIMEOUT by the next cs_device_status or recon_solve.
 * ---------------------------------------------------------------------------------------- */
cs_status sketched_maps(const float* S, const float* maps_rot, int64_t D, int C, int V, int Sn,
                        int precision, float* maps_s, void* stream);

/* ------------------------------------------------------------------------------------------
 * recon_solve: Algorithm 1 (coil sketching) or, with sketch disabled, the plain full-coil
 * solver, on one plan.  Runs on `stream` and SYNCHRONISES before returning (it fills stats).
 *
 * problem: y [C][N] k-space (density-compensated data y = W^1/2 k for non-Cartesian),
 *          maps [C][image], lambda, reg (CS_REG_L2 -> CG, CS_REG_L1_WAVELET -> FISTA with a
 *          periodised db4 transform, `wavelet_levels` levels, CS_REG_L1_TV -> PDHG
 *          (Chambolle & Pock 2011, theta = 1) on lambda ||T x||_1, T the forward differences
 *          along every image axis with periodic wrap, the l1 norm summing complex moduli
 *          (Sec. 2.1); each PDHG data step prox_{tau f} is solved by `cg_iters` CG iterations
 *          started at the current iterate; the dual variable starts at zero and is carried
 *          from one sketched sub-problem to the next).
 * params:  T outer iterations, K inner iterations, V, S, sketch distribution/normalisation,
 *          seed (or a caller-given sketch array), whether to run coil PCA first, the FISTA
 *          step (0 = estimate 1/L by `power_iters` power iterations on the first sketched
 *          normal operator, from the caller's start vector), whether to capture one outer
 *          iteration as a CUDA graph, an optional learned warm start and an optional trace.
 * x_inout: initial estimate on input (x^0), x^T on output.
 * workspace: the solver's device vectors live in a workspace owned by the plan; it is
 *          allocated on the first call and grown when a later call needs more (every call on a
 *          plan shares it, so calls on one plan must not overlap).  cs_plan_destroy frees it.
 * ---------------------------------------------------------------------------------------- */
typedef struct cs_unet cs_unet;   /* the warm-start network (ws_net_create, below) */

/* Fields of one trace record (cs_solve_params.trace): one record per outer iteration of
 * Algorithm 1 (plain solver: one per iteration), written on the device inside the loop.      */
enum {
    CS_TRACE_GRAD2 = 0,      /* ||d||^2 of the true gradient d = A^H (A x^t - y) at x^t (plain
                                solver: ||gradient||^2 at the point the iteration evaluates it) */
    CS_TRACE_OBJECTIVE = 1,  /* 1/2 ||A x^t - y||^2 + g(x^t) at the start of the outer iteration
                                (plain FISTA: at its gradient point); NaN unless trace_objective,
                                and NaN for l1-TV                                              */
    CS_TRACE_ACCEPT = 2,     /* warm start: 1 accepted, 0 rejected; -1 without a warm start    */
    CS_TRACE_DIST2 = 3,      /* ||x^{t+1} - x_ref||^2 / ||x_ref||^2 after the iteration; -1
                                without x_ref                                                 */
    CS_TRACE_TIME_NS = 4,    /* device clock (%globaltimer, ns) at the end of the iteration    */
    CS_TRACE_STEP_L = 5,     /* FISTA: the eigenvalue estimate L whose 1/L is the iteration's step
                                (constant unless step_per_outer); 0 when the step was given    */
    CS_TRACE_FIELDS = 6
};

typedef struct {
    const float* y;          /* [C][N]                                                       */
    const float* maps;       /* [C][image]                                                   */
    int C;
    float lambda;
    int reg;                 /* CS_REG_L2 | CS_REG_L1_WAVELET | CS_REG_L1_TV                  */
    int wavelet_levels;      /* db4 levels for CS_REG_L1_WAVELET (every axis divisible by 2^levels) */
} cs_problem;

typedef struct {
    int T;                   /* outer iterations                                             */
    int K;                   /* inner iterations per sub-problem (plain solver: total)        */
    int sketch;              /* 1 = coil sketching (Algorithm 1), 0 = plain full-coil solver  */
    int V, S;                /* high-energy virtual coils kept, sketched coils (C^ = V + S)   */
    int dist, norm;          /* CS_GAUSSIAN | CS_RADEMACHER, CS_NORM_*                        */
    uint64_t seed;
    const float* sketches;   /* optional device [T][S][C-V]; NULL = draw with sketch_draw      */
    int do_pca;              /* 1 = coil PCA + rotation of maps and data first                */
    int precision;           /* CS_PREC_FP32 | CS_PREC_BF16_SPLIT for the sketched maps        */
    float step;              /* FISTA step eta; 0 = 1/L from power iteration                  */
    int power_iters;         /* power iterations for L (default 20)                          */
    const float* power_v0;   /* device [image] start vector for the power iteration (may be NULL
                                only when step > 0)                                           */
    int use_graph;           /* capture one outer iteration (sketched) or one inner iteration
                                (plain) as a CUDA graph and replay it                         */
    float* iterates;         /* optional device [T][image]: x^t after every outer iteration
                                (plain solver: [K][image], after every iteration)             */
    int cg_iters;            /* CS_REG_L1_TV: CG iterations per PDHG data step (0 = 5)         */
    float tv_tau, tv_sigma;  /* CS_REG_L1_TV: PDHG primal/dual steps; 0 = 0.99 / sqrt(4 ndim)
                                each (tau sigma ||T||^2 < 1 with ||T||^2 = 4 ndim)            */
    int init;                /* 1 = Algorithm 1's classical-sketch initialisation before the T
                                outer iterations: x <- argmin 1/2 ||S^0 A x - S^0 y||^2 + g(x),
                                K iterations of the sub-problem solver from x^0 (the sketched
                                gradient in place of the true one); S^0 is sketch block T, so
                                a caller-given `sketches` array then holds T + 1 blocks; the
                                FISTA step comes from S^0's model.  Ignored without sketch.   */
    /* Comparators of the paper's Sec. 3.3 (plain solver, sketch = 0):                         */
    int keep;                /* aggressive coil compression: solve with only the first `keep`
                                (virtual, after do_pca) coils; 0 = all                         */
    int sgd_batch;           /* > 0: AccProxSGD (l1-wavelets only) with coil batches of this size:
                                K iterations x^{k+1} = prox(z - alpha_k (C'/B) sum_batch
                                A_c^H (A_c z - y_c)), Nesterov (FISTA) momentum, alpha_k =
                                max(sgd_beta^k, sgd_min) alpha_0, alpha_0 = 1/L of the C'-coil
                                normal operator (power iteration, or 1/step), C' = coils used  */
    const int* sgd_coils;    /* device int [K][sgd_batch]: the coil indices of every batch (in
                                [0, C')), drawn by the caller; checked on the host              */
    float sgd_beta, sgd_min; /* step decay and floor (fractions of alpha_0); 0 = 0.99 and 0.1    */
    /* Learned warm start (not in the paper; sketched l1-wavelet solves only): at every outer
     * iteration the network predicts a start x^ from (x^t, d); the sub-problem objective of
     * Eq. 9-10 is evaluated at x^ and at x^t on the device, and FISTA starts from x^ only when
     * its objective is lower, else from x^t (Algorithm 1 unchanged).  The decision never leaves
     * the device, so the outer iteration stays one captured graph.  Image sizes must be
     * multiples of 4 (the network pools twice).  NULL = no warm start.                       */
    cs_unet* warm;
    /* Optional trace (any solver): x_ref (device [image], may be NULL) is the reference of the
     * CS_TRACE_DIST2 field; trace (HOST array of [T][CS_TRACE_FIELDS] doubles for the sketched
     * solver, [K][CS_TRACE_FIELDS] for the plain solver) receives the records when recon_solve
     * returns; trace_objective = 1 adds the objective field (one extra full forward operator per
     * record).  NULL trace = nothing recorded and nothing extra launched.                    */
    const float* x_ref;
    double* trace;
    int trace_objective;
    /* Sketched FISTA with step = 0: the step 1/L comes from power_iters power iterations on the
     * first sub-problem's sketched normal operator and is reused (Sec. 3.3).  step_per_outer > 0
     * re-estimates L at every outer iteration instead, by that many power iterations on the
     * iteration's own sketched operator started from the previous eigenvector estimate (on the
     * device, inside the captured outer iteration).  0 = reuse (default).                     */
    int step_per_outer;
} cs_solve_params;

typedef struct {
    double L;                /* step-size eigenvalue estimate (FISTA) or 0                   */
    double final_rr;         /* CG: last squared residual norm (FP64); FISTA: 0              */
    int outer_done;          /* outer iterations run                                         */
    int graph_used;          /* 1 if the loop body ran as a replayed CUDA graph              */
    double ms_total;         /* device time of the whole solve (CUDA events)                 */
    double ms_pca;           /* device time of coil PCA + rotations                           */
    int warm_accepted;       /* outer iterations whose warm start was accepted               */
} cs_stats;

cs_status recon_solve(const cs_plan* plan, const cs_problem* problem, const cs_solve_params* params,
                      float* x_inout, cs_stats* stats, void* stream);

/* ------------------------------------------------------------------------------------------
 * recon_solve_batched: many independent reconstructions (e.g. the 2D slices of a volume, each
 * with its own size, plan, maps and data; the paper reconstructs slices separately, Sec. 3.1-3.2)
 * in one call.  Every item has its own plan (plans must be distinct); the solves share `params`
 * (sketches are drawn per item from params->seed; params->sketches and params->iterates must be
 * NULL).  The items are forked onto a pool of streams and joined on `stream`; with
 * params->use_graph all of them are captured once into ONE CUDA graph (cached for identical
 * calls) and launched with a single cudaGraphLaunch.  Synchronises; stats (optional) is an array
 * of nslices entries.  For FISTA with step == 0 every item gives its own power-iteration start
 * vector (power_v0 of the item, the size of its image).
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    cs_plan* plan;
    cs_problem problem;
    float* x_inout;          /* device [image of this plan]                                  */
    const float* power_v0;   /* device [image of this plan] or NULL                          */
} cs_batch_item;

cs_status recon_solve_batched(int nslices, const cs_batch_item* items, const cs_solve_params* params,
                              cs_stats* stats, void* stream);

/* ------------------------------------------------------------------------------------------
 * Pseudo-replica noise statistics (the paper's Sec. 3.2 inverse g-factor analysis, after
 * Pruessmann et al. and Robson et al.): recons are K reconstructions of noisy copies of one
 * acquisition, complex64 [K][D] device arrays.  cs_noise_std: std_out[i] = sqrt(mean_k |x_k[i] -
 * mean_k x_k[i]|^2) (float [D]); cs_inverse_gfactor: inv_g[i] = std_full[i] sqrt(R) / std_R[i]
 * (float [D]).  Computed in FP64 per pixel, summing the replicas in order.  Asynchronous.
 * ---------------------------------------------------------------------------------------- */
cs_status cs_noise_std(const float* recons, int K, int64_t D, float* std_out, void* stream);
cs_status cs_inverse_gfactor(const float* recons_R, const float* recons_full, int K, int64_t D, float R, float* inv_g,
                             void* stream);

/* ------------------------------------------------------------------------------------------
 * Sub-problem pieces for callers that drive Algorithm 1 themselves (e.g. with a warm start).
 * sketched_subproblem_solve: K iterations (CG for CS_REG_L2, FISTA with step `step` for
 *   CS_REG_L1_WAVELET) on the sketched sub-problem of Eq. 9-10,
 *   min_x 1/2 ||A_S (x - x^t)||^2 + Re<x, d> + g(x),
 *   starting from x_inout (x^t itself when x_inout == xt, else a warm start); x_inout receives
 *   the result.  Sketched maps as in sketched_normal_apply.  Asynchronous.
 * cs_subproblem_objective: the value of that objective at u (host double; synchronises).
 * cs_power_iteration: largest eigenvalue of A_S^H A_S from v0 (host double; synchronises).
 * ---------------------------------------------------------------------------------------- */
cs_status sketched_subproblem_solve(const cs_plan* plan, const float* d, const float* xt, float* x_inout,
                                    const float* maps_v, int V, const float* maps_s, int S, float lambda,
                                    int reg, int wavelet_levels, int K, float step, void* stream);
cs_status cs_subproblem_objective(const cs_plan* plan, const float* u, const float* xt, const float* d,
                                  const float* maps_v, int V, const float* maps_s, int S, float lambda,
                                  int reg, int wavelet_levels, double* value, void* stream);
cs_status cs_power_iteration(const cs_plan* plan, const float* v0, const float* maps_v, int V,
                             const float* maps_s, int S, int iters, double* L, void* stream);

/* ------------------------------------------------------------------------------------------
 * Learned warm start (not in the paper): a 3D U-Net maps the sub-problem's (x^t, d) to a
 * correction of x^t; its prediction is used as the sub-problem's starting point only when the
 * sub-problem objective confirms it.  Activations are voxel-major, channels fastest, FP32.
 * cs_nn_conv3d: 3x3x3 convolution, zero padding 1, as a BF16 implicit GEMM on the tensor cores
 *   (tcgen05, FP32 accumulation in tensor memory): out[v][coff + n] = bias[n] +
 *   sum_{tap, c} in[v + s off(tap)][c] W[n][tap * cin + c] (+ ReLU), s = -1 when flip (the data
 *   gradient, with weights packed transposed), else +1.  `packed` is [npad][kpad] BF16 from
 *   cs_nn_pack_weights (npad in {16, 32, 64}, kpad >= 27 cin, multiple of 16; 16-byte aligned).
 * cs_nn_conv3d_wgrad: gw[co][tap][ci] += sum_v gout[v][co] in[v + off(tap)][ci] as a BF16 implicit
 *   GEMM on the tensor cores (in and gout rounded to BF16, FP32 accumulation; voxels are the
 *   reduction, partial sums added in a fixed order, so the result is bit-reproducible); gb += sum_v
 *   gout in FP32.
 * cs_nn_conv1(_bwd): 1x1x1 layer; cs_nn_relu_bwd: g *= (act > 0); cs_nn_mse: loss += mean sq.
 *   error, g = its gradient; cs_nn_adam: one Adam step (step >= 1).
 * cs_nn_features / target / apply: network input [x^t / s, d eta / s] with s the RMS of
 *   (x^t, eta d) (ss receives ||x^t||^2 + eta^2 ||d||^2), training target (x_sub - x^t) / s,
 *   prediction x^t + s delta.
 * cs_nn_status: synchronise and report a bounded tensor-core wait that gave up.
 * U-Net pieces (coarse sizes nz, ny, nx; fine = 2x each; child a = 4 dz + 2 dy + dx):
 * cs_nn_maxpool2: out[v][c] = max over the 2x2x2 children of v of in, idx[v][c] = the first child
 *   reaching it; cs_nn_maxpool2_bwd: gin (fine) = g routed to the argmax child, zero elsewhere.
 * cs_nn_upconv2: stride-2 transposed convolution (kernel 2): out[child a of v][coff + co] =
 *   b[co] + sum_ci in[v][ci] w[co][a][ci] (w [cout][8][cin], FP32 on CUDA cores);
 *   cs_nn_upconv2_bwd: gin[v][ci] = sum_{a, co} gout[child a][goff + co] w[co][a][ci] (if gin),
 *   gw[co][a][ci] += sum_v gout[child a][goff + co] in[v][ci] and gb += sum gout (if gw).
 * cs_nn_slice: dst[v][doff + j] (+)= src[v][soff + j] for j < n (concatenation and its split).
 * cs_nn_conv3d_wgrad and cs_nn_upconv2_bwd take cin, cout <= 128; cs_nn_upconv2 takes cin <= 1024
 * (CS_ERR_UNSUPPORTED_SIZE above).  The 3x3x3 convolution reads a halo brick per tile when cin is
 * a multiple of 4 and `in` is 16-byte aligned, else builds the im2col rows per voxel; both give
 * the same result.
 * ---------------------------------------------------------------------------------------- */
cs_status cs_nn_pack_weights(const float* w, int cout, int cin, int transpose, unsigned short* packed,
                             int npad, int kpad, void* stream);
cs_status cs_nn_conv3d(const float* in, int nz, int ny, int nx, int cin, const unsigned short* packed,
                       int npad, int kpad, int nout, const float* bias, int relu, int flip, float* out,
                       int ldo, int coff, void* stream);
cs_status cs_nn_conv3d_wgrad(const float* in, const float* gout, int nz, int ny, int nx, int cin, int cout,
                             float* gw, float* gb, void* stream);
cs_status cs_nn_relu_bwd(const float* act, float* g, int64_t n, void* stream);
cs_status cs_nn_conv1(const float* in, int64_t nvox, int cin, int cout, const float* w, const float* b,
                      float* out, void* stream);
cs_status cs_nn_conv1_bwd(const float* in, const float* gout, int64_t nvox, int cin, int cout, const float* w,
                          float* gin, float* gw, float* gb, void* stream);
cs_status cs_nn_mse(const float* out, const float* tgt, int64_t n, float* g, float* loss, void* stream);
cs_status cs_nn_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                     float eps, int step, void* stream);
cs_status cs_nn_features(const float* xt, const float* d, int64_t n, float eta, float* ss, float* f,
                         void* stream);
cs_status cs_nn_target(const float* xt, const float* xs, int64_t n, const float* ss, float* tgt, void* stream);
cs_status cs_nn_apply(const float* xt, const float* delta, int64_t n, const float* ss, float* out, void* stream);
cs_status cs_nn_status(void* stream);
cs_status cs_nn_maxpool2(const float* in, int nz, int ny, int nx, int C, float* out, unsigned char* idx,
                         void* stream);
cs_status cs_nn_maxpool2_bwd(const float* g, const unsigned char* idx, int nz, int ny, int nx, int C, float* gin,
                             void* stream);
cs_status cs_nn_upconv2(const float* in, int nz, int ny, int nx, int cin, const float* w, const float* b,
                        int cout, float* out, int ldo, int coff, void* stream);
cs_status cs_nn_upconv2_bwd(const float* in, const float* gout, int ldg, int goff, int nz, int ny, int nx,
                            int cin, const float* w, int cout, float* gin, float* gw, float* gb, void* stream);
/* cs_crop3d: dst = the box [origin, origin + box) of a complex64 volume src of size dims (host
 * int[3] each, z, y, x); the box must lie inside the volume (CS_ERR_INVALID_ARG otherwise).  Used
 * to train the warm start on crops of large volumes. */
cs_status cs_crop3d(const float* src, const int* dims, const int* origin, const int* box, float* dst, void* stream);
cs_status cs_nn_slice(const float* src, int lds, int soff, int n, float* dst, int ldd, int doff, int64_t nvox,
                      int accumulate, void* stream);

/* Self-test of the bounded-wait protocol of the kernels that wait on mbarriers (tensor-core
 * contractions and convolutions, tensor-copy FFT passes): one block waits on a barrier, polling
 * at most `limit` times (1 .. 2^24); with arrive = 1 the barrier completes and the call returns
 * CS_OK, with arrive = 0 nothing arrives, the wait gives up on its own, the block records it in
 * a device flag and exits normally, and the call returns CS_ERR_TIMEOUT (the context stays
 * usable).  Synchronous. */
cs_status cs_wait_selftest(int arrive, int64_t limit, void* stream);

/* ------------------------------------------------------------------------------------------
 * The warm-start network as a library object (built from the pieces above; not in the paper).
 * ws_net_create: a U-Net of widths c1/c2/c3 (multiples of 4, c1, c2 <= 32, c3 <= 64; the
 *   default 16/32/64), He-normal weights from a Mersenne twister seeded by `seed` (Box-Muller),
 *   zero biases and zero Adam state, on the current device.  The handle owns all its device
 *   memory (parameters, gradients, Adam moments, packed BF16 weights, activation buffers sized
 *   for the last volume) and ws_net_destroy frees it.
 * ws_net_infer: xhat = x^t + s U-Net([x^t / s, eta d / s]) with s the RMS of (x^t, eta d); xt,
 *   d, xhat complex64 [nz][ny][nx] device arrays, dims = {nz, ny, nx} on the host, each a
 *   positive multiple of 4 (else CS_ERR_UNSUPPORTED_SIZE).  Asynchronous on `stream`.
 * ws_net_train_step: one Adam step (lr; beta 0.9 / 0.999, eps 1e-8) on the mean squared error
 *   between the network output and (x_target - x^t) / s for one volume (x_target: complex64,
 *   the sub-problem solved tightly from x^t); `loss` (device float, nullable) receives the loss
 *   before the step.  Asynchronous on `stream`.
 * ws_net_param: parameter `index` (0..25: the (w, b) pairs of e1a, e1b, e2a, e2b, b1, b2,
 *   u2, d2a, d2b, u1, d1a, d1b, out; w [cout][27][cin], [cout][8][cin] or [2][c1]) of array
 *   `which` (0 parameters, 1 last gradients, 2 / 3 Adam first / second moments): copied from
 *   the device array `src` when non-null, then to `dst` when non-null; *numel receives its size.
 * ws_net_save / ws_net_load: parameters, Adam moments and step count in a binary file (magic
 *   "CSUNET1", widths, step, then every array); loading checks the widths.  Synchronous.
 * ---------------------------------------------------------------------------------------- */
cs_status ws_net_create(int c1, int c2, int c3, uint64_t seed, cs_unet** out);
cs_status ws_net_destroy(cs_unet* net);
cs_status ws_net_infer(cs_unet* net, const float* xt, const float* d, const int* dims, float eta, float* xhat,
                       void* stream);
cs_status ws_net_train_step(cs_unet* net, const float* xt, const float* d, const float* target, const int* dims,
                            float eta, float lr, float* loss, void* stream);
cs_status ws_net_param(cs_unet* net, int which, int index, const float* src, float* dst, int64_t* numel,
                       void* stream);
cs_status ws_net_save(cs_unet* net, const char* path);
cs_status ws_net_load(cs_unet* net, const char* path);

/* ------------------------------------------------------------------------------------------
 * Regulariser building blocks (Sec. 2.1, l1-wavelets with a unitary Psi), exposed for testing:
 * periodised orthonormal db4 analysis/synthesis over all axes of an image, `levels` levels,
 * Mallat corner layout, and the complex soft threshold z max(0, 1 - tau/|z|).
 * ---------------------------------------------------------------------------------------- */
cs_status wavelet_fwd(const float* x, int ndim, const int* dims, int levels, float* c, void* stream);
cs_status wavelet_inv(const float* c, int ndim, const int* dims, int levels, float* x, void* stream);
cs_status soft_threshold(float* z, int64_t n, float tau, void* stream);

/* Host-side FP64 Hermitian eigensolver used by coil_pca's device kernel (same algorithm, same
 * source), exposed so that the Jacobi rotations can be checked without a GPU.
 *   A: host [n][n] complex128 (re, im interleaved, row-major, Hermitian), n <= 64.
 *   evecs: host [n][n] complex128 (column k = eigenvector k), evals: host [n], descending. */
cs_status cs_hermitian_eig_host(const double* A, int n, double* evecs, double* evals);

#ifdef __cplusplus
}
#endif

#endif /* COILSKETCH_H */
