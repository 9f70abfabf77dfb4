/*
 * sbqa.h -- C ABI of the GB300 (sm_103a) Simulated Bifurcation Quantum
 * Annealing hot path.
 *
 * Method: Pawlowski, Tarasiuk, Tuziemski, Pawela, Gardas, "Simulated
 * Bifurcation Quantum Annealing", arXiv 2604.01050.
 *
 * Notation.  The paper's R Trotter replicas of one run are called P here,
 * and R counts the independent runs ("repetitions" of the auto-tuning in
 * Sec. II B).  One run has P replicas coupled along a periodic
 * imaginary-time ring; runs never interact.
 *
 * Everything below is plain C: pointers, sizes, status codes.  No function
 * throws.  Status: SBQA_OK (0) or a negative SBQA_ERR_* code;
 * sbqa_strerror() names it and sbqa_last_error() gives the detail message of
 * the calling thread's last failure.
 *
 * Ownership.  The library copies every input array during the call that
 * receives it; the caller keeps ownership of its buffers and may free them
 * when the call returns.  Output buffers are owned by the caller and must
 * hold the documented number of elements.  A problem handle owns all device
 * memory it allocates and releases it in sbqa_destroy(), which keeps the
 * released blocks in a process-wide cache for later handles (a few GiB per
 * device at most; sbqa_release_cached_memory() returns them to the driver).
 *
 * Threads and streams.  Calls on one handle must not overlap (no internal
 * lock); different handles are independent.  Device work of a handle is
 * issued on the stream given to sbqa_run()/sbqa_run_begin() (NULL = the
 * legacy default stream); the device is the one current when the handle was
 * created.
 */
#ifndef SBQA_H
#define SBQA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------- */
#define SBQA_OK 0
#define SBQA_ERR_INVALID_ARG -1  /* bad size, NULL where required, bad enum   */
#define SBQA_ERR_NOT_SYMMETRIC -2 /* J != J^T, nonzero diagonal, bad CSR      */
#define SBQA_ERR_NOT_FINITE -3   /* NaN / Inf in J, h or parameters           */
#define SBQA_ERR_OOM -4          /* device or host allocation failed          */
#define SBQA_ERR_CUDA -5         /* a CUDA runtime call failed                */
#define SBQA_ERR_STATE -6        /* call out of order (e.g. get_best before run) */
#define SBQA_ERR_UNSUPPORTED -7  /* valid request the library does not serve  */
#define SBQA_ERR_TIMEOUT -8      /* a bounded device wait gave up             */

/* ---- enums ------------------------------------------------------------ */
/* Precision of the coupling product G = J . f(X) (Sec. II A, Eq. 7).  The
 * positions and momenta are FP32 in every mode; f(X) is in {-1, 0, +1}. */
#define SBQA_PREC_AUTO 0  /* EXACT if J is integer with |J_ij| <= 256, else
                             FP32                                             */
#define SBQA_PREC_FP32 1  /* J in FP32, FP32 accumulation (CUDA cores)         */
#define SBQA_PREC_EXACT 2 /* integer J (|J_ij| <= 256): J.f(X) computed exactly
                             (int8 adds or exact FP32 sums on CUDA cores; for
                             dense J with N >= 256 tcgen05 tensor cores, e4m3
                             operands for |J_ij| <= 16 and bfloat16 above,
                             FP32 accumulation of integers below 2^24)       */
#define SBQA_PREC_BF16 3  /* J rounded to bfloat16 (round to nearest even),
                             FP32 accumulation; dense J with N >= 256 runs on
                             tcgen05 tensor cores (kind::f16).  With the
                             ballistic form f(x) = x, dense J on the tensor
                             cores takes x as two bfloat16 terms, hi =
                             bf16(x) and lo = bf16(x - hi), so each x_j
                             enters the product to 2^-16 relative           */

/* Form of f in Eq. 7. */
#define SBQA_VARIANT_THRESHOLD 0 /* f(x) = 0 if |x| <= Delta(t), else sign(x) (Eq. 8) */
#define SBQA_VARIANT_BALLISTIC 1 /* f(x) = x: the bSB form of SBM (Sec. II A), with
                                    the replica coupling of Eq. 7 unchanged   */

typedef struct sbqa_problem sbqa_problem;

/* ---- problem ---------------------------------------------------------- */
/*
 * Ising instance of Sec. II A (Eqs. 1-2): symmetric couplings J with zero
 * diagonal and fields h; the energy minimised is
 *     E(s) = - sum_{i<j} J_ij s_i s_j - sum_i h_i s_i        (Eq. 4 sign).
 *
 * sbqa_create_problem_dense
 *   n    number of spins, 1 <= n <= 65536
 *   J    host, n*n doubles, row-major; must be symmetric with zero diagonal
 *        and finite (exact equality J_ij == J_ji is required)
 *   h    host, n doubles, or NULL for h = 0
 *   out  receives the new handle (NULL on failure)
 * Errors: INVALID_ARG, NOT_SYMMETRIC, NOT_FINITE, OOM, CUDA.
 */
int sbqa_create_problem_dense(int32_t n, const double *J, const double *h,
                              sbqa_problem **out);

/*
 * sbqa_create_problem_csr: the same instance in compressed sparse rows.
 *   n        number of spins, 1 <= n <= 2^31 - 1
 *   nnz      number of stored entries (both triangles), 0 <= nnz < 2^31
 *   row_ptr  host, n+1 int64, row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz
 *   col_idx  host, nnz int32, strictly increasing within a row, no diagonal
 *   val      host, nnz doubles; the pattern and values must be symmetric
 *   h        host, n doubles, or NULL
 * Errors: INVALID_ARG, NOT_SYMMETRIC (also for unsorted/duplicate columns
 * or a diagonal entry), NOT_FINITE, OOM, CUDA.
 */
int sbqa_create_problem_csr(int32_t n, int64_t nnz, const int64_t *row_ptr,
                            const int32_t *col_idx, const double *val,
                            const double *h, sbqa_problem **out);

/* Releases every resource of the handle (NULL is ignored).  Waits for the
 * handle's outstanding device work first.  Its device blocks go to the
 * library's cache of device memory (see below), not back to the driver. */
void sbqa_destroy(sbqa_problem *p);

/* Returns every device block held in the library's cache of released
 * problem buffers (on all devices) to the driver.  Handles created later
 * allocate afresh.  Safe at any time: cached blocks are not in use.  Returns
 * SBQA_OK, or SBQA_ERR_CUDA if a cudaFree failed (the remaining blocks are
 * still released). */
int sbqa_release_cached_memory(void);

typedef struct {
    int32_t n;          /* spins                                           */
    int32_t is_dense;   /* 1 if created from a dense matrix                */
    int64_t nnz;        /* stored nonzero couplings (both triangles)       */
    int32_t is_integer; /* all J_ij and h_i are integers                   */
    int32_t max_abs_j;  /* max |J_ij| if integer, else -1                  */
    double c0_auto;     /* default c0 = 0.5 sqrt(n / sum_ij J_ij^2)        */
    int32_t step_kernel;  /* coupling-product kernel of the last run: 0 CSR
                             per step, 1 dense CUDA cores, 2 dense tcgen05
                             FP8 per step (128 x 256 tiles when the padded
                             column count is a multiple of 256, else 128 x
                             128), 3 the one-launch small dense solver, 4 the
                             persistent CSR solver (one cooperative launch
                             for all steps), 5 the persistent dense tcgen05
                             solver (x, y resident in tensor memory), 6 CSR
                             and 7 dense CUDA cores for the ballistic form
                             f(x) = x, 8 the persistent dense tcgen05
                             solver with its K loop split across the two
                             CTAs of a cluster (128 x 256 tiles), 9 the
                             persistent dense tcgen05 solver on CTA pairs
                             sharing M=256 MMAs (2-CTA clusters, tcgen05
                             cta_group::2); 10 dense tcgen05 with bfloat16
                             operands per step (128 x 128 tiles), 11 its
                             persistent solver; 12 and 13 the same for the
                             ballistic form (x as bfloat16 hi + lo); 14
                             the persistent CSR solver of the ballistic
                             form; 15 the persistent dense tcgen05 solver
                             with packed e2m1 operands (kind::mxf4, unit
                             scale factors) and J resident in shared
                             memory, 16 its paired form (2-CTA clusters
                             sharing M=256 MMAs); -1 none                    */
    int32_t step_variant; /* CSR kernel variant picked by the autotuner:
                             0-5: 4 << (v % 3) consecutive replica columns
                             per lane, v >= 3 with one wave of blocks
                             looping over the (row, column chunk) items;
                             6, 7: the ELL form of rows of degree <= 8 (4
                             or 8 columns per lane); -1 before the first
                             run                                          */
    float variant_ms[8];  /* autotuner timing of each CSR variant (ms per
                             step; 0 = not timed / not eligible); for the
                             dense tcgen05 path [0] is the per-step kernel */
    float persistent_ms;  /* autotuner timing of the persistent solver of
                             the path in use, CSR or dense tcgen05 (ms per
                             step; 0 = not timed / not eligible)          */
    int32_t j_on_device;  /* 1: a dense J of N >= 1024 read by the GPU from
                             the caller's array (systems where the GPU
                             reaches pageable host memory through the
                             host's page tables), with its checks and
                             statistics, and the library's copy kept in
                             device memory; 0: read on the host            */
} sbqa_problem_info;

int sbqa_get_problem_info(const sbqa_problem *p, sbqa_problem_info *info);

/* ---- schedule --------------------------------------------------------- */
/*
 * Parameters of the equations of motion (Sec. II A, Eqs. 5-8) and of the
 * per-run auto-tuning (Sec. II B).
 *   a0           a_0 of Eqs. 6-7 (default 1)
 *   c0           c_0 of Eq. 7; <= 0 selects c0_auto (default 0)
 *   dt           time step of the symplectic Euler integrator (default 0.5);
 *                step n runs at t/T = n / steps
 *   gamma0       Gamma_x(0) of Eq. 5 (default 1)
 *   delta_slope  Delta(t) = delta_slope * t/T (Eq. 8 threshold; default 0.7)
 *   init_amp     initial x, y uniform in [-init_amp, init_amp) (default 0.1)
 *   jperp_enable 1: J_perp(t) of Eq. 5; 0: J_perp = 0 (plain SB per replica)
 *   variant      SBQA_VARIANT_THRESHOLD (SBQA, Eq. 8) or
 *                SBQA_VARIANT_BALLISTIC (f(x) = x; the product runs on FP32
 *                positions: CSR kernels for sparse J, the CUDA-core kernel
 *                for dense J, or, with SBQA_PREC_BF16 and dense N >= 256,
 *                the tensor cores with x as bfloat16 hi + lo; not served by
 *                the batching engine)
 *   precision    SBQA_PREC_*
 *   eval_every   0: read out only after the last step; K > 0: also after
 *                every step n with (n+1) % K == 0, keeping the best so far
 *   n_runs       length of beta and alpha (must equal R of the run)
 *   kernel_select  0 = let the autotuner choose between the per-step
 *                kernels and the persistent solver (default); 1 = per-step
 *                kernels; 2 = the persistent solver when the instance
 *                qualifies, else per-step.  CSR qualifies with degree <= 8
 *                and R*P a multiple of 128; the dense tensor-core
 *                path when its 128 x 128 tiles (padded N x padded R*P) fit
 *                the device at once (one per SM).  3 + v (v = 0..7) forces
 *                per-step CSR kernel variant v (see step_variant); 11 forces
 *                the persistent CSR solver in the mode that caches whole
 *                rows (otherwise taken only when the items outnumber its
 *                cache; when the rows outnumber it too, a warp caches the
 *                items that fit and reads the neighbours of the rest from
 *                the ELL form every step); 12 = as 2, but the dense tensor-core solver keeps
 *                its 128 x 128 tiles instead of splitting the K loop across
 *                2-CTA clusters (taken by default when padded N and padded
 *                R*P are multiples of 256); with 1 or 12 no cluster kernel
 *                is launched at all; 13 = the dense tensor-core
 *                solver on CTA pairs that share M=256 MMAs (padded N a
 *                multiple of 256; with kernel_select 0 the autotuner times
 *                it beside the others); 14 = the dense tensor-core
 *                solver with packed e2m1 operands (integer |J_ij| <= 4,
 *                padded N <= 2304: each CTA keeps its 128 rows of J in
 *                shared memory and only f streams in), on CTA pairs that
 *                share M=256 MMAs where padded N is a multiple of 256,
 *                else as 12; 15 = the same solver without clusters; with
 *                kernel_select 0 the autotuner times both forms beside the
 *                others.
 *                For the ballistic form on CSR, 2
 *                takes its persistent solver when each warp's share of the
 *                (row, 128-column) items fits its cache (degree <= 8), 0
 *                times it beside the per-step kernel, any other value keeps
 *                the per-step kernel.  Results are identical whichever
 *                kernel runs.
 *   beta, alpha  host, n_runs doubles each: per-run inverse temperature and
 *                schedule exponent (the auto-tuning draws them from
 *                [0.5,1.5] x [0.5,1.0]); beta > 0, alpha > 0
 * The library copies beta and alpha.  Errors: INVALID_ARG, NOT_FINITE.
 */
typedef struct {
    double a0;
    double c0;
    double dt;
    double gamma0;
    double delta_slope;
    double init_amp;
    int32_t jperp_enable;
    int32_t variant;
    int32_t precision;
    int32_t eval_every;
    int32_t n_runs;
    int32_t kernel_select;
    const double *beta;
    const double *alpha;
} sbqa_params;

/* Fills the defaults listed above (beta = alpha = NULL, n_runs = 0, which
 * sbqa_set_schedule reads as beta = alpha = 1 for every run). */
void sbqa_default_params(sbqa_params *p);

int sbqa_set_schedule(sbqa_problem *p, const sbqa_params *params);

/* ---- run -------------------------------------------------------------- */
/*
 * sbqa_run: the whole hot path, asynchronously on `stream`
 * (a cudaStream_t, NULL = legacy default stream):
 *   initial state from SplitMix64 keyed by (seed, run r, replica k, spin i)
 *   -> `steps` steps of Eqs. 6-7 with the wall rule
 *   -> sign readout, energies of all R*P replicas, per-run best.
 *   steps  >= 0 (0 reads out the initial state)
 *   P      Trotter replicas per run, 1 <= P <= 128 (the periodic ring of
 *          Eqs. 6-7 closes at P for any P; a run occupies the next power of
 *          two of replica columns on the device, the rest being padding
 *          that no replica reads; P > 128 gives UNSUPPORTED)
 *   R      runs, >= 1, R * (P rounded up to a power of two) <= 2^20; must
 *          equal params.n_runs when beta and alpha were given
 * Errors: STATE (no schedule), INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 * Device buffers for the state are allocated on first use for a given
 * (P, R) and reused by later runs of the same shape.
 */
int sbqa_run(sbqa_problem *p, int32_t steps, int32_t P, int32_t R,
             uint64_t seed, void *stream);

/* The same run split at step boundaries (checkpoint / resume):
 * begin = initial state and tables, advance = the next n_steps steps
 * (clamped to the anneal's end, with readouts per eval_every),
 * finish = final readout.  begin + advance(steps) + finish is exactly
 * sbqa_run. */
int sbqa_run_begin(sbqa_problem *p, int32_t steps, int32_t P, int32_t R,
                   uint64_t seed, void *stream);
int sbqa_run_advance(sbqa_problem *p, int32_t n_steps);
int sbqa_run_finish(sbqa_problem *p);

/* Waits for the handle's device work. */
int sbqa_synchronize(sbqa_problem *p);

/* ---- results (synchronising, host buffers) ---------------------------- */
/*
 * Per-run best over replicas (and over readouts when eval_every > 0), the
 * answer of the auto-tuned solver ("return the best solution from all
 * repetitions", Sec. II B).  Any pointer may be NULL.
 *   spins       R*N int8 (+1/-1), run-major
 *   energy      R doubles (exact for integer instances)
 *   energy_int  R int64 (filled only for integer instances)
 *   replica     R int32, the replica k of the best readout (lowest k on ties)
 *   step        R int32, the step index after which it was read (-1 = the
 *               initial state; the earliest readout wins ties)
 * Errors: STATE (no finished readout), CUDA.
 */
int sbqa_get_best(sbqa_problem *p, int8_t *spins, double *energy,
                  int64_t *energy_int, int32_t *replica, int32_t *step);

/* Energies of all R*P replicas at the last readout, run-major [r][k]. */
int sbqa_get_energies(sbqa_problem *p, double *energy, int64_t *energy_int);

/*
 * State access for tests and checkpoints, layout [r][k][i] (R*P*N floats).
 * get_state returns the positions/momenta after `*step_done` steps.
 * set_state replaces them and sets the number of completed steps to
 * step_done (0 <= step_done <= steps of the current run); the next
 * advance continues from there.
 */
int sbqa_get_state(sbqa_problem *p, float *x, float *y, int32_t *step_done);
int sbqa_set_state(sbqa_problem *p, const float *x, const float *y,
                   int32_t step_done);

/* ---- batching engine ---------------------------------------------------- */
/*
 * Continuous batching of many solves on one GPU (no counterpart in the
 * paper, which runs the repetitions of one instance in parallel, Sec. II B;
 * the engine extends that to many instances).  A request is a problem handle
 * (with its schedule set) plus steps, P, R and seed; its result is the
 * per-run best of sbqa_get_best.  Requests are admitted in arrival order
 * whenever a slot and room in the engine's device arena are free; their
 * state stays resident in the arena; at every sbqa_engine_step all active
 * requests advance by up to `chunk_steps` steps (CSR requests together in
 * one batched launch per step); finished requests are read out and leave.
 * A request's result is bit-identical to sbqa_run of the same request.
 * The problem handles must outlive their requests.  One engine is driven by
 * one host thread.
 *
 * sbqa_engine_create
 *   arena_bytes  device memory reserved for request state (>= 1 MiB)
 *   max_slots    requests active at the same time (1..4096)
 *   chunk_steps  steps per sbqa_engine_step (>= 1)
 * Errors: INVALID_ARG, OOM.
 */
typedef struct sbqa_engine sbqa_engine;

int sbqa_engine_create(int64_t arena_bytes, int32_t max_slots,
                       int32_t chunk_steps, sbqa_engine **out);
void sbqa_engine_destroy(sbqa_engine *e);

/* How the engine runs the chunks of small dense requests on the tensor cores
 * (fewer 128 x 128 tiles than one wave of the persistent solver holds):
 *   1 (default)  together, one cooperative launch of the batched persistent
 *                solver per group of equal operand form and run width, on
 *                the engine's stream before the CSR requests' chunk
 *   0            each on a stream of its own slot, one per-step kernel launch
 *                per step, beside the CSR requests' chunk
 * Results are the same either way.  Takes effect at the next
 * sbqa_engine_step.  Errors: INVALID_ARG. */
int sbqa_engine_set_dense_batching(sbqa_engine *e, int32_t on);

/* Queues a request; *id receives its number (0, 1, ... in submit order).
 * steps >= 1; P and R as for sbqa_run.  Errors: STATE (no schedule),
 * INVALID_ARG, UNSUPPORTED, OOM (request larger than the arena). */
int sbqa_engine_submit(sbqa_engine *e, sbqa_problem *p, int32_t steps,
                       int32_t P, int32_t R, uint64_t seed, int32_t *id);

/* Admits what fits, advances every active request by up to chunk_steps
 * steps on `stream` (a cudaStream_t), reads out the finished ones and waits
 * for the device.  *n_done receives how many finished; the first `cap` of
 * their ids go to done_ids (host, may be NULL when cap = 0).
 * Errors: CUDA, TIMEOUT.  TIMEOUT means that a bounded device wait of at
 * least one finished request gave up: every finished request (failed or
 * not) has still left its slot and arena space and is listed in done_ids;
 * sbqa_engine_result returns TIMEOUT for the failed ones and the results of
 * the others; the engine keeps serving. */
int sbqa_engine_step(sbqa_engine *e, void *stream, int32_t *n_done,
                     int32_t *done_ids, int32_t cap);

/* Result of a finished request (host buffers, any may be NULL):
 * spins R*N int8, energy R doubles, energy_int R int64 (integer instances),
 * replica R int32 -- as sbqa_get_best.  Errors: INVALID_ARG, STATE (not
 * finished), TIMEOUT (the request failed, see sbqa_engine_step). */
int sbqa_engine_result(sbqa_engine *e, int32_t id, int8_t *spins,
                       double *energy, int64_t *energy_int,
                       int32_t *replica);

typedef struct {
    int32_t queued, active, finished;
    int64_t arena_bytes, arena_used;
    int64_t updates_issued; /* replica-spin updates advanced so far */
    int64_t kernels_launched; /* kernels the engine has launched so far */
    int64_t batched_updates;  /* replica-spin updates of the CSR requests, advanced
                                 by the batched step kernel */
    double batched_ms;        /* device time of those batched launches (CUDA
                                 events around each chunk's launches; dense
                                 requests may run beside them) */
    int64_t dense_batched_launches; /* cooperative launches that advanced the
                                       chunks of several small dense
                                       tensor-core requests together */
    int64_t dense_batched_chunks;   /* request chunks advanced by those launches */
    int64_t dense_e2m1_requests;    /* dense requests served by the solver with
                                       packed e2m1 operands (integer |J| <= 4) */
} sbqa_engine_stats_t;

int sbqa_engine_stats(const sbqa_engine *e, sbqa_engine_stats_t *s);

/* ---- energies without device allocation -------------------------------- */
/*
 * sbqa_energies_csr_noalloc -- Ising energies of caller-supplied spin
 * configurations for a CSR instance, using no device allocation at all.
 * The paper has no counterpart: this is a service entry point for callers
 * that cannot call cudaMalloc where they need energies, e.g. code that is in
 * the middle of capturing a CUDA graph (allocation is not a capturable
 * operation), real-time loops that must never block in the allocator, and
 * host frameworks that own all device memory through their own pool.
 *
 * Every pointer except `stream` is a DEVICE pointer owned by the caller:
 *   n         spins, >= 1
 *   row_ptr   int32[n+1], col_idx int32[nnz]: the CSR pattern (as in
 *             sbqa_create_problem_csr, symmetric, no diagonal; not re-checked)
 *   val_i32 / val_f64   couplings, exactly one non-NULL: int32 for integer
 *             instances (exact int64 energies), double otherwise
 *   h_i64 / h_f64       fields matching the value type, or NULL for h = 0
 *   spins     int8 [n][ld], +1/-1; column c (0 <= c < count) is one
 *             configuration (the spin-major layout of the solver's state)
 *   ld        row stride of spins in bytes, >= count
 *   count     number of configurations, >= 1
 *   energy_int  int64[count] or NULL (integer instances only)
 *   energy    double[count]; required for real instances, optional otherwise
 *   stream    cudaStream_t (NULL = legacy default stream); the call is
 *             asynchronous on it
 * E(s) = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i, summed in a fixed order
 * (the same as the solver's readout), so results match sbqa_get_energies.
 *
 * Memory: the partial sums live in one file-scope device array of 4 MiB that
 * is part of the library image; every GPU that loads the library reserves it
 * until the process exits.  A call needs ceil(n/32) * ceil(count/128)*128
 * partial sums of 8 bytes; larger requests fail with SBQA_ERR_UNSUPPORTED
 * (e.g. n = 4096 allows up to 4096 configurations).  Nothing is allocated,
 * freed or cleared: every scratch entry that is read was written earlier in
 * the same call.
 * All calls share that array and it keeps the last call's contents, so calls
 * whose kernels overlap on the GPU (different streams, or several host
 * threads) race and must be ordered by the caller.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * Errors: INVALID_ARG, UNSUPPORTED (size beyond the scratch), CUDA.
 */
int sbqa_energies_csr_noalloc(int32_t n, const int32_t *row_ptr,
                              const int32_t *col_idx, const int32_t *val_i32,
                              const double *val_f64, const int64_t *h_i64,
                              const double *h_f64, const int8_t *spins,
                              int32_t ld, int32_t count, int64_t *energy_int,
                              double *energy, void *stream);

/* ---- errors ----------------------------------------------------------- */
const char *sbqa_strerror(int status);
/* Detail message of the calling thread's last failed call ("" if none). */
const char *sbqa_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int sbqa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SBQA_H */
