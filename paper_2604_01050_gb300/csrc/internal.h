// internal.h -- declarations shared by the translation units of libsbqa.
//
// Device layout of one run batch (C = R * P columns, column c = r * P + k,
// padded to Cp, a multiple of 128 so that one warp owns 128 whole columns
// and therefore whole runs, because P divides 32):
//   x, y   float  [N][Cp]   positions / momenta, spin-major
//   F[2]   uint8  [N][Cp]   f(x) + 1 in {0, 1, 2} for the current / next step
// Per-step FP32 coefficients (host FP64 -> FP32, one table entry per step):
//   ka[n]      dt * (a0 - a_n) / P       (a_n = n / S, Sec. II A)
//   dl[n]      Delta_n = delta_slope * n / S   (n = 0..S, Eq. 8)
//   kj[n][r]   dt * J_perp(t_n) for run r  (Eq. 5)
//   kc, kx     dt * c0 / P,  dt * a0 / P
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace sbqa {

constexpr int kColsPerWarp = 128;  // 32 lanes x 4 columns
constexpr int kMaxReplicas = 128;  // Trotter replicas per run: a run's columns never leave a warp's 128

// Columns a run of P replicas occupies: the smallest power of two >= P
// (replica k of run r is column r * width + k; the rest of the run is padding).
inline int run_width(int P) {
  int w = 1;
  while (w < P) w <<= 1;
  return w;
}
constexpr int kColsPerLane = 4;

enum ValKind : int { VAL_PM1 = 0, VAL_F32 = 1, VAL_BF16 = 2 };

struct StepTables {
  const float *ka;  // [S]
  const float *dl;  // [S + 1]
  const float *kj;  // [S][R]
  float kc, kx;
  int S, R;
};

struct StateView {
  // P: columns per run (a power of two, the kernels' template width); Pr: the
  // run's Trotter replicas (1 <= Pr <= P), columns r * P + k for k < Pr; the
  // columns k >= Pr of a run are padding that no replica reads
  int N, C, Cp, P, R;
  int Pr;
  float *x, *y;
  uint8_t *F[2];  // f(x) + 1 codes, double-buffered by step parity
  float *Fx[2];   // f(x) = x copies of the ballistic form (null otherwise)
  int8_t *Sg;     // [N][Cp] readout spins sign(x), +1 for x >= 0
  // F buffer holding the codes of step n (selected without indexing the
  // array, which would put the kernel argument in local memory)
  __host__ __device__ uint8_t *f_of(int n) const { return (n & 1) ? F[1] : F[0]; }
  __host__ __device__ float *fx_of(int n) const { return (n & 1) ? Fx[1] : Fx[0]; }
};

struct CsrView {
  const int32_t *row_ptr;  // [N + 1]
  const int32_t *col;      // [nnz] (VAL_PM1: each row's +1 entries first)
  const void *val;         // float (F32) or bf16 (BF16); unused for VAL_PM1
  const int32_t *npos;     // VAL_PM1: number of +1 entries of each row
  const float *h;          // [N], never null (zeros when h = 0)
  int kind;
  // ELL form of rows with degree <= kEllSlots (null when not built): slots
  // [N][kEllSlots] of columns and values (the CSR kernel's entry order, zero
  // padded) and (degree, +1 count) per row
  const int32_t *ell_col;
  const float *ell_val;
  const int32_t *ell_meta;
};

constexpr int kEllSlots = 8;

struct DenseView {
  const float *J;  // [N][N] row-major, FP32 (exact for integers)
  const float *h;  // [N]
};

// Readout: energies of s = sign(x) for every column.
struct EnergyView {
  int is_integer;
  // sparse: row_ptr/col from CsrView with FP64 or int values below
  const double *val_f64;   // [nnz] (sparse) or [N][N] (dense), real instances
  const int32_t *val_i32;  // [nnz] or [N][N], integer instances
  const double *h_f64;     // [N]
  const int64_t *h_i64;    // [N]
};

struct BestView {
  int64_t *e_int;        // [Cp] energies of the last readout (integer)
  double *e_f64;         // [Cp] (real instances, also filled for integer)
  int64_t *part_int;     // [nblk][Cp] partial sums
  double *part_f64;      // [nblk][Cp]
  int nblk;              // row blocks of the energy kernel
  int64_t *best_e_int;   // [R]
  double *best_e;        // [R]
  int32_t *best_k;       // [R]
  int32_t *best_step;    // [R]
  int8_t *best_spins;    // [R][N]
  int32_t *have_best;    // [R]
};

// Records msg as the calling thread's detail message (sbqa_last_error) and
// returns code.
int set_error(int code, const std::string &msg);

// All steps of a +-1 CSR run batch in one cooperative launch with a bounded
// grid barrier between steps (solve_persistent.cu).
int persistent_blocks();
int persistent_barrier_words();  // size of the barrier counter buffer
// 0: not eligible; 1: items cached per warp; 2: whole rows cached per warp
// (force_rows: rows whenever they fit); 3: items, as many cached per warp as
// fit and the rest read from the ELL arrays every step (ell: the ELL form
// exists); kind = the CSR value kind
int persistent_mode(int N, int Cp, int max_degree, int kind, int blocks, bool force_rows, bool ell);
cudaError_t launch_solve_csr_persistent(const StateView &s, const CsrView &J, const StepTables &t, int n_begin,
                                        int n_end, unsigned *bar, int *err, int blocks, int mode, cudaStream_t st);
// The ballistic form f(x) = x in one cooperative launch (items of 128 columns
// cached per warp; f buffers Fx in FP32): eligible when the items fit the
// cache (persistent_bsb_ok); results equal launch_step_csr_bsb bit for bit.
bool persistent_bsb_ok(int N, int Cp, int max_degree, int kind, int blocks);
cudaError_t launch_solve_csr_persistent_bsb(const StateView &s, const CsrView &J, const StepTables &t, int n_begin,
                                            int n_end, unsigned *bar, int *err, int blocks, cudaStream_t st);

// Steps of a dense integer run on the tensor cores in one cooperative launch,
// x and y resident in tensor memory, per-tile step flags between CTAs
// (step_dense_tc.cu).  flags holds tc_persistent_flag_count() counters.
int tc_persistent_blocks();
bool tc_persistent_eligible(int Kp, int Cp, int blocks);
size_t tc_persistent_flag_count(int Kp, int Cp);
// The same with the K loop split across the two CTAs of a cluster (128 x 256
// output tiles; Kp and Cp multiples of 256); blocks = co-resident CTAs in
// 2-CTA clusters (tc_split_blocks()).
int tc_split_blocks();
bool tc_split_eligible(int Kp, int Cp, int blocks);
cudaError_t launch_solve_dense_tc_split(const void *plan, const StateView &s, int Kp, int *err, const float *h,
                                        const StepTables &t, int n_begin, int n_end, uint32_t *flags,
                                        cudaStream_t st);
cudaError_t launch_solve_dense_tc_persistent(const void *plan, const StateView &s, int Kp, int *err, const float *h,
                                             const StepTables &t, int n_begin, int n_end, uint32_t *flags,
                                             cudaStream_t st);

// Dense J read by the GPU from the caller's host array (ingest_dense.cu),
// where the GPU reaches pageable host memory through the host's page tables;
// one pass, each entry read once.  Per row: max |J_ij|, the sum of squares,
// the nonzeros and the flags below; d8 / d64 [N][N] receive the byte copy
// (int(v) for v in [-128, 127], else 0) and the FP64 copy; part holds
// ingest_part_count(N) per-tile partials; *asym becomes nonzero when J != J^T.
struct IngestRow {
  double mx, s2;
  int32_t nnz;
  uint32_t flags;
};
constexpr uint32_t kIngestFinite = 1, kIngestDiagZero = 2, kIngestInteger = 4, kIngestPm1 = 8;
bool ingest_on_device_possible();
size_t ingest_part_count(int n);
cudaError_t launch_ingest_dense(const double *J, int n, int8_t *d8, double *d64, IngestRow *part, IngestRow *rows,
                                int *asym, cudaStream_t st);
// Device forms from the device copy (d8 when it holds J, else d64): padded
// e4m3 (|J_ij| <= 16) and bfloat16 operands [Kp][Kp], and flat [N][N] forms.
constexpr int kFlatI32 = 0, kFlatF64 = 1, kFlatF32 = 2, kFlatBf16InF32 = 3;
cudaError_t launch_tc_j8_from_device(const int8_t *d8, int n, int Kp, uint8_t *out, cudaStream_t st);
cudaError_t launch_tc_jbf16_from_device(const int8_t *d8, const double *d64, int n, int Kp, uint16_t *out,
                                        cudaStream_t st);
cudaError_t launch_flat_from_device(const int8_t *d8, const double *d64, size_t m, int form, void *out,
                                    cudaStream_t st);

// Several dense problems' chunks in one cooperative launch of the persistent
// tensor-core solver (solve_dense_tc_batched.cu): one CTA per 128 x 128 tile
// of each problem, tiles of one problem consecutive; the problems of a batch
// share the operand form, the run width P and the ring form.  A batch holds
// at most cap_reqs problems and cap_tiles tiles (at most tc_batch_blocks()
// for one launch).  tc_batch_add returns cudaErrorInvalidValue for a problem
// that does not fit (tc_batch_fits) or has no persistent form.
struct TcBatch;
cudaError_t tc_batch_create(TcBatch **out, int cap_reqs, int cap_tiles);
void tc_batch_destroy(TcBatch *b);
void tc_batch_clear(TcBatch *b);
int tc_batch_tiles(const TcBatch *b);
int tc_batch_size(const TcBatch *b);
bool tc_batch_fits(const TcBatch *b, const void *plan, const StateView &s, int Kp);
// hold_step: test hook, the request's tile (0, 0) leaves its step counter
// unpublished after that step, so its other tiles' waits run out (-1: never)
cudaError_t tc_batch_add(TcBatch *b, const void *plan, const StateView &s, int Kp, int *err, const float *h,
                         const StepTables &t, int n_begin, int n_end, int hold_step = -1);
cudaError_t tc_batch_launch(TcBatch *b, cudaStream_t st);
cudaError_t tc_batch_set_attributes();
int tc_batch_blocks();

// The persistent dense solver with the product in packed e2m1 on the
// block-scaled tensor cores (tcgen05.mma kind::mxf4, unit scale factors;
// solve_dense_tc_f4.cu): integer |J_ij| <= 4, a CTA's J rows resident in
// shared memory (Kp <= 2304).  J4 [Kp][Kh] and FT4 [2][Cp][Kh] bytes, Kh =
// tc_f4_row_bytes(Kp), two spins per byte; the same flags, step protocol and
// results (bit for bit) as launch_solve_dense_tc_persistent.
int tc_f4_row_bytes(int Kp);
int tc_f4_blocks();
bool tc_f4_eligible(int Kp, int Cp, int blocks);
cudaError_t tc_f4_set_attributes();
bool tc4_plan_make(void **plan, const void *J4, void *FT4, int Kp, int Cp);
void tc4_plan_free(void *plan);
cudaError_t launch_j4_from_j8(const uint8_t *J8, int Kp, uint8_t *J4, cudaStream_t st);
cudaError_t launch_f_to_ft4(const StateView &s, int which, uint8_t *FT4, int Kp, int buffer, cudaStream_t st);
cudaError_t launch_solve_dense_tc_f4(const void *plan, const StateView &s, int Kp, int *err, const float *h,
                                     const StepTables &t, int n_begin, int n_end, uint32_t *flags, cudaStream_t st);
// Its batched form for many small problems in one cooperative launch (the
// engine): the same protocol as TcBatch below; tc_f4_blocks() covers its
// occupancy and attributes.
struct Tc4Batch;
cudaError_t tc4_batch_create(Tc4Batch **out, int cap_reqs, int cap_tiles);
void tc4_batch_destroy(Tc4Batch *b);
void tc4_batch_clear(Tc4Batch *b);
int tc4_batch_size(const Tc4Batch *b);
bool tc4_batch_fits(const Tc4Batch *b, const StateView &s, int Kp);
cudaError_t tc4_batch_add(Tc4Batch *b, const void *plan4, const StateView &s, int Kp, int *err, const float *h,
                          const StepTables &t, int n_begin, int n_end, int hold_step = -1);
cudaError_t tc4_batch_launch(Tc4Batch *b, cudaStream_t st);
// Its paired form: the CTAs of row tiles 2p, 2p + 1 share M=256 MMAs (2-CTA
// clusters, tcgen05 cta_group::2) and each stages half of every f tile, so a
// step's f tiles are in flight at once; padded N a multiple of 256, blocks
// = co-resident CTAs in 2-CTA clusters (tc_f4_pair_blocks()).
int tc_f4_pair_blocks();
bool tc_f4_pair_eligible(int Kp, int Cp, int blocks);
cudaError_t launch_solve_dense_tc_f4_pair(const void *plan, const StateView &s, int Kp, int *err, const float *h,
                                          const StepTables &t, int n_begin, int n_end, uint32_t *flags,
                                          cudaStream_t st);

// The persistent dense solver on 2-CTA clusters sharing M=256 MMAs
// (tcgen05 cta_group::2; step_dense_tc.cu): padded N a multiple of 256,
// row-tile pairs x column tiles co-resident as clusters (tc_pair_blocks()).
// Same flags and results as launch_solve_dense_tc_persistent.
int tc_pair_blocks();
bool tc_pair_eligible(int Kp, int Cp, int blocks);
cudaError_t launch_solve_dense_tc_pair(const void *plan, const StateView &s, int Kp, int *err, const float *h,
                                       const StepTables &t, int n_begin, int n_end, uint32_t *flags,
                                       cudaStream_t st);

// Ballistic form f(x) = x (step_bsb.cu): CSR and dense CUDA-core steps, and
// the copy x -> Fx[which] that starts the f buffers.
cudaError_t launch_step_csr_bsb(const StateView &s, const CsrView &J, const StepTables &t, int n, cudaStream_t st);
cudaError_t launch_step_dense_bsb(const StateView &s, const DenseView &J, const StepTables &t, int n,
                                  cudaStream_t st);
cudaError_t launch_copy_fx(const StateView &s, int which, cudaStream_t st);

// Whole solve of a small integer dense instance in one launch (solve_small.cu).
struct SmallArgs {
  int N, P, R, S, Cp;
  uint64_t seed;
  float amp, kc, kx;
  const float *J;        // [N][N] FP32
  const float *ka, *dl, *kj;
  const float *h;        // [N]
  const int32_t *J_i32;  // [N][N]
  const int64_t *h_i64;  // [N]
  float *x, *y;          // [N][Cp]
  int8_t *Sg;
  int64_t *e_int;
  double *e_f64;
  int64_t *best_e_int;
  double *best_e;
  int32_t *best_k, *best_step, *have_best;
  int8_t *best_spins;
};
bool small_eligible(int N, int P, int S);
cudaError_t launch_solve_small(const SmallArgs &a, cudaStream_t st);

// One active request of the batching engine (device copy, read by the
// batched step kernel).
struct SlotDesc {
  const int32_t *row_ptr, *col, *npos;  // CSR (col in the step kernel's order)
  const int32_t *ell_col, *ell_meta;    // ELL form of rows of degree <= 8 (null when not built)
  const float *ell_val;
  const void *val;
  const float *h;
  int kind;
  int N, C, Cp, P, R, S;
  int Pr;  // replicas of a run (P: its column width, a power of two)
  float *x, *y;
  uint8_t *F0, *F1;
  const float *ka, *dl, *kj;
  float kc, kx;
  int n0;  // steps completed before the current chunk
  int W;   // replica columns per lane: 8 (ELL form: units of two rows on half warps) or 4 (a row per warp)
  int wide;  // ELL form with Cp a multiple of 256: units of one row x 256 columns on a whole warp
};

// 128 replica columns (colgroup) of 2 spin rows (a unit, W = 8), 256 columns of one row (a wide unit), or
// 128 columns of 8 rows (an item, W = 4) of one slot.
struct WorkItem {
  int slot, row0, colgroup, pad;
};

// ---- launchers (return cudaGetLastError() of the launch) ----
cudaError_t launch_init(const StateView &s, uint64_t seed, float amp, float delta0,
                        cudaStream_t st);
cudaError_t launch_refresh_f(const StateView &s, int which, float delta, cudaStream_t st);
// variant v: 4 << v consecutive columns per lane (picked per problem shape by
// the autotuner in api.cu); valid when Cp is a multiple of 32 * (4 << v).
int csr_step_variants();
bool csr_step_variant_ok(int variant, int Cp, bool has_ell);
cudaError_t launch_step_csr(const StateView &s, const CsrView &J, const StepTables &t,
                            int n, int variant, cudaStream_t st);
cudaError_t launch_step_dense(const StateView &s, const DenseView &J, const StepTables &t,
                              int n, cudaStream_t st);
// Dense couplings on tcgen05 (step_dense_tc.cu).  Operand forms (op):
// 0 = integer J and f codes in e4m3, 1 = J rounded to bfloat16 and f codes in
// bfloat16, 2 = the ballistic form, J in bfloat16 and x as bfloat16 hi + lo.
// The plan holds the TMA descriptors of J [Kp][Kp] and FT [2][Cp][Kp] (of the
// operand type; for op 2 the lo terms follow the hi terms) and of the state
// x, y [N][Cp] (FP32) of one run batch.
constexpr int kTcOpF8 = 0, kTcOpBf16 = 1, kTcOpBsb = 2;
size_t tc_ft_bytes(int Kp, int Cp, int op);  // bytes of FT
size_t tc_j_bytes(int Kp, int op);           // bytes of J
bool tc_plan_make(void **plan, const void *J, void *FT, int Kp, int Cp, float *x, float *y, int N, int op);
void tc_plan_free(void *plan);
int tc_op_of(const void *plan);
cudaError_t tc_set_attributes();  // dynamic shared memory limit of the tcgen05 kernels
cudaError_t launch_step_dense_tc(const void *plan, const StateView &s, int Kp, uint8_t *FT, int *err,
                                 const float *h, const StepTables &t, int n, cudaStream_t st);
// FT buffer `buffer` from the f codes of F buffer `which` (op 0, 1) or from x (op 2)
cudaError_t launch_f_to_ft(const StateView &s, int which, uint8_t *FT, int Kp, int buffer, int op, cudaStream_t st);

// All steps j0 .. j1 - 1 of a chunk for every active CSR slot in one
// cooperative launch of `grid` blocks (step_batched.cu; at most
// batched_persistent_blocks(), the co-resident count).  items: first
// counts[0] units of 2 rows x 128 columns of slots in ELL form (W = 8), then
// counts[1] items of 8 rows x 128 columns of the others (W = 4); counts in
// device memory.  bar holds grid_barrier_words() counters (zeroed here); a
// barrier that gives up records code 4 in *err.
int batched_persistent_blocks();
int batched_grid(int64_t tasks);  // blocks for `tasks` warp tasks (units, or rows of items), at most one wave
cudaError_t launch_solve_batched(const SlotDesc *slots, int n_slots, const WorkItem *items, const int *counts,
                                 int grid, int j0, int j1, unsigned *bar, int *err, cudaStream_t st);

int energy_row_blocks(int N);
// Readout energies of an integer dense instance on the tensor cores: the sign
// codes go into FT buffer `buffer` (one the next step does not read), then
// one FP8 GEMM with the row-block partial sums in its epilogue
// (step_dense_tc.cu, init_readout.cu).
cudaError_t launch_energy_partials_tc(const void *plan, const StateView &s, int Kp, uint8_t *FT, int b, int *err,
                                      const int64_t *h_i64, int64_t *part, int nblk, cudaStream_t st);
cudaError_t launch_energy_dense_tc(const void *plan, const StateView &s, int Kp, uint8_t *FT, int buffer, int *err,
                                   const EnergyView &E, const BestView &b, cudaStream_t st);
// sign(x) into Sg, energies of every column into b.e_int / b.e_f64.
cudaError_t launch_energy_csr(const StateView &s, const CsrView &J, const EnergyView &E,
                              const BestView &b, cudaStream_t st);
cudaError_t launch_energy_dense(const StateView &s, const EnergyView &E, const BestView &b,
                                cudaStream_t st);
cudaError_t launch_best(const StateView &s, const EnergyView &E, const BestView &b, int step,
                        cudaStream_t st);
cudaError_t launch_reset_best(const StateView &s, const BestView &b, cudaStream_t st);

}  // namespace sbqa
