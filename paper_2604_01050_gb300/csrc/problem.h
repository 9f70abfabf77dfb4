// problem.h -- the problem handle shared by the host side of the library
// (api.cu: single solves; engine.cu: the batching engine).
#pragma once
#include <cstdint>
#include <cstring>
#include <memory>
#include <new>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sbqa.h"
#include "internal.h"

namespace sbqa {

// Process-wide cache of large host blocks (api.cu): arrays of 1 MiB and more
// (copies of J, staging of device uploads) are kept after use, up to a cap,
// so that the next handle of a similar size writes into pages that are
// already mapped instead of faulting in fresh ones (64 MB for the byte copy
// of a dense J at N = 8192).  Size classes are multiples of 1 MiB.
constexpr size_t kHostCacheMin = size_t(1) << 20;
void *hostcache_get(size_t bytes);          // a block of at least `bytes`; nullptr when out of memory
void hostcache_put(void *p, size_t bytes);  // `bytes` as given to hostcache_get

// Allocator that leaves value-initialised elements uninitialised, for host
// arrays that are filled right after they are sized (a dense J of 8192^2
// doubles is 512 MB); blocks of 1 MiB and more come from the host cache.
template <typename T>
struct NoInitAlloc : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <typename U>
  NoInitAlloc(const NoInitAlloc<U> &) {}
  T *allocate(size_t count) {
    const size_t bytes = count * sizeof(T);
    if (bytes < kHostCacheMin) return std::allocator<T>::allocate(count);
    void *q = hostcache_get(bytes);
    if (!q) throw std::bad_alloc();
    return static_cast<T *>(q);
  }
  void deallocate(T *q, size_t count) {
    const size_t bytes = count * sizeof(T);
    if (bytes < kHostCacheMin) std::allocator<T>::deallocate(q, count);
    else hostcache_put(q, bytes);
  }
  template <typename U, typename... A>
  void construct(U *q, A &&...a) {
    if constexpr (sizeof...(A) == 0) ::new (static_cast<void *>(q)) U;
    else ::new (static_cast<void *>(q)) U(std::forward<A>(a)...);
  }
};
template <typename T>
using HostVec = std::vector<T, NoInitAlloc<T>>;

// Process-wide cache of released device blocks (api.cu).  A handle created
// after another of the same shape takes its buffers from here instead of from
// cudaMalloc, and a destroyed handle's buffers come back here instead of going
// to cudaFree.  Blocks are kept per device and size class (powers of two up to
// 1 MiB, then multiples of 2 MiB) up to a cap per device; a cudaMalloc that
// fails for lack of memory empties the cache of that device and is tried once
// more.  devcache_put must only see blocks that no queued or running work can
// still use.  sbqa_release_cached_memory() empties the cache.
cudaError_t devcache_get(void **p, size_t bytes, size_t *got);
void devcache_put(void *p, size_t bytes);
bool devcache_trim();  // cudaFree of every cached block; false if one failed

template <typename T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;      // elements the block holds (at least the count asked for)
  size_t bytes = 0;  // its size class
  cudaError_t alloc(size_t count) {
    if (count <= n && p) return cudaSuccess;
    release();
    if (count == 0) return cudaSuccess;
    void *q = nullptr;
    size_t got = 0;
    const cudaError_t e = devcache_get(&q, count * sizeof(T), &got);
    if (e != cudaSuccess) return e;
    p = static_cast<T *>(q);
    n = got / sizeof(T);
    bytes = got;
    return cudaSuccess;
  }
  // idle: the caller has synchronized the device, so no work still uses the
  // block; otherwise this waits for the device first, as cudaFree would.
  void release(bool idle = false) {
    if (p) {
      if (!idle) cudaDeviceSynchronize();
      devcache_put(p, bytes);
    }
    p = nullptr;
    n = 0;
    bytes = 0;
  }
};

}  // namespace sbqa

using sbqa::BestView;
using sbqa::CsrView;
using sbqa::DenseView;
using sbqa::EnergyView;
using sbqa::StateView;
using sbqa::StepTables;
using sbqa::VAL_BF16;
using sbqa::VAL_F32;
using sbqa::VAL_PM1;

struct sbqa_problem {
  int device = 0;
  int32_t n = 0;
  bool dense = false;
  int64_t nnz = 0;
  bool is_integer = false, is_pm1 = false, j_integer = false;
  int32_t max_abs_j = -1;
  int32_t max_degree = 0;
  double c0_auto = 0.5;
  bool h_zero = true;

  // host copies (CSR for sparse, row-major for dense)
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col;
  sbqa::HostVec<double> val;  // CSR values or dense N*N (empty when val_i8 holds the dense copy)
  sbqa::HostVec<int8_t> val_i8;  // dense integer J with |J_ij| <= 127, one byte per entry
  // dense J read by the GPU from the caller's array: the library's copy is on
  // the device (d_jcopy_i8 for integer |J_ij| <= 127, else the FP64 values in
  // d_e_f64) and the host copies above stay empty
  bool j_on_device = false;
  sbqa::DevBuf<int8_t> d_jcopy_i8;
  size_t jcount() const {
    if (j_on_device) return size_t(n) * size_t(n);
    return val_i8.empty() ? val.size() : val_i8.size();
  }
  double jv(size_t e) const { return val_i8.empty() ? val[e] : double(val_i8[e]); }
  std::vector<double> h;

  // device: product operands
  sbqa::DevBuf<int32_t> d_row_ptr, d_col;
  sbqa::DevBuf<int32_t> d_col_pm1, d_npos;  // +-1 rows with the +1 entries first
  sbqa::DevBuf<float> d_val_f32;
  sbqa::DevBuf<__nv_bfloat16> d_val_bf16;
  sbqa::DevBuf<float> d_dense_f32;  // dense J for the CUDA-core path
  int dense_prec = -1;        // precision the dense FP32 copy was built for
  // dense J on the tensor cores, padded to Kp: e4m3 (integer |J| <= 16) or
  // bfloat16 copies (operand form tc_op: sbqa::kTcOp*)
  bool use_tc = false;
  int tc_op = 0;
  int j_tc_op = -1;  // operand form the device copy d_J8 holds (-1: none)
  int Kp = 0;
  sbqa::DevBuf<uint8_t> d_J8, d_FT;
  void *tc_plan = nullptr;
  const void *tc_plan_ft = nullptr;  // FT buffer the plan was made for
  const void *tc_plan_x = nullptr;   // state buffer the plan was made for
  int tc_plan_cp = 0;
  sbqa::DevBuf<int> d_err;
  sbqa::DevBuf<float> d_h;
  // device: readout operands
  sbqa::DevBuf<int32_t> d_e_i32;
  sbqa::DevBuf<double> d_e_f64;
  sbqa::DevBuf<int64_t> d_h_i64;
  sbqa::DevBuf<double> d_h_f64;

  // schedule
  bool have_params = false;
  uint64_t params_version = 0;  // bumped by every sbqa_set_schedule
  // the schedule tables on the device were built for this (S, P, R, schedule, buffers)
  struct TablesKey {
    int S = -1, P = -1, R = -1;
    uint64_t version = 0;
    const void *ka = nullptr, *dl = nullptr, *kj = nullptr;
    bool operator==(const TablesKey &o) const {
      return S == o.S && P == o.P && R == o.R && version == o.version && ka == o.ka && dl == o.dl && kj == o.kj;
    }
  } tables_key;
  sbqa_params prm{};
  std::vector<double> beta, alpha;

  // run state
  int S = 0, P = 0, R = 0, C = 0, Cp = 0;
  int Ps = 0;  // columns per run: run_width(P); C = R * Ps
  int step_done = 0;
  bool small_path = false;  // the last sbqa_run used the one-launch small solver
  bool begun = false, finished = false;
  cudaStream_t stream = nullptr;
  int kind = VAL_F32;  // sparse value kind in use
  int csr_variant = -1;  // CSR step kernel variant chosen by the autotuner (-1 = not yet)
  float variant_ms[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  bool use_persistent = false;  // autotuner: one cooperative launch for all steps
  float persistent_ms = 0.f;    // its timing per step
  int persist_blocks = 0;
  sbqa::DevBuf<unsigned> d_bar;  // grid barrier counter of the persistent kernel
  int csr_variant_cp = -1, csr_variant_kind = -1, csr_variant_select = -1;
  // dense tcgen05: per-step kernel or the persistent solver (autotuned per Cp and kernel_select)
  bool use_tc_persistent = false;
  float tc_step_ms = 0.f, tc_persistent_ms = 0.f;
  int tc_persist_blocks = 0;
  int tc_split_blocks = -1;      // co-resident CTAs in 2-CTA clusters (-1: not queried yet)
  bool tc_split_failed = false;  // the cluster launch was refused: plain persistent solver
  bool use_tc_split = false;     // the persistent dense solver runs split-K (autotuner's or caller's choice)
  int tc_pair_blocks = -1;       // co-resident CTAs of the paired solver in 2-CTA clusters (-1: not queried yet)
  bool tc_pair_failed = false;   // its cluster launch was refused or misshaped: not used again on this handle
  bool use_tc_pair = false;      // the persistent dense solver runs on CTA pairs sharing M=256 MMAs
  int tc_select_cp = -1, tc_select = -1, tc_select_p = -1;
  sbqa::DevBuf<uint32_t> d_tc_flags;  // per-tile step counters of the persistent solver
  // the persistent solver in packed e2m1 (integer |J_ij| <= 4, J rows resident in shared memory)
  sbqa::DevBuf<uint8_t> d_J4, d_FT4;
  void *tc4_plan = nullptr;
  const void *tc4_plan_ft = nullptr, *tc4_plan_j = nullptr;
  int tc4_plan_cp = 0;
  int tc_f4_blocks = -1;  // co-resident CTAs of the e2m1 solver (-1: not queried yet)
  bool use_tc_f4 = false;
  int tc_f4_pair_blocks = -1;     // co-resident CTAs of its paired form in 2-CTA clusters
  bool tc_f4_pair_failed = false;  // the paired form's cluster launch was refused or misshaped
  bool use_tc_f4_pair = false;
  sbqa::DevBuf<float> d_x, d_y;
  sbqa::DevBuf<uint8_t> d_F0, d_F1;
  // ELL slots of rows with degree <= 8 (built for value kind ell_kind)
  sbqa::DevBuf<int32_t> d_ell_col, d_ell_meta;
  sbqa::DevBuf<float> d_ell_val;
  int ell_kind = -1;
  sbqa::DevBuf<float> d_Fx0, d_Fx1;  // f(x) = x buffers of the ballistic form
  sbqa::DevBuf<int8_t> d_Sg;
  sbqa::DevBuf<float> d_ka, d_dl, d_kj;
  sbqa::DevBuf<int64_t> d_ei, d_part_i, d_best_ei;
  sbqa::DevBuf<double> d_ef, d_part_f, d_best_e;
  sbqa::DevBuf<int32_t> d_best_k, d_best_step, d_have;
  sbqa::DevBuf<int8_t> d_best_spins;
  StepTables tables{};

  // cached graph of the step loop + readouts of a full run
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;
  struct Key {
    int S = -1, P = -1, R = -1, eval = -1, kind = -1, dense = -1, tc = -1, variant = -1, fvar = -1;
    float kc = 0.f, kx = 0.f;  // step constants are kernel arguments in the graph
    const void *x = nullptr, *kj = nullptr;
    bool operator==(const Key &o) const {
      return S == o.S && P == o.P && R == o.R && eval == o.eval && kind == o.kind &&
             dense == o.dense && tc == o.tc && variant == o.variant && fvar == o.fvar && x == o.x && kj == o.kj &&
             std::memcmp(&kc, &o.kc, sizeof(float)) == 0 && std::memcmp(&kx, &o.kx, sizeof(float)) == 0;
    }
  } graph_key;

  ~sbqa_problem();  // waits for the device, releases every buffer (api.cu)

  bool ballistic() const { return prm.variant == SBQA_VARIANT_BALLISTIC; }

  bool tc_persistent_ok() const {
    return use_tc && tc_plan && sbqa::tc_persistent_eligible(Kp, Cp, tc_persist_blocks);
  }

  // the instance qualifies for the split-K persistent solver on 2-CTA clusters
  bool tc_split_possible() const {
    return tc_persistent_ok() && tc_op == sbqa::kTcOpF8 && Ps <= 32 && P == Ps && prm.kernel_select != 12 &&
           prm.kernel_select != 13 &&
           !tc_split_failed &&
           sbqa::tc_split_eligible(Kp, Cp, tc_split_blocks);
  }
  bool tc_split_ok() const { return use_tc_split && tc_split_possible(); }

  // the instance qualifies for the paired persistent solver (autotuned, or kernel_select 13)
  bool tc_pair_possible() const {
    return tc_persistent_ok() && tc_op == sbqa::kTcOpF8 && Ps <= 32 && P == Ps &&
           (prm.kernel_select == 0 || prm.kernel_select == 13) &&
           !tc_pair_failed &&
           sbqa::tc_pair_eligible(Kp, Cp, tc_pair_blocks);
  }
  bool tc_pair_ok() const { return use_tc_pair && tc_pair_possible(); }

  // the instance qualifies for the persistent solver with e2m1 operands (autotuned, or kernel_select 14, 15)
  bool tc_f4_possible() const {
    return tc_persistent_ok() && tc_op == sbqa::kTcOpF8 && j_integer && max_abs_j <= 4 &&
           (prm.kernel_select == 0 || prm.kernel_select == 14 || prm.kernel_select == 15) &&
           sbqa::tc_f4_eligible(Kp, Cp, tc_f4_blocks);
  }
  bool tc_f4_ok() const { return use_tc_f4 && tc4_plan && tc_f4_possible(); }
  // ... and for its paired form (not with kernel_select 15)
  bool tc_f4_pair_possible() const {
    return tc_f4_possible() && prm.kernel_select != 15 && !tc_f4_pair_failed &&
           sbqa::tc_f4_pair_eligible(Kp, Cp, tc_f4_pair_blocks);
  }
  bool tc_f4_pair_ok() const { return use_tc_f4_pair && tc_f4_ok() && tc_f4_pair_possible(); }

  int persist_mode() const {
    return sbqa::persistent_mode(n, Cp, max_degree, kind, persist_blocks, prm.kernel_select == 11,
                                 ell_kind == kind && d_ell_col.p != nullptr);
  }

  bool persistent_ok() const {
    if (dense) return false;
    if (ballistic()) return sbqa::persistent_bsb_ok(n, Cp, max_degree, kind, persist_blocks);
    return persist_mode() != 0;
  }

  StateView state() const {
    StateView s;
    s.N = n; s.C = C; s.Cp = Cp; s.P = Ps; s.R = R; s.Pr = P;
    s.x = d_x.p; s.y = d_y.p;
    s.F[0] = d_F0.p; s.F[1] = d_F1.p;
    s.Fx[0] = d_Fx0.p; s.Fx[1] = d_Fx1.p;
    s.Sg = d_Sg.p;
    return s;
  }
  // CSR in the caller's entry order (the readout pairs it with the value arrays)
  CsrView csr_readout() const {
    CsrView v = csr();
    v.col = d_col.p;
    return v;
  }
  CsrView csr() const {
    CsrView v;
    v.row_ptr = d_row_ptr.p; v.h = d_h.p; v.kind = kind; v.npos = d_npos.p;
    v.col = kind == VAL_PM1 ? d_col_pm1.p : d_col.p;
    v.val = kind == VAL_F32 ? static_cast<const void *>(d_val_f32.p)
                            : static_cast<const void *>(d_val_bf16.p);
    const bool ell = ell_kind == kind && d_ell_col.p;
    v.ell_col = ell ? d_ell_col.p : nullptr;
    v.ell_val = ell ? d_ell_val.p : nullptr;
    v.ell_meta = ell ? d_ell_meta.p : nullptr;
    return v;
  }
  EnergyView energy() const {
    EnergyView e;
    e.is_integer = is_integer ? 1 : 0;
    e.val_i32 = d_e_i32.p; e.val_f64 = d_e_f64.p; e.h_i64 = d_h_i64.p; e.h_f64 = d_h_f64.p;
    return e;
  }
  BestView best() const {
    BestView b;
    b.e_int = d_ei.p; b.e_f64 = d_ef.p; b.part_int = d_part_i.p; b.part_f64 = d_part_f.p;
    b.nblk = sbqa::energy_row_blocks(n);
    b.best_e_int = d_best_ei.p; b.best_e = d_best_e.p; b.best_k = d_best_k.p;
    b.best_step = d_best_step.p; b.best_spins = d_best_spins.p; b.have_best = d_have.p;
    return b;
  }
};

namespace sbqa {

// Host helpers implemented in api.cu, used by the engine.
int problem_check_run(sbqa_problem *p, int32_t steps, int32_t P, int32_t R);
// Device copies of J in the form the current precision needs.
int problem_prepare_values(sbqa_problem *p);
// FP64 schedule of Sec. II A rounded to the FP32 step coefficients, written to
// ka[S], dl[S+1], kj[S][R] (device) on st; *t receives the table view.
int problem_build_tables(const sbqa_problem *p, int S, int P, int R, float *ka, float *dl, float *kj,
                         StepTables *t, cudaStream_t st);
CsrView problem_csr_view(const sbqa_problem *p);
CsrView problem_csr_readout_view(const sbqa_problem *p);
EnergyView problem_energy_view(const sbqa_problem *p);
DenseView problem_dense_view(const sbqa_problem *p);

}  // namespace sbqa
