// engine.cu -- continuous-batching engine for many SBQA solves on one GPU.
//
// Requests (a problem handle with its schedule + steps, P, R, seed) queue in
// arrival order.  At every chunk boundary the engine admits queued requests
// while a slot and room in its device arena are free (strict FIFO), builds
// their schedule tables and initial state, and then advances every active
// request by up to `chunk` steps: all CSR requests together in one
// cooperative launch for the whole chunk (k_solve_batched over a work list
// of 8-row x 128- or 256-column items, a bounded grid barrier between steps;
// each slot keeps its own step index on the device, so the launch is
// captured once in a CUDA graph and replayed every chunk), dense requests
// with the persistent tensor-core solver (one launch per chunk) when their
// tiles fill a good part of the device, else per-step kernels on their
// slot's stream.
// A request whose last step falls inside the chunk is read out (energies of
// all replicas, best per run), its result copied to the host and its slot
// and arena space released.  Each element is computed exactly as by
// sbqa_run, so a request's result does not depend on what else is running.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <deque>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sbqa.h"
#include "grid_sync.cuh"
#include "internal.h"
#include "problem.h"

using namespace sbqa;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over one device allocation, free blocks coalesced.
struct Arena {
  uint8_t *base = nullptr;
  size_t bytes = 0;
  std::map<size_t, size_t> free_blocks;  // offset -> size
  size_t used = 0;

  bool alloc(size_t n, size_t *off) {
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, o = it->first;
        free_blocks.erase(it);
        if (rest) free_blocks[o + n] = rest;
        used += n;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    used -= n;
    auto it = free_blocks.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_blocks.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_blocks.erase(nx);
    }
    if (it != free_blocks.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_blocks.erase(it);
      }
    }
  }
};

// FAILED: a bounded device wait of the request gave up; it left its slot and
// arena space like a finished request and has no result.
enum ReqState { QUEUED = 0, ACTIVE = 1, DONE = 2, FAILED = 3 };

struct Request {
  int id = -1;
  sbqa_problem *prob = nullptr;
  int S = 0, P = 0, R = 0, C = 0, Cp = 0, nblk = 0;
  uint64_t seed = 0;
  int state = QUEUED;
  int slot = -1;
  int n0 = 0;  // steps done
  size_t off = 0, bytes = 0;
  // carved device buffers
  float *x, *y, *ka, *dl, *kj;
  uint8_t *F0, *F1, *FT;
  uint8_t *FT4 = nullptr;  // packed e2m1 f buffers of the e2m1 dense solver (f4 requests)
  bool f4 = false;         // a dense request on the e2m1 solver (integer |J| <= 4, its tiles co-resident)
  void *tc4_plan = nullptr;
  int8_t *Sg, *best_spins;
  int64_t *ei, *part_i, *best_ei;
  double *ef, *part_f, *best_e;
  int32_t *best_k, *best_step, *have;
  int *err;
  uint32_t *tc_flags;  // per-tile step counters of the persistent dense solver (dense tensor-core requests)
  bool on_side = false;  // this chunk runs on the slot's side stream
  StepTables tables{};
  void *tc_plan = nullptr;
  // results (host)
  std::vector<int8_t> spins;
  std::vector<double> energy;
  std::vector<int64_t> energy_int;
  std::vector<int32_t> replica;

  StateView state_view() const {
    StateView s;
    s.N = prob->n; s.C = C; s.Cp = Cp; s.P = run_width(P); s.R = R; s.Pr = P;
    s.x = x; s.y = y; s.F[0] = F0; s.F[1] = F1; s.Sg = Sg;
    s.Fx[0] = s.Fx[1] = nullptr;
    return s;
  }
  BestView best_view() const {
    BestView b;
    b.e_int = ei; b.e_f64 = ef; b.part_int = part_i; b.part_f64 = part_f; b.nblk = nblk;
    b.best_e_int = best_ei; b.best_e = best_e; b.best_k = best_k; b.best_step = best_step;
    b.best_spins = best_spins; b.have_best = have;
    return b;
  }
};

}  // namespace

struct sbqa_engine {
  int device = 0;
  Arena arena;
  int max_slots = 0, chunk = 0;
  std::vector<Request> reqs;
  std::deque<int> queue;
  std::vector<int> slot_req;  // slot -> request id, -1 free
  SlotDesc *d_slots = nullptr;
  WorkItem *d_items = nullptr;
  int *d_n_items = nullptr;  // [units, items] of the work list (device)
  size_t items_cap = 0;
  int sms = 0;
  int64_t steps_done_total = 0;  // replica-spin updates issued, for statistics
  int64_t kernels_launched = 0;  // kernels this engine has launched, for statistics
  int64_t batched_updates = 0;   // updates of CSR requests advanced by the batched kernel
  double batched_ms = 0.0;       // device time of the batched launches
  cudaEvent_t batched_t0 = nullptr, batched_t1 = nullptr;
  // the CSR requests' chunk: one cooperative launch (k_solve_batched), captured
  // once in a CUDA graph and replayed every chunk while its grid size and
  // work-list buffer stay the same (the slots' step indices live on the device)
  unsigned *d_bar = nullptr;  // grid barrier counters
  int *d_err = nullptr;       // error flag of the batched launch
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t csr_graph = nullptr;
  int csr_graph_grid = 0;
  const void *csr_graph_items = nullptr;
  bool csr_graph_refused = false;  // capture of the cooperative launch was refused: launch it directly
  int tc_blocks = -1;              // co-resident CTAs of the persistent dense solver
  int64_t graph_launches = 0;
  // small dense tensor-core requests: their chunks in one cooperative launch
  // per group of equal operand form and run width (solve_dense_tc_batched.cu)
  TcBatch *tcb = nullptr;
  Tc4Batch *tc4b = nullptr;  // the same for the requests on the e2m1 solver
  int f4_blocks = -1;        // co-resident CTAs of the e2m1 solvers (-1: not queried yet)
  bool dense_batching = true;
  int64_t dense_batched_launches = 0, dense_batched_chunks = 0;
  int64_t dense_e2m1_requests = 0;  // requests admitted on the e2m1 solver
  // dense requests run their chunk on a stream of their slot (created on first
  // use), so small dense problems share the GPU instead of queueing
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> side_done;
  cudaEvent_t chunk_start = nullptr;

  ~sbqa_engine() {
    cudaDeviceSynchronize();
    if (csr_graph) cudaGraphExecDestroy(csr_graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (d_bar) cudaFree(d_bar);
    if (d_err) cudaFree(d_err);
    for (cudaStream_t x : side)
      if (x) cudaStreamDestroy(x);
    for (cudaEvent_t x : side_done)
      if (x) cudaEventDestroy(x);
    if (chunk_start) cudaEventDestroy(chunk_start);
    tc_batch_destroy(tcb);
    tc4_batch_destroy(tc4b);
    if (batched_t0) cudaEventDestroy(batched_t0);
    if (batched_t1) cudaEventDestroy(batched_t1);
    for (auto &r : reqs) {
      if (r.tc_plan) tc_plan_free(r.tc_plan);
      if (r.tc4_plan) tc4_plan_free(r.tc4_plan);
    }
    if (arena.base) cudaFree(arena.base);
    if (d_slots) cudaFree(d_slots);
    if (d_items) cudaFree(d_items);
    if (d_n_items) cudaFree(d_n_items);
  }
};

namespace {

#define ENG_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return set_error(e_ == cudaErrorMemoryAllocation ? SBQA_ERR_OOM : SBQA_ERR_CUDA,          \
                       std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

size_t request_bytes(const sbqa_problem *p, int S, int P, int R, bool tc, int Kp, bool f4) {
  const int C = R * run_width(P), Cp = (C + kColsPerWarp - 1) / kColsPerWarp * kColsPerWarp;
  const size_t N = size_t(p->n), NC = N * Cp;
  const size_t nblk = size_t(energy_row_blocks(p->n));
  size_t b = 0;
  b += align_up(NC * 4) * 2;               // x, y
  b += align_up(NC) * 3;                   // F0, F1, Sg
  b += align_up(size_t(std::max(S, 1)) * 4) + align_up(size_t(S + 1) * 4) + align_up(size_t(std::max(S, 1)) * R * 4);
  b += align_up(size_t(Cp) * 8) * 2;       // energies
  b += align_up(nblk * Cp * 8);            // partial sums
  b += align_up(size_t(R) * 8) * 2 + align_up(size_t(R) * 4) * 3 + align_up(size_t(R) * N);
  b += align_up(4);                        // error flag
  if (tc) b += align_up(tc_ft_bytes(Kp, Cp, p->tc_op)) + align_up(tc_persistent_flag_count(Kp, Cp) * 4);
  if (f4) b += align_up(size_t(2) * Cp * tc_f4_row_bytes(Kp));
  return b;
}

void carve(Request &r, uint8_t *base, bool tc, int Kp) {
  const size_t N = size_t(r.prob->n), NC = N * r.Cp;
  size_t o = 0;
  auto take = [&](size_t n) {
    uint8_t *p = base + o;
    o += align_up(n);
    return p;
  };
  r.x = reinterpret_cast<float *>(take(NC * 4));
  r.y = reinterpret_cast<float *>(take(NC * 4));
  r.F0 = take(NC);
  r.F1 = take(NC);
  r.Sg = reinterpret_cast<int8_t *>(take(NC));
  r.ka = reinterpret_cast<float *>(take(size_t(std::max(r.S, 1)) * 4));
  r.dl = reinterpret_cast<float *>(take(size_t(r.S + 1) * 4));
  r.kj = reinterpret_cast<float *>(take(size_t(std::max(r.S, 1)) * r.R * 4));
  r.ei = reinterpret_cast<int64_t *>(take(size_t(r.Cp) * 8));
  r.ef = reinterpret_cast<double *>(take(size_t(r.Cp) * 8));
  uint8_t *part = take(size_t(r.nblk) * r.Cp * 8);
  r.part_i = reinterpret_cast<int64_t *>(part);
  r.part_f = reinterpret_cast<double *>(part);
  r.best_ei = reinterpret_cast<int64_t *>(take(size_t(r.R) * 8));
  r.best_e = reinterpret_cast<double *>(take(size_t(r.R) * 8));
  r.best_k = reinterpret_cast<int32_t *>(take(size_t(r.R) * 4));
  r.best_step = reinterpret_cast<int32_t *>(take(size_t(r.R) * 4));
  r.have = reinterpret_cast<int32_t *>(take(size_t(r.R) * 4));
  r.best_spins = reinterpret_cast<int8_t *>(take(size_t(r.R) * N));
  r.err = reinterpret_cast<int *>(take(4));
  r.FT = tc ? take(tc_ft_bytes(Kp, r.Cp, r.prob->tc_op)) : nullptr;
  r.tc_flags = tc ? reinterpret_cast<uint32_t *>(take(tc_persistent_flag_count(Kp, r.Cp) * 4)) : nullptr;
  r.FT4 = r.f4 ? take(size_t(2) * r.Cp * tc_f4_row_bytes(Kp)) : nullptr;
}

// A dense request runs on the e2m1 solver when its couplings are integers |J| <= 4 (exact in e2m1),
// the e4m3 form is in use, its tiles fit the device at once and the problem's kernel_select allows
// it (0, 14 or 15); decided at submission, so that the arena holds its packed f buffers.
bool request_f4(sbqa_engine *e, const sbqa_problem *p, int P, int R) {
  if (!p->dense || !p->use_tc || p->tc_op != kTcOpF8 || !p->j_integer || p->max_abs_j > 4) return false;
  const int ks = p->prm.kernel_select;
  if (ks != 0 && ks != 14 && ks != 15) return false;
  const int C = R * run_width(P), Cp = (C + kColsPerWarp - 1) / kColsPerWarp * kColsPerWarp;
  if (e->f4_blocks < 0) e->f4_blocks = tc_f4_blocks();
  return tc_f4_eligible(p->Kp, Cp, e->f4_blocks);
}

int admit(sbqa_engine *e, Request &r, int slot, cudaStream_t st) {
  sbqa_problem *p = r.prob;
  const bool tc = p->use_tc;
  r.C = r.R * run_width(r.P);  // a run's columns: P replicas, then padding up to a power of two
  r.Cp = (r.C + kColsPerWarp - 1) / kColsPerWarp * kColsPerWarp;
  r.nblk = energy_row_blocks(p->n);
  carve(r, e->arena.base + r.off, tc, p->Kp);
  int rc = problem_build_tables(p, r.S, r.P, r.R, r.ka, r.dl, r.kj, &r.tables, st);
  if (rc != SBQA_OK) return rc;
  if (tc) {
    if (!tc_plan_make(&r.tc_plan, p->d_J8.p, r.FT, p->Kp, r.Cp, r.x, r.y, p->n, p->tc_op))
      return set_error(SBQA_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    ENG_CUDA(tc_set_attributes());
  }
  if (r.f4) {
    // the problem's packed J (once per problem), this request's plan and zeroed f buffers (the
    // bytes past Kp that no tile writes stay zero)
    const int Kh = tc_f4_row_bytes(p->Kp);
    if (!p->d_J4.p) {
      ENG_CUDA(p->d_J4.alloc(size_t(p->Kp) * Kh));
      ENG_CUDA(launch_j4_from_j8(p->d_J8.p, p->Kp, p->d_J4.p, st));
      ++e->kernels_launched;
    }
    if (!tc4_plan_make(&r.tc4_plan, p->d_J4.p, r.FT4, p->Kp, r.Cp))
      return set_error(SBQA_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    ENG_CUDA(cudaMemsetAsync(r.FT4, 0, size_t(2) * r.Cp * Kh, st));
  }
  const StateView s = r.state_view();
  ENG_CUDA(cudaMemsetAsync(r.err, 0, sizeof(int), st));
  ENG_CUDA(launch_init(s, r.seed, float(p->prm.init_amp), 0.0f, st));
  if (tc) ENG_CUDA(launch_f_to_ft(s, 0, r.FT, p->Kp, 0, p->tc_op, st));
  if (r.f4) {
    ENG_CUDA(launch_f_to_ft4(s, 0, r.FT4, p->Kp, 0, st));
    ++e->dense_e2m1_requests;
  }
  ENG_CUDA(launch_reset_best(s, r.best_view(), st));
  e->kernels_launched += (tc ? 3 : 2) + (r.f4 ? 1 : 0);
  r.slot = slot;
  r.n0 = 0;
  r.state = ACTIVE;
  e->slot_req[slot] = r.id;
  return SBQA_OK;
}

SlotDesc slot_desc(const Request &r) {
  const sbqa_problem *p = r.prob;
  const CsrView v = problem_csr_view(p);
  SlotDesc d{};
  d.row_ptr = v.row_ptr; d.col = v.col; d.npos = v.npos; d.val = v.val; d.h = v.h; d.kind = v.kind;
  d.ell_col = v.ell_col; d.ell_meta = v.ell_meta; d.ell_val = v.ell_val;
  d.N = p->n; d.C = r.C; d.Cp = r.Cp; d.P = run_width(r.P); d.Pr = r.P; d.R = r.R; d.S = r.S;
  d.x = r.x; d.y = r.y; d.F0 = r.F0; d.F1 = r.F1;
  d.ka = r.ka; d.dl = r.dl; d.kj = r.kj; d.kc = r.tables.kc; d.kx = r.tables.kx;
  d.n0 = r.n0;
  d.W = d.ell_col ? 8 : 4;
  d.wide = d.ell_col && r.Cp % 256 == 0 ? 1 : 0;
  return d;
}

int readout(sbqa_engine *e, Request &r, cudaStream_t st) {
  (void)e;
  sbqa_problem *p = r.prob;
  const StateView s = r.state_view();
  const EnergyView ev = problem_energy_view(p);
  // the tensor-core readout needs integer energies (J and h); a non-integer h
  // takes the FP64 CUDA-core readout (the product still runs on the tensor cores)
  const bool tc = p->dense && r.tc_plan && p->is_integer && p->tc_op == kTcOpF8;
  cudaError_t err = tc ? launch_energy_dense_tc(r.tc_plan, s, p->Kp, r.FT, (r.S - 1) & 1, r.err, ev, r.best_view(), st)
                       : p->dense ? launch_energy_dense(s, ev, r.best_view(), st)
                                  : launch_energy_csr(s, problem_csr_readout_view(p), ev, r.best_view(), st);
  if (err == cudaSuccess) err = launch_best(s, ev, r.best_view(), r.S - 1, st);
  e->kernels_launched += tc ? 5 : 4;  // signs, (sign codes,) energies, their final sums, best
  if (err != cudaSuccess) return set_error(SBQA_ERR_CUDA, std::string("engine readout: ") + cudaGetErrorString(err));
  r.spins.resize(size_t(r.R) * p->n);
  r.energy.resize(r.R);
  r.energy_int.assign(r.R, 0);
  r.replica.resize(r.R);
  ENG_CUDA(cudaMemcpyAsync(r.spins.data(), r.best_spins, r.spins.size(), cudaMemcpyDeviceToHost, st));
  ENG_CUDA(cudaMemcpyAsync(r.energy.data(), r.best_e, r.R * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (p->is_integer)
    ENG_CUDA(cudaMemcpyAsync(r.energy_int.data(), r.best_ei, r.R * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  ENG_CUDA(cudaMemcpyAsync(r.replica.data(), r.best_k, r.R * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  return SBQA_OK;
}

// Dense tensor-core requests with at least this many 128 x 128 tiles (most
// of the device's 152 SMs) run a chunk on the persistent solver; smaller
// ones take per-step kernels on their slot's stream, where they overlap with
// other work (a persistent solver of a few dozen tiles would run alone on
// the engine stream, which serialises the cooperative launches).
constexpr int kPersistMinTiles = 112;

// The captured graph of the CSR chunk launch for `grid` blocks (recaptured
// when the grid size or the work-list buffer changes).  A capture that the
// runtime refuses leaves e->csr_graph null, and the chunk is launched directly.
int csr_chunk_graph(sbqa_engine *e, int grid) {
  if (e->csr_graph_refused) return SBQA_OK;
  if (e->csr_graph && e->csr_graph_grid == grid && e->csr_graph_items == e->d_items) return SBQA_OK;
  if (e->csr_graph) {
    cudaGraphExecDestroy(e->csr_graph);
    e->csr_graph = nullptr;
  }
  if (!e->cap_stream) ENG_CUDA(cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking));
  ENG_CUDA(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = launch_solve_batched(e->d_slots, e->max_slots, e->d_items, e->d_n_items, grid, 0, e->chunk,
                                         e->d_bar, e->d_err, e->cap_stream);
  cudaGraph_t graph = nullptr;
  const cudaError_t err2 = cudaStreamEndCapture(e->cap_stream, &graph);
  cudaGraphExec_t exec = nullptr;
  if (err == cudaSuccess && err2 == cudaSuccess) err = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (err != cudaSuccess || err2 != cudaSuccess || !exec) {
    cudaGetLastError();  // the refusal is not an error of the engine: launch directly from now on
    e->csr_graph_refused = true;
    return SBQA_OK;
  }
  e->csr_graph = exec;
  e->csr_graph_grid = grid;
  e->csr_graph_items = e->d_items;
  return SBQA_OK;
}

}  // namespace

extern "C" {

int sbqa_engine_set_dense_batching(sbqa_engine *e, int32_t on) {
  if (!e || (on != 0 && on != 1)) return set_error(SBQA_ERR_INVALID_ARG, "need an engine and on = 0 or 1");
  e->dense_batching = on != 0;
  return SBQA_OK;
}

int sbqa_engine_create(int64_t arena_bytes, int32_t max_slots, int32_t chunk_steps, sbqa_engine **out) {
  if (!out) return set_error(SBQA_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (arena_bytes < (1 << 20) || max_slots < 1 || max_slots > 4096 || chunk_steps < 1)
    return set_error(SBQA_ERR_INVALID_ARG, "need arena_bytes >= 1 MiB, 1 <= max_slots <= 4096, chunk_steps >= 1");
  auto *e = new (std::nothrow) sbqa_engine();
  if (!e) return set_error(SBQA_ERR_OOM, "host allocation");
  cudaGetDevice(&e->device);
  e->max_slots = max_slots;
  e->chunk = chunk_steps;
  e->slot_req.assign(max_slots, -1);
  auto fail_free = [&](int code, const std::string &m) {
    delete e;
    return set_error(code, m);
  };
  if (cudaMalloc(&e->arena.base, size_t(arena_bytes)) != cudaSuccess) return fail_free(SBQA_ERR_OOM, "engine arena");
  e->arena.bytes = size_t(arena_bytes);
  e->arena.free_blocks[0] = size_t(arena_bytes);
  if (cudaMalloc(&e->d_slots, sizeof(SlotDesc) * max_slots) != cudaSuccess ||
      cudaMalloc(&e->d_n_items, 2 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&e->d_bar, sizeof(unsigned) * grid_barrier_words()) != cudaSuccess ||
      cudaMalloc(&e->d_err, sizeof(int)) != cudaSuccess || cudaMemset(e->d_err, 0, sizeof(int)) != cudaSuccess)
    return fail_free(SBQA_ERR_OOM, "engine tables");
  cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, e->device);
  *out = e;
  return SBQA_OK;
}

void sbqa_engine_destroy(sbqa_engine *e) { delete e; }

int sbqa_engine_submit(sbqa_engine *e, sbqa_problem *p, int32_t steps, int32_t P, int32_t R, uint64_t seed,
                       int32_t *id) {
  if (!e || !p || !id) return set_error(SBQA_ERR_INVALID_ARG, "null argument");
  int rc = problem_check_run(p, steps, P, R);
  if (rc != SBQA_OK) return rc;
  if (steps < 1) return set_error(SBQA_ERR_INVALID_ARG, "engine requests need steps >= 1");
  if (p->prm.variant != SBQA_VARIANT_THRESHOLD)
    return set_error(SBQA_ERR_UNSUPPORTED, "the engine serves the thresholded f (Eq. 8) only");
  if ((rc = problem_prepare_values(p)) != SBQA_OK) return rc;
  Request r;
  r.id = int(e->reqs.size());
  r.prob = p;
  r.S = steps; r.P = P; r.R = R; r.seed = seed;
  r.f4 = request_f4(e, p, P, R);
  r.bytes = request_bytes(p, steps, P, R, p->use_tc, p->Kp, r.f4);
  if (r.bytes > e->arena.bytes) return set_error(SBQA_ERR_OOM, "request larger than the engine arena");
  e->reqs.push_back(std::move(r));
  e->queue.push_back(e->reqs.back().id);
  *id = e->reqs.back().id;
  return SBQA_OK;
}

// The chunks of the small dense tensor-core requests: grouped by operand form,
// run width and ring form (one kernel instance each), every group in as few
// cooperative launches as the co-resident CTAs allow, all on st one after
// another (no two cooperative grids ever wait for each other's blocks).
static int dense_batches(sbqa_engine *e, std::vector<int> &ids, cudaStream_t st) {
  if (!e->tcb) ENG_CUDA(tc_batch_create(&e->tcb, std::min(e->max_slots, e->tc_blocks), e->tc_blocks));
  auto key = [&](int id) {
    const Request &r = e->reqs[id];
    return std::make_tuple(r.prob->tc_op, run_width(r.P), r.P != run_width(r.P));
  };
  std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return key(a) < key(b); });
  tc_batch_clear(e->tcb);
  auto flush = [&]() -> int {
    if (tc_batch_size(e->tcb) == 0) return SBQA_OK;
    const cudaError_t err = tc_batch_launch(e->tcb, st);
    if (err != cudaSuccess) return set_error(SBQA_ERR_CUDA, std::string("engine dense batch: ") + cudaGetErrorString(err));
    ++e->kernels_launched;
    ++e->dense_batched_launches;
    e->dense_batched_chunks += tc_batch_size(e->tcb);
    tc_batch_clear(e->tcb);
    return SBQA_OK;
  };
  int rc;
  // test hook: SBQA_TEST_ENGINE_HOLD_DENSE=id makes that request's tile (0, 0) leave its step
  // counter unpublished after the chunk's first step, so that its other tiles' bounded waits
  // run out on the device (not for production use)
  const char *hold_hook = std::getenv("SBQA_TEST_ENGINE_HOLD_DENSE");
  const int hold_id = hold_hook ? std::atoi(hold_hook) : -1;
  for (int id : ids) {
    Request &r = e->reqs[id];
    const sbqa_problem *p = r.prob;
    const StateView sv = r.state_view();
    if (!tc_batch_fits(e->tcb, r.tc_plan, sv, p->Kp) && (rc = flush()) != SBQA_OK) return rc;
    const int steps_now = std::min(e->chunk, r.S - r.n0);
    const cudaError_t err = tc_batch_add(e->tcb, r.tc_plan, sv, p->Kp, r.err, p->d_h.p, r.tables, r.n0,
                                         r.n0 + steps_now, id == hold_id ? r.n0 : -1);
    if (err != cudaSuccess) return set_error(SBQA_ERR_CUDA, std::string("engine dense batch: ") + cudaGetErrorString(err));
  }
  return flush();
}

// The chunks of the small requests on the e2m1 solver: grouped by run width
// and ring form, every group in as few cooperative launches as the
// co-resident CTAs allow, on st one after another.
static int dense_batches_f4(sbqa_engine *e, std::vector<int> &ids, cudaStream_t st) {
  if (!e->tc4b) ENG_CUDA(tc4_batch_create(&e->tc4b, std::min(e->max_slots, e->f4_blocks), e->f4_blocks));
  auto key = [&](int id) {
    const Request &r = e->reqs[id];
    return std::make_pair(run_width(r.P), r.P != run_width(r.P));
  };
  std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return key(a) < key(b); });
  tc4_batch_clear(e->tc4b);
  auto flush = [&]() -> int {
    if (tc4_batch_size(e->tc4b) == 0) return SBQA_OK;
    const cudaError_t err = tc4_batch_launch(e->tc4b, st);
    if (err != cudaSuccess) return set_error(SBQA_ERR_CUDA, std::string("engine dense batch: ") + cudaGetErrorString(err));
    ++e->kernels_launched;
    ++e->dense_batched_launches;
    e->dense_batched_chunks += tc4_batch_size(e->tc4b);
    tc4_batch_clear(e->tc4b);
    return SBQA_OK;
  };
  int rc;
  // test hook: as in dense_batches
  const char *hold_hook = std::getenv("SBQA_TEST_ENGINE_HOLD_DENSE");
  const int hold_id = hold_hook ? std::atoi(hold_hook) : -1;
  for (int id : ids) {
    Request &r = e->reqs[id];
    const sbqa_problem *p = r.prob;
    const StateView sv = r.state_view();
    if (!tc4_batch_fits(e->tc4b, sv, p->Kp) && (rc = flush()) != SBQA_OK) return rc;
    const int steps_now = std::min(e->chunk, r.S - r.n0);
    const cudaError_t err = tc4_batch_add(e->tc4b, r.tc4_plan, sv, p->Kp, r.err, p->d_h.p, r.tables, r.n0,
                                          r.n0 + steps_now, id == hold_id ? r.n0 : -1);
    if (err != cudaSuccess) return set_error(SBQA_ERR_CUDA, std::string("engine dense batch: ") + cudaGetErrorString(err));
  }
  return flush();
}

int sbqa_engine_step(sbqa_engine *e, void *stream, int32_t *n_done, int32_t *done_ids, int32_t cap) {
  if (!e || !n_done) return set_error(SBQA_ERR_INVALID_ARG, "null argument");
  *n_done = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc;
  // 1. admission, strict FIFO: by slot and arena room
  while (!e->queue.empty()) {
    Request &r = e->reqs[e->queue.front()];
    int slot = -1;
    for (int q = 0; q < e->max_slots; ++q)
      if (e->slot_req[q] < 0) {
        slot = q;
        break;
      }
    if (slot < 0 || !e->arena.alloc(r.bytes, &r.off)) break;
    e->queue.pop_front();
    if ((rc = admit(e, r, slot, st)) != SBQA_OK) return rc;
  }
  // 2. slot table and work list of the CSR requests
  std::vector<SlotDesc> slots(e->max_slots);
  std::vector<WorkItem> items;
  std::vector<int> dense_active, ell_slots, other_slots;
  for (int q = 0; q < e->max_slots; ++q) {
    if (e->slot_req[q] < 0) continue;
    Request &r = e->reqs[e->slot_req[q]];
    slots[q] = slot_desc(r);
    if (r.prob->dense) dense_active.push_back(r.id);
    else (slots[q].W == 8 ? ell_slots : other_slots).push_back(q);
  }
  // units of the ELL slots first, ordered by the code they run (run width,
  // coupling kind, ring form), so that a warp's contiguous share mostly runs one
  // form; then the 8-row items of the other slots
  std::stable_sort(ell_slots.begin(), ell_slots.end(), [&](int a, int b) {
    const SlotDesc &x = slots[a], &y = slots[b];
    return std::make_tuple(x.wide, x.P, x.kind != VAL_PM1, x.Pr != x.P) <
           std::make_tuple(y.wide, y.P, y.kind != VAL_PM1, y.Pr != y.P);
  });
  for (int q : ell_slots) {
    const bool wide = slots[q].wide != 0;  // one row x 256 columns, or two rows x 128
    for (int g = 0; g < slots[q].Cp / (wide ? 256 : kColsPerWarp); ++g)
      for (int r0 = 0; r0 < slots[q].N; r0 += wide ? 1 : 2) items.push_back(WorkItem{q, r0, g, 0});
  }
  int counts[2] = {int(items.size()), 0};
  for (int q : other_slots)
    for (int g = 0; g < slots[q].Cp / kColsPerWarp; ++g)
      for (int r0 = 0; r0 < slots[q].N; r0 += 8) items.push_back(WorkItem{q, r0, g, 0});
  counts[1] = int(items.size()) - counts[0];
  if (items.size() > e->items_cap) {
    if (e->d_items) cudaFree(e->d_items);
    e->d_items = nullptr;
    e->items_cap = std::max(items.size(), e->items_cap * 2);
    ENG_CUDA(cudaMalloc(&e->d_items, e->items_cap * sizeof(WorkItem)));
  }
  const int n_items = int(items.size());
  ENG_CUDA(cudaMemcpyAsync(e->d_slots, slots.data(), slots.size() * sizeof(SlotDesc), cudaMemcpyHostToDevice, st));
  if (n_items)
    ENG_CUDA(cudaMemcpyAsync(e->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, st));
  ENG_CUDA(cudaMemcpyAsync(e->d_n_items, counts, sizeof(counts), cudaMemcpyHostToDevice, st));
  // 3. the chunk: the dense requests on their slots' streams (after everything
  //    issued on `st` so far: admission, tables), one batched launch per step
  //    for all CSR requests on `st`; `st` then waits for the dense streams
  if (!dense_active.empty()) {
    if (!e->chunk_start) ENG_CUDA(cudaEventCreateWithFlags(&e->chunk_start, cudaEventDisableTiming));
    ENG_CUDA(cudaEventRecord(e->chunk_start, st));
    if (e->side.empty()) {
      e->side.assign(e->max_slots, nullptr);
      e->side_done.assign(e->max_slots, nullptr);
    }
  }
  std::vector<int> batch_ids, batch_f4_ids;
  for (int id : dense_active) {
    Request &r = e->reqs[id];
    const int steps_now = std::min(e->chunk, r.S - r.n0);
    const sbqa_problem *p = r.prob;
    if (r.f4) {  // the e2m1 solver: with the other small ones in one launch, or alone
      const int f4_tiles = (p->Kp / 128) * (r.Cp / 128);
      if (e->dense_batching && f4_tiles < kPersistMinTiles) {
        batch_f4_ids.push_back(id);
        continue;
      }
      const cudaError_t err = launch_solve_dense_tc_f4(r.tc4_plan, r.state_view(), p->Kp, r.err, p->d_h.p, r.tables,
                                                       r.n0, r.n0 + steps_now, r.tc_flags, st);
      if (err != cudaSuccess) return set_error(SBQA_ERR_CUDA, std::string("engine dense chunk: ") + cudaGetErrorString(err));
      ++e->kernels_launched;
      continue;
    }
    // a tensor-core request whose tiles fill a good part of the device runs its chunk on the
    // persistent solver (one launch); cooperative launches all go to `st`, one after another,
    // so no two of them ever wait for each other's blocks
    const int tiles = p->use_tc ? (p->Kp / 128) * (r.Cp / 128) : 0;
    if (p->use_tc && e->tc_blocks < 0) {
      ENG_CUDA(tc_set_attributes());
      ENG_CUDA(tc_batch_set_attributes());
      e->tc_blocks = std::min(tc_persistent_blocks(), tc_batch_blocks());
    }
    if (p->use_tc && tiles >= kPersistMinTiles && tc_persistent_eligible(p->Kp, r.Cp, e->tc_blocks)) {
      const cudaError_t err = launch_solve_dense_tc_persistent(r.tc_plan, r.state_view(), p->Kp, r.err, p->d_h.p,
                                                               r.tables, r.n0, r.n0 + steps_now, r.tc_flags, st);
      if (err != cudaSuccess) return set_error(SBQA_ERR_CUDA, std::string("engine dense chunk: ") + cudaGetErrorString(err));
      ++e->kernels_launched;
      continue;
    }
    if (e->dense_batching && p->use_tc && tc_persistent_eligible(p->Kp, r.Cp, e->tc_blocks)) {
      batch_ids.push_back(id);  // with the other small tensor-core requests, below
      continue;
    }
    cudaStream_t &ds = e->side[r.slot];
    cudaEvent_t &dv = e->side_done[r.slot];
    if (!ds) ENG_CUDA(cudaStreamCreateWithFlags(&ds, cudaStreamNonBlocking));
    if (!dv) ENG_CUDA(cudaEventCreateWithFlags(&dv, cudaEventDisableTiming));
    ENG_CUDA(cudaStreamWaitEvent(ds, e->chunk_start, 0));
    for (int j = 0; j < steps_now; ++j) {
      const int n = r.n0 + j;
      cudaError_t err;
      if (p->use_tc)
        err = launch_step_dense_tc(r.tc_plan, r.state_view(), p->Kp, r.FT, r.err, p->d_h.p, r.tables, n, ds);
      else
        err = launch_step_dense(r.state_view(), problem_dense_view(p), r.tables, n, ds);
      if (err != cudaSuccess) return set_error(SBQA_ERR_CUDA, std::string("engine step: ") + cudaGetErrorString(err));
      ++e->kernels_launched;
    }
    ENG_CUDA(cudaEventRecord(dv, ds));
    r.on_side = true;
  }
  if (!batch_ids.empty() && (rc = dense_batches(e, batch_ids, st)) != SBQA_OK) return rc;
  if (!batch_f4_ids.empty() && (rc = dense_batches_f4(e, batch_f4_ids, st)) != SBQA_OK) return rc;
  if (n_items) {
    if (!e->batched_t0) {
      ENG_CUDA(cudaEventCreate(&e->batched_t0));
      ENG_CUDA(cudaEventCreate(&e->batched_t1));
    }
    // every CSR request's chunk in one cooperative launch, replayed from a captured graph
    // a warp per task (a unit, or a row of an item), at most one co-resident wave
    const int grid = batched_grid(int64_t(counts[0]) + 8 * int64_t(counts[1]));
    if ((rc = csr_chunk_graph(e, grid)) != SBQA_OK) return rc;
    ENG_CUDA(cudaEventRecord(e->batched_t0, st));
    if (e->csr_graph) {
      ENG_CUDA(cudaGraphLaunch(e->csr_graph, st));
      ++e->graph_launches;
    } else {
      ENG_CUDA(launch_solve_batched(e->d_slots, e->max_slots, e->d_items, e->d_n_items, grid, 0, e->chunk, e->d_bar,
                                    e->d_err, st));
    }
    ++e->kernels_launched;
    ENG_CUDA(cudaEventRecord(e->batched_t1, st));
  }
  for (int id : dense_active) {
    Request &r = e->reqs[id];
    if (r.on_side) ENG_CUDA(cudaStreamWaitEvent(st, e->side_done[r.slot], 0));
    r.on_side = false;
  }
  // 4. retire the requests that finished inside the chunk
  std::vector<int> finished;
  for (int q = 0; q < e->max_slots; ++q) {
    if (e->slot_req[q] < 0) continue;
    Request &r = e->reqs[e->slot_req[q]];
    const int done_now = std::min(e->chunk, r.S - r.n0);
    e->steps_done_total += int64_t(done_now) * r.prob->n * r.R * r.P;
    if (!r.prob->dense) e->batched_updates += int64_t(done_now) * r.prob->n * r.R * r.P;
    r.n0 += done_now;
    if (r.n0 >= r.S) {
      if ((rc = readout(e, r, st)) != SBQA_OK) return rc;
      finished.push_back(r.id);
    }
  }
  ENG_CUDA(cudaStreamSynchronize(st));
  int csr_err = 0;  // the batched launch's grid barrier gave up: every CSR request of the chunk fails
  if (n_items) {
    float ms = 0.f;
    ENG_CUDA(cudaEventElapsedTime(&ms, e->batched_t0, e->batched_t1));
    e->batched_ms += ms;
    ENG_CUDA(cudaMemcpy(&csr_err, e->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (csr_err) {
      ENG_CUDA(cudaMemset(e->d_err, 0, sizeof(int)));
      for (int q = 0; q < e->max_slots; ++q) {
        if (e->slot_req[q] < 0) continue;
        Request &r = e->reqs[e->slot_req[q]];
        if (r.prob->dense || std::find(finished.begin(), finished.end(), r.id) != finished.end()) continue;
        finished.push_back(r.id);  // retired below as failed
      }
    }
  }
  // Every finished request leaves its slot and arena space, also one whose
  // device wait gave up: it is retired as FAILED and the others still
  // complete; TIMEOUT is returned once all of them are retired.
  const char *fail_hook = std::getenv("SBQA_TEST_ENGINE_FAIL_REQUEST");
  const int fail_id = fail_hook ? std::atoi(fail_hook) : -1;
  std::string failed_ids;
  for (int id : finished) {
    Request &r = e->reqs[id];
    int err = 0;
    ENG_CUDA(cudaMemcpy(&err, r.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (id == fail_id) err = 1;  // test hook: the request's device error word as a failed wait leaves it
    if (csr_err && !r.prob->dense) err = 1;
    if (r.tc_plan) {
      tc_plan_free(r.tc_plan);
      r.tc_plan = nullptr;
    }
    if (r.tc4_plan) {
      tc4_plan_free(r.tc4_plan);
      r.tc4_plan = nullptr;
    }
    e->slot_req[r.slot] = -1;
    e->arena.release(r.off, r.bytes);
    r.state = err ? FAILED : DONE;
    if (err) failed_ids += (failed_ids.empty() ? "" : ", ") + std::to_string(id);
    if (*n_done < cap && done_ids) done_ids[*n_done] = id;
    ++*n_done;
  }
  if (!failed_ids.empty())
    return set_error(SBQA_ERR_TIMEOUT, "a bounded device wait gave up in request(s) " + failed_ids +
                                           "; they were retired without a result, the others completed");
  return SBQA_OK;
}

int sbqa_engine_result(sbqa_engine *e, int32_t id, int8_t *spins, double *energy, int64_t *energy_int,
                       int32_t *replica) {
  if (!e || id < 0 || id >= int(e->reqs.size())) return set_error(SBQA_ERR_INVALID_ARG, "unknown request");
  const Request &r = e->reqs[id];
  if (r.state == FAILED)
    return set_error(SBQA_ERR_TIMEOUT, "request " + std::to_string(id) + " failed: a bounded device wait gave up");
  if (r.state != DONE) return set_error(SBQA_ERR_STATE, "request not finished");
  if (spins) std::memcpy(spins, r.spins.data(), r.spins.size());
  if (energy) std::memcpy(energy, r.energy.data(), r.energy.size() * sizeof(double));
  if (energy_int) std::memcpy(energy_int, r.energy_int.data(), r.energy_int.size() * sizeof(int64_t));
  if (replica) std::memcpy(replica, r.replica.data(), r.replica.size() * sizeof(int32_t));
  return SBQA_OK;
}

int sbqa_engine_stats(const sbqa_engine *e, sbqa_engine_stats_t *s) {
  if (!e || !s) return set_error(SBQA_ERR_INVALID_ARG, "null argument");
  s->queued = int32_t(e->queue.size());
  s->active = 0;
  for (int q : e->slot_req) s->active += q >= 0;
  s->finished = 0;
  for (const auto &r : e->reqs) s->finished += r.state == DONE || r.state == FAILED;
  s->arena_bytes = int64_t(e->arena.bytes);
  s->arena_used = int64_t(e->arena.used);
  s->updates_issued = e->steps_done_total;
  s->kernels_launched = e->kernels_launched;
  s->batched_updates = e->batched_updates;
  s->batched_ms = e->batched_ms;
  s->dense_batched_launches = e->dense_batched_launches;
  s->dense_batched_chunks = e->dense_batched_chunks;
  s->dense_e2m1_requests = e->dense_e2m1_requests;
  return SBQA_OK;
}

}  // extern "C"
