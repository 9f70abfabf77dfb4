// api.cu -- host side of the C ABI declared in include/sbqa.h.
//
// Responsibilities: validate and copy the Ising instance (Sec. II A,
// Eqs. 1-2: symmetric J, zero diagonal), pick the coupling-product path,
// build the FP64 schedule tables of Sec. II A (a(t) = t/T, Gamma_x(t) and
// J_perp(t) of Eq. 5, Delta(t) of Eq. 8) and round them to FP32, own the
// device buffers, and issue the hot-path kernels on the caller's stream.
// The step loop of a full run is captured once per shape in a CUDA graph and
// replayed.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <type_traits>
#include <vector>

#include <unistd.h>

#include "../../include/sbqa.h"
#include "internal.h"
#include "problem.h"

using namespace sbqa;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};


#define SBQA_CUDA(call)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? SBQA_ERR_OOM : SBQA_ERR_CUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

}  // namespace

int sbqa::set_error(int code, const std::string &msg) { return fail(code, msg); }

// ---------------------------------------------------------------- device block cache
namespace {

constexpr size_t kCacheCapBytes = size_t(4) << 30;  // per device

struct DevCache {
  std::mutex mu;
  std::map<int, std::multimap<size_t, void *>> blocks;  // device -> (size class, block)
  std::map<int, size_t> held;                           // device -> bytes held
};

DevCache &devcache() {
  static DevCache *c = new DevCache();  // never destroyed: blocks are left to the driver at exit
  return *c;
}

size_t size_class(size_t bytes) {
  if (bytes <= (size_t(1) << 20)) {
    size_t c = 512;
    while (c < bytes) c <<= 1;
    return c;
  }
  const size_t g = size_t(2) << 20;
  return (bytes + g - 1) / g * g;
}

// cudaFree of every cached block of device dev (every device if dev < 0);
// the caller holds the lock.  False if a cudaFree failed.
bool trim_locked(DevCache &c, int dev) {
  bool ok = true;
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto &kv : c.blocks) {
    if (dev >= 0 && kv.first != dev) continue;
    if (!kv.second.empty()) cudaSetDevice(kv.first);
    for (auto &b : kv.second) ok = cudaFree(b.second) == cudaSuccess && ok;
    kv.second.clear();
    c.held[kv.first] = 0;
  }
  cudaSetDevice(cur);
  return ok;
}

}  // namespace

// ---------------------------------------------------------------- host block cache
namespace {

constexpr size_t kHostCacheCap = size_t(2) << 30;

struct HostCache {
  std::mutex mu;
  std::multimap<size_t, void *> blocks;  // size class -> block
  size_t held = 0;
};

HostCache &hostcache() {
  static HostCache *c = new HostCache();  // never destroyed: blocks are left to the OS at exit
  return *c;
}

size_t host_class(size_t bytes) { return (bytes + kHostCacheMin - 1) / kHostCacheMin * kHostCacheMin; }

}  // namespace

void *sbqa::hostcache_get(size_t bytes) {
  const size_t cls = host_class(bytes);
  HostCache &c = hostcache();
  {
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.blocks.find(cls);
    if (it != c.blocks.end()) {
      void *q = it->second;
      c.blocks.erase(it);
      c.held -= cls;
      return q;
    }
  }
  void *q = std::malloc(cls);
  if (!q) {  // give the cached blocks back and try once more
    std::lock_guard<std::mutex> lk(c.mu);
    for (auto &b : c.blocks) std::free(b.second);
    c.blocks.clear();
    c.held = 0;
    q = std::malloc(cls);
  }
  return q;
}

void sbqa::hostcache_put(void *p, size_t bytes) {
  if (!p) return;
  const size_t cls = host_class(bytes);
  HostCache &c = hostcache();
  std::lock_guard<std::mutex> lk(c.mu);
  if (c.held + cls > kHostCacheCap) {
    std::free(p);
    return;
  }
  c.blocks.emplace(cls, p);
  c.held += cls;
}

cudaError_t sbqa::devcache_get(void **p, size_t bytes, size_t *got) {
  const size_t cls = size_class(bytes);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  DevCache &c = devcache();
  {
    std::lock_guard<std::mutex> lk(c.mu);
    auto &m = c.blocks[dev];
    auto it = m.find(cls);
    if (it != m.end()) {
      *p = it->second;
      *got = cls;
      m.erase(it);
      c.held[dev] -= cls;
      return cudaSuccess;
    }
  }
  e = cudaMalloc(p, cls);
  if (e == cudaErrorMemoryAllocation) {  // give the cached blocks back and try once more
    cudaGetLastError();
    {
      std::lock_guard<std::mutex> lk(c.mu);
      trim_locked(c, dev);
    }
    e = cudaMalloc(p, cls);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  *got = cls;
  return cudaSuccess;
}

void sbqa::devcache_put(void *p, size_t bytes) {
  if (!p) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  DevCache &c = devcache();
  std::lock_guard<std::mutex> lk(c.mu);
  if (c.held[dev] + bytes > kCacheCapBytes) {
    cudaFree(p);
    return;
  }
  c.blocks[dev].emplace(bytes, p);
  c.held[dev] += bytes;
}

bool sbqa::devcache_trim() {
  DevCache &c = devcache();
  std::lock_guard<std::mutex> lk(c.mu);
  return trim_locked(c, -1);
}

sbqa_problem::~sbqa_problem() {
  DeviceGuard g(device);
  cudaDeviceSynchronize();  // no kernel of this handle may still use the buffers
  if (graph) cudaGraphExecDestroy(graph);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  if (tc_plan) tc_plan_free(tc_plan);
  if (tc4_plan) tc4_plan_free(tc4_plan);
  d_J8.release(true); d_FT.release(true); d_err.release(true);
  d_row_ptr.release(true); d_col.release(true); d_col_pm1.release(true); d_npos.release(true); d_val_f32.release(true);
  d_val_bf16.release(true); d_dense_f32.release(true); d_h.release(true); d_e_i32.release(true);
  d_e_f64.release(true); d_h_i64.release(true); d_h_f64.release(true); d_x.release(true); d_y.release(true);
  d_jcopy_i8.release(true);
  d_F0.release(true); d_F1.release(true); d_Fx0.release(true); d_Fx1.release(true); d_Sg.release(true);
  d_ell_col.release(true); d_ell_meta.release(true); d_ell_val.release(true); d_ka.release(true); d_dl.release(true);
  d_kj.release(true); d_ei.release(true); d_part_i.release(true); d_best_ei.release(true); d_ef.release(true);
  d_part_f.release(true); d_best_e.release(true); d_best_k.release(true); d_best_step.release(true);
  d_have.release(true); d_best_spins.release(true); d_bar.release(true); d_tc_flags.release(true);
  d_J4.release(true); d_FT4.release(true);
}



namespace {

constexpr int kTcMinN = 256;  // smaller dense instances stay on the CUDA-core kernel
constexpr int kIngestMinN = 1024;  // dense J from N = 1024 on is read by the GPU where it can
// EXACT precision takes integer J up to this magnitude: the products are exact
// in bfloat16 (and e4m3 up to 16) and every partial sum, an integer below
// 256 N < 2^24 for N < 65536, is exact in FP32
constexpr int kExactMaxAbsJ = 256;

bool finite_all(const double *v, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// Round a double to the nearest bfloat16 (ties to even), returned as bits.
uint16_t bf16_bits_rne(double v) {
  if (v == 0.0) return std::signbit(v) ? 0x8000u : 0u;
  int e;
  const double m = std::frexp(v, &e);           // |m| in [0.5, 1)
  const double q = std::nearbyint(std::ldexp(m, 8));  // 8 significant bits
  const float f = float(std::ldexp(q, e - 8));  // exact in FP32 for normal range
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return uint16_t(u >> 16);
}

// Host threads of parallel_tasks: up to 15 workers beside the calling
// thread, started on first use and kept for the life of the process (a job
// wakes them instead of creating threads).  One job at a time; its tasks go
// to whichever thread takes the next index.
class HostPool {
 public:
  static HostPool &get() {
    static HostPool pool;
    return pool;
  }
  template <class Fn>
  void run(int64_t n_tasks, Fn &fn) {
    if (started_ && getpid() != owner_) {  // a forked child: the workers stayed in the parent
      for (int64_t t = 0; t < n_tasks; ++t) fn(t, 0);
      return;
    }
    std::lock_guard<std::mutex> job(job_mu_);
    if (!started_) start();
    {
      std::lock_guard<std::mutex> l(mu_);
      invoke_ = [](void *c, int64_t t) { (*static_cast<Fn *>(c))(t, 0); };
      ctx_ = &fn;
      n_ = n_tasks;
      next_.store(0);
      busy_ = int(th_->size());
      ++gen_;
    }
    cv_.notify_all();
    for (int64_t t; (t = next_.fetch_add(1)) < n_tasks;) fn(t, 0);
    std::unique_lock<std::mutex> l(mu_);
    done_cv_.wait(l, [&] { return busy_ == 0; });  // every worker is past this job
  }
  ~HostPool() {
    // a forked child leaves the parent's thread handles alone (none runs here)
    if (!started_ || getpid() != owner_) return;
    {
      std::lock_guard<std::mutex> l(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto &x : *th_) x.join();
    delete th_;
  }

 private:
  void start() {
    started_ = true;
    owner_ = getpid();
    const unsigned hw = std::thread::hardware_concurrency();
    const int T = int(std::max(1u, std::min(hw ? hw : 1u, 16u)));
    th_ = new std::vector<std::thread>();
    for (int w = 1; w < T; ++w) th_->emplace_back([this] { loop(); });
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      std::unique_lock<std::mutex> l(mu_);
      cv_.wait(l, [&] { return stop_ || gen_ != seen; });
      if (stop_) return;
      seen = gen_;
      void (*invoke)(void *, int64_t) = invoke_;
      void *ctx = ctx_;
      const int64_t n = n_;
      l.unlock();
      for (int64_t t; (t = next_.fetch_add(1)) < n;) invoke(ctx, t);
      l.lock();
      if (--busy_ == 0) done_cv_.notify_one();
    }
  }
  std::mutex job_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  std::vector<std::thread> *th_ = nullptr;  // released only by the process that started them
  std::atomic<bool> started_{false};
  bool stop_ = false;
  pid_t owner_ = 0;
  void (*invoke_)(void *, int64_t) = nullptr;
  void *ctx_ = nullptr;
  int64_t n_ = 0;
  std::atomic<int64_t> next_{0};
  int busy_ = 0;
  uint64_t gen_ = 0;
};

// Runs fn(task, 0) for task = 0 .. n_tasks-1 on the host pool; the split
// never changes a result, because each task writes only its own outputs.
template <class Fn>
void parallel_tasks(int64_t n_tasks, Fn fn) {
  if (n_tasks <= 1) {
    for (int64_t t = 0; t < n_tasks; ++t) fn(t, 0);
    return;
  }
  HostPool::get().run(n_tasks, fn);
}

// Statistics of the stored couplings (merged in a fixed order of blocks).
struct JStats {
  bool j_int = true, pm1 = true;
  double mx = 0.0, s2 = 0.0;
  void add(double v) {
    if (v == 0.0) return;
    if (v != std::nearbyint(v)) j_int = false;
    if (std::fabs(v) != 1.0) pm1 = false;
    mx = std::max(mx, std::fabs(v));
    s2 += v * v;
  }
  void merge(const JStats &o) {  // in a fixed order, so the sums do not depend on threads
    j_int = j_int && o.j_int;
    pm1 = pm1 && o.pm1;
    mx = std::max(mx, o.mx);
    s2 += o.s2;
  }
};

void finish_analysis(sbqa_problem *p, JStats js);

void finish_analysis(sbqa_problem *p, JStats js) {
  bool j_int = js.j_int, pm1 = js.pm1, h_int = true;
  const double mx = js.mx, s2 = js.s2;
  if (mx > 1e6) j_int = false;
  for (double v : p->h)
    if (v != std::nearbyint(v) || std::fabs(v) > 1e12) h_int = false;
  p->j_integer = j_int;
  p->is_integer = j_int && h_int;  // energies exact in int64
  p->is_pm1 = pm1;                 // every stored J_ij is +1 or -1
  p->max_abs_j = j_int ? int32_t(mx) : -1;
  p->c0_auto = s2 > 0.0 ? 0.5 * std::sqrt(double(p->n) / s2) : 0.5;
  p->h_zero = true;
  for (double v : p->h)
    if (v != 0.0) p->h_zero = false;
}

int upload_common(sbqa_problem *p) {
  const int N = p->n;
  std::vector<float> hf(N, 0.f);
  for (int i = 0; i < N; ++i) hf[i] = p->h.empty() ? 0.f : float(p->h[i]);
  SBQA_CUDA(p->d_h.alloc(N));
  SBQA_CUDA(cudaMemcpy(p->d_h.p, hf.data(), N * sizeof(float), cudaMemcpyHostToDevice));
  if (p->is_integer) {
    std::vector<int64_t> hi(N, 0);
    for (int i = 0; i < N; ++i) hi[i] = p->h.empty() ? 0 : int64_t(std::llround(p->h[i]));
    SBQA_CUDA(p->d_h_i64.alloc(N));
    SBQA_CUDA(cudaMemcpy(p->d_h_i64.p, hi.data(), N * sizeof(int64_t), cudaMemcpyHostToDevice));
  } else {
    std::vector<double> hd(N, 0.0);
    for (int i = 0; i < N; ++i) hd[i] = p->h.empty() ? 0.0 : p->h[i];
    SBQA_CUDA(p->d_h_f64.alloc(N));
    SBQA_CUDA(cudaMemcpy(p->d_h_f64.p, hd.data(), N * sizeof(double), cudaMemcpyHostToDevice));
  }
  return SBQA_OK;
}

int upload_readout_values(sbqa_problem *p) {
  const size_t m = p->jcount();
  if (m == 0 || (p->is_integer ? p->d_e_i32.p != nullptr : p->d_e_f64.p != nullptr)) return SBQA_OK;
  if (p->j_on_device) {  // converted from the device copy
    const int8_t *d8 = p->d_jcopy_i8.p;
    if (p->is_integer) {
      SBQA_CUDA(p->d_e_i32.alloc(m));
      SBQA_CUDA(launch_flat_from_device(d8, p->d_e_f64.p, m, kFlatI32, p->d_e_i32.p, nullptr));
    } else {  // integer J beside a real h (a real J's FP64 copy is already d_e_f64)
      SBQA_CUDA(p->d_e_f64.alloc(m));
      SBQA_CUDA(launch_flat_from_device(d8, nullptr, m, kFlatF64, p->d_e_f64.p, nullptr));
    }
    SBQA_CUDA(cudaStreamSynchronize(nullptr));
    return SBQA_OK;
  }
  const int64_t blk = 1 << 16, tasks = (int64_t(m) + blk - 1) / blk;
  if (p->is_integer) {
    HostVec<int32_t> vi(m);
    parallel_tasks(tasks, [&](int64_t t, int64_t) {
      const size_t e1 = std::min(m, size_t(t + 1) * blk);
      if (!p->val_i8.empty())
        for (size_t e = size_t(t) * blk; e < e1; ++e) vi[e] = p->val_i8[e];
      else
        for (size_t e = size_t(t) * blk; e < e1; ++e) vi[e] = int32_t(std::llround(p->val[e]));
    });
    SBQA_CUDA(p->d_e_i32.alloc(m));
    SBQA_CUDA(cudaMemcpy(p->d_e_i32.p, vi.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice));
  } else if (!p->val_i8.empty()) {  // integer J beside a real h
    HostVec<double> vd(m);
    parallel_tasks(tasks, [&](int64_t t, int64_t) {
      const size_t e1 = std::min(m, size_t(t + 1) * blk);
      for (size_t e = size_t(t) * blk; e < e1; ++e) vd[e] = p->val_i8[e];
    });
    SBQA_CUDA(p->d_e_f64.alloc(m));
    SBQA_CUDA(cudaMemcpy(p->d_e_f64.p, vd.data(), m * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    SBQA_CUDA(p->d_e_f64.alloc(m));
    SBQA_CUDA(cudaMemcpy(p->d_e_f64.p, p->val.data(), m * sizeof(double), cudaMemcpyHostToDevice));
  }
  return SBQA_OK;
}

// Sparse value array for the requested precision; sets p->kind.
int prepare_sparse_values(sbqa_problem *p, int precision) {
  const size_t m = p->val.size();
  int kind;
  if (precision == SBQA_PREC_BF16) kind = VAL_BF16;
  else if (precision == SBQA_PREC_FP32) kind = VAL_F32;
  else if (p->is_pm1 && p->max_degree <= 127) kind = VAL_PM1;
  else kind = VAL_F32;
  if (precision == SBQA_PREC_EXACT && (!p->j_integer || p->max_abs_j > kExactMaxAbsJ))
    return fail(SBQA_ERR_UNSUPPORTED, "EXACT precision needs integer J with |J_ij| <= 256");
  p->kind = kind;
  if (kind == VAL_PM1 && !p->d_npos.p) {
    // each row: columns of the +1 entries, then of the -1 entries
    std::vector<int32_t> col(m), npos(p->n);
    parallel_tasks((int64_t(p->n) + 4095) / 4096, [&](int64_t task, int64_t) {
      const int i1 = std::min<int64_t>(p->n, (task + 1) * 4096);
      for (int i = int(task) * 4096; i < i1; ++i) {
        int64_t w = p->row_ptr[i];
        for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e)
          if (p->val[e] > 0) col[w++] = p->col[e];
        npos[i] = int32_t(w - p->row_ptr[i]);
        for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e)
          if (p->val[e] < 0) col[w++] = p->col[e];
      }
    });
    SBQA_CUDA(p->d_npos.alloc(p->n));
    SBQA_CUDA(cudaMemcpy(p->d_npos.p, npos.data(), p->n * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (m) {
      SBQA_CUDA(p->d_col_pm1.alloc(m));
      SBQA_CUDA(cudaMemcpy(p->d_col_pm1.p, col.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
  } else if (kind == VAL_F32 && !p->d_val_f32.p && m) {
    std::vector<float> v(m);
    parallel_tasks((int64_t(m) + 65535) / 65536, [&](int64_t task, int64_t) {
      const size_t e1 = std::min<size_t>(m, size_t(task + 1) * 65536);
      for (size_t e = size_t(task) * 65536; e < e1; ++e) v[e] = float(p->val[e]);
    });
    SBQA_CUDA(p->d_val_f32.alloc(m));
    SBQA_CUDA(cudaMemcpy(p->d_val_f32.p, v.data(), m * sizeof(float), cudaMemcpyHostToDevice));
  } else if (kind == VAL_BF16 && !p->d_val_bf16.p && m) {
    std::vector<uint16_t> v(m);
    parallel_tasks((int64_t(m) + 65535) / 65536, [&](int64_t task, int64_t) {
      const size_t e1 = std::min<size_t>(m, size_t(task + 1) * 65536);
      for (size_t e = size_t(task) * 65536; e < e1; ++e) v[e] = bf16_bits_rne(p->val[e]);
    });
    SBQA_CUDA(p->d_val_bf16.alloc(m));
    SBQA_CUDA(cudaMemcpy(p->d_val_bf16.p, v.data(), m * 2, cudaMemcpyHostToDevice));
  }
  if (p->max_degree <= kEllSlots && p->ell_kind != kind && p->n > 0) {
    // ELL slots: each row's entries in the order the CSR kernels sum them
    // (+1 entries first for +-1 J), values as the kernels see them (FP32, or
    // BF16 widened exactly), zero padding; (degree, +1 count) per row
    const int N = p->n;
    std::vector<int32_t> ec(size_t(N) * kEllSlots, 0), meta(size_t(N) * 2, 0);
    std::vector<float> ev(kind == VAL_PM1 ? 0 : size_t(N) * kEllSlots, 0.f);
    parallel_tasks((int64_t(N) + 4095) / 4096, [&](int64_t task, int64_t) {
    const int i1 = std::min<int64_t>(N, (task + 1) * 4096);
    for (int i = int(task) * 4096; i < i1; ++i) {
      const int64_t e0 = p->row_ptr[i], e1 = p->row_ptr[i + 1];
      int w = 0, npos = 0;
      if (kind == VAL_PM1) {
        for (int64_t e = e0; e < e1; ++e)
          if (p->val[e] > 0) ec[size_t(i) * kEllSlots + w++] = p->col[e];
        npos = w;
        for (int64_t e = e0; e < e1; ++e)
          if (p->val[e] < 0) ec[size_t(i) * kEllSlots + w++] = p->col[e];
      } else {
        for (int64_t e = e0; e < e1; ++e, ++w) {
          ec[size_t(i) * kEllSlots + w] = p->col[e];
          float v;
          if (kind == VAL_BF16) {
            const uint32_t bits = uint32_t(bf16_bits_rne(p->val[e])) << 16;
            std::memcpy(&v, &bits, sizeof(v));
          } else {
            v = float(p->val[e]);
          }
          ev[size_t(i) * kEllSlots + w] = v;
        }
        npos = w;
      }
      meta[2 * size_t(i)] = w;
      meta[2 * size_t(i) + 1] = npos;
    }
    });
    SBQA_CUDA(p->d_ell_col.alloc(ec.size()));
    SBQA_CUDA(cudaMemcpy(p->d_ell_col.p, ec.data(), ec.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    SBQA_CUDA(p->d_ell_meta.alloc(meta.size()));
    SBQA_CUDA(cudaMemcpy(p->d_ell_meta.p, meta.data(), meta.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (!ev.empty()) {
      SBQA_CUDA(p->d_ell_val.alloc(ev.size()));
      SBQA_CUDA(cudaMemcpy(p->d_ell_val.p, ev.data(), ev.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    p->ell_kind = kind;
  }
  return SBQA_OK;
}

// e4m3 bits of a small integer (|v| <= 16, exact): 1.mmm x 2^e, bias 7.
uint8_t e4m3_of_int(int v) {
  if (v == 0) return 0;
  const uint8_t sign = v < 0 ? 0x80 : 0x00;
  int a = v < 0 ? -v : v, e = 0;
  while ((a >> (e + 1)) != 0) ++e;          // a in [2^e, 2^(e+1))
  const int mant = ((a << 3) >> e) & 7;     // 3 fraction bits (exact for a <= 16)
  return uint8_t(sign | ((e + 7) << 3) | mant);
}

// bfloat16 copy of J for the tensor cores (operand forms kTcOpBf16 and
// kTcOpBsb): round to nearest even from the FP64 values (exact for integers
// |J_ij| <= 256), zero padding to Kp.
int prepare_tc_values_bf16(sbqa_problem *p) {
  const int N = p->n, Kp = (N + 127) / 128 * 128;
  if (p->j_on_device) {
    SBQA_CUDA(p->d_J8.alloc(size_t(Kp) * Kp * 2));
    SBQA_CUDA(launch_tc_jbf16_from_device(p->d_jcopy_i8.p, p->d_e_f64.p, N, Kp,
                                          reinterpret_cast<uint16_t *>(p->d_J8.p), nullptr));
    SBQA_CUDA(cudaStreamSynchronize(nullptr));
    p->Kp = Kp;
    p->j_tc_op = p->tc_op;
    return SBQA_OK;
  }
  HostVec<uint16_t> jb(size_t(Kp) * Kp);
  parallel_tasks(Kp, [&](int64_t i, int64_t) {
    uint16_t *out = jb.data() + size_t(i) * Kp;
    if (i >= N) {
      std::memset(out, 0, size_t(Kp) * 2);
      return;
    }
    for (int j = 0; j < N; ++j) out[j] = bf16_bits_rne(p->jv(size_t(i) * N + j));
    std::memset(out + N, 0, size_t(Kp - N) * 2);
  });
  SBQA_CUDA(p->d_J8.alloc(jb.size() * 2));
  SBQA_CUDA(cudaMemcpy(p->d_J8.p, jb.data(), jb.size() * 2, cudaMemcpyHostToDevice));
  p->Kp = Kp;
  p->j_tc_op = p->tc_op;
  return SBQA_OK;
}

int prepare_tc_values(sbqa_problem *p) {
  const bool bf = p->tc_op != kTcOpF8;
  if (p->d_J8.p && (p->j_tc_op == p->tc_op || (bf && p->j_tc_op != kTcOpF8))) {
    p->j_tc_op = p->tc_op;
    return SBQA_OK;
  }
  if (bf) return prepare_tc_values_bf16(p);
  const int N = p->n, Kp = (N + 127) / 128 * 128;
  if (p->j_on_device) {  // integer |J_ij| <= 16: the byte copy is on the device
    SBQA_CUDA(p->d_J8.alloc(size_t(Kp) * Kp));
    SBQA_CUDA(launch_tc_j8_from_device(p->d_jcopy_i8.p, N, Kp, p->d_J8.p, nullptr));
    SBQA_CUDA(cudaStreamSynchronize(nullptr));
    p->Kp = Kp;
    p->j_tc_op = kTcOpF8;
    return SBQA_OK;
  }
  HostVec<uint8_t> j8(size_t(Kp) * Kp);  // every byte is written below (zeros in the padding)
  uint8_t lut[33];  // e4m3 of -16 .. 16 (the tensor-core path takes |J_ij| <= 16)
  for (int v = -16; v <= 16; ++v) lut[v + 16] = e4m3_of_int(v);
  parallel_tasks(Kp, [&](int64_t i, int64_t) {
    uint8_t *out = j8.data() + size_t(i) * Kp;
    if (i >= N) {
      std::memset(out, 0, size_t(Kp));
      return;
    }
    if (!p->val_i8.empty()) {
      const int8_t *row = p->val_i8.data() + size_t(i) * N;
      for (int j = 0; j < N; ++j) out[j] = lut[row[j] + 16];  // |J_ij| <= 16, checked when J was analysed
    } else {
      const double *row = p->val.data() + size_t(i) * N;
      for (int j = 0; j < N; ++j) out[j] = lut[int(row[j]) + 16];
    }
    std::memset(out + N, 0, size_t(Kp - N));
  });
  SBQA_CUDA(p->d_J8.alloc(j8.size()));
  SBQA_CUDA(cudaMemcpy(p->d_J8.p, j8.data(), j8.size(), cudaMemcpyHostToDevice));
  p->Kp = Kp;
  p->j_tc_op = kTcOpF8;
  return SBQA_OK;
}

int prepare_dense_values(sbqa_problem *p, int precision) {
  if (precision == SBQA_PREC_EXACT && (!p->j_integer || p->max_abs_j > kExactMaxAbsJ))
    return fail(SBQA_ERR_UNSUPPORTED, "EXACT precision needs integer J with |J_ij| <= 256");
  // Tensor-core forms (N >= kTcMinN):
  //  e4m3   exact: integer |J| <= 16 with the thresholded f in {-1, 0, 1}
  //  bf16   exact for integer |J| <= 256 (AUTO, EXACT), or J rounded to
  //         bfloat16 (BF16), with the thresholded f
  //  bsb    the ballistic form f(x) = x with BF16: J rounded to bfloat16, x as
  //         bfloat16 hi + lo
  const bool exactish = precision == SBQA_PREC_AUTO || precision == SBQA_PREC_EXACT;
  int op = -1;
  if (p->n >= kTcMinN) {
    if (p->ballistic()) {
      if (precision == SBQA_PREC_BF16) op = kTcOpBsb;
    } else if (exactish && p->j_integer && p->max_abs_j <= 16) {
      op = kTcOpF8;
    } else if ((exactish && p->j_integer && p->max_abs_j <= kExactMaxAbsJ) || precision == SBQA_PREC_BF16) {
      op = kTcOpBf16;
    }
  }
  p->use_tc = op >= 0;
  if (p->use_tc) {
    if (p->tc_op != op && p->tc_plan) {  // the plan's maps are of the other operand type
      tc_plan_free(p->tc_plan);
      p->tc_plan = nullptr;
    }
    p->tc_op = op;
    // the readout runs on the tensor cores too when its energies are integers
    // and the product is e4m3; otherwise on the CUDA cores (exact int64 or FP64)
    const int rc = prepare_tc_values(p);
    if (rc != SBQA_OK || (p->is_integer && op == kTcOpF8)) return rc;
    return upload_readout_values(p);
  }
  {
    const int rc = upload_readout_values(p);
    if (rc != SBQA_OK) return rc;
  }
  const int want = precision == SBQA_PREC_BF16 ? SBQA_PREC_BF16 : SBQA_PREC_FP32;
  if (p->d_dense_f32.p && p->dense_prec == want) return SBQA_OK;
  const size_t m = p->jcount();
  if (p->j_on_device) {
    SBQA_CUDA(p->d_dense_f32.alloc(m));
    SBQA_CUDA(launch_flat_from_device(p->d_jcopy_i8.p, p->d_e_f64.p, m,
                                      want == SBQA_PREC_BF16 ? kFlatBf16InF32 : kFlatF32, p->d_dense_f32.p, nullptr));
    SBQA_CUDA(cudaStreamSynchronize(nullptr));
    p->dense_prec = want;
    return SBQA_OK;
  }
  HostVec<float> v(m);
  const int64_t blk = 1 << 16;
  parallel_tasks((int64_t(m) + blk - 1) / blk, [&](int64_t t, int64_t) {
    const size_t e1 = std::min(m, size_t(t + 1) * blk);
    for (size_t e = size_t(t) * blk; e < e1; ++e) {
      if (want == SBQA_PREC_BF16) {
        const uint32_t u = uint32_t(bf16_bits_rne(p->jv(e))) << 16;
        std::memcpy(&v[e], &u, 4);
      } else {
        v[e] = float(p->jv(e));
      }
    }
  });
  SBQA_CUDA(p->d_dense_f32.alloc(m));
  SBQA_CUDA(cudaMemcpy(p->d_dense_f32.p, v.data(), m * sizeof(float), cudaMemcpyHostToDevice));
  p->dense_prec = want;
  return SBQA_OK;
}

// Per-device memo of the solvers' co-resident block counts: the occupancy
// queries (and the shared-memory attributes the first one sets, which last
// for the context) cost tens of microseconds each, and every new handle
// would repeat them.
int memo_blocks(int (*query)()) {
  static std::mutex mu;
  static std::map<std::pair<int, int (*)()>, int> memo;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return query();
  std::lock_guard<std::mutex> lk(mu);
  auto it = memo.find({dev, query});
  if (it != memo.end()) return it->second;
  const int v = query();
  memo[{dev, query}] = v;
  return v;
}

// The tensor-core kernels' shared-memory limits, set once per device (they last for the context).
int tc_attributes_once() { return tc_set_attributes() == cudaSuccess ? 1 : 0; }

int alloc_run(sbqa_problem *p, int S, int P, int R) {
  const int Ps = run_width(P);  // a run's columns: P replicas, then padding up to a power of two
  const int C = R * Ps;
  const int Cp = (C + kColsPerWarp - 1) / kColsPerWarp * kColsPerWarp;
  const size_t NC = size_t(p->n) * Cp;
  SBQA_CUDA(p->d_x.alloc(NC));
  SBQA_CUDA(p->d_y.alloc(NC));
  SBQA_CUDA(p->d_F0.alloc(NC));
  SBQA_CUDA(p->d_F1.alloc(NC));
  if (p->ballistic() && !p->use_tc) {  // the tensor-core form keeps f(x) = x in its FT buffers
    SBQA_CUDA(p->d_Fx0.alloc(NC));
    SBQA_CUDA(p->d_Fx1.alloc(NC));
    SBQA_CUDA(cudaMemsetAsync(p->d_Fx1.p, 0, NC * sizeof(float), p->stream));
  }
  SBQA_CUDA(p->d_Sg.alloc(NC));
  SBQA_CUDA(p->d_ka.alloc(size_t(std::max(S, 1))));
  SBQA_CUDA(p->d_dl.alloc(size_t(S) + 1));
  SBQA_CUDA(p->d_kj.alloc(size_t(std::max(S, 1)) * R));
  SBQA_CUDA(p->d_ei.alloc(Cp));
  SBQA_CUDA(p->d_ef.alloc(Cp));
  const size_t parts = size_t(energy_row_blocks(p->n)) * Cp;
  if (p->is_integer) SBQA_CUDA(p->d_part_i.alloc(parts));
  else SBQA_CUDA(p->d_part_f.alloc(parts));
  SBQA_CUDA(p->d_best_ei.alloc(R));
  SBQA_CUDA(p->d_best_e.alloc(R));
  SBQA_CUDA(p->d_best_k.alloc(R));
  SBQA_CUDA(p->d_best_step.alloc(R));
  SBQA_CUDA(p->d_have.alloc(R));
  SBQA_CUDA(p->d_best_spins.alloc(size_t(R) * p->n));
  SBQA_CUDA(p->d_err.alloc(1));
  SBQA_CUDA(cudaMemsetAsync(p->d_err.p, 0, sizeof(int), p->stream));  // no trial launch reads a stale code
  p->S = S; p->P = P; p->R = R; p->C = C; p->Cp = Cp; p->Ps = Ps;
  if (p->use_tc) {
    SBQA_CUDA(p->d_FT.alloc(tc_ft_bytes(p->Kp, Cp, p->tc_op)));
    if (!p->tc_plan || p->tc_plan_ft != p->d_FT.p || p->tc_plan_cp != Cp || p->tc_plan_x != p->d_x.p ||
        tc_op_of(p->tc_plan) != p->tc_op) {
      if (p->tc_plan) tc_plan_free(p->tc_plan);
      p->tc_plan = nullptr;
      if (!tc_plan_make(&p->tc_plan, p->d_J8.p, p->d_FT.p, p->Kp, Cp, p->d_x.p, p->d_y.p, p->n, p->tc_op))
        return fail(SBQA_ERR_CUDA, "cuTensorMapEncodeTiled failed");
      if (memo_blocks(tc_attributes_once) != 1) return fail(SBQA_ERR_CUDA, "cudaFuncSetAttribute failed");
      p->tc_plan_ft = p->d_FT.p;
      p->tc_plan_cp = Cp;
      p->tc_plan_x = p->d_x.p;
    }
  }
  return SBQA_OK;
}

// The FP64 tables cost S * R transcendental evaluations on the host (640 000
// for 10^4 steps of 64 runs), so they are rebuilt only when the run shape, the
// schedule or the buffers change.
int build_tables(sbqa_problem *p) {
  sbqa_problem::TablesKey key;
  key.S = p->S; key.P = p->P; key.R = p->R; key.version = p->params_version;
  key.ka = p->d_ka.p; key.dl = p->d_dl.p; key.kj = p->d_kj.p;
  if (key == p->tables_key) return SBQA_OK;
  const int rc = problem_build_tables(p, p->S, p->P, p->R, p->d_ka.p, p->d_dl.p, p->d_kj.p, &p->tables, p->stream);
  p->tables_key = rc == SBQA_OK ? key : sbqa_problem::TablesKey{};
  return rc;
}

cudaError_t issue_step(sbqa_problem *p, int n, cudaStream_t st) {
  const StateView s = p->state();
  if (p->use_tc) return launch_step_dense_tc(p->tc_plan, s, p->Kp, p->d_FT.p, p->d_err.p, p->d_h.p, p->tables, n, st);
  if (p->ballistic()) {
    if (p->dense) {
      DenseView d;
      d.J = p->d_dense_f32.p;
      d.h = p->d_h.p;
      return launch_step_dense_bsb(s, d, p->tables, n, st);
    }
    return launch_step_csr_bsb(s, p->csr(), p->tables, n, st);
  }
  if (p->dense) {
    DenseView d;
    d.J = p->d_dense_f32.p;
    d.h = p->d_h.p;
    return launch_step_dense(s, d, p->tables, n, st);
  }
  return launch_step_csr(s, p->csr(), p->tables, n, p->csr_variant < 0 ? 0 : p->csr_variant, st);
}

// Device time per launch of `reps` launches issued by issue(stream), replayed
// as one CUDA graph (as a solve replays its step launches), so launch
// overhead on the host does not bias the comparison with the persistent
// solvers.  One untimed replay first.
template <class Issue>
static int time_per_launch_in_graph(sbqa_problem *p, int reps, Issue issue, float *ms_per_launch) {
  if (!p->cap_stream) SBQA_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  SBQA_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int w = 0; w < reps && e == cudaSuccess; ++w) e = issue(p->cap_stream);
  const cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(SBQA_ERR_CUDA, std::string("autotuner capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(SBQA_ERR_CUDA, std::string("autotuner instantiate: ") + cudaGetErrorString(e));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, p->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e0, p->stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, p->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return fail(SBQA_ERR_CUDA, std::string("autotuner timing: ") + cudaGetErrorString(e));
  *ms_per_launch = ms / reps;
  return SBQA_OK;
}

// Autotuner of the CSR step kernel: times every variant on this problem's
// shape (a few launches each, on the freshly allocated state buffers, before
// the initial state is written) and keeps the fastest.  Results are cached
// per handle and shape; skipped while the stream is being captured.
// Process-wide memory of the autotuner's results.  The choice depends only on
// the device and the problem's shape, so a new handle of a shape already tuned
// on this device skips the timing launches.
struct TuneKey {
  int dev, dense, n, kind, Cp, P, select, max_degree, Kp;
  int64_t nnz;
  bool operator<(const TuneKey &o) const {
    return std::tie(dev, dense, n, kind, Cp, P, select, max_degree, Kp, nnz) <
           std::tie(o.dev, o.dense, o.n, o.kind, o.Cp, o.P, o.select, o.max_degree, o.Kp, o.nnz);
  }
};
struct TuneResult {
  int csr_variant = 0;
  bool use_persistent = false, use_tc_persistent = false, use_tc_split = false, use_tc_pair = false,
       use_tc_f4 = false, use_tc_f4_pair = false;
  float variant_ms[8] = {};
  float persistent_ms = 0.f, tc_step_ms = 0.f, tc_persistent_ms = 0.f;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneResult> g_tune;

TuneKey tune_key(const sbqa_problem *p) {
  TuneKey k;
  k.dev = p->device; k.dense = p->dense ? 1 : 0; k.n = p->n; k.kind = p->dense ? -1 - (p->use_tc ? p->tc_op : 8) : p->kind; k.Cp = p->Cp;
  if (p->ballistic()) k.kind += 16;  // the ballistic form's choices are its own
  if (p->dense && p->use_tc && p->tc_f4_possible()) k.kind -= 32;  // the e2m1 solver is a candidate
  k.P = p->P; k.select = p->prm.kernel_select; k.max_degree = p->max_degree; k.Kp = p->Kp; k.nnz = p->nnz;
  return k;
}

bool tune_lookup(const sbqa_problem *p, TuneResult *r) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(tune_key(p));
  if (it == g_tune.end()) return false;
  *r = it->second;
  return true;
}

void tune_store(const sbqa_problem *p, const TuneResult &r) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[tune_key(p)] = r;
}

// The ballistic form has one per-step kernel and, where the items fit the
// cache, the persistent solver: kernel_select 1 keeps the per-step kernel, 2
// the persistent solver, 0 times both (a few steps each) and keeps the faster.
int autotune_csr_bsb(sbqa_problem *p) {
  if (p->csr_variant < 0) p->csr_variant = 0;
  const int sel = p->prm.kernel_select;
  if (p->csr_variant_cp == p->Cp && p->csr_variant_kind == p->kind && p->csr_variant_select == sel) return SBQA_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  SBQA_CUDA(cudaStreamIsCapturing(p->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return SBQA_OK;
  p->use_persistent = false;
  p->persistent_ms = 0.f;
  if (p->persist_blocks == 0) p->persist_blocks = memo_blocks(persistent_blocks);
  if (p->S > 0 && (sel == 0 || sel == 2) && p->persistent_ok()) {
    SBQA_CUDA(p->d_bar.alloc(persistent_barrier_words()));
    TuneResult known;
    const StateView s = p->state();
    const CsrView J = p->csr();
    if (sel == 2) {
      p->use_persistent = true;
    } else if (tune_lookup(p, &known)) {
      p->variant_ms[0] = known.variant_ms[0];
      p->persistent_ms = known.persistent_ms;
      p->use_persistent = known.use_persistent;
    } else {
      const int reps = 8, steps = std::min(p->S, 64);
      float step_ms = 0.f;
      int rc = time_per_launch_in_graph(
          p, reps, [&](cudaStream_t st) { return launch_step_csr_bsb(s, J, p->tables, 0, st); }, &step_ms);
      if (rc != SBQA_OK) return rc;
      cudaEvent_t e0, e1;
      SBQA_CUDA(cudaEventCreate(&e0));
      SBQA_CUDA(cudaEventCreate(&e1));
      cudaError_t e = launch_solve_csr_persistent_bsb(s, J, p->tables, 0, std::min(p->S, 4), p->d_bar.p, p->d_err.p,
                                                      p->persist_blocks, p->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, p->stream);
      if (e == cudaSuccess)
        e = launch_solve_csr_persistent_bsb(s, J, p->tables, 0, steps, p->d_bar.p, p->d_err.p, p->persist_blocks,
                                            p->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      SBQA_CUDA(e);
      SBQA_CUDA(cudaMemsetAsync(p->d_err.p, 0, sizeof(int), p->stream));
      p->variant_ms[0] = step_ms;
      p->persistent_ms = ms / steps;
      p->use_persistent = p->persistent_ms < step_ms;
      TuneResult r;
      r.variant_ms[0] = step_ms;
      r.persistent_ms = p->persistent_ms;
      r.use_persistent = p->use_persistent;
      tune_store(p, r);
    }
  }
  p->csr_variant_cp = p->Cp;
  p->csr_variant_kind = p->kind;
  p->csr_variant_select = sel;
  return SBQA_OK;
}

int autotune_csr(sbqa_problem *p) {
  if (p->dense) return SBQA_OK;
  if (p->ballistic()) return autotune_csr_bsb(p);
  if (p->csr_variant >= 0 && p->csr_variant_cp == p->Cp && p->csr_variant_kind == p->kind &&
      p->csr_variant_select == p->prm.kernel_select)
    return SBQA_OK;
  p->csr_variant_select = p->prm.kernel_select;
  if (p->prm.kernel_select >= 3 && p->prm.kernel_select <= 10) {  // a forced per-step variant
    const int v = p->prm.kernel_select - 3;
    p->csr_variant = csr_step_variant_ok(v, p->Cp, p->csr().ell_col != nullptr) ? v : 0;
    p->csr_variant_cp = p->Cp;
    p->csr_variant_kind = p->kind;
    p->use_persistent = false;
    return SBQA_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  SBQA_CUDA(cudaStreamIsCapturing(p->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return SBQA_OK;
  if (p->persist_blocks == 0) p->persist_blocks = memo_blocks(persistent_blocks);
  TuneResult known;
  if (p->S > 0 && tune_lookup(p, &known)) {
    p->csr_variant = known.csr_variant;
    for (int v = 0; v < 8; ++v) p->variant_ms[v] = known.variant_ms[v];
    p->persistent_ms = known.persistent_ms;
    p->use_persistent = known.use_persistent && p->persistent_ok();
    if (p->use_persistent) SBQA_CUDA(p->d_bar.alloc(persistent_barrier_words()));
    p->csr_variant_cp = p->Cp;
    p->csr_variant_kind = p->kind;
    return SBQA_OK;
  }
  const StateView s = p->state();
  const CsrView J = p->csr();
  const int nv = csr_step_variants(), reps = 8;
  float best_ms = 1e30f;
  int best = 0;
  const int n = 0;
  for (int v = 0; v < nv && p->S > 0; ++v) {
    if (!csr_step_variant_ok(v, p->Cp, J.ell_col != nullptr)) continue;
    float ms = 0.f;
    const int rc = time_per_launch_in_graph(
        p, reps, [&](cudaStream_t st) { return launch_step_csr(s, J, p->tables, n, v, st); }, &ms);
    if (rc != SBQA_OK) return rc;
    if (v < 8) p->variant_ms[v] = ms;
    ms *= reps;
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  // the persistent kernel: a few steps in one cooperative launch
  cudaEvent_t e0, e1;
  SBQA_CUDA(cudaEventCreate(&e0));
  SBQA_CUDA(cudaEventCreate(&e1));
  p->use_persistent = false;
  p->persistent_ms = 0.f;
  if (p->persist_blocks == 0) p->persist_blocks = memo_blocks(persistent_blocks);
  if ((p->prm.kernel_select == 2 || p->prm.kernel_select >= 11) && p->S > 0 &&
      p->persistent_ok()) {
    SBQA_CUDA(p->d_bar.alloc(persistent_barrier_words()));
    p->use_persistent = true;
  } else if (p->prm.kernel_select == 0 && p->S > 0 && p->persistent_ok()) {
    SBQA_CUDA(p->d_bar.alloc(persistent_barrier_words()));
    const int steps = std::min(p->S, 64);
    SBQA_CUDA(launch_solve_csr_persistent(s, J, p->tables, 0, std::min(p->S, 4), p->d_bar.p, p->d_err.p,
                                          p->persist_blocks, p->persist_mode(), p->stream));
    SBQA_CUDA(cudaEventRecord(e0, p->stream));
    SBQA_CUDA(launch_solve_csr_persistent(s, J, p->tables, 0, steps, p->d_bar.p, p->d_err.p, p->persist_blocks,
                                          p->persist_mode(), p->stream));
    SBQA_CUDA(cudaEventRecord(e1, p->stream));
    SBQA_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    SBQA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    p->persistent_ms = ms / steps;
    p->use_persistent = p->persistent_ms < best_ms / reps;
    SBQA_CUDA(cudaMemsetAsync(p->d_err.p, 0, sizeof(int), p->stream));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->csr_variant = best;
  p->csr_variant_cp = p->Cp;
  p->csr_variant_kind = p->kind;
  if (p->S > 0) {
    TuneResult r;
    r.csr_variant = best;
    for (int v = 0; v < 8; ++v) r.variant_ms[v] = p->variant_ms[v];
    r.persistent_ms = p->persistent_ms;
    r.use_persistent = p->use_persistent;
    tune_store(p, r);
  }
  return SBQA_OK;
}

// Steps [n0, n1) of the persistent dense tcgen05 solver: on CTA pairs, split-K
// across 2-CTA clusters, or with 128 x 128 tiles, as chosen.
cudaError_t launch_tc_persistent(sbqa_problem *p, const StateView &s, int n0, int n1, cudaStream_t st) {
  if (p->tc_f4_ok())
    return p->tc_f4_pair_ok()
               ? launch_solve_dense_tc_f4_pair(p->tc4_plan, s, p->Kp, p->d_err.p, p->d_h.p, p->tables, n0, n1,
                                               p->d_tc_flags.p, st)
               : launch_solve_dense_tc_f4(p->tc4_plan, s, p->Kp, p->d_err.p, p->d_h.p, p->tables, n0, n1,
                                          p->d_tc_flags.p, st);
  if (p->tc_pair_ok())
    return launch_solve_dense_tc_pair(p->tc_plan, s, p->Kp, p->d_err.p, p->d_h.p, p->tables, n0, n1,
                                      p->d_tc_flags.p, st);
  if (p->tc_split_ok())
    return launch_solve_dense_tc_split(p->tc_plan, s, p->Kp, p->d_err.p, p->d_h.p, p->tables, n0, n1,
                                       p->d_tc_flags.p, st);
  return launch_solve_dense_tc_persistent(p->tc_plan, s, p->Kp, p->d_err.p, p->d_h.p, p->tables, n0, n1,
                                          p->d_tc_flags.p, st);
}

// Operands of the e2m1 solver: J4 from the e4m3 copy of J (once per
// problem), FT4 for the run's column count (zeroed, so the bytes past Kp
// that no tile writes stay zero), and their tensor maps.
int prepare_tc_f4(sbqa_problem *p) {
  const int Kh = tc_f4_row_bytes(p->Kp);
  if (!p->d_J4.p) {
    SBQA_CUDA(p->d_J4.alloc(size_t(p->Kp) * Kh));
    SBQA_CUDA(launch_j4_from_j8(p->d_J8.p, p->Kp, p->d_J4.p, p->stream));
  }
  SBQA_CUDA(p->d_FT4.alloc(size_t(2) * p->Cp * Kh));
  if (!p->tc4_plan || p->tc4_plan_ft != p->d_FT4.p || p->tc4_plan_cp != p->Cp || p->tc4_plan_j != p->d_J4.p) {
    SBQA_CUDA(cudaMemsetAsync(p->d_FT4.p, 0, size_t(2) * p->Cp * Kh, p->stream));
    if (p->tc4_plan) tc4_plan_free(p->tc4_plan);
    p->tc4_plan = nullptr;
    if (!tc4_plan_make(&p->tc4_plan, p->d_J4.p, p->d_FT4.p, p->Kp, p->Cp))
      return fail(SBQA_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    p->tc4_plan_ft = p->d_FT4.p;
    p->tc4_plan_j = p->d_J4.p;
    p->tc4_plan_cp = p->Cp;
  }
  return SBQA_OK;
}

// Autotuner of the dense tensor-core path: times the per-step kernel, the
// persistent solver with 128 x 128 tiles and, where the instance qualifies,
// the split-K and the paired persistent solvers (same state buffers, before
// the initial state is written) and keeps the fastest.  kernel_select 1
// forces the per-step kernel, 2 the persistent solver (split-K where it
// qualifies), 12 the persistent solver with 128 x 128 tiles, 13 the paired
// persistent solver where it qualifies, 14 the e2m1 solver where it
// qualifies (its paired form where that qualifies; else as 12), 15 the e2m1
// solver without clusters (else as 12).  Cached per handle, column count, replica count
// and selection, and process-wide per instance shape.
int autotune_tc(sbqa_problem *p) {
  if (!p->use_tc) {
    p->use_tc_persistent = p->use_tc_split = p->use_tc_pair = p->use_tc_f4 = p->use_tc_f4_pair = false;
    return SBQA_OK;
  }
  if (p->tc_select_cp == p->Cp && p->tc_select == p->prm.kernel_select && p->tc_select_p == p->P) return SBQA_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  SBQA_CUDA(cudaStreamIsCapturing(p->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return SBQA_OK;
  p->use_tc_persistent = p->use_tc_split = p->use_tc_pair = p->use_tc_f4 = p->use_tc_f4_pair = false;
  p->tc_step_ms = p->tc_persistent_ms = 0.f;
  if (p->tc_persist_blocks == 0) p->tc_persist_blocks = memo_blocks(tc_persistent_blocks);
  if (p->tc_split_blocks < 0) p->tc_split_blocks = memo_blocks(tc_split_blocks);
  if (p->tc_pair_blocks < 0) p->tc_pair_blocks = memo_blocks(tc_pair_blocks);
  if (p->tc_f4_blocks < 0) p->tc_f4_blocks = memo_blocks(tc_f4_blocks);
  if (p->tc_f4_pair_blocks < 0) p->tc_f4_pair_blocks = memo_blocks(tc_f4_pair_blocks);
  const int sel = p->prm.kernel_select;
  if (sel != 1 && p->S > 0 && p->tc_persistent_ok()) {
    SBQA_CUDA(p->d_tc_flags.alloc(tc_persistent_flag_count(p->Kp, p->Cp)));
    if (p->tc_f4_possible()) {
      const int frc = prepare_tc_f4(p);
      if (frc != SBQA_OK) return frc;
    }
    SBQA_CUDA(cudaMemsetAsync(p->d_err.p, 0, sizeof(int), p->stream));  // read after the trial launches
    // a cluster launch the device refuses, or one that does not arrive as 2-CTA
    // clusters (the kernel then reports ERR_CLUSTER_SHAPE before touching
    // anything, e.g. under a profiler's replay), leaves the plain persistent
    // solver: a zero-step launch of each cluster solver checks that first
    auto probe = [&](bool *use, bool *failed) -> int {
      *use = true;
      SBQA_CUDA(cudaMemsetAsync(p->d_err.p, 0, sizeof(int), p->stream));
      if (launch_tc_persistent(p, p->state(), 0, 0, p->stream) != cudaSuccess) {
        cudaGetLastError();
        *failed = true;
      } else {
        int err = 0;
        SBQA_CUDA(cudaMemcpyAsync(&err, p->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
        SBQA_CUDA(cudaStreamSynchronize(p->stream));
        if (err != 0) {
          *failed = true;
          SBQA_CUDA(cudaMemsetAsync(p->d_err.p, 0, sizeof(int), p->stream));
        }
      }
      *use = false;
      return SBQA_OK;
    };
    // a kernel_select that names a solver without clusters (1, 12) launches
    // no cluster solver at all, not even the probe
    int prc = SBQA_OK;
    if ((sel == 0 || sel == 2) && p->tc_split_possible() &&
        (prc = probe(&p->use_tc_split, &p->tc_split_failed)) != SBQA_OK)
      return prc;
    if ((sel == 0 || sel == 13) && p->tc_pair_possible() &&
        (prc = probe(&p->use_tc_pair, &p->tc_pair_failed)) != SBQA_OK)
      return prc;
    if ((sel == 0 || sel == 14) && p->tc_f4_pair_possible()) {
      p->use_tc_f4 = true;
      prc = probe(&p->use_tc_f4_pair, &p->tc_f4_pair_failed);
      p->use_tc_f4 = false;
      if (prc != SBQA_OK) return prc;
    }
    TuneResult known;
    if (sel == 2 || sel == 12 || sel == 13 || sel == 14 || sel == 15) {
      p->use_tc_persistent = true;
      p->use_tc_split = sel == 2 && p->tc_split_possible();
      p->use_tc_pair = sel == 13 && p->tc_pair_possible();
      p->use_tc_f4 = (sel == 14 || sel == 15) && p->tc_f4_possible();
      p->use_tc_f4_pair = sel == 14 && p->tc_f4_pair_possible();
    } else if (tune_lookup(p, &known)) {
      p->use_tc_persistent = known.use_tc_persistent;
      p->use_tc_split = known.use_tc_split;
      p->use_tc_pair = known.use_tc_pair;
      p->use_tc_f4 = known.use_tc_f4;
      p->use_tc_f4_pair = known.use_tc_f4_pair;
      p->tc_step_ms = known.tc_step_ms;
      p->tc_persistent_ms = known.tc_persistent_ms;
    } else {
      const StateView s = p->state();
      float ms = 0.f;
      const int rc = time_per_launch_in_graph(
          p, 8,
          [&](cudaStream_t st) {
            return launch_step_dense_tc(p->tc_plan, s, p->Kp, p->d_FT.p, p->d_err.p, p->d_h.p, p->tables, 0, st);
          },
          &ms);
      if (rc != SBQA_OK) return rc;
      p->tc_step_ms = ms;
      // the persistent candidates: 128 x 128 tiles, then split-K, CTA pairs and e2m1 where they qualify
      const int steps = std::min(p->S, 64);
      float best_persistent = 0.f;
      int best_cand = 0;
      for (int cand = 0; cand < 5; ++cand) {
        if ((cand == 1 && !p->tc_split_possible()) || (cand == 2 && !p->tc_pair_possible()) ||
            (cand == 3 && !p->tc_f4_possible()) || (cand == 4 && !p->tc_f4_pair_possible()))
          continue;
        p->use_tc_split = cand == 1;
        p->use_tc_pair = cand == 2;
        p->use_tc_f4 = cand >= 3;
        p->use_tc_f4_pair = cand == 4;
        cudaEvent_t e0, e1;
        SBQA_CUDA(cudaEventCreate(&e0));
        SBQA_CUDA(cudaEventCreate(&e1));
        cudaError_t e = launch_tc_persistent(p, s, 0, std::min(p->S, 4), p->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, p->stream);
        if (e == cudaSuccess) e = launch_tc_persistent(p, s, 0, steps, p->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        SBQA_CUDA(e);
        // a cluster solver (split-K, CTA pairs, e2m1 pairs) must beat the best
        // single-CTA one by a margin: at shapes where they tie (N=2000, R*P=1024)
        // a 64-step trial picks either by noise
        auto cluster = [](int c) { return c == 1 || c == 2 || c == 4; };
        const float margin = cluster(cand) && !cluster(best_cand) ? 0.97f : 1.f;
        if (cand == 0 || ms / steps < best_persistent * margin) {
          best_persistent = ms / steps;
          best_cand = cand;
        }
      }
      p->use_tc_split = best_cand == 1;
      p->use_tc_pair = best_cand == 2;
      p->use_tc_f4 = best_cand >= 3;
      p->use_tc_f4_pair = best_cand == 4;
      p->tc_persistent_ms = best_persistent;
      p->use_tc_persistent = p->tc_persistent_ms < p->tc_step_ms;
      int err = 0;
      SBQA_CUDA(cudaMemcpy(&err, p->d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
      if (err != 0) return fail(SBQA_ERR_TIMEOUT, "a bounded device wait gave up (code " + std::to_string(err) + ")");
      TuneResult r;
      r.use_tc_persistent = p->use_tc_persistent;
      r.use_tc_split = p->use_tc_split;
      r.use_tc_pair = p->use_tc_pair;
      r.use_tc_f4 = p->use_tc_f4;
      r.use_tc_f4_pair = p->use_tc_f4_pair;
      r.tc_step_ms = p->tc_step_ms;
      r.tc_persistent_ms = p->tc_persistent_ms;
      tune_store(p, r);
    }
  }
  p->tc_select_cp = p->Cp;
  p->tc_select = p->prm.kernel_select;
  p->tc_select_p = p->P;
  return SBQA_OK;
}

cudaError_t issue_readout(sbqa_problem *p, int step, cudaStream_t st) {
  const StateView s = p->state();
  // integer dense instances (J and h) on the tensor cores: the sign codes take
  // the FT buffer of step `step`, which the next step does not read
  cudaError_t e = p->dense ? (p->use_tc && p->tc_plan && p->is_integer && p->tc_op == kTcOpF8 ? launch_energy_dense_tc(p->tc_plan, s, p->Kp, p->d_FT.p,
                                                                               step & 1, p->d_err.p, p->energy(),
                                                                               p->best(), st)
                                                      : launch_energy_dense(s, p->energy(), p->best(), st))
                           : launch_energy_csr(s, p->csr_readout(), p->energy(), p->best(), st);
  if (e != cudaSuccess) return e;
  return launch_best(s, p->energy(), p->best(), step, st);
}

// Steps [n0, n1) with the intermediate readouts of eval_every.
cudaError_t issue_range(sbqa_problem *p, int n0, int n1, cudaStream_t st) {
  const int K = p->prm.eval_every;
  const bool tc_persist = p->use_tc_persistent && p->tc_persistent_ok();
  if (tc_persist || (p->use_persistent && p->persistent_ok())) {
    // one cooperative launch per stretch between readouts
    int n = n0;
    while (n < n1) {
      int stop = n1;
      if (K > 0) stop = std::min(n1, (n / K + 1) * K);
      cudaError_t e = tc_persist      ? launch_tc_persistent(p, p->state(), n, stop, st)
                      : p->ballistic() ? launch_solve_csr_persistent_bsb(p->state(), p->csr(), p->tables, n, stop,
                                                                          p->d_bar.p, p->d_err.p, p->persist_blocks, st)
                                       : launch_solve_csr_persistent(p->state(), p->csr(), p->tables, n, stop,
                                                                     p->d_bar.p, p->d_err.p, p->persist_blocks,
                                                                     p->persist_mode(), st);
      if (e != cudaSuccess) return e;
      const int last = stop - 1;
      if (K > 0 && (last + 1) % K == 0 && last != p->S - 1) {
        e = issue_readout(p, last, st);
        if (e != cudaSuccess) return e;
      }
      n = stop;
    }
    return cudaSuccess;
  }
  for (int n = n0; n < n1; ++n) {
    cudaError_t e = issue_step(p, n, st);
    if (e != cudaSuccess) return e;
    if (K > 0 && (n + 1) % K == 0 && n != p->S - 1) {
      e = issue_readout(p, n, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

int check_run_args(sbqa_problem *p, int32_t steps, int32_t P, int32_t R) {
  if (!p) return fail(SBQA_ERR_INVALID_ARG, "null problem");
  if (!p->have_params) return fail(SBQA_ERR_STATE, "sbqa_set_schedule has not been called");
  if (steps < 0) return fail(SBQA_ERR_INVALID_ARG, "steps must be >= 0");
  if (P < 1) return fail(SBQA_ERR_INVALID_ARG, "P must be >= 1");
  if (P > kMaxReplicas) return fail(SBQA_ERR_UNSUPPORTED, "P must be at most 128");
  if (R < 1 || int64_t(R) * run_width(P) > (1 << 20))
    return fail(SBQA_ERR_INVALID_ARG, "need 1 <= R and R * (P rounded up to a power of two) <= 2^20");
  if (!p->beta.empty() && int(p->beta.size()) != R)
    return fail(SBQA_ERR_INVALID_ARG, "R differs from params.n_runs");
  return SBQA_OK;
}

}  // namespace

// ---- helpers shared with the batching engine (problem.h) ----
int sbqa::problem_check_run(sbqa_problem *p, int32_t steps, int32_t P, int32_t R) {
  return check_run_args(p, steps, P, R);
}

int sbqa::problem_prepare_values(sbqa_problem *p) {
  DeviceGuard g(p->device);
  return p->dense ? prepare_dense_values(p, p->prm.precision) : prepare_sparse_values(p, p->prm.precision);
}

// FP64 schedule of Sec. II A rounded to the FP32 step coefficients.
int sbqa::problem_build_tables(const sbqa_problem *p, int S, int P, int R, float *d_ka, float *d_dl, float *d_kj,
                               StepTables *t, cudaStream_t st) {
  const sbqa_params &q = p->prm;
  const double c0 = q.c0 > 0.0 ? q.c0 : p->c0_auto;
  std::vector<float> ka(std::max(S, 1), 0.f), dl(S + 1), kj(size_t(std::max(S, 1)) * R, 0.f);
  for (int n = 0; n <= S; ++n) {
    const double tau = S > 0 ? double(n) / double(S) : 0.0;
    dl[n] = float(q.delta_slope * tau);                 // Delta(t) = 0.7 t/T
    if (n < S) ka[n] = float(q.dt * (q.a0 - tau) / P);  // a(t) = t/T
  }
  // S * R transcendental evaluations (640 000 for 10^4 steps of 64 runs), in
  // blocks of steps over the host threads; each entry is computed alone
  constexpr int kStepsPerTask = 64;
  parallel_tasks((int64_t(S) + kStepsPerTask - 1) / kStepsPerTask, [&](int64_t task, int64_t) {
    const int n1 = std::min(S, int(task + 1) * kStepsPerTask);
    for (int n = int(task) * kStepsPerTask; n < n1; ++n) {
      const double tau = double(n) / double(S);
      for (int r = 0; r < R; ++r) {
        double jp = 0.0;
        if (q.jperp_enable) {
          const double b = p->beta.empty() ? 1.0 : p->beta[r];
          const double a = p->alpha.empty() ? 1.0 : p->alpha[r];
          const double gam = q.gamma0 * (std::pow(1.0 - tau, a) + 1e-5);  // Gamma_x(t), Eq. 5
          jp = -std::log(std::tanh(b * gam / P)) / (2.0 * b);           // J_perp(t), Eq. 5
        }
        kj[size_t(n) * R + r] = float(q.dt * jp);
      }
    }
  });
  SBQA_CUDA(cudaMemcpyAsync(d_ka, ka.data(), ka.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  SBQA_CUDA(cudaMemcpyAsync(d_dl, dl.data(), dl.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  SBQA_CUDA(cudaMemcpyAsync(d_kj, kj.data(), kj.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  t->ka = d_ka;
  t->dl = d_dl;
  t->kj = d_kj;
  t->kc = float(q.dt * c0 / P);
  t->kx = float(q.dt * q.a0 / P);
  t->S = S;
  t->R = R;
  return SBQA_OK;
}

// sbqa_create_problem_dense with the checks, statistics and the library's
// copy of J made on the GPU from the caller's array (ingest_dense.cu): the
// same errors, in the same order, and the same analysis as the host pass
// (each row's sum of squares added per 32-column tile, the tiles in order,
// then the rows in row order).
static int create_dense_on_device(int32_t n, const double *J, const double *h, sbqa_problem **out) {
  const size_t m = size_t(n) * n;
  sbqa_problem *p = new (std::nothrow) sbqa_problem();
  if (!p) return fail(SBQA_ERR_OOM, "host allocation");
  cudaGetDevice(&p->device);
  DevBuf<int8_t> d8;
  DevBuf<double> d64;
  DevBuf<IngestRow> drows, dpart;
  DevBuf<int> dasym;
  std::vector<IngestRow> rows(n);
  int asym = 0;
  auto cuda_fail = [&](cudaError_t e) {
    d8.release(); d64.release(); drows.release(); dpart.release(); dasym.release();
    delete p;
    return fail(e == cudaErrorMemoryAllocation ? SBQA_ERR_OOM : SBQA_ERR_CUDA,
                std::string("dense J on the device: ") + cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = d8.alloc(m)) != cudaSuccess || (e = d64.alloc(m)) != cudaSuccess || (e = drows.alloc(n)) != cudaSuccess ||
      (e = dpart.alloc(ingest_part_count(n))) != cudaSuccess || (e = dasym.alloc(1)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = launch_ingest_dense(J, n, d8.p, d64.p, dpart.p, drows.p, dasym.p, nullptr)) != cudaSuccess ||
      (e = cudaMemcpy(rows.data(), drows.p, size_t(n) * sizeof(IngestRow), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(&asym, dasym.p, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e);
  drows.release(true);
  dpart.release(true);
  dasym.release(true);
  bool finite = !h || finite_all(h, n), diag = true;
  int64_t nnz = 0;
  int32_t maxdeg = 0;
  JStats js;
  for (const IngestRow &r : rows) {
    finite = finite && (r.flags & kIngestFinite);
    diag = diag && (r.flags & kIngestDiagZero);
    js.j_int = js.j_int && (r.flags & kIngestInteger);
    js.pm1 = js.pm1 && (r.flags & kIngestPm1);
    js.mx = std::max(js.mx, r.mx);
    js.s2 += r.s2;
    nnz += r.nnz;
    maxdeg = std::max(maxdeg, r.nnz);
  }
  auto reject = [&](int code, const char *msg) {
    d8.release(true); d64.release(true);
    delete p;
    return fail(code, msg);
  };
  if (!finite) return reject(SBQA_ERR_NOT_FINITE, "J or h not finite");
  if (!diag) return reject(SBQA_ERR_NOT_SYMMETRIC, "nonzero diagonal");
  if (asym) return reject(SBQA_ERR_NOT_SYMMETRIC, "J != J^T");
  p->n = n;
  p->dense = true;
  p->j_on_device = true;
  if (js.j_int && js.mx <= 127.0) {
    p->d_jcopy_i8 = d8;
    d64.release(true);
  } else {
    p->d_e_f64 = d64;  // the FP64 values (also the readout's copy)
    d8.release(true);
  }
  d8 = DevBuf<int8_t>();
  d64 = DevBuf<double>();
  if (h) p->h.assign(h, h + n);
  p->nnz = nnz;
  p->max_degree = maxdeg;
  finish_analysis(p, js);
  const int rc = upload_common(p);
  if (rc != SBQA_OK) {
    delete p;
    return rc;
  }
  *out = p;
  return SBQA_OK;
}

CsrView sbqa::problem_csr_view(const sbqa_problem *p) { return p->csr(); }
CsrView sbqa::problem_csr_readout_view(const sbqa_problem *p) { return p->csr_readout(); }
EnergyView sbqa::problem_energy_view(const sbqa_problem *p) { return p->energy(); }
DenseView sbqa::problem_dense_view(const sbqa_problem *p) {
  DenseView d;
  d.J = p->d_dense_f32.p;
  d.h = p->d_h.p;
  return d;
}

extern "C" {

int sbqa_version(void) { return 100; }

const char *sbqa_last_error(void) { return g_last_error.c_str(); }

const char *sbqa_strerror(int status) {
  switch (status) {
    case SBQA_OK: return "ok";
    case SBQA_ERR_INVALID_ARG: return "invalid argument";
    case SBQA_ERR_NOT_SYMMETRIC: return "couplings not symmetric / malformed";
    case SBQA_ERR_NOT_FINITE: return "non-finite value";
    case SBQA_ERR_OOM: return "out of memory";
    case SBQA_ERR_CUDA: return "CUDA error";
    case SBQA_ERR_STATE: return "call out of order";
    case SBQA_ERR_UNSUPPORTED: return "unsupported request";
    case SBQA_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

void sbqa_default_params(sbqa_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->a0 = 1.0;
  p->c0 = 0.0;
  p->dt = 0.5;
  p->gamma0 = 1.0;
  p->delta_slope = 0.7;
  p->init_amp = 0.1;
  p->jperp_enable = 1;
  p->variant = SBQA_VARIANT_THRESHOLD;
  p->precision = SBQA_PREC_AUTO;
  p->eval_every = 0;
  p->n_runs = 0;
  p->beta = nullptr;
  p->alpha = nullptr;
}

int sbqa_create_problem_dense(int32_t n, const double *J, const double *h, sbqa_problem **out) {
  if (!out) return fail(SBQA_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (n < 1 || n > 65536 || !J) return fail(SBQA_ERR_INVALID_ARG, "need 1 <= n <= 65536 and J != NULL");
  // test hook: SBQA_TEST_HOST_INGEST=1 keeps the host pass where the GPU could
  // read J itself (not for production use)
  if (n >= kIngestMinN && ingest_on_device_possible() && !std::getenv("SBQA_TEST_HOST_INGEST"))
    return create_dense_on_device(n, J, h, out);
  const size_t m = size_t(n) * n;
  // One pass over blocks of 64 rows, spread over host threads: finiteness, the
  // diagonal, row degrees and the value statistics of each block, and the
  // symmetry of its tiles against their mirror tiles (64 x 64, so the
  // transposed reads stay in cache).
  constexpr int kB = 64;
  const int nb = (n + kB - 1) / kB;
  struct Block {
    bool finite = true, diag = true, sym = true;
    int64_t nnz = 0;
    int32_t maxdeg = 0;
    JStats js;
  };
  std::vector<Block> blocks(nb);
  // The library's copy: one byte per entry, filled in the same pass, which is
  // the whole copy when J turns out integer with |J_ij| <= 127 (the FP64 copy
  // is made afterwards otherwise).
  HostVec<int8_t> vals8(m);
  parallel_tasks(nb, [&](int64_t b, int64_t) {
    Block &B = blocks[b];
    const int i0 = int(b) * kB, i1 = std::min(n, i0 + kB);
    // accumulators in locals: J (double) and the byte copy could alias the
    // fields of B, which would force a store and reload per element
    JStats js;
    bool finite_b = true, diag_b = true, sym_b = true;
    int64_t nnz_b = 0;
    int32_t maxdeg_b = 0;
    for (int i = i0; i < i1; ++i) {
      const double *row = J + size_t(i) * n;
      int8_t *row8 = vals8.data() + size_t(i) * n;
      int32_t d = 0;
      bool fin = true;
      for (int j = 0; j < n; ++j) {
        const double v = row[j];
        fin &= std::isfinite(v);
        d += v != 0.0;
        js.add(v);
        row8[j] = int8_t(v >= -128.0 && v <= 127.0 ? int(v) : 0);
      }
      finite_b = finite_b && fin;
      if (row[i] != 0.0) diag_b = false;
      nnz_b += d;
      maxdeg_b = std::max(maxdeg_b, d);
    }
    for (int jb = int(b); jb < nb && sym_b; ++jb) {
      const int j0 = jb * kB, j1 = std::min(n, j0 + kB);
      bool same = true;
      for (int i = i0; i < i1; ++i)
        for (int j = std::max(j0, i + 1); j < j1; ++j) same &= J[size_t(i) * n + j] == J[size_t(j) * n + i];
      sym_b = same;
    }
    B.js = js;
    B.finite = finite_b;
    B.diag = diag_b;
    B.sym = sym_b;
    B.nnz = nnz_b;
    B.maxdeg = maxdeg_b;
  });
  bool finite = !h || finite_all(h, n), diag = true, sym = true;
  int64_t nnz = 0;
  int32_t maxdeg = 0;
  JStats js;
  for (const Block &B : blocks) {
    finite = finite && B.finite;
    diag = diag && B.diag;
    sym = sym && B.sym;
    nnz += B.nnz;
    maxdeg = std::max(maxdeg, B.maxdeg);
    js.merge(B.js);
  }
  if (!finite) return fail(SBQA_ERR_NOT_FINITE, "J or h not finite");
  if (!diag) return fail(SBQA_ERR_NOT_SYMMETRIC, "nonzero diagonal");
  if (!sym) return fail(SBQA_ERR_NOT_SYMMETRIC, "J != J^T");
  sbqa_problem *p = new (std::nothrow) sbqa_problem();
  if (!p) return fail(SBQA_ERR_OOM, "host allocation");
  cudaGetDevice(&p->device);
  p->n = n;
  p->dense = true;
  if (js.j_int && js.mx <= 127.0) {
    p->val_i8 = std::move(vals8);
  } else {
    vals8 = HostVec<int8_t>();
    p->val.resize(m);
    parallel_tasks(nb, [&](int64_t b, int64_t) {
      const int i0 = int(b) * kB, i1 = std::min(n, i0 + kB);
      std::memcpy(p->val.data() + size_t(i0) * n, J + size_t(i0) * n, size_t(i1 - i0) * n * sizeof(double));
    });
  }
  if (h) p->h.assign(h, h + n);
  p->nnz = nnz;
  p->max_degree = maxdeg;
  finish_analysis(p, js);
  // the readout values of the CUDA-core energy kernel are uploaded when a
  // schedule leaves the tensor cores (prepare_dense_values)
  int rc = upload_common(p);
  if (rc != SBQA_OK) {
    delete p;
    return rc;
  }
  *out = p;
  return SBQA_OK;
}

int sbqa_create_problem_csr(int32_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col_idx,
                            const double *val, const double *h, sbqa_problem **out) {
  if (!out) return fail(SBQA_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (n < 1 || nnz < 0 || nnz >= (int64_t(1) << 31) || !row_ptr || (nnz > 0 && (!col_idx || !val)))
    return fail(SBQA_ERR_INVALID_ARG, "bad sizes or null arrays");
  if (row_ptr[0] != 0 || row_ptr[n] != nnz) return fail(SBQA_ERR_NOT_SYMMETRIC, "row_ptr ends do not match nnz");
  for (int i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return fail(SBQA_ERR_NOT_SYMMETRIC, "row_ptr decreasing");
  // One pass over blocks of rows spread over the host threads: finiteness and
  // the value statistics, indices in range, sorted and off the diagonal, and
  // the partner (j, i) of every entry holding the same value.  The errors keep
  // the precedence of separate passes: non-finite values first, then the first
  // index error in row order, then asymmetry.
  constexpr int kRowsPerTask = 4096;
  const int64_t tasks = (int64_t(n) + kRowsPerTask - 1) / kRowsPerTask;
  struct Block {
    bool finite = true, sym = true;
    int err = SBQA_OK;
    const char *msg = nullptr;
    int32_t maxdeg = 0;
    JStats js;
  };
  std::vector<Block> blocks(static_cast<size_t>(tasks));
  parallel_tasks(tasks, [&](int64_t task, int64_t) {
    Block B;
    const int i1 = int(std::min<int64_t>(n, (task + 1) * kRowsPerTask));
    for (int i = int(task) * kRowsPerTask; i < i1; ++i) {
      const int64_t e0 = row_ptr[i], e1 = row_ptr[i + 1];
      B.maxdeg = std::max<int32_t>(B.maxdeg, int32_t(e1 - e0));
      for (int64_t e = e0; e < e1; ++e) {
        const double v = val[e];
        B.finite = B.finite && std::isfinite(v);
        B.js.add(v);
      }
      if (B.err != SBQA_OK) continue;
      for (int64_t e = e0; e < e1 && B.err == SBQA_OK; ++e) {
        const int32_t j = col_idx[e];
        if (j < 0 || j >= n) B.err = SBQA_ERR_INVALID_ARG, B.msg = "column index out of range";
        else if (j == i) B.err = SBQA_ERR_NOT_SYMMETRIC, B.msg = "diagonal entry in CSR";
        else if (e > e0 && col_idx[e - 1] >= j) B.err = SBQA_ERR_NOT_SYMMETRIC, B.msg = "unsorted or duplicate columns";
      }
      if (B.err != SBQA_OK || !B.sym) continue;
      for (int64_t e = e0; e < e1; ++e) {  // the row's columns are valid: the partner lookups stay in range
        const int32_t j = col_idx[e];
        const int32_t *b = col_idx + row_ptr[j], *en = col_idx + row_ptr[j + 1];
        const int32_t *it = std::lower_bound(b, en, i);
        if (it == en || *it != i || val[row_ptr[j] + (it - b)] != val[e]) {
          B.sym = false;
          break;
        }
      }
    }
    blocks[size_t(task)] = B;
  });
  bool finite = !h || finite_all(h, n), sym = true;
  int32_t maxdeg = 0;
  JStats js_all;
  const Block *first_err = nullptr;
  for (const Block &B : blocks) {  // in row order: the same results whatever the threads
    finite = finite && B.finite;
    sym = sym && B.sym;
    maxdeg = std::max(maxdeg, B.maxdeg);
    js_all.merge(B.js);
    if (!first_err && B.err != SBQA_OK) first_err = &B;
  }
  if (!finite) return fail(SBQA_ERR_NOT_FINITE, "J or h not finite");
  if (first_err) return fail(first_err->err, first_err->msg);
  if (!sym) return fail(SBQA_ERR_NOT_SYMMETRIC, "J != J^T");
  sbqa_problem *p = new (std::nothrow) sbqa_problem();
  if (!p) return fail(SBQA_ERR_OOM, "host allocation");
  cudaGetDevice(&p->device);
  p->n = n;
  p->dense = false;
  p->nnz = nnz;
  p->max_degree = maxdeg;
  p->row_ptr.assign(row_ptr, row_ptr + n + 1);
  p->col.assign(col_idx, col_idx + nnz);
  p->val.assign(val, val + nnz);
  if (h) p->h.assign(h, h + n);
  finish_analysis(p, js_all);
  std::vector<int32_t> rp32(n + 1);
  for (int i = 0; i <= n; ++i) rp32[i] = int32_t(row_ptr[i]);
  auto upload = [&]() -> int {
    SBQA_CUDA(p->d_row_ptr.alloc(n + 1));
    SBQA_CUDA(cudaMemcpy(p->d_row_ptr.p, rp32.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (nnz) {
      SBQA_CUDA(p->d_col.alloc(nnz));
      SBQA_CUDA(cudaMemcpy(p->d_col.p, col_idx, nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    int rc = upload_common(p);
    if (rc == SBQA_OK) rc = upload_readout_values(p);
    return rc;
  };
  const int rc = upload();
  if (rc != SBQA_OK) {
    delete p;
    return rc;
  }
  *out = p;
  return SBQA_OK;
}

void sbqa_destroy(sbqa_problem *p) { delete p; }

int sbqa_release_cached_memory(void) {
  return sbqa::devcache_trim() ? SBQA_OK : fail(SBQA_ERR_CUDA, "cudaFree of a cached block failed");
}

int sbqa_get_problem_info(const sbqa_problem *p, sbqa_problem_info *info) {
  if (!p || !info) return fail(SBQA_ERR_INVALID_ARG, "null argument");
  info->n = p->n;
  info->is_dense = p->dense ? 1 : 0;
  info->nnz = p->nnz;
  info->is_integer = p->is_integer ? 1 : 0;
  info->max_abs_j = p->max_abs_j;
  info->c0_auto = p->c0_auto;
  const bool tc_pers = p->use_tc && p->use_tc_persistent && p->tc_persistent_ok();
  int tc_kernel =
      tc_pers ? (p->tc_f4_ok() ? (p->tc_f4_pair_ok() ? 16 : 15) : p->tc_pair_ok() ? 9 : p->tc_split_ok() ? 8 : 5)
              : 2;
  if (p->tc_op == kTcOpBf16) tc_kernel = tc_pers ? 11 : 10;
  if (p->tc_op == kTcOpBsb) tc_kernel = tc_pers ? 13 : 12;
  info->step_kernel = !p->begun ? -1
                     : p->use_tc ? tc_kernel
                     : p->ballistic() ? (p->dense ? 7 : p->use_persistent && p->persistent_ok() ? 14 : 6)
                     : p->small_path ? 3
                     : (p->dense ? 1 : (p->use_persistent ? 4 : 0));
  info->persistent_ms = p->use_tc ? p->tc_persistent_ms : p->persistent_ms;
  info->step_variant = p->dense ? -1 : p->csr_variant;
  for (int v = 0; v < 8; ++v) info->variant_ms[v] = p->use_tc ? (v == 0 ? p->tc_step_ms : 0.f) : p->variant_ms[v];
  info->j_on_device = p->j_on_device ? 1 : 0;
  return SBQA_OK;
}

int sbqa_set_schedule(sbqa_problem *p, const sbqa_params *q) {
  if (!p || !q) return fail(SBQA_ERR_INVALID_ARG, "null argument");
  const double v[6] = {q->a0, q->c0, q->dt, q->gamma0, q->delta_slope, q->init_amp};
  if (!finite_all(v, 6)) return fail(SBQA_ERR_NOT_FINITE, "non-finite parameter");
  if (q->a0 <= 0 || q->dt <= 0 || q->gamma0 <= 0 || q->delta_slope < 0 || q->init_amp < 0 || q->init_amp > 1)
    return fail(SBQA_ERR_INVALID_ARG, "need a0, dt, gamma0 > 0, delta_slope >= 0, 0 <= init_amp <= 1");
  if (q->variant != SBQA_VARIANT_THRESHOLD && q->variant != SBQA_VARIANT_BALLISTIC)
    return fail(SBQA_ERR_INVALID_ARG, "variant must be SBQA_VARIANT_THRESHOLD or SBQA_VARIANT_BALLISTIC");
  if (q->precision < SBQA_PREC_AUTO || q->precision > SBQA_PREC_BF16) return fail(SBQA_ERR_INVALID_ARG, "bad precision");
  if (q->precision == SBQA_PREC_EXACT && (!p->j_integer || p->max_abs_j > kExactMaxAbsJ))
    return fail(SBQA_ERR_UNSUPPORTED, "EXACT precision needs integer J with |J_ij| <= 256");
  if (q->eval_every < 0 || q->n_runs < 0) return fail(SBQA_ERR_INVALID_ARG, "negative eval_every or n_runs");
  if (q->kernel_select < 0 || q->kernel_select > 15) return fail(SBQA_ERR_INVALID_ARG, "kernel_select must be 0..15");
  if (q->n_runs > 0 && (!q->beta || !q->alpha)) return fail(SBQA_ERR_INVALID_ARG, "beta/alpha missing");
  std::vector<double> beta, alpha;
  if (q->n_runs > 0) {
    if (!finite_all(q->beta, q->n_runs) || !finite_all(q->alpha, q->n_runs)) return fail(SBQA_ERR_NOT_FINITE, "beta/alpha");
    for (int r = 0; r < q->n_runs; ++r)
      if (q->beta[r] <= 0 || q->alpha[r] <= 0) return fail(SBQA_ERR_INVALID_ARG, "beta, alpha must be > 0");
    beta.assign(q->beta, q->beta + q->n_runs);
    alpha.assign(q->alpha, q->alpha + q->n_runs);
  }
  p->prm = *q;
  p->prm.beta = nullptr;
  p->prm.alpha = nullptr;
  p->beta.swap(beta);
  p->alpha.swap(alpha);
  p->have_params = true;
  ++p->params_version;
  return SBQA_OK;
}

int sbqa_run_begin(sbqa_problem *p, int32_t steps, int32_t P, int32_t R, uint64_t seed, void *stream) {
  int rc = check_run_args(p, steps, P, R);
  if (rc != SBQA_OK) return rc;
  DeviceGuard g(p->device);
  p->small_path = false;
  p->stream = static_cast<cudaStream_t>(stream);
  p->begun = p->finished = false;
  rc = p->dense ? prepare_dense_values(p, p->prm.precision) : prepare_sparse_values(p, p->prm.precision);
  if (rc != SBQA_OK) return rc;
  if ((rc = alloc_run(p, steps, P, R)) != SBQA_OK) return rc;
  if ((rc = build_tables(p)) != SBQA_OK) return rc;
  if ((rc = autotune_csr(p)) != SBQA_OK) return rc;
  if ((rc = autotune_tc(p)) != SBQA_OK) return rc;
  const StateView s = p->state();
  SBQA_CUDA(cudaMemsetAsync(p->d_err.p, 0, sizeof(int), p->stream));
  SBQA_CUDA(launch_init(s, seed, float(p->prm.init_amp), 0.0f, p->stream));
  if (p->use_tc) SBQA_CUDA(launch_f_to_ft(s, 0, p->d_FT.p, p->Kp, 0, p->tc_op, p->stream));
  if (p->tc_f4_ok()) SBQA_CUDA(launch_f_to_ft4(s, 0, p->d_FT4.p, p->Kp, 0, p->stream));
  if (p->ballistic() && !p->use_tc) SBQA_CUDA(launch_copy_fx(s, 0, p->stream));
  SBQA_CUDA(launch_reset_best(s, p->best(), p->stream));
  p->step_done = 0;
  p->begun = true;
  return SBQA_OK;
}

int sbqa_run_advance(sbqa_problem *p, int32_t n_steps) {
  if (!p) return fail(SBQA_ERR_INVALID_ARG, "null problem");
  if (!p->begun || p->finished) return fail(SBQA_ERR_STATE, "no run in progress");
  if (n_steps < 0) return fail(SBQA_ERR_INVALID_ARG, "n_steps must be >= 0");
  DeviceGuard g(p->device);
  const int n1 = int(std::min<int64_t>(int64_t(p->step_done) + n_steps, p->S));
  SBQA_CUDA(issue_range(p, p->step_done, n1, p->stream));
  p->step_done = n1;
  return SBQA_OK;
}

int sbqa_run_finish(sbqa_problem *p) {
  if (!p) return fail(SBQA_ERR_INVALID_ARG, "null problem");
  if (!p->begun || p->finished) return fail(SBQA_ERR_STATE, "no run in progress");
  if (p->step_done != p->S) return fail(SBQA_ERR_STATE, "run has steps left");
  DeviceGuard g(p->device);
  SBQA_CUDA(issue_readout(p, p->S - 1, p->stream));
  p->finished = true;
  return SBQA_OK;
}

int sbqa_run(sbqa_problem *p, int32_t steps, int32_t P, int32_t R, uint64_t seed, void *stream) {
  // small integer dense instances: the whole solve in one launch
  if (p && p->have_params && p->dense && p->is_integer && p->prm.eval_every == 0 &&
      !p->ballistic() && check_run_args(p, steps, P, R) == SBQA_OK && run_width(P) == P && P <= 32 &&
      small_eligible(p->n, P, steps)) {
    DeviceGuard g(p->device);
    p->stream = static_cast<cudaStream_t>(stream);
    p->begun = p->finished = false;
    int rc = prepare_dense_values(p, p->prm.precision);
    if (rc == SBQA_OK && !p->use_tc) {
      if ((rc = alloc_run(p, steps, P, R)) != SBQA_OK) return rc;
      if ((rc = build_tables(p)) != SBQA_OK) return rc;
      SmallArgs a{};
      a.N = p->n; a.P = P; a.R = R; a.S = steps; a.Cp = p->Cp; a.seed = seed;
      a.amp = float(p->prm.init_amp); a.kc = p->tables.kc; a.kx = p->tables.kx;
      a.J = p->d_dense_f32.p; a.ka = p->d_ka.p; a.dl = p->d_dl.p; a.kj = p->d_kj.p; a.h = p->d_h.p;
      a.J_i32 = p->d_e_i32.p; a.h_i64 = p->d_h_i64.p;
      a.x = p->d_x.p; a.y = p->d_y.p; a.Sg = p->d_Sg.p; a.e_int = p->d_ei.p; a.e_f64 = p->d_ef.p;
      a.best_e_int = p->d_best_ei.p; a.best_e = p->d_best_e.p; a.best_k = p->d_best_k.p;
      a.best_step = p->d_best_step.p; a.have_best = p->d_have.p; a.best_spins = p->d_best_spins.p;
      SBQA_CUDA(cudaMemsetAsync(p->d_err.p, 0, sizeof(int), p->stream));
      SBQA_CUDA(launch_solve_small(a, p->stream));
      p->step_done = steps;
      p->begun = p->finished = true;
      p->small_path = true;
      return SBQA_OK;
    }
    if (rc != SBQA_OK) return rc;
  }
  int rc = sbqa_run_begin(p, steps, P, R, seed, stream);
  if (rc != SBQA_OK) return rc;
  DeviceGuard g(p->device);
  if ((p->use_persistent && p->persistent_ok()) || (p->use_tc_persistent && p->tc_persistent_ok())) {
    // no graph: one launch covers the steps
    SBQA_CUDA(issue_range(p, 0, steps, p->stream));
    SBQA_CUDA(issue_readout(p, steps - 1, p->stream));
    p->step_done = steps;
    p->finished = true;
    return SBQA_OK;
  }
  sbqa_problem::Key key;
  key.S = steps; key.P = P; key.R = R; key.eval = p->prm.eval_every; key.kind = p->kind;
  key.dense = p->dense ? 1 : 0; key.x = p->d_x.p; key.kj = p->d_kj.p;
  key.kc = p->tables.kc; key.kx = p->tables.kx; key.tc = p->use_tc ? 1 + p->tc_op : 0; key.variant = p->csr_variant;
  key.fvar = p->prm.variant;
  if (!(p->graph && p->graph_key == key)) {
    if (p->graph) {
      cudaGraphExecDestroy(p->graph);
      p->graph = nullptr;
    }
    if (!p->cap_stream) SBQA_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    SBQA_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = issue_range(p, 0, steps, p->cap_stream);
    if (e == cudaSuccess) e = issue_readout(p, steps - 1, p->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(SBQA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&p->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      p->graph = nullptr;
      return fail(SBQA_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    p->graph_key = key;
  }
  SBQA_CUDA(cudaGraphLaunch(p->graph, p->stream));
  p->step_done = steps;
  p->finished = true;
  return SBQA_OK;
}

int sbqa_synchronize(sbqa_problem *p) {
  if (!p) return fail(SBQA_ERR_INVALID_ARG, "null problem");
  DeviceGuard g(p->device);
  SBQA_CUDA(p->stream ? cudaStreamSynchronize(p->stream) : cudaDeviceSynchronize());
  SBQA_CUDA(cudaGetLastError());
  if (p->d_err.p) {
    int err = 0;
    SBQA_CUDA(cudaMemcpy(&err, p->d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (err != 0) return fail(SBQA_ERR_TIMEOUT, "a bounded device wait gave up (code " + std::to_string(err) + ")");
  }
  return SBQA_OK;
}

int sbqa_get_best(sbqa_problem *p, int8_t *spins, double *energy, int64_t *energy_int, int32_t *replica,
                  int32_t *step) {
  if (!p) return fail(SBQA_ERR_INVALID_ARG, "null problem");
  if (!p->finished) return fail(SBQA_ERR_STATE, "no finished readout");
  int rc = sbqa_synchronize(p);
  if (rc != SBQA_OK) return rc;
  DeviceGuard g(p->device);
  const int R = p->R;
  if (spins) SBQA_CUDA(cudaMemcpy(spins, p->d_best_spins.p, size_t(R) * p->n, cudaMemcpyDeviceToHost));
  if (energy) SBQA_CUDA(cudaMemcpy(energy, p->d_best_e.p, R * sizeof(double), cudaMemcpyDeviceToHost));
  if (energy_int && p->is_integer)
    SBQA_CUDA(cudaMemcpy(energy_int, p->d_best_ei.p, R * sizeof(int64_t), cudaMemcpyDeviceToHost));
  if (replica) SBQA_CUDA(cudaMemcpy(replica, p->d_best_k.p, R * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (step) SBQA_CUDA(cudaMemcpy(step, p->d_best_step.p, R * sizeof(int32_t), cudaMemcpyDeviceToHost));
  return SBQA_OK;
}

int sbqa_get_energies(sbqa_problem *p, double *energy, int64_t *energy_int) {
  if (!p) return fail(SBQA_ERR_INVALID_ARG, "null problem");
  if (!p->finished) return fail(SBQA_ERR_STATE, "no finished readout");
  int rc = sbqa_synchronize(p);
  if (rc != SBQA_OK) return rc;
  DeviceGuard g(p->device);
  // device energies by column r * Ps + k; the caller gets [r][k] for k < P
  auto gather = [&](auto *out, const auto *dev) -> int {
    using T = std::remove_pointer_t<decltype(out)>;
    std::vector<T> buf(size_t(p->C));
    SBQA_CUDA(cudaMemcpy(buf.data(), dev, size_t(p->C) * sizeof(T), cudaMemcpyDeviceToHost));
    for (int r = 0; r < p->R; ++r)
      for (int k = 0; k < p->P; ++k) out[size_t(r) * p->P + k] = buf[size_t(r) * p->Ps + k];
    return SBQA_OK;
  };
  if (energy && (rc = gather(energy, p->d_ef.p)) != SBQA_OK) return rc;
  if (energy_int && p->is_integer && (rc = gather(energy_int, p->d_ei.p)) != SBQA_OK) return rc;
  return SBQA_OK;
}

int sbqa_get_state(sbqa_problem *p, float *x, float *y, int32_t *step_done) {
  if (!p) return fail(SBQA_ERR_INVALID_ARG, "null problem");
  if (!p->begun) return fail(SBQA_ERR_STATE, "no run");
  int rc = sbqa_synchronize(p);
  if (rc != SBQA_OK) return rc;
  DeviceGuard g(p->device);
  const size_t NC = size_t(p->n) * p->Cp;
  std::vector<float> buf(NC);
  float *outs[2] = {x, y};
  const float *src[2] = {p->d_x.p, p->d_y.p};
  for (int w = 0; w < 2; ++w) {
    if (!outs[w]) continue;
    SBQA_CUDA(cudaMemcpy(buf.data(), src[w], NC * sizeof(float), cudaMemcpyDeviceToHost));
    for (int r = 0; r < p->R; ++r)
      for (int k = 0; k < p->P; ++k) {
        const size_t c = size_t(r) * p->Ps + k, o = (size_t(r) * p->P + k) * p->n;
        for (int i = 0; i < p->n; ++i) outs[w][o + i] = buf[size_t(i) * p->Cp + c];
      }
  }
  if (step_done) *step_done = p->step_done;
  return SBQA_OK;
}

int sbqa_set_state(sbqa_problem *p, const float *x, const float *y, int32_t step_done) {
  if (!p || !x || !y) return fail(SBQA_ERR_INVALID_ARG, "null argument");
  if (!p->begun) return fail(SBQA_ERR_STATE, "no run");
  if (step_done < 0 || step_done > p->S) return fail(SBQA_ERR_INVALID_ARG, "step_done out of range");
  int rc = sbqa_synchronize(p);
  if (rc != SBQA_OK) return rc;
  DeviceGuard g(p->device);
  const size_t NC = size_t(p->n) * p->Cp;
  std::vector<float> bx(NC, 0.f), by(NC, 0.f);  // padding columns of a run stay at zero
  for (int r = 0; r < p->R; ++r)
    for (int k = 0; k < p->P; ++k) {
      const size_t c = size_t(r) * p->Ps + k, o = (size_t(r) * p->P + k) * p->n;
      for (int i = 0; i < p->n; ++i) {
        bx[size_t(i) * p->Cp + c] = x[o + i];
        by[size_t(i) * p->Cp + c] = y[o + i];
      }
    }
  SBQA_CUDA(cudaMemcpy(p->d_x.p, bx.data(), NC * sizeof(float), cudaMemcpyHostToDevice));
  SBQA_CUDA(cudaMemcpy(p->d_y.p, by.data(), NC * sizeof(float), cudaMemcpyHostToDevice));
  const double tau = p->S > 0 ? double(step_done) / double(p->S) : 0.0;
  SBQA_CUDA(launch_refresh_f(p->state(), step_done & 1, float(p->prm.delta_slope * tau), p->stream));
  if (p->use_tc)
    SBQA_CUDA(launch_f_to_ft(p->state(), step_done & 1, p->d_FT.p, p->Kp, step_done & 1, p->tc_op, p->stream));
  if (p->tc_f4_ok())
    SBQA_CUDA(launch_f_to_ft4(p->state(), step_done & 1, p->d_FT4.p, p->Kp, step_done & 1, p->stream));
  if (p->ballistic() && !p->use_tc) SBQA_CUDA(launch_copy_fx(p->state(), step_done & 1, p->stream));
  p->step_done = step_done;
  p->finished = false;
  return SBQA_OK;
}

}  // extern "C"
