// solve_persistent.cu -- all steps of a CSR run batch in one cooperative launch.
//
// For rows of degree <= 8 (+-1, FP32 or BF16 couplings).  The grid is exactly
// as large as can be co-resident; every warp owns fixed work items (spin row,
// chunk of 32 W replica columns, W = 4 or 8) for the whole anneal --
// individual items, or whole rows with all their chunks when the items
// outnumber the cache.  Before the first step a warp copies the column
// indices (and signs or values) of its rows into shared memory, so a step
// needs no index loads: per item it gathers the f codes of the (at most 8)
// neighbours and the x, y of its columns, sums (same arithmetic and order as
// k_step_csr), updates and writes x, y and the next codes.  The codes
// written by other blocks are read through L2 (ld.global.cg), never the
// non-coherent path.  Between steps all blocks meet at a grid barrier; the
// wait is bounded (1 s, or at once when another block has already failed):
// a block that gives up records an error and stops stepping, so a broken
// grid ends with a status the host reads.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "grid_sync.cuh"
#include "step_common.cuh"

namespace sbqa {

constexpr int kPersistMaxDeg = 8;
constexpr size_t kPersistSmem = 46080;  // per block: under the 48 KB default with the static barrier flag

struct PersistArgs {
  StateView s;
  const int32_t *row_ptr, *col, *npos;  // CSR (+-1: each row's +1 entries first)
  const void *val;                      // FP32 or BF16 values (not +-1)
  const float *h;
  // ELL form (mode 3: the items beyond a warp's cache read their neighbours here)
  const int32_t *ell_col, *ell_meta;
  const float *ell_val;
  StepTables t;
  int n_begin, n_end;
  unsigned *bar;  // grid barrier counters (persistent_barrier_words(), zeroed before the launch)
  int *err;       // error flag
  int skip_step;  // test hook: block 0 does not arrive at the barrier after this step (-1: never)
  int cache_cap;  // items (or rows) a warp caches at most
};

// Cache entries.  Items mode: one (row, chunk) item.  Rows mode: one row; its
// index is gw + q * warps for the warp's q-th row.  (degree | +1 count << 8)
// packed in degpos; values only for FP32 / BF16 couplings.
template <bool VALS>
struct ItemEntry {
  int32_t col[kPersistMaxDeg];
  int32_t row, chunk;
  uint32_t degpos;
};
template <>
struct ItemEntry<true> {
  int32_t col[kPersistMaxDeg];
  float val[kPersistMaxDeg];
  int32_t row, chunk;
  uint32_t degpos;
};
template <bool VALS>
struct RowEntry {
  int32_t col[kPersistMaxDeg];
  uint32_t degpos;
};
template <>
struct RowEntry<true> {
  int32_t col[kPersistMaxDeg];
  float val[kPersistMaxDeg];
  uint32_t degpos;
};

template <bool ROWS, bool VALS>
struct Cache {
  using Entry = typename std::conditional<ROWS, RowEntry<VALS>, ItemEntry<VALS>>::type;
  static constexpr int kPerWarp = int(kPersistSmem / 8 / sizeof(Entry));
};

// W bytes of f codes (one 4- or 8-byte load through L2: other blocks wrote
// these codes in this launch).
template <int W>
struct Codes;
template <>
struct Codes<4> {
  uint32_t w[1];
  __device__ __forceinline__ void load(const uint8_t *p) { w[0] = __ldcg(reinterpret_cast<const uint32_t *>(p)); }
  __device__ __forceinline__ void zero(uint32_t z) { w[0] = z; }
};
template <>
struct Codes<8> {
  uint32_t w[2];
  __device__ __forceinline__ void load(const uint8_t *p) {
    const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(p));
    w[0] = v.x;
    w[1] = v.y;
  }
  __device__ __forceinline__ void zero(uint32_t z) { w[0] = w[1] = z; }
};

// One item: x, y of the lane's W columns and the f codes of the row's
// neighbours for those columns (issued together), the coupling sums (+-1:
// packed code sums per sign; otherwise FP32 FMAs in entry order, as
// k_step_csr), the update and the stores.
// LPI lanes own one item of LPI * W columns: the whole warp (32), or half of
// it (16: the warp works on two items at once, lanes 16-31 on the second;
// act = false leaves a half without an item idle but in the shuffles).
template <int P, int KIND, int W, bool GEN, int LPI = 32>
__device__ __forceinline__ void persist_item(const PersistArgs &a, int i, int chunk, const int32_t *col,
                                             const float *val, uint32_t degpos, const uint8_t *Fin, uint8_t *Fout,
                                             float ka, float dnext, int n, int lane, bool act = true) {
  const StateView &s = a.s;
  const int deg = act ? int(degpos & 0xffu) : 0, npos = int(degpos >> 8);
  const int c0 = chunk * LPI * W + (lane % LPI) * W;
  const size_t off = size_t(i) * s.Cp + c0;
  float xs[W], ys[W];
#pragma unroll
  for (int u = 0; u < W / 4; ++u) {
    const float4 xa = *reinterpret_cast<const float4 *>(s.x + off + 4 * u);
    const float4 ya = *reinterpret_cast<const float4 *>(s.y + off + 4 * u);
    xs[4 * u] = xa.x; xs[4 * u + 1] = xa.y; xs[4 * u + 2] = xa.z; xs[4 * u + 3] = xa.w;
    ys[4 * u] = ya.x; ys[4 * u + 1] = ya.y; ys[4 * u + 2] = ya.z; ys[4 * u + 3] = ya.w;
  }
  Codes<W> f[kPersistMaxDeg];
#pragma unroll
  for (int e = 0; e < kPersistMaxDeg; ++e) {
    if (e < deg) f[e].load(Fin + size_t(col[e]) * s.Cp + c0);
    else f[e].zero(KIND == VAL_PM1 ? 0u : kFZero4);
  }
  float G[W];
  if constexpr (KIND == VAL_PM1) {
    uint32_t ap[W / 4], am[W / 4];
#pragma unroll
    for (int q = 0; q < W / 4; ++q) ap[q] = am[q] = 0;
#pragma unroll
    for (int e = 0; e < kPersistMaxDeg; ++e) {
      if (e < npos) {
#pragma unroll
        for (int q = 0; q < W / 4; ++q) ap[q] += f[e].w[q];
      } else {
#pragma unroll
        for (int q = 0; q < W / 4; ++q) am[q] += f[e].w[q];
      }
    }
    const int bias = (deg - npos) - npos;  // codes carry f + 1; missing entries add 0
#pragma unroll
    for (int c = 0; c < W; ++c)
      G[c] = float(int((ap[c / 4] >> (8 * (c % 4))) & 0xffu) - int((am[c / 4] >> (8 * (c % 4))) & 0xffu) + bias);
  } else {
#pragma unroll
    for (int c = 0; c < W; ++c) G[c] = 0.f;
#pragma unroll
    for (int e = 0; e < kPersistMaxDeg; ++e) {
      if (e < deg) {
        const float w = val[e];
        acc_codes<W>(G, w, f[e].w);
      }
    }
  }
  // an idle half takes part in the ring shuffles only (a column past C stores nothing)
  sb_updateW<P, W, GEN>(s, a.t, ka, dnext, n, i, act ? c0 : s.C, G, __ldg(a.h + i), xs, ys, Fout);
}

template <int KIND>
__device__ __forceinline__ float entry_value(const PersistArgs &a, int e) {
  if constexpr (KIND == VAL_F32) return static_cast<const float *>(a.val)[e];
  else return __bfloat162float(static_cast<const __nv_bfloat16 *>(a.val)[e]);
}

// ROWS = false: warp items (row, chunk) cached; true: whole rows cached.
// LPI = 16 (items mode, W = 8): a half warp per item of 128 columns, two
// items per warp at a time -- twice the items in flight per warp and half the
// per-item instructions of W = 4 on a whole warp, same arithmetic per column.
template <int P, bool ROWS, int KIND, int W, int LPI = 32>
__global__ void __launch_bounds__(256, 4) k_solve_csr_persistent(PersistArgs a) {
  constexpr bool VALS = KIND != VAL_PM1;
  using C = Cache<ROWS, VALS>;
  using Entry = typename C::Entry;
  extern __shared__ int32_t s_cache[];  // [8 warps][C::kPerWarp] entries
  const StateView &s = a.s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunks = s.Cp / (LPI * W);
  const int warps_total = gridDim.x * 8;
  const int gw = blockIdx.x * 8 + warp;
  Entry *mine = reinterpret_cast<Entry *>(s_cache) + warp * C::kPerWarp;
  int my_count = 0;
  const int n_units = ROWS ? s.N : s.N * chunks;
  const int cap = C::kPerWarp < a.cache_cap ? C::kPerWarp : a.cache_cap;
  for (int u = gw; u < n_units && my_count < cap; u += warps_total, ++my_count) {
    if (lane == 0) {
      const int row = ROWS ? u : u / chunks;
      const int e0 = a.row_ptr[row], e1 = a.row_ptr[row + 1];
      Entry &m = mine[my_count];
      if constexpr (!ROWS) {
        m.row = row;
        m.chunk = u - row * chunks;
      }
      m.degpos = uint32_t(e1 - e0) | (uint32_t(KIND == VAL_PM1 ? a.npos[row] : e1 - e0) << 8);
      for (int q = 0; q < kPersistMaxDeg; ++q) {
        m.col[q] = q < e1 - e0 ? a.col[e0 + q] : 0;
        if constexpr (VALS) m.val[q] = q < e1 - e0 ? entry_value<KIND>(a, e0 + q) : 0.f;
      }
    }
  }
  __syncwarp();
  unsigned k = 0;
  // replica counts below the run width take the general ring (one form per launch)
  const bool gen = P > 2 && s.Pr != P;
  for (int n = a.n_begin; n < a.n_end; ++n) {
    const uint8_t *Fin = s.f_of(n);
    uint8_t *Fout = s.f_of(n + 1);
    const float ka = __ldg(a.t.ka + n), dnext = __ldg(a.t.dl + n + 1);
    for (int q = 0; q < my_count; ++q) {
      const Entry &m = mine[q];
      const float *val = nullptr;
      if constexpr (VALS) val = m.val;
      if constexpr (ROWS) {
        for (int ch = 0; ch < chunks; ++ch) {
          if (gen)
            persist_item<P, KIND, W, true>(a, gw + q * warps_total, ch, m.col, val, m.degpos, Fin, Fout, ka, dnext,
                                           n, lane);
          else
            persist_item<P, KIND, W, false>(a, gw + q * warps_total, ch, m.col, val, m.degpos, Fin, Fout, ka, dnext,
                                            n, lane);
        }
      } else if constexpr (LPI == 32) {
        if (gen)
          persist_item<P, KIND, W, true>(a, m.row, m.chunk, m.col, val, m.degpos, Fin, Fout, ka, dnext, n, lane);
        else
          persist_item<P, KIND, W, false>(a, m.row, m.chunk, m.col, val, m.degpos, Fin, Fout, ka, dnext, n, lane);
      } else {
        // lanes 16-31 take the next entry (idle past the warp's last one)
        const int qq = q + (lane >> 4);
        const bool act = qq < my_count;
        const Entry &mh = mine[act ? qq : q];
        const float *valh = nullptr;
        if constexpr (VALS) valh = mh.val;
        if (gen)
          persist_item<P, KIND, W, true, LPI>(a, mh.row, mh.chunk, mh.col, valh, mh.degpos, Fin, Fout, ka, dnext, n,
                                              lane, act);
        else
          persist_item<P, KIND, W, false, LPI>(a, mh.row, mh.chunk, mh.col, valh, mh.degpos, Fin, Fout, ka, dnext,
                                               n, lane, act);
        ++q;  // two entries per pass
      }
    }
    if constexpr (!ROWS) {
      // items past the warp's cache (mode 3): neighbours from the ELL arrays
      for (int u0 = gw + my_count * warps_total; u0 < n_units; u0 += (32 / LPI) * warps_total) {
        const int uh = u0 + (LPI == 16 ? (lane >> 4) * warps_total : 0);
        const bool act = uh < n_units;
        const int u = act ? uh : u0;
        const int row = u / chunks, ch = u - row * chunks;
        const int2 meta = __ldg(reinterpret_cast<const int2 *>(a.ell_meta) + row);
        const uint32_t dp = uint32_t(meta.x) | (uint32_t(KIND == VAL_PM1 ? meta.y : meta.x) << 8);
        const int32_t *colp = a.ell_col + size_t(row) * kPersistMaxDeg;
        const float *valp = VALS ? a.ell_val + size_t(row) * kPersistMaxDeg : nullptr;
        if (gen)
          persist_item<P, KIND, W, true, LPI>(a, row, ch, colp, valp, dp, Fin, Fout, ka, dnext, n, lane, act);
        else
          persist_item<P, KIND, W, false, LPI>(a, row, ch, colp, valp, dp, Fin, Fout, ka, dnext, n, lane, act);
      }
    }
    if (!grid_barrier(a.bar, ++k, a.err, n == a.skip_step && blockIdx.x == 0)) break;
  }
}

// The ballistic form f(x) = x (the bSB choice named in Sec. II A): the same
// persistent scheme in items mode with items of 128 columns on whole warps
// (4 columns per lane), gathering the neighbours' FP32 positions of the step
// before (written by other blocks: read through L2).  The sum runs over the
// row's eight cache slots in order, a zero weight and a zero position past the
// degree -- the sequence of fused multiply-adds of k_step_csr_bsb -- and the
// update is sb_update4_bsb, so results equal the per-step kernel bit for bit.
template <int P, int KIND>
__global__ void __launch_bounds__(256, 4) k_solve_csr_persistent_bsb(PersistArgs a) {
  constexpr bool VALS = KIND != VAL_PM1;
  using C = Cache<false, VALS>;
  using Entry = typename C::Entry;
  extern __shared__ int32_t s_cache[];
  const StateView &s = a.s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunks = s.Cp / kColsPerWarp;
  const int warps_total = gridDim.x * 8;
  const int gw = blockIdx.x * 8 + warp;
  Entry *mine = reinterpret_cast<Entry *>(s_cache) + warp * C::kPerWarp;
  int my_count = 0;
  const int n_units = s.N * chunks;
  const int cap = C::kPerWarp < a.cache_cap ? C::kPerWarp : a.cache_cap;
  for (int u = gw; u < n_units && my_count < cap; u += warps_total, ++my_count) {
    if (lane == 0) {
      const int row = u / chunks;
      const int e0 = a.row_ptr[row], e1 = a.row_ptr[row + 1];
      Entry &m = mine[my_count];
      m.row = row;
      m.chunk = u - row * chunks;
      m.degpos = uint32_t(e1 - e0) | (uint32_t(KIND == VAL_PM1 ? a.npos[row] : e1 - e0) << 8);
      for (int q = 0; q < kPersistMaxDeg; ++q) {
        m.col[q] = q < e1 - e0 ? a.col[e0 + q] : 0;
        if constexpr (VALS) m.val[q] = q < e1 - e0 ? entry_value<KIND>(a, e0 + q) : 0.f;
      }
    }
  }
  __syncwarp();
  unsigned k = 0;
  for (int n = a.n_begin; n < a.n_end; ++n) {
    const float *Fin = s.fx_of(n);
    float *Fout = s.fx_of(n + 1);
    for (int q = 0; q < my_count; ++q) {
      const Entry &m = mine[q];
      const int i = m.row, c4 = m.chunk * kColsPerWarp + lane * 4;
      const size_t off = size_t(i) * s.Cp + c4;
      const float4 xv = *reinterpret_cast<const float4 *>(s.x + off);
      const float4 yv = *reinterpret_cast<const float4 *>(s.y + off);
      const int deg = int(m.degpos & 0xffu), npos = int(m.degpos >> 8);
      float4 f[kPersistMaxDeg];
#pragma unroll
      for (int e = 0; e < kPersistMaxDeg; ++e)
        f[e] = e < deg ? __ldcg(reinterpret_cast<const float4 *>(Fin + size_t(m.col[e]) * s.Cp + c4))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
      float g[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int e = 0; e < kPersistMaxDeg; ++e) {
        float w = 0.f;
        if (e < deg) {
          if constexpr (VALS) w = m.val[e];
          else w = e < npos ? 1.f : -1.f;
        }
        g[0] = fmaf(w, f[e].x, g[0]);
        g[1] = fmaf(w, f[e].y, g[1]);
        g[2] = fmaf(w, f[e].z, g[2]);
        g[3] = fmaf(w, f[e].w, g[3]);
      }
      sb_update4_bsb<P>(s, a.t, n, i, c4, g, __ldg(a.h + i), xv, yv, Fout);
    }
    if (!grid_barrier(a.bar, ++k, a.err, n == a.skip_step && blockIdx.x == 0)) break;
  }
}

template <int KIND>
static const void *persistent_bsb_fn_k(int P) {
  switch (P) {
    case 1: return (const void *)k_solve_csr_persistent_bsb<1, KIND>;
    case 2: return (const void *)k_solve_csr_persistent_bsb<2, KIND>;
    case 4: return (const void *)k_solve_csr_persistent_bsb<4, KIND>;
    case 8: return (const void *)k_solve_csr_persistent_bsb<8, KIND>;
    case 16: return (const void *)k_solve_csr_persistent_bsb<16, KIND>;
    case 32: return (const void *)k_solve_csr_persistent_bsb<32, KIND>;
    case 64: return (const void *)k_solve_csr_persistent_bsb<64, KIND>;
    case 128: return (const void *)k_solve_csr_persistent_bsb<128, KIND>;
    default: return nullptr;
  }
}

static const void *persistent_bsb_fn(int P, int kind) {
  switch (kind) {
    case VAL_PM1: return persistent_bsb_fn_k<VAL_PM1>(P);
    case VAL_F32: return persistent_bsb_fn_k<VAL_F32>(P);
    default: return persistent_bsb_fn_k<VAL_BF16>(P);
  }
}

// Items mode with 128-column items (W = 4 on a whole warp) runs as W = 8 on
// half warps (LPI = 16); rows mode and 256-column items keep LPI = 32.
template <bool ROWS, int KIND, int W>
static const void *persistent_fn_p(int P) {
  constexpr bool HALF = !ROWS && W == 4;
  constexpr int WK = HALF ? 8 : W, LPI = HALF ? 16 : 32;
  switch (P) {
    case 1: return (const void *)k_solve_csr_persistent<1, ROWS, KIND, WK, LPI>;
    case 2: return (const void *)k_solve_csr_persistent<2, ROWS, KIND, WK, LPI>;
    case 4: return (const void *)k_solve_csr_persistent<4, ROWS, KIND, WK, LPI>;
    case 8: return (const void *)k_solve_csr_persistent<8, ROWS, KIND, WK, LPI>;
    case 16: return (const void *)k_solve_csr_persistent<16, ROWS, KIND, WK, LPI>;
    case 32: return (const void *)k_solve_csr_persistent<32, ROWS, KIND, WK, LPI>;
    case 64: return (const void *)k_solve_csr_persistent<64, ROWS, KIND, WK, LPI>;
    case 128: return (const void *)k_solve_csr_persistent<128, ROWS, KIND, WK, LPI>;
    default: return nullptr;
  }
}

template <bool ROWS, int W>
static const void *persistent_fn_k(int P, int kind) {
  switch (kind) {
    case VAL_PM1: return persistent_fn_p<ROWS, VAL_PM1, W>(P);
    case VAL_F32: return persistent_fn_p<ROWS, VAL_F32, W>(P);
    default: return persistent_fn_p<ROWS, VAL_BF16, W>(P);
  }
}

static const void *persistent_fn(int P, bool rows, int kind, int W) {
  if (W == 8) return rows ? persistent_fn_k<true, 8>(P, kind) : persistent_fn_k<false, 8>(P, kind);
  return rows ? persistent_fn_k<true, 4>(P, kind) : persistent_fn_k<false, 4>(P, kind);
}

static int per_warp(bool rows, int kind) {
  const bool vals = kind != VAL_PM1;
  if (rows) return vals ? Cache<true, true>::kPerWarp : Cache<true, false>::kPerWarp;
  return vals ? Cache<false, true>::kPerWarp : Cache<false, false>::kPerWarp;
}

// W = 8 columns per lane when R * P allows it, else 4.
static int persist_w(int Cp) { return Cp % 256 == 0 ? 8 : (Cp % 128 == 0 ? 4 : 0); }

int persistent_barrier_words() { return int(kBarStride * (kBarGroups + 1)); }

// Test hook: SBQA_TEST_PERSIST_CACHE=k caches at most k items or rows per
// warp, so that small instances take mode 3 (not for production use).
static int cache_cap_hook() {
  const char *v = std::getenv("SBQA_TEST_PERSIST_CACHE");
  const int k = v ? std::atoi(v) : 0;
  return k > 0 ? k : (1 << 30);
}

int persistent_blocks() {
  int dev = 0, sms = 0, best = 1 << 30;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the smallest co-resident count over all instantiations, so any of them fits the grid
  const int Ps[8] = {1, 2, 4, 8, 16, 32, 64, 128};
  for (int P : Ps)
    for (int kind = 0; kind < 3; ++kind)
      for (int rows = 0; rows < 2; ++rows)
        for (int W = 4; W <= 8; W += 4) {
          int per_sm = 0;
          if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_fn(P, rows != 0, kind, W), 256,
                                                            kPersistSmem) != cudaSuccess)
            return 0;
          best = per_sm < best ? per_sm : best;
        }
  for (int P : Ps)
    for (int kind = 0; kind < 3; ++kind) {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_bsb_fn(P, kind), 256, kPersistSmem) !=
          cudaSuccess)
        return 0;
      best = per_sm < best ? per_sm : best;
    }
  return sms * best;
}

bool persistent_bsb_ok(int N, int Cp, int max_degree, int kind, int blocks) {
  if (blocks <= 0 || max_degree > kPersistMaxDeg || Cp % kColsPerWarp != 0) return false;
  return (long long)N * (Cp / kColsPerWarp) <= (long long)blocks * 8 * std::min<long long>(per_warp(false, kind),
                                                                                         cache_cap_hook());
}

cudaError_t launch_solve_csr_persistent_bsb(const StateView &s, const CsrView &J, const StepTables &t, int n_begin,
                                            int n_end, unsigned *bar, int *err, int blocks, cudaStream_t st) {
  PersistArgs a;
  a.s = s;
  a.row_ptr = J.row_ptr;
  a.col = J.col;
  a.npos = J.npos;
  a.val = J.val;
  a.h = J.h;
  a.ell_col = J.ell_col;
  a.ell_meta = J.ell_meta;
  a.ell_val = J.ell_val;
  a.t = t;
  a.n_begin = n_begin;
  a.n_end = n_end;
  a.bar = bar;
  a.err = err;
  const char *skip = std::getenv("SBQA_TEST_SKIP_BARRIER_STEP");
  a.skip_step = skip ? std::atoi(skip) : -1;
  a.cache_cap = cache_cap_hook();
  const void *fn = persistent_bsb_fn(s.P, J.kind);
  if (!fn || !persistent_bsb_ok(s.N, s.Cp, kPersistMaxDeg, J.kind, blocks)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(bar, 0, persistent_barrier_words() * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  void *args[] = {&a};
  return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(256), args, kPersistSmem, st);
}


int persistent_mode(int N, int Cp, int max_degree, int kind, int blocks, bool force_rows, bool ell) {
  const int W = persist_w(Cp);
  if (blocks <= 0 || max_degree > kPersistMaxDeg || W == 0) return 0;
  const long long warps = (long long)blocks * 8, cap = cache_cap_hook();
  if (!force_rows && (long long)N * (Cp / (32 * W)) <= warps * std::min<long long>(per_warp(false, kind), cap)) return 1;
  if ((long long)N <= warps * std::min<long long>(per_warp(true, kind), cap)) return 2;
  if (!force_rows && ell) return 3;
  return 0;
}

cudaError_t launch_solve_csr_persistent(const StateView &s, const CsrView &J, const StepTables &t, int n_begin,
                                        int n_end, unsigned *bar, int *err, int blocks, int mode, cudaStream_t st) {
  PersistArgs a;
  a.s = s;
  a.row_ptr = J.row_ptr;
  a.col = J.col;
  a.npos = J.npos;
  a.val = J.val;
  a.h = J.h;
  a.ell_col = J.ell_col;
  a.ell_meta = J.ell_meta;
  a.ell_val = J.ell_val;
  a.t = t;
  a.n_begin = n_begin;
  a.n_end = n_end;
  a.bar = bar;
  a.err = err;
  // test hook for the barrier timeout: SBQA_TEST_SKIP_BARRIER_STEP=n makes block 0
  // skip its arrival after step n of a launch that runs it (not for production use)
  const char *skip = std::getenv("SBQA_TEST_SKIP_BARRIER_STEP");
  a.skip_step = skip ? std::atoi(skip) : -1;
  a.cache_cap = cache_cap_hook();
  void *args[] = {&a};
  const int W = persist_w(s.Cp);
  const void *fn = (mode == 1 || mode == 2 || mode == 3) && W ? persistent_fn(s.P, mode == 2, J.kind, W) : nullptr;
  if (!fn || (mode == 3 && (!J.ell_col || !J.ell_meta || (J.kind != VAL_PM1 && !J.ell_val))))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(bar, 0, persistent_barrier_words() * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(256), args, kPersistSmem, st);
}

}  // namespace sbqa
