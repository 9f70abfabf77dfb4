// solve_persistent.cu -- all steps of a CSR run batch in one cooperative launch.
//
// For +-1 couplings with row degree <= 8.  The grid is exactly as large as
// can be co-resident; every warp owns fixed work items (spin row, chunk of
// 32 W replica columns) for the whole anneal -- individual items, or whole
// rows with all their chunks when the items outnumber the cache.  Before the
// first step a warp copies the column indices and signs of its rows into
// shared memory, so a step needs no index loads: per item it gathers the f codes of the
// (at most 8) neighbours and the x, y of its columns, sums, updates (same
// arithmetic as k_step_csr) and writes x, y and the next codes.  The codes
// written by other blocks are read through L2 (ld.global.cg), never the
// non-coherent path.  Between
// steps all blocks meet at a grid barrier (a counter in global memory); the
// wait is bounded: after kBarrierSpins polls a block records an error and
// stops stepping, so a broken grid ends with a status the host reads.
#include "step_common.cuh"

namespace sbqa {

constexpr int kPersistMaxDeg = 8;
constexpr int kPersistW = 8;                   // columns per lane
constexpr int kPersistMaxItems = 120;  // items per warp in shared memory: 45 KB per block, under the 48 KB default
constexpr unsigned kBarrierSpins = 1u << 24;  // polls per grid barrier (with backoff: seconds)
// Two-level grid barrier: blocks arrive on one of kBarGroups group counters
// (each on its own 128-byte line); the last arrival of a group adds one to
// the global counter, which every block polls.  Counter words: global at 0,
// group g at kBarStride * (g + 1).
constexpr unsigned kBarGroups = 32, kBarStride = 32;

struct PersistArgs {
  StateView s;
  const int32_t *row_ptr, *col, *npos;  // +-1 CSR, each row's +1 entries first
  const float *h;
  StepTables t;
  int n_begin, n_end;
  unsigned *bar;  // grid barrier counters (persistent_barrier_words(), zeroed before the launch)
  int *err;       // error flag
};

struct ItemIdx {
  int32_t col[kPersistMaxDeg];
  int32_t row, chunk, deg, npos;
};

// Rows mode (more items than the item cache holds): a warp owns whole rows,
// gw + q * warps for q = 0, 1, ..., and walks all column chunks of each; only
// the row's neighbours and (degree | +1 count << 8) are cached.
constexpr int kPersistMaxRows = 150;  // 36 B each: 43 KB per block
struct RowIdx {
  int32_t col[kPersistMaxDeg];
  uint32_t degpos;
};

__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned k, int *err) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    const unsigned G = gridDim.x < kBarGroups ? gridDim.x : kBarGroups;
    const unsigned g = blockIdx.x % G;
    const unsigned size_g = (gridDim.x - g + G - 1) / G;  // blocks b with b % G == g
    __threadfence();
    const unsigned old = atomicAdd(bar + kBarStride * (g + 1), 1u);
    if (old + 1 == size_g * k) {  // last arrival of the group
      __threadfence();
      atomicAdd(bar, 1u);
    }
    const unsigned target = G * k;
    unsigned v = 0;
    unsigned it = 0;
    for (; it < kBarrierSpins; ++it) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      __nanosleep(it < 64 ? 32 : 128);
    }
    s_ok = it < kBarrierSpins;
    if (!s_ok) atomicCAS(err, 0, 4);
  }
  __syncthreads();
  return s_ok != 0;
}

// One item: x, y of the lane's columns and the f codes of the row's
// neighbours for those columns (issued together), packed code sums per sign
// (as k_step_csr), the update and the stores.
template <int P>
__device__ __forceinline__ void persist_item(const PersistArgs &a, int i, int chunk, const int32_t *col, int deg,
                                             int npos, const uint8_t *Fin, uint8_t *Fout, float ka, float dnext,
                                             int n, int lane) {
  const StateView &s = a.s;
  const int c0 = chunk * 32 * kPersistW + lane * kPersistW;
  const size_t off = size_t(i) * s.Cp + c0;
  float xs[kPersistW], ys[kPersistW];
#pragma unroll
  for (int u = 0; u < kPersistW / 4; ++u) {
    const float4 xa = *reinterpret_cast<const float4 *>(s.x + off + 4 * u);
    const float4 ya = *reinterpret_cast<const float4 *>(s.y + off + 4 * u);
    xs[4 * u] = xa.x; xs[4 * u + 1] = xa.y; xs[4 * u + 2] = xa.z; xs[4 * u + 3] = xa.w;
    ys[4 * u] = ya.x; ys[4 * u + 1] = ya.y; ys[4 * u + 2] = ya.z; ys[4 * u + 3] = ya.w;
  }
  uint2 f[kPersistMaxDeg];
#pragma unroll
  for (int e = 0; e < kPersistMaxDeg; ++e)
    f[e] = e < deg ? __ldcg(reinterpret_cast<const uint2 *>(Fin + size_t(col[e]) * s.Cp + c0))
                   : make_uint2(0u, 0u);  // L2 loads: other blocks wrote these codes in this launch
  uint32_t ap0 = 0, ap1 = 0, am0 = 0, am1 = 0;
#pragma unroll
  for (int e = 0; e < kPersistMaxDeg; ++e) {
    if (e < npos) {
      ap0 += f[e].x;
      ap1 += f[e].y;
    } else {
      am0 += f[e].x;
      am1 += f[e].y;
    }
  }
  const int bias = (deg - npos) - npos;  // codes carry f + 1
  float G[kPersistW];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    G[c] = float(int((ap0 >> (8 * c)) & 0xffu) - int((am0 >> (8 * c)) & 0xffu) + bias);
    G[4 + c] = float(int((ap1 >> (8 * c)) & 0xffu) - int((am1 >> (8 * c)) & 0xffu) + bias);
  }
  sb_updateW<P, kPersistW>(s, a.t, ka, dnext, n, i, c0, G, __ldg(a.h + i), xs, ys, Fout);
}

// ROWS = false: warp items (row, chunk) cached; true: whole rows cached.
template <int P, bool ROWS>
__global__ void __launch_bounds__(256, 4) k_solve_csr_persistent(PersistArgs a) {
  extern __shared__ int32_t s_cache[];  // [8 warps][kPersistMaxItems] ItemIdx or [8][kPersistMaxRows] RowIdx
  const StateView &s = a.s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunks = s.Cp / (32 * kPersistW);
  const int warps_total = gridDim.x * 8;
  const int gw = blockIdx.x * 8 + warp;
  ItemIdx *items = reinterpret_cast<ItemIdx *>(s_cache) + warp * kPersistMaxItems;
  RowIdx *rows = reinterpret_cast<RowIdx *>(s_cache) + warp * kPersistMaxRows;
  int my_count = 0;
  if constexpr (ROWS) {
    for (int row = gw; row < s.N && my_count < kPersistMaxRows; row += warps_total, ++my_count) {
      if (lane == 0) {
        const int e0 = a.row_ptr[row], e1 = a.row_ptr[row + 1];
        RowIdx &m = rows[my_count];
        m.degpos = uint32_t(e1 - e0) | (uint32_t(a.npos[row]) << 8);
        for (int q = 0; q < kPersistMaxDeg; ++q) m.col[q] = q < e1 - e0 ? a.col[e0 + q] : 0;
      }
    }
  } else {
    const int n_items = s.N * chunks;
    for (int it = gw; it < n_items && my_count < kPersistMaxItems; it += warps_total, ++my_count) {
      if (lane == 0) {
        const int row = it / chunks;
        const int e0 = a.row_ptr[row], e1 = a.row_ptr[row + 1];
        ItemIdx &m = items[my_count];
        m.row = row;
        m.chunk = it - row * chunks;
        m.deg = e1 - e0;
        m.npos = a.npos[row];
        for (int q = 0; q < kPersistMaxDeg; ++q) m.col[q] = q < m.deg ? a.col[e0 + q] : 0;
      }
    }
  }
  __syncwarp();
  unsigned k = 0;
  for (int n = a.n_begin; n < a.n_end; ++n) {
    const uint8_t *Fin = s.f_of(n);
    uint8_t *Fout = s.f_of(n + 1);
    const float ka = __ldg(a.t.ka + n), dnext = __ldg(a.t.dl + n + 1);
    for (int q = 0; q < my_count; ++q) {
      if constexpr (ROWS) {
        const RowIdx &m = rows[q];
        const int deg = int(m.degpos & 0xffu), npos = int(m.degpos >> 8);
        for (int ch = 0; ch < chunks; ++ch)
          persist_item<P>(a, gw + q * warps_total, ch, m.col, deg, npos, Fin, Fout, ka, dnext, n, lane);
      } else {
        const ItemIdx &m = items[q];
        persist_item<P>(a, m.row, m.chunk, m.col, m.deg, m.npos, Fin, Fout, ka, dnext, n, lane);
      }
    }
    if (!grid_barrier(a.bar, ++k, a.err)) break;
  }
}

constexpr size_t kPersistSmem = 8 * (kPersistMaxItems * sizeof(ItemIdx) > kPersistMaxRows * sizeof(RowIdx)
                                         ? kPersistMaxItems * sizeof(ItemIdx)
                                         : kPersistMaxRows * sizeof(RowIdx));

template <bool ROWS>
static const void *persistent_fn(int P) {
  switch (P) {
    case 1: return (const void *)k_solve_csr_persistent<1, ROWS>;
    case 2: return (const void *)k_solve_csr_persistent<2, ROWS>;
    case 4: return (const void *)k_solve_csr_persistent<4, ROWS>;
    case 8: return (const void *)k_solve_csr_persistent<8, ROWS>;
    case 16: return (const void *)k_solve_csr_persistent<16, ROWS>;
    case 32: return (const void *)k_solve_csr_persistent<32, ROWS>;
    default: return nullptr;
  }
}

int persistent_barrier_words() { return int(kBarStride * (kBarGroups + 1)); }

int persistent_blocks() {
  int dev = 0, sms = 0, best = 1 << 30;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the smallest co-resident count over all replica counts and both modes
  const int Ps[6] = {1, 2, 4, 8, 16, 32};
  for (int P : Ps)
    for (int rows = 0; rows < 2; ++rows) {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rows ? persistent_fn<true>(P) : persistent_fn<false>(P),
                                                        256, kPersistSmem) != cudaSuccess)
        return 0;
      best = per_sm < best ? per_sm : best;
    }
  return sms * best;
}

int persistent_mode(int N, int Cp, int max_degree, int blocks, bool force_rows) {
  if (blocks <= 0 || max_degree > kPersistMaxDeg || Cp % (32 * kPersistW) != 0) return 0;
  const long long warps = (long long)blocks * 8;
  if (!force_rows && (long long)N * (Cp / (32 * kPersistW)) <= warps * kPersistMaxItems) return 1;
  if ((long long)N <= warps * kPersistMaxRows) return 2;
  return 0;
}

cudaError_t launch_solve_csr_persistent(const StateView &s, const CsrView &J, const StepTables &t, int n_begin,
                                        int n_end, unsigned *bar, int *err, int blocks, int mode, cudaStream_t st) {
  PersistArgs a;
  a.s = s;
  a.row_ptr = J.row_ptr;
  a.col = J.col;
  a.npos = J.npos;
  a.h = J.h;
  a.t = t;
  a.n_begin = n_begin;
  a.n_end = n_end;
  a.bar = bar;
  a.err = err;
  void *args[] = {&a};
  const void *fn = mode == 2 ? persistent_fn<true>(s.P) : persistent_fn<false>(s.P);
  if (!fn || (mode != 1 && mode != 2)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(bar, 0, persistent_barrier_words() * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(256), args, kPersistSmem, st);
}

}  // namespace sbqa
