// step_batched.cu -- the steps of many CSR instances of uneven size in one
// launch (the batching engine's chunk kernel).
//
// Every active request owns a slot: its CSR couplings (and their ELL form for
// rows of degree <= 8), its state buffers, its schedule tables and the number
// of steps it had completed when the current chunk of steps started.  The
// engine lists the work of all active slots: units of 2 spin rows x 128
// replica columns for slots in ELL form (1 row x 256 columns when the
// slot's padded width is a multiple of 256; first, ordered by unit shape,
// run width and coupling kind) and items of 8 rows x 128 columns for the
// others.  One
// cooperative launch runs all steps of a chunk; a bounded grid barrier
// separates the steps.  At the start of the launch every warp takes a
// contiguous share of the units and keeps their neighbour columns, coupling
// values, degrees and fields in shared memory for the whole chunk; each step
// it runs them on half warps (one row of a unit per half, 8 columns per lane;
// a wide unit on the whole warp), units beyond its shared-memory share from
// global memory.  The items of the
// other slots are spread over all warps, a row per warp (4 columns per lane).
// The arithmetic per element is the one of k_step_csr (same gathers, same
// sums in the same order, same update), so a request gives bit-identical
// results alone and in any mix.
#include "grid_sync.cuh"
#include "step_common.cuh"

namespace sbqa {

// Step j of the chunk of a slot whose n0 steps were done before the chunk.
template <int P>
__device__ __forceinline__ void batched_row_csr(const SlotDesc &d, int n, int i, int c4, float4 xv, float4 yv,
                                                float hi) {
  const int lane = threadIdx.x & 31;
  StateView s;
  s.N = d.N; s.C = d.C; s.Cp = d.Cp; s.P = P; s.R = d.R; s.Pr = d.Pr;
  s.x = d.x; s.y = d.y; s.F[0] = d.F0; s.F[1] = d.F1; s.Sg = nullptr;
  s.Fx[0] = s.Fx[1] = nullptr;
  StepTables t;
  t.ka = d.ka; t.dl = d.dl; t.kj = d.kj; t.kc = d.kc; t.kx = d.kx; t.S = d.S; t.R = d.R;
  const uint8_t *Fc = s.f_of(n) + c4;
  uint8_t *Fout = s.f_of(n + 1);
  const int e0 = __ldg(d.row_ptr + i), e1 = __ldg(d.row_ptr + i + 1);
  float G[4];
  if (d.kind == VAL_PM1) {
    const int ep = e0 + __ldg(d.npos + i);
    uint32_t ap = 0, am = 0;
    for (int base = e0; base < e1; base += 32) {
      const int cnt = min(32, e1 - base);
      const int my_col = lane < cnt ? __ldg(d.col + base + lane) : 0;
      for (int q = 0; q < cnt; q += 8) {
        uint32_t f4[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = __shfl_sync(0xffffffffu, my_col, q + u);
          f4[u] = (q + u < cnt) ? __ldcg(reinterpret_cast<const uint32_t *>(Fc + size_t(j) * d.Cp)) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (base + q + u < ep) ap += f4[u];
          else am += f4[u];
        }
      }
    }
    const int bias = (e1 - ep) - (ep - e0);
#pragma unroll
    for (int q = 0; q < 4; ++q) G[q] = float(int((ap >> (8 * q)) & 0xffu) - int((am >> (8 * q)) & 0xffu) + bias);
  } else {
    float g[4] = {0.f, 0.f, 0.f, 0.f};
    for (int base = e0; base < e1; base += 32) {
      const int cnt = min(32, e1 - base);
      int my_col = 0;
      float my_w = 0.f;
      if (lane < cnt) {
        my_col = __ldg(d.col + base + lane);
        my_w = d.kind == VAL_F32 ? __ldg(static_cast<const float *>(d.val) + base + lane)
                                 : __bfloat162float(static_cast<const __nv_bfloat16 *>(d.val)[base + lane]);
      }
      for (int q = 0; q < cnt; q += 8) {
        uint32_t f4[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = __shfl_sync(0xffffffffu, my_col, q + u);
          f4[u] = (q + u < cnt) ? __ldcg(reinterpret_cast<const uint32_t *>(Fc + size_t(j) * d.Cp)) : kFZero4;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float w = __shfl_sync(0xffffffffu, my_w, q + u);
          acc_codes<4>(g, w, &f4[u]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) G[c] = g[c];
  }
  if (P > 2 && d.Pr != P) sb_update4<P, true>(s, t, n, i, c4, G, hi, xv, yv, Fout);
  else sb_update4<P, false>(s, t, n, i, c4, G, hi, xv, yv, Fout);
}

// Neighbours of two rows of a unit, kept in shared memory for a chunk.
struct BatchEntry {
  int slot, row0, chunk;
  uint32_t degpos[2];  // per row: degree | +1 count (VAL_PM1) << 8; 0 for a row past N
  float h[2];
  int32_t col[2][kEllSlots];
  float val[2][kEllSlots];  // FP32 / BF16 couplings (unused for VAL_PM1)
  int pad;
};
static_assert(sizeof(BatchEntry) % 16 == 0, "entries start on 16-byte boundaries");

constexpr int kBatchThreads = 256, kBatchWarps = kBatchThreads / 32, kBatchBlocksPerSM = 3;
constexpr int kBatchEntriesPerWarp = 48;  // x 160 B per warp: 61.4 KB of shared memory per block of 8 warps
constexpr int kBatchSmem = kBatchWarps * kBatchEntriesPerWarp * int(sizeof(BatchEntry));

// One row of a unit on a half warp (8 columns per lane): the gathers of its
// neighbours' codes, the sums in the CSR kernel's order, the update.  col and
// val point at the row's entries in shared memory or in the slot's ELL
// arrays; act = false for the second row of a unit that ends past N (the
// half repeats the first row's loads and stores nothing).
template <int P, bool PM1, bool GEN>
__device__ __forceinline__ void batched_unit_row(const SlotDesc &d, int n, int row, bool act, int c0, int deg,
                                                 int npos, const int32_t *col, const float *val, float hi) {
  constexpr int W = 8;
  StateView s;
  s.N = d.N; s.C = d.C; s.Cp = d.Cp; s.P = P; s.R = d.R; s.Pr = d.Pr;
  s.x = d.x; s.y = d.y; s.F[0] = d.F0; s.F[1] = d.F1; s.Sg = nullptr;
  s.Fx[0] = s.Fx[1] = nullptr;
  StepTables t;
  t.ka = d.ka; t.dl = d.dl; t.kj = d.kj; t.kc = d.kc; t.kx = d.kx; t.S = d.S; t.R = d.R;
  const size_t off = size_t(row) * d.Cp + c0;
  float xs[W], ys[W];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const float4 xa = *reinterpret_cast<const float4 *>(d.x + off + 4 * u);
    const float4 ya = *reinterpret_cast<const float4 *>(d.y + off + 4 * u);
    xs[4 * u] = xa.x; xs[4 * u + 1] = xa.y; xs[4 * u + 2] = xa.z; xs[4 * u + 3] = xa.w;
    ys[4 * u] = ya.x; ys[4 * u + 1] = ya.y; ys[4 * u + 2] = ya.z; ys[4 * u + 3] = ya.w;
  }
  const uint8_t *Fc = s.f_of(n) + c0;
  uint32_t f4[kEllSlots][2];
#pragma unroll
  for (int e = 0; e < kEllSlots; ++e) {
    if (e < deg) {
      const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(Fc + size_t(col[e]) * d.Cp));
      f4[e][0] = v.x;
      f4[e][1] = v.y;
    } else {
      f4[e][0] = f4[e][1] = PM1 ? 0u : kFZero4;
    }
  }
  float G[W];
  if constexpr (PM1) {
    uint32_t ap[2] = {0u, 0u}, am[2] = {0u, 0u};
#pragma unroll
    for (int e = 0; e < kEllSlots; ++e) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (e < npos) ap[q] += f4[e][q];
        else am[q] += f4[e][q];
      }
    }
    const int bias = (deg - npos) - npos;  // codes carry f + 1; padding slots hold 0
#pragma unroll
    for (int c = 0; c < W; ++c)
      G[c] = float(int((ap[c / 4] >> (8 * (c % 4))) & 0xffu) - int((am[c / 4] >> (8 * (c % 4))) & 0xffu) + bias);
  } else {
#pragma unroll
    for (int c = 0; c < W; ++c) G[c] = 0.f;
#pragma unroll
    for (int e = 0; e < kEllSlots; ++e) {
      if (e < deg) acc_codes<W>(G, val[e], f4[e]);
    }
  }
  const float ka = __ldg(d.ka + n), dnext = __ldg(d.dl + n + 1);
  // an idle half takes part in the ring shuffles only (a column past C stores nothing)
  sb_updateW<P, W, GEN>(s, t, ka, dnext, n, row, act ? c0 : d.C, G, hi, xs, ys, s.f_of(n + 1));
}

template <int P>
__device__ __forceinline__ void batched_unit_p(const SlotDesc &d, int n, int row, bool act, int c0, int deg, int npos,
                                               const int32_t *col, const float *val, float hi) {
  const bool gen = P > 2 && d.Pr != P;
  if (d.kind == VAL_PM1) {
    if (gen) batched_unit_row<P, true, true>(d, n, row, act, c0, deg, npos, col, val, hi);
    else batched_unit_row<P, true, false>(d, n, row, act, c0, deg, npos, col, val, hi);
  } else {
    if (gen) batched_unit_row<P, false, true>(d, n, row, act, c0, deg, npos, col, val, hi);
    else batched_unit_row<P, false, false>(d, n, row, act, c0, deg, npos, col, val, hi);
  }
}

// The lane's row of a unit (both halves of a warp run the same slot, so
// every branch on the slot is warp-uniform).
__device__ __forceinline__ void batched_unit(const SlotDesc &d, int n, int row, bool act, int c0, int deg, int npos,
                                             const int32_t *col, const float *val, float hi) {
  switch (d.P) {
    case 1: batched_unit_p<1>(d, n, row, act, c0, deg, npos, col, val, hi); break;
    case 2: batched_unit_p<2>(d, n, row, act, c0, deg, npos, col, val, hi); break;
    case 4: batched_unit_p<4>(d, n, row, act, c0, deg, npos, col, val, hi); break;
    case 8: batched_unit_p<8>(d, n, row, act, c0, deg, npos, col, val, hi); break;
    case 16: batched_unit_p<16>(d, n, row, act, c0, deg, npos, col, val, hi); break;
    case 32: batched_unit_p<32>(d, n, row, act, c0, deg, npos, col, val, hi); break;
    case 64: batched_unit_p<64>(d, n, row, act, c0, deg, npos, col, val, hi); break;
    default: batched_unit_p<128>(d, n, row, act, c0, deg, npos, col, val, hi); break;
  }
}

// A row of an item of a slot without ELL form, on a whole warp.
__device__ __forceinline__ void batched_item_row(const SlotDesc &d, int n, int row, int c4) {
  const size_t off = size_t(row) * d.Cp + c4;
  const float4 xv = *reinterpret_cast<const float4 *>(d.x + off);
  const float4 yv = *reinterpret_cast<const float4 *>(d.y + off);
  const float hi = __ldg(d.h + row);
  switch (d.P) {
    case 1: batched_row_csr<1>(d, n, row, c4, xv, yv, hi); break;
    case 2: batched_row_csr<2>(d, n, row, c4, xv, yv, hi); break;
    case 4: batched_row_csr<4>(d, n, row, c4, xv, yv, hi); break;
    case 8: batched_row_csr<8>(d, n, row, c4, xv, yv, hi); break;
    case 16: batched_row_csr<16>(d, n, row, c4, xv, yv, hi); break;
    case 32: batched_row_csr<32>(d, n, row, c4, xv, yv, hi); break;
    case 64: batched_row_csr<64>(d, n, row, c4, xv, yv, hi); break;
    default: batched_row_csr<128>(d, n, row, c4, xv, yv, hi); break;
  }
}

constexpr int kBatchSmemSlots = 64;  // slot descriptors kept in shared memory (more: read from global)

// The slot descriptors into shared memory (when they fit).
__device__ __forceinline__ const SlotDesc *stage_slots(SlotDesc *s_slots, const SlotDesc *slots, int n_slots) {
  if (n_slots > kBatchSmemSlots) return slots;
  const int words = n_slots * int(sizeof(SlotDesc) / 4);
  for (int q = threadIdx.x; q < words; q += blockDim.x)
    reinterpret_cast<uint32_t *>(s_slots)[q] = reinterpret_cast<const uint32_t *>(slots)[q];
  __syncthreads();
  return s_slots;
}

// Entry `m` of unit w: the neighbours of its two rows (lanes 0-15: columns,
// 16-31: values), then degrees and fields.
__device__ __forceinline__ void fill_entry(BatchEntry &m, const SlotDesc *D, const WorkItem &w, int lane) {
  const SlotDesc &d = D[w.slot];
  const int h = (lane >> 3) & 1, e = lane & 7, row = w.row0 + h;
  const bool ok = row < d.N;
  if (lane < 16) m.col[h][e] = ok ? __ldg(d.ell_col + size_t(row) * kEllSlots + e) : 0;
  else m.val[h][e] = (ok && d.kind != VAL_PM1) ? __ldg(d.ell_val + size_t(row) * kEllSlots + e) : 0.f;
  if (lane < 2) {
    const int r = w.row0 + lane;
    const int2 meta = r < d.N ? __ldg(reinterpret_cast<const int2 *>(d.ell_meta) + r) : make_int2(0, 0);
    m.degpos[lane] = uint32_t(meta.x) | (uint32_t(meta.y) << 8);
    m.h[lane] = r < d.N ? __ldg(d.h + r) : 0.f;
  }
  if (lane == 0) {
    m.slot = w.slot;
    m.row0 = w.row0;
    m.chunk = w.colgroup;
  }
}

// Steps j0 .. j1 - 1 of the chunk for every active slot in one cooperative
// launch (the grid exactly co-resident).  counts[0] = units (2 rows x 128
// columns of slots in ELL form, items[0 .. counts[0])), counts[1] = items of
// 8 rows x 128 columns of the other slots (after the units).  Each slot keeps
// its own step index n0 + j, and a slot past its last step does nothing.  The
// f codes other blocks wrote in the step before are read through L2.  A
// barrier that gives up records error code 4 in *err and every block stops
// stepping.
__global__ void __launch_bounds__(kBatchThreads, kBatchBlocksPerSM)
    k_solve_batched(const SlotDesc *slots, int n_slots, const WorkItem *items, const int *counts, int j0, int j1,
                    unsigned *bar, int *err) {
  __shared__ SlotDesc s_slots[kBatchSmemSlots];
  extern __shared__ BatchEntry s_entries[];
  const SlotDesc *D = stage_slots(s_slots, slots, n_slots);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_units = counts[0], n_items = counts[1];
  const int warps = gridDim.x * kBatchWarps, gw = blockIdx.x * kBatchWarps + warp;
  // this warp's units: a contiguous share (neighbouring units run the same code)
  const int u_begin = int(int64_t(n_units) * gw / warps), u_end = int(int64_t(n_units) * (gw + 1) / warps);
  const int cached = min(u_end - u_begin, kBatchEntriesPerWarp);
  BatchEntry *mine = s_entries + warp * kBatchEntriesPerWarp;
  for (int q = 0; q < cached; ++q) fill_entry(mine[q], D, items[u_begin + q], lane);
  __syncwarp();
  const int h = lane >> 4, c_lane = (lane & 15) * 8;
  unsigned k = 0;
  for (int j = j0; j < j1; ++j) {
    for (int q = 0; q < cached; ++q) {
      const BatchEntry &m = mine[q];
      const SlotDesc &d = D[m.slot];
      const int n = d.n0 + j;
      if (n >= d.S) continue;  // the request has finished (warp-uniform)
      if (d.wide) {  // one row, 256 columns on the whole warp (the entry's first row)
        const uint32_t dp = m.degpos[0];
        batched_unit(d, n, m.row0, true, m.chunk * 256 + lane * 8, int(dp & 0xffu), int(dp >> 8), m.col[0], m.val[0],
                     m.h[0]);
        continue;
      }
      const bool act = m.row0 + h < d.N;
      const uint32_t dp = m.degpos[h];
      batched_unit(d, n, act ? m.row0 + h : m.row0, act, m.chunk * kColsPerWarp + c_lane, act ? int(dp & 0xffu) : 0,
                   int(dp >> 8), m.col[h], m.val[h], m.h[h]);
    }
    for (int u = u_begin + cached; u < u_end; ++u) {  // past this warp's shared-memory share
      const WorkItem w = items[u];
      const SlotDesc &d = D[w.slot];
      const int n = d.n0 + j;
      if (n >= d.S) continue;
      if (d.wide) {
        const int2 meta = __ldg(reinterpret_cast<const int2 *>(d.ell_meta) + w.row0);
        batched_unit(d, n, w.row0, true, w.colgroup * 256 + lane * 8, meta.x, meta.y,
                     d.ell_col + size_t(w.row0) * kEllSlots, d.ell_val + size_t(w.row0) * kEllSlots,
                     __ldg(d.h + w.row0));
        continue;
      }
      const bool act = w.row0 + h < d.N;
      const int row = act ? w.row0 + h : w.row0;
      const int2 meta = __ldg(reinterpret_cast<const int2 *>(d.ell_meta) + row);
      batched_unit(d, n, row, act, w.colgroup * kColsPerWarp + c_lane, act ? meta.x : 0, meta.y,
                   d.ell_col + size_t(row) * kEllSlots, d.ell_val + size_t(row) * kEllSlots, __ldg(d.h + row));
    }
    for (int r = gw; r < n_items * 8; r += warps) {  // the other slots' rows, a row per warp
      const WorkItem w = items[n_units + (r >> 3)];
      const SlotDesc &d = D[w.slot];
      const int n = d.n0 + j, row = w.row0 + (r & 7);
      if (n >= d.S || row >= d.N) continue;
      batched_item_row(d, n, row, w.colgroup * kColsPerWarp + lane * 4);
    }
    if (j + 1 < j1 && !grid_barrier(bar, ++k, err)) break;
  }
}

int batched_grid(int64_t tasks) {
  const int64_t blocks = (tasks + kBatchWarps - 1) / kBatchWarps;
  const int most = batched_persistent_blocks();
  return int(blocks < 1 ? 1 : (blocks < most ? blocks : (most > 0 ? most : 1)));
}

int batched_persistent_blocks() {
  static int blocks = -1;
  if (blocks < 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute((const void *)k_solve_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kBatchSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_batched, kBatchThreads, kBatchSmem) !=
            cudaSuccess)
      per_sm = 0;
    blocks = sms * per_sm;
  }
  return blocks;
}

cudaError_t launch_solve_batched(const SlotDesc *slots, int n_slots, const WorkItem *items, const int *counts,
                                 int grid, int j0, int j1, unsigned *bar, int *err, cudaStream_t st) {
  if (batched_persistent_blocks() <= 0) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaMemsetAsync(bar, 0, grid_barrier_words() * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  void *args[] = {(void *)&slots, (void *)&n_slots, (void *)&items, (void *)&counts, (void *)&j0, (void *)&j1,
                  (void *)&bar, (void *)&err};
  return cudaLaunchCooperativeKernel((const void *)k_solve_batched, dim3(grid), dim3(kBatchThreads), args, kBatchSmem,
                                     st);
}

}  // namespace sbqa
