// step_batched.cu -- one SBQA step for many CSR instances of uneven size in a
// single launch (the batching engine's kernel).
//
// Every active request owns a slot: its CSR couplings (and their ELL form for
// rows of degree <= 8), its state buffers, its schedule tables and the number
// of steps it had completed when the current chunk of steps started.  The
// engine lists the work of all active slots as items of 8 spin rows x 128
// replica columns; one wave of blocks walks the item list (a warp per row of
// an item), so one launch advances every request by one step whatever the
// mix.  The slot descriptors sit in shared memory, and a warp issues the
// loads of its next row (work item two ahead, then x, y, h and the ELL
// columns) before it gathers and updates the current one, so the memory
// latency of one row overlaps the work of the previous one.  The arithmetic
// per element is the one of k_step_csr (same gathers, same sums in the same
// order, same update), so a request gives bit-identical results alone and in
// any mix.
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

// Loads of one row of a work item, issued ahead of its use.
struct RowFetch {
  int slot, row, n, c0;  // row < 0: nothing to do (past N, or the request has finished)
  int col;               // lane < 8: ELL column of entry `lane`
  float val;             // lane < 8: its value (FP32 / BF16 couplings)
  int2 meta;             // (degree, +1 count)
  float hi;
  float ka, dnext;       // this step's schedule values of the slot
  float kj[4];           // J_perp of the runs of the lane's columns (W = 4)
  float4 x[2], y[2];     // x, y of the lane's W columns
};

__device__ __forceinline__ void fetch_row(RowFetch &f, const SlotDesc *D, const WorkItem &w, int sub, int j, int lane) {
  const SlotDesc &d = D[w.slot];
  f.slot = w.slot;
  f.row = w.row0 + sub;
  f.n = d.n0 + j;
  if (f.row >= d.N || f.n >= d.S) {  // warp-uniform
    f.row = -1;
    return;
  }
  const int W = d.W;
  f.c0 = w.colgroup * 32 * W + lane * W;
  const size_t off = size_t(f.row) * d.Cp + f.c0;
  f.x[0] = *reinterpret_cast<const float4 *>(d.x + off);
  f.y[0] = *reinterpret_cast<const float4 *>(d.y + off);
  if (W == 8) {
    f.x[1] = *reinterpret_cast<const float4 *>(d.x + off + 4);
    f.y[1] = *reinterpret_cast<const float4 *>(d.y + off + 4);
  }
  f.hi = __ldg(d.h + f.row);
  f.ka = __ldg(d.ka + f.n);
  f.dnext = __ldg(d.dl + f.n + 1);
  if (W == 4) {
    const float *kjn = d.kj + size_t(f.n) * d.R;
    const int lp = __ffs(d.P) - 1;  // P (the run's column width) is a power of two
    if (d.P >= 4) {
      const float k = f.c0 < d.C ? __ldg(kjn + (f.c0 >> lp)) : 0.f;
      f.kj[0] = f.kj[1] = f.kj[2] = f.kj[3] = k;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) f.kj[q] = (f.c0 + q < d.C) ? __ldg(kjn + ((f.c0 + q) >> lp)) : 0.f;
    }
  }
  if (d.ell_col) {
    if (lane < kEllSlots) {
      f.col = __ldg(d.ell_col + size_t(f.row) * kEllSlots + lane);
      if (d.kind != VAL_PM1) f.val = __ldg(d.ell_val + size_t(f.row) * kEllSlots + lane);
    }
    f.meta = __ldg(reinterpret_cast<const int2 *>(d.ell_meta) + f.row);
  }
}

// The W = 4 update's per-lane constants of a row, from its prefetched values
// (as LaneConsts::load computes them).
template <int P>
__device__ __forceinline__ LaneConsts<P> lane_consts(const SlotDesc &d, const RowFetch &f) {
  LaneConsts<P> L;
  L.kc2 = make_float2(d.kc, d.kc);
  L.mka2 = make_float2(-f.ka, -f.ka);
  L.kx2 = make_float2(d.kx, d.kx);
  L.dnext = f.dnext;
#pragma unroll
  for (int q = 0; q < 4; ++q) L.kj[q] = f.kj[q];
  L.active = f.c0 < d.C;
  L.Pr = d.Pr;
  return L;
}

// One row from its ELL slots with W columns per lane: the gathers of its (at
// most 8) neighbours, the sums in the CSR kernel's order, the update.
template <int P, int W>
__device__ __forceinline__ void batched_row_ell(const SlotDesc &d, const RowFetch &f) {
  StateView s;
  s.N = d.N; s.C = d.C; s.Cp = d.Cp; s.P = P; s.R = d.R; s.Pr = d.Pr;
  s.x = d.x; s.y = d.y; s.F[0] = d.F0; s.F[1] = d.F1; s.Sg = nullptr;
  s.Fx[0] = s.Fx[1] = nullptr;
  const uint8_t *Fc = s.f_of(f.n) + f.c0;
  const int deg = f.meta.x, npos = f.meta.y;
  const bool pm1 = d.kind == VAL_PM1;
  uint32_t f4[kEllSlots][W / 4];
#pragma unroll
  for (int e = 0; e < kEllSlots; ++e) {
    const int j = __shfl_sync(0xffffffffu, f.col, e);
    if (e < deg) {
      if constexpr (W == 8) {
        const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(Fc + size_t(j) * d.Cp));
        f4[e][0] = v.x;
        f4[e][1] = v.y;
      } else {
        f4[e][0] = __ldcg(reinterpret_cast<const uint32_t *>(Fc + size_t(j) * d.Cp));
      }
    } else {
#pragma unroll
      for (int q = 0; q < W / 4; ++q) f4[e][q] = pm1 ? 0u : kFZero4;
    }
  }
  float G[W];
  if (pm1) {
    uint32_t ap[W / 4], am[W / 4];
#pragma unroll
    for (int q = 0; q < W / 4; ++q) ap[q] = am[q] = 0;
#pragma unroll
    for (int e = 0; e < kEllSlots; ++e) {
#pragma unroll
      for (int q = 0; q < W / 4; ++q) {
        if (e < npos) ap[q] += f4[e][q];
        else am[q] += f4[e][q];
      }
    }
    const int bias = (deg - npos) - npos;  // codes carry f + 1; padding slots hold 0
#pragma unroll
    for (int c = 0; c < W; ++c)
      G[c] = float(int((ap[c / 4] >> (8 * (c % 4))) & 0xffu) - int((am[c / 4] >> (8 * (c % 4))) & 0xffu) + bias);
  } else {
    float g[W];
#pragma unroll
    for (int c = 0; c < W; ++c) g[c] = 0.f;
#pragma unroll
    for (int e = 0; e < kEllSlots; ++e) {
      const float w = __shfl_sync(0xffffffffu, f.val, e);
      if (e < deg) {
        acc_codes<W>(g, w, f4[e]);
      }
    }
#pragma unroll
    for (int c = 0; c < W; ++c) G[c] = g[c];
  }
  if constexpr (W == 4) {
    if (P > 2 && d.Pr != P)
      sb_update4c<P, true>(s, lane_consts<P>(d, f), f.row, f.c0, G, f.hi, f.x[0], f.y[0], s.f_of(f.n + 1));
    else
      sb_update4c<P, false>(s, lane_consts<P>(d, f), f.row, f.c0, G, f.hi, f.x[0], f.y[0], s.f_of(f.n + 1));
  } else {
    StepTables t;
    t.ka = d.ka; t.dl = d.dl; t.kj = d.kj; t.kc = d.kc; t.kx = d.kx; t.S = d.S; t.R = d.R;
    float xs[8] = {f.x[0].x, f.x[0].y, f.x[0].z, f.x[0].w, f.x[1].x, f.x[1].y, f.x[1].z, f.x[1].w};
    float ys[8] = {f.y[0].x, f.y[0].y, f.y[0].z, f.y[0].w, f.y[1].x, f.y[1].y, f.y[1].z, f.y[1].w};
    if (P > 2 && d.Pr != P) sb_updateW<P, 8, true>(s, t, f.ka, f.dnext, f.n, f.row, f.c0, G, f.hi, xs, ys, s.f_of(f.n + 1));
    else sb_updateW<P, 8, false>(s, t, f.ka, f.dnext, f.n, f.row, f.c0, G, f.hi, xs, ys, s.f_of(f.n + 1));
  }
}

template <int P>
__device__ __forceinline__ void batched_row(const SlotDesc &d, const RowFetch &f) {
  if (!d.ell_col) batched_row_csr<P>(d, f.n, f.row, f.c0, f.x[0], f.y[0], f.hi);
  else if (d.W == 8) batched_row_ell<P, 8>(d, f);
  else batched_row_ell<P, 4>(d, f);
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

// Step j of the chunk for every active slot: the warps of the grid walk the
// rows of the work items (a warp per row; the next row's loads go out before
// this row's gathers).  A warp with no row returns from here only.
__device__ __forceinline__ void batched_pass(const SlotDesc *D, const WorkItem *items, int total, int j) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stride = gridDim.x * 8;
  int u = blockIdx.x * 8 + warp;
  if (u >= total) return;  // whole warp
  RowFetch pf;
  pf.col = 0;
  pf.val = 0.f;
  fetch_row(pf, D, items[u >> 3], u & 7, j, lane);
  WorkItem w_after = u + stride < total ? items[(u + stride) >> 3] : WorkItem{0, 0, 0, 0};
  for (; u < total; u += stride) {
    const RowFetch cur = pf;
    const int nx = u + stride;
    if (nx < total) {  // warp-uniform: the next row's loads go out before this row's gathers
      fetch_row(pf, D, w_after, nx & 7, j, lane);
      if (nx + stride < total) w_after = items[(nx + stride) >> 3];
    }
    if (cur.row < 0) continue;
    const SlotDesc &d = D[cur.slot];
    switch (d.P) {
      case 1: batched_row<1>(d, cur); break;
      case 2: batched_row<2>(d, cur); break;
      case 4: batched_row<4>(d, cur); break;
      case 8: batched_row<8>(d, cur); break;
      case 16: batched_row<16>(d, cur); break;
      case 32: batched_row<32>(d, cur); break;
      case 64: batched_row<64>(d, cur); break;
      default: batched_row<128>(d, cur); break;
    }
  }
}

__global__ void __launch_bounds__(256, 2) k_step_batched(const SlotDesc *slots, int n_slots, const WorkItem *items,
                                                      const int *n_items, int j) {
  __shared__ SlotDesc s_slots[kBatchSmemSlots];
  const SlotDesc *D = stage_slots(s_slots, slots, n_slots);
  batched_pass(D, items, *n_items * 8, j);
}

// Steps j0 .. j1 - 1 of the chunk for every active slot in one cooperative
// launch (the grid exactly co-resident): one pass per step, the bounded grid
// barrier between steps (each slot keeps its own step index n0 + j, and a
// slot past its last step has no rows).  The f codes other blocks wrote in
// the step before are read through L2.  A barrier that gives up records
// error code 4 in *err and every block stops stepping.
__global__ void __launch_bounds__(256, 2) k_solve_batched(const SlotDesc *slots, int n_slots, const WorkItem *items,
                                                       const int *n_items, int j0, int j1, unsigned *bar, int *err) {
  __shared__ SlotDesc s_slots[kBatchSmemSlots];
  const SlotDesc *D = stage_slots(s_slots, slots, n_slots);
  const int total = *n_items * 8;
  unsigned k = 0;
  for (int j = j0; j < j1; ++j) {
    batched_pass(D, items, total, j);
    if (j + 1 < j1 && !grid_barrier(bar, ++k, err)) break;
  }
}

int batched_blocks_per_sm() {
  static int per_sm = 0;
  if (per_sm == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_batched, 256, 0) != cudaSuccess ||
                      per_sm < 1))
    per_sm = 1;
  return per_sm;
}

cudaError_t launch_step_batched(const SlotDesc *slots, int n_slots, const WorkItem *items, const int *n_items,
                                int grid, int j, cudaStream_t st) {
  k_step_batched<<<grid, 256, 0, st>>>(slots, n_slots, items, n_items, j);
  return cudaGetLastError();
}

int batched_persistent_blocks() {
  static int blocks = -1;
  if (blocks < 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_batched, 256, 0) != cudaSuccess) per_sm = 0;
    blocks = sms * per_sm;
  }
  return blocks;
}

cudaError_t launch_solve_batched(const SlotDesc *slots, int n_slots, const WorkItem *items, const int *n_items,
                                 int grid, int j0, int j1, unsigned *bar, int *err, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bar, 0, grid_barrier_words() * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  void *args[] = {(void *)&slots, (void *)&n_slots, (void *)&items, (void *)&n_items, (void *)&j0, (void *)&j1,
                  (void *)&bar, (void *)&err};
  return cudaLaunchCooperativeKernel((const void *)k_solve_batched, dim3(grid), dim3(256), args, 0, st);
}

}  // namespace sbqa
