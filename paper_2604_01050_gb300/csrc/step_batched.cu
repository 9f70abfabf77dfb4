// step_batched.cu -- one SBQA step for many CSR instances of uneven size in a
// single launch (the batching engine's kernel).
//
// Every active request owns a slot: its CSR couplings, its state buffers,
// its schedule tables and the number of steps it had completed when the
// current chunk of steps started.  The engine lists the work of all active
// slots as items of 8 spin rows x 128 replica columns; a persistent grid
// walks the item list, so one launch advances every request by one step
// whatever the mix.  The arithmetic per element is the one of k_step_csr
// (same gathers, same sums in the same order, same update), so a request
// gives bit-identical results alone and in any mix.
#include "step_common.cuh"

namespace sbqa {

// Step j of the chunk of a slot whose n0 steps were done before the chunk.
template <int P>
__device__ __forceinline__ void batched_rows(const SlotDesc &d, int n, int r0, int c4) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  StateView s;
  s.N = d.N; s.C = d.C; s.Cp = d.Cp; s.P = P; s.R = d.R;
  s.x = d.x; s.y = d.y; s.F[0] = d.F0; s.F[1] = d.F1; s.Sg = nullptr;
  s.Fx[0] = s.Fx[1] = nullptr;
  StepTables t;
  t.ka = d.ka; t.dl = d.dl; t.kj = d.kj; t.kc = d.kc; t.kx = d.kx; t.S = d.S; t.R = d.R;
  const uint8_t *Fc = s.f_of(n) + c4;
  uint8_t *Fout = s.f_of(n + 1);
  const int i = r0 + warp;
  if (i >= d.N) return;  // warp-uniform
  const size_t off = size_t(i) * d.Cp + c4;
  const float4 xv = *reinterpret_cast<const float4 *>(d.x + off);
  const float4 yv = *reinterpret_cast<const float4 *>(d.y + off);
  const float hi = __ldg(d.h + i);
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
          f4[u] = (q + u < cnt) ? __ldg(reinterpret_cast<const uint32_t *>(Fc + size_t(j) * d.Cp)) : 0u;
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
          f4[u] = (q + u < cnt) ? __ldg(reinterpret_cast<const uint32_t *>(Fc + size_t(j) * d.Cp)) : kFZero4;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float w = __shfl_sync(0xffffffffu, my_w, q + u);
#pragma unroll
          for (int c = 0; c < 4; ++c) g[c] = fmaf(w, fdec(f4[u], c), g[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) G[c] = g[c];
  }
  sb_update4<P>(s, t, n, i, c4, G, hi, xv, yv, Fout);
}

__global__ void __launch_bounds__(256, 3) k_step_batched(const SlotDesc *slots, const WorkItem *items,
                                                      const int *n_items, int j) {
  const int total = *n_items;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const WorkItem w = items[it];
    const SlotDesc &d = slots[w.slot];
    const int n = d.n0 + j;
    if (n >= d.S) continue;  // block-uniform: this request is done
    const int c4 = w.colgroup * kColsPerWarp + (threadIdx.x & 31) * kColsPerLane;
    switch (d.P) {
      case 1: batched_rows<1>(d, n, w.row0, c4); break;
      case 2: batched_rows<2>(d, n, w.row0, c4); break;
      case 4: batched_rows<4>(d, n, w.row0, c4); break;
      case 8: batched_rows<8>(d, n, w.row0, c4); break;
      case 16: batched_rows<16>(d, n, w.row0, c4); break;
      default: batched_rows<32>(d, n, w.row0, c4); break;
    }
  }
}

cudaError_t launch_step_batched(const SlotDesc *slots, const WorkItem *items, const int *n_items, int grid, int j,
                                cudaStream_t st) {
  k_step_batched<<<grid, 256, 0, st>>>(slots, items, n_items, j);
  return cudaGetLastError();
}

}  // namespace sbqa
