// step_sparse.cu -- one SBQA step for CSR couplings (Sec. II A, Eq. 7 with a
// sparse J), the coupling product and the update fused in one kernel.
//
// A warp owns one spin row i and 128 replica columns (4 per lane).  The row's
// (col, J) entries are read once per warp (uniform broadcast loads); for each
// entry the lane reads 4 bytes of F (f(x) of the neighbour spin for its 4
// columns).  Accumulation:
//   VAL_PM1   J = +-1: packed byte adds (__vadd4 / __vsub4), exact while the
//             row degree is <= 127 (checked on the host)
//   VAL_F32   FP32 J, FP32 accumulation (exact for small-integer J)
//   VAL_BF16  bfloat16 J, FP32 accumulation
// Memory per update: x, y read + write (16 B) + F write (1 B); F gathers and
// the CSR arrays are shared by all columns of a row and mostly hit in cache.
#include "step_common.cuh"

namespace sbqa {

template <int KIND>
__device__ __forceinline__ float load_val(const void *val, int e) {
  if constexpr (KIND == VAL_PM1) return float(__ldg(static_cast<const int8_t *>(val) + e));
  else if constexpr (KIND == VAL_F32) return __ldg(static_cast<const float *>(val) + e);
  else return __bfloat162float(static_cast<const __nv_bfloat16 *>(val)[e]);
}

template <int P, int KIND>
__global__ void __launch_bounds__(256) k_step_csr(StateView s, CsrView J, StepTables t, int n) {
  const int warps_per_row = s.Cp / kColsPerWarp;
  const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int i = wid / warps_per_row;
  if (i >= s.N) return;  // whole warp leaves together
  const int lane = threadIdx.x & 31;
  const int c4 = (wid - i * warps_per_row) * kColsPerWarp + lane * kColsPerLane;
  const int8_t *Fin = s.f_of(n);
  int8_t *Fout = s.f_of(n + 1);
  // state loads first: they do not depend on the product
  const size_t off = size_t(i) * s.Cp + c4;
  const float4 xv = *reinterpret_cast<const float4 *>(s.x + off);
  const float4 yv = *reinterpret_cast<const float4 *>(s.y + off);
  const float hi = __ldg(J.h + i);
  const int e0 = __ldg(J.row_ptr + i), deg = __ldg(J.row_ptr + i + 1) - e0;
  const int8_t *Fc = Fin + c4;
  uint32_t acc = 0;                  // VAL_PM1: 4 packed int8 sums
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
  // The row's (col, J) entries are read 32 at a time, one per lane, and
  // broadcast by shuffle; the F gathers of 8 entries are issued together.
  for (int base = 0; base < deg; base += 32) {
    const int cnt = min(32, deg - base);
    int my_col = 0;
    float my_w = 0.f;
    if (lane < cnt) {
      my_col = __ldg(J.col + e0 + base + lane);
      my_w = load_val<KIND>(J.val, e0 + base + lane);
    }
    for (int q = 0; q < cnt; q += 8) {
      uint32_t f4[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = __shfl_sync(0xffffffffu, my_col, q + u);
        f4[u] = (q + u < cnt) ? __ldg(reinterpret_cast<const uint32_t *>(Fc + size_t(j) * s.Cp)) : 0u;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float w = __shfl_sync(0xffffffffu, my_w, q + u);
        if constexpr (KIND == VAL_PM1) {
          acc = (w > 0.f) ? __vadd4(acc, f4[u]) : __vsub4(acc, f4[u]);  // f4 = 0 past the row end
        } else {
          g0 = fmaf(w, sbyte(f4[u], 0), g0);
          g1 = fmaf(w, sbyte(f4[u], 1), g1);
          g2 = fmaf(w, sbyte(f4[u], 2), g2);
          g3 = fmaf(w, sbyte(f4[u], 3), g3);
        }
      }
    }
  }
  float G[4];
  if constexpr (KIND == VAL_PM1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) G[q] = sbyte(acc, q);
  } else {
    G[0] = g0; G[1] = g1; G[2] = g2; G[3] = g3;
  }
  sb_update4<P>(s, t, n, i, c4, G, hi, xv, yv, Fout);
}

template <int P>
static cudaError_t launch_p(const StateView &s, const CsrView &J, const StepTables &t, int n,
                            cudaStream_t st) {
  const long long warps = (long long)s.N * (s.Cp / kColsPerWarp);
  const unsigned blocks = unsigned((warps + 7) / 8);
  switch (J.kind) {
    case VAL_PM1: k_step_csr<P, VAL_PM1><<<blocks, 256, 0, st>>>(s, J, t, n); break;
    case VAL_F32: k_step_csr<P, VAL_F32><<<blocks, 256, 0, st>>>(s, J, t, n); break;
    default: k_step_csr<P, VAL_BF16><<<blocks, 256, 0, st>>>(s, J, t, n); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_step_csr(const StateView &s, const CsrView &J, const StepTables &t, int n,
                            cudaStream_t st) {
  switch (s.P) {
    case 1: return launch_p<1>(s, J, t, n, st);
    case 2: return launch_p<2>(s, J, t, n, st);
    case 4: return launch_p<4>(s, J, t, n, st);
    case 8: return launch_p<8>(s, J, t, n, st);
    case 16: return launch_p<16>(s, J, t, n, st);
    case 32: return launch_p<32>(s, J, t, n, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sbqa
