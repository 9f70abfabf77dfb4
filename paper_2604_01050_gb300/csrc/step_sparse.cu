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
  const int e0 = J.row_ptr[i], e1 = J.row_ptr[i + 1];
  float G[4];
  if constexpr (KIND == VAL_PM1) {
    const int8_t *v = static_cast<const int8_t *>(J.val);
    uint32_t acc = 0;
    for (int e = e0; e < e1; ++e) {
      const int j = __ldg(J.col + e);
      const uint32_t f4 = __ldg(reinterpret_cast<const uint32_t *>(Fin + size_t(j) * s.Cp + c4));
      acc = (__ldg(v + e) > 0) ? __vadd4(acc, f4) : __vsub4(acc, f4);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) G[q] = sbyte(acc, q);
  } else {
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
    for (int e = e0; e < e1; ++e) {
      const int j = __ldg(J.col + e);
      float w;
      if constexpr (KIND == VAL_F32) {
        w = __ldg(static_cast<const float *>(J.val) + e);
      } else {
        w = __bfloat162float(static_cast<const __nv_bfloat16 *>(J.val)[e]);
      }
      const uint32_t f4 = __ldg(reinterpret_cast<const uint32_t *>(Fin + size_t(j) * s.Cp + c4));
      g0 = fmaf(w, sbyte(f4, 0), g0);
      g1 = fmaf(w, sbyte(f4, 1), g1);
      g2 = fmaf(w, sbyte(f4, 2), g2);
      g3 = fmaf(w, sbyte(f4, 3), g3);
    }
    G[0] = g0; G[1] = g1; G[2] = g2; G[3] = g3;
  }
  sb_update4<P>(s, t, n, i, c4, G, __ldg(J.h + i), Fout);
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
