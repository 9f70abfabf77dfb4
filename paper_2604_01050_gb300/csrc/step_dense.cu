// step_dense.cu -- one SBQA step for dense couplings on the CUDA cores
// (Sec. II A, Eq. 7, G = J f(X) with an N x N matrix), product and update
// fused.  This is the general dense path (any real J in FP32, small-integer J
// exactly); the tensor-core path for integer J lives in step_dense_tc.cu.
//
// Tile: 32 spin rows x 128 replica columns per block of 8 warps; each warp
// owns 4 rows, each lane 4 rows x 4 columns of accumulators.  The K loop
// stages a 32 x 32 block of J (FP32) and a 32 x 128 block of F (int8) in
// shared memory.  128 aligned columns hold whole runs, so the epilogue's
// replica-ring shuffles stay inside the warp.
#include "step_common.cuh"

namespace sbqa {

constexpr int kDenseBM = 32;
constexpr int kDenseBK = 32;

template <int P>
__global__ void __launch_bounds__(256) k_step_dense(StateView s, DenseView J, StepTables t, int n) {
  __shared__ float Js[kDenseBM][kDenseBK + 1];
  __shared__ __align__(16) uint8_t Fs[kDenseBK][kColsPerWarp];
  const int row0 = blockIdx.y * kDenseBM;
  const int col0 = blockIdx.x * kColsPerWarp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint8_t *Fin = s.f_of(n);
  uint8_t *Fout = s.f_of(n + 1);
  const int N = s.N;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;

  for (int k0 = 0; k0 < N; k0 += kDenseBK) {
    // J tile: 1024 floats, 4 per thread
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = threadIdx.x + q * 256;
      const int r = idx >> 5, k = idx & 31;
      const int gi = row0 + r, gk = k0 + k;
      Js[r][k] = (gi < N && gk < N) ? __ldg(J.J + size_t(gi) * N + gk) : 0.f;
    }
    // F tile: 32 rows of 128 bytes, 16 bytes per thread
    {
      const int r = threadIdx.x >> 3, seg = (threadIdx.x & 7) * 16;
      const int gk = k0 + r;
      uint4 v = make_uint4(kFZero4, kFZero4, kFZero4, kFZero4);  // f = 0 past the last spin
      if (gk < N) v = __ldg(reinterpret_cast<const uint4 *>(Fin + size_t(gk) * s.Cp + col0 + seg));
      *reinterpret_cast<uint4 *>(&Fs[r][seg]) = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kDenseBK; ++k) {
      const uint32_t f4 = *reinterpret_cast<const uint32_t *>(&Fs[k][lane * 4]);
      const float f0 = fdec(f4, 0), f1 = fdec(f4, 1), f2 = fdec(f4, 2), f3 = fdec(f4, 3);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float w = Js[warp * 4 + a][k];
        acc[a][0] = fmaf(w, f0, acc[a][0]);
        acc[a][1] = fmaf(w, f1, acc[a][1]);
        acc[a][2] = fmaf(w, f2, acc[a][2]);
        acc[a][3] = fmaf(w, f3, acc[a][3]);
      }
    }
    __syncthreads();
  }
  const int c4 = col0 + lane * 4;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = row0 + warp * 4 + a;
    if (i < N) sb_update4<P>(s, t, n, i, c4, acc[a], __ldg(J.h + i), Fout);
  }
}

template <int P>
static cudaError_t launch_p(const StateView &s, const DenseView &J, const StepTables &t, int n,
                            cudaStream_t st) {
  dim3 grid(s.Cp / kColsPerWarp, (s.N + kDenseBM - 1) / kDenseBM);
  k_step_dense<P><<<grid, 256, 0, st>>>(s, J, t, n);
  return cudaGetLastError();
}

cudaError_t launch_step_dense(const StateView &s, const DenseView &J, const StepTables &t, int n,
                              cudaStream_t st) {
  switch (s.P) {
    case 1: return launch_p<1>(s, J, t, n, st);
    case 2: return launch_p<2>(s, J, t, n, st);
    case 4: return launch_p<4>(s, J, t, n, st);
    case 8: return launch_p<8>(s, J, t, n, st);
    case 16: return launch_p<16>(s, J, t, n, st);
    case 32: return launch_p<32>(s, J, t, n, st);
    case 64: return launch_p<64>(s, J, t, n, st);
    case 128: return launch_p<128>(s, J, t, n, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sbqa
