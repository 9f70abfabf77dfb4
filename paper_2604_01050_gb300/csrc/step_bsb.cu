// step_bsb.cu -- one step of the ballistic form of the machine, f(x) = x
// (the bSB choice of SBM named in Sec. II A; SBQA itself uses the threshold
// f of Eq. 8).  The coupling product then runs on real positions:
//   G_{i,c} = sum_j J_ij x_{j,c}
// so the f buffers hold FP32 copies of x, double-buffered by step parity like
// the codes of the thresholded form (neighbours read x of step n while the
// owning row writes x of step n + 1).  The update -- momentum, position, wall
// -- is the same arithmetic as sb_update4; the value stored for the next
// product is the new x itself.
//
//   k_step_csr_bsb    one warp per (spin row, 128 replica columns), 4 columns
//                     per lane; 8 neighbour gathers (16 bytes each) in flight;
//                     FP32 accumulation in the row's CSR order
//   k_step_dense_bsb  32 rows x 128 columns per block; J (FP32) and x (FP32)
//                     tiles staged in shared memory
// Memory per update: x, y read + write (16 B) + f write (4 B); the gathers of
// neighbour f (4 B per coupling) mostly hit in L2.
#include "step_common.cuh"

namespace sbqa {

template <int KIND>
__device__ __forceinline__ float bsb_weight(const CsrView &J, int e, int ep) {
  if constexpr (KIND == VAL_PM1) return e < ep ? 1.f : -1.f;
  else if constexpr (KIND == VAL_F32) return __ldg(static_cast<const float *>(J.val) + e);
  else return __bfloat162float(static_cast<const __nv_bfloat16 *>(J.val)[e]);
}

template <int P, int KIND>
__global__ void __launch_bounds__(256) k_step_csr_bsb(StateView s, CsrView J, StepTables t, int n) {
  constexpr int U = 8;  // gathers in flight per lane
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= s.N) return;  // whole warp
  const int c4 = blockIdx.y * kColsPerWarp + lane * 4;
  const size_t off = size_t(i) * s.Cp + c4;
  const float4 xv = *reinterpret_cast<const float4 *>(s.x + off);
  const float4 yv = *reinterpret_cast<const float4 *>(s.y + off);
  const int e0 = __ldg(J.row_ptr + i), e1 = __ldg(J.row_ptr + i + 1);
  const int ep = (KIND == VAL_PM1) ? e0 + __ldg(J.npos + i) : e1;
  const float *Fc = s.fx_of(n) + c4;
  float g[4] = {0.f, 0.f, 0.f, 0.f};
  for (int base = e0; base < e1; base += 32) {
    const int cnt = min(32, e1 - base);
    int my_col = 0;
    float my_w = 0.f;
    if (lane < cnt) {
      my_col = __ldg(J.col + base + lane);
      my_w = bsb_weight<KIND>(J, base + lane, ep);
    }
    for (int q = 0; q < cnt; q += U) {  // q + u <= 31: q is a multiple of U below cnt <= 32
      float4 f[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = __shfl_sync(0xffffffffu, my_col, q + u);
        f[u] = (q + u < cnt) ? __ldg(reinterpret_cast<const float4 *>(Fc + size_t(j) * s.Cp))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float w = __shfl_sync(0xffffffffu, my_w, q + u);  // 0 past the row end
        g[0] = fmaf(w, f[u].x, g[0]);
        g[1] = fmaf(w, f[u].y, g[1]);
        g[2] = fmaf(w, f[u].z, g[2]);
        g[3] = fmaf(w, f[u].w, g[3]);
      }
    }
  }
  sb_update4_bsb<P>(s, t, n, i, c4, g, __ldg(J.h + i), xv, yv, s.fx_of(n + 1));
}

constexpr int kBsbBM = 32, kBsbBK = 32;

template <int P>
__global__ void __launch_bounds__(256) k_step_dense_bsb(StateView s, DenseView J, StepTables t, int n) {
  __shared__ float Js[kBsbBM][kBsbBK + 1];
  __shared__ __align__(16) float Fs[kBsbBK][kColsPerWarp];
  const int row0 = blockIdx.y * kBsbBM;
  const int col0 = blockIdx.x * kColsPerWarp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float *Fin = s.fx_of(n);
  const int N = s.N;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int k0 = 0; k0 < N; k0 += kBsbBK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // J tile: 1024 floats, 4 per thread
      const int idx = threadIdx.x + q * 256;
      const int r = idx >> 5, k = idx & 31;
      const int gi = row0 + r, gk = k0 + k;
      Js[r][k] = (gi < N && gk < N) ? __ldg(J.J + size_t(gi) * N + gk) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // f tile: 32 rows x 128 floats, 4 float4 per thread
      const int idx = threadIdx.x + q * 256;
      const int r = idx >> 5, seg = (idx & 31) * 4;
      const int gk = k0 + r;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);  // f = 0 past the last spin
      if (gk < N) v = __ldg(reinterpret_cast<const float4 *>(Fin + size_t(gk) * s.Cp + col0 + seg));
      *reinterpret_cast<float4 *>(&Fs[r][seg]) = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kBsbBK; ++k) {
      const float4 f = *reinterpret_cast<const float4 *>(&Fs[k][lane * 4]);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float w = Js[warp * 4 + a][k];
        acc[a][0] = fmaf(w, f.x, acc[a][0]);
        acc[a][1] = fmaf(w, f.y, acc[a][1]);
        acc[a][2] = fmaf(w, f.z, acc[a][2]);
        acc[a][3] = fmaf(w, f.w, acc[a][3]);
      }
    }
    __syncthreads();
  }
  const int c4 = col0 + lane * 4;
  float *Fout = s.fx_of(n + 1);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = row0 + warp * 4 + a;
    if (i < N) {
      const size_t off = size_t(i) * s.Cp + c4;
      const float4 xv = *reinterpret_cast<const float4 *>(s.x + off);
      const float4 yv = *reinterpret_cast<const float4 *>(s.y + off);
      sb_update4_bsb<P>(s, t, n, i, c4, acc[a], __ldg(J.h + i), xv, yv, Fout);
    }
  }
}

__global__ void k_copy_fx(const float *x, float *fx, size_t count) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < count) fx[e] = x[e];
}

template <int P>
static cudaError_t launch_csr_p(const StateView &s, const CsrView &J, const StepTables &t, int n, cudaStream_t st) {
  const dim3 blocks(unsigned((s.N + 7) / 8), unsigned(s.Cp / kColsPerWarp));
  switch (J.kind) {
    case VAL_PM1: k_step_csr_bsb<P, VAL_PM1><<<blocks, 256, 0, st>>>(s, J, t, n); break;
    case VAL_F32: k_step_csr_bsb<P, VAL_F32><<<blocks, 256, 0, st>>>(s, J, t, n); break;
    default: k_step_csr_bsb<P, VAL_BF16><<<blocks, 256, 0, st>>>(s, J, t, n); break;
  }
  return cudaGetLastError();
}

template <int P>
static cudaError_t launch_dense_p(const StateView &s, const DenseView &J, const StepTables &t, int n,
                                  cudaStream_t st) {
  const dim3 grid(unsigned(s.Cp / kColsPerWarp), unsigned((s.N + kBsbBM - 1) / kBsbBM));
  k_step_dense_bsb<P><<<grid, 256, 0, st>>>(s, J, t, n);
  return cudaGetLastError();
}

cudaError_t launch_step_csr_bsb(const StateView &s, const CsrView &J, const StepTables &t, int n, cudaStream_t st) {
  switch (s.P) {
    case 1: return launch_csr_p<1>(s, J, t, n, st);
    case 2: return launch_csr_p<2>(s, J, t, n, st);
    case 4: return launch_csr_p<4>(s, J, t, n, st);
    case 8: return launch_csr_p<8>(s, J, t, n, st);
    case 16: return launch_csr_p<16>(s, J, t, n, st);
    case 32: return launch_csr_p<32>(s, J, t, n, st);
    case 64: return launch_csr_p<64>(s, J, t, n, st);
    case 128: return launch_csr_p<128>(s, J, t, n, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step_dense_bsb(const StateView &s, const DenseView &J, const StepTables &t, int n,
                                  cudaStream_t st) {
  switch (s.P) {
    case 1: return launch_dense_p<1>(s, J, t, n, st);
    case 2: return launch_dense_p<2>(s, J, t, n, st);
    case 4: return launch_dense_p<4>(s, J, t, n, st);
    case 8: return launch_dense_p<8>(s, J, t, n, st);
    case 16: return launch_dense_p<16>(s, J, t, n, st);
    case 32: return launch_dense_p<32>(s, J, t, n, st);
    case 64: return launch_dense_p<64>(s, J, t, n, st);
    case 128: return launch_dense_p<128>(s, J, t, n, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_copy_fx(const StateView &s, int which, cudaStream_t st) {
  const size_t count = size_t(s.N) * s.Cp;
  if (count == 0) return cudaSuccess;
  k_copy_fx<<<unsigned((count + 255) / 256), 256, 0, st>>>(s.x, s.fx_of(which), count);
  return cudaGetLastError();
}

}  // namespace sbqa
