// solve_small.cu -- a whole solve of a small dense instance in one launch.
//
// For N <= 128 and P * N <= 1024 (and 2 P <= N) one CTA holds one run: J
// (FP32, N x N) and
// f(X) (N x P), and the run's schedule in shared memory, and the state (one
// (spin, replica) element per thread) in registers for all steps.
// Each step: G = J f(X) from shared memory (exact: integer terms), the update of Sec. II A Eqs. 6-7 with the
// wall rule and the threshold of Eq. 8, the ring neighbours by warp shuffle
// (P divides 32, thread t = i * P + k).  At the end the CTA reads out the
// exact int64 energies of its P replicas, the best replica and its spins, and
// writes the final state.  Results equal the per-step path bit for bit.
// Served for integer instances (exact energies in any summation order).
#include <cfloat>
#include <climits>

#include "step_common.cuh"

namespace sbqa {

__device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1ull) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float uni(uint64_t z, float amp) {
  return __fmul_rn(float(int(z >> 40) - 8388608) * 0x1p-23f, amp);
}

template <int P>
__global__ void __launch_bounds__(1024) k_solve_small(SmallArgs a) {
  extern __shared__ float sh[];
  const int N = a.N, S = a.S;
  const int ldj = N + 1;                // padded rows: the four spins of a warp hit four banks
  float *sJ = sh;                       // [N][N + 1]
  float *sF = sJ + N * ldj;             // [2][N][P] f values
  float *sKa = sF + 2 * N * P;          // [S]
  float *sDl = sKa + S;                 // [S + 1]
  float *sKj = sDl + S + 1;             // [S] of this run
  const size_t red_off = (size_t(N * ldj + 2 * N * P + 3 * S + 1) * sizeof(float) + 7) & ~size_t(7);
  double *sRed = reinterpret_cast<double *>(reinterpret_cast<char *>(sh) + red_off);  // [P + 1]
  const int r = blockIdx.x, t = threadIdx.x;
  const int k = t % P, i = t / P;
  const bool live = i < N;
  for (int q = t; q < N * N; q += blockDim.x) sJ[(q / N) * ldj + q % N] = a.J[q];
  for (int q = t; q < S; q += blockDim.x) {
    sKa[q] = a.ka[q];
    sKj[q] = a.kj[size_t(q) * a.R + r];
  }
  for (int q = t; q <= S; q += blockDim.x) sDl[q] = a.dl[q];
  // initial state, same counter layout as k_init
  float x = 0.f, y = 0.f;
  const int c = r * P + k;
  if (live) {
    const uint64_t el = uint64_t(c) * uint64_t(N) + uint64_t(i);
    x = uni(sm64(a.seed, 2ull * el), a.amp);
    y = uni(sm64(a.seed, 2ull * el + 1ull), a.amp);
    sF[i * P + k] = float(int(fcode(x, 0.f)) - 1);
  }
  const float hi = live ? a.h[i] : 0.f;
  __syncthreads();
  const int lane = t & 31;
  const int src_l = (k == 0) ? lane + P - 1 : lane - 1;
  const int src_r = (k == P - 1) ? lane - P + 1 : lane + 1;
  for (int n = 0; n < S; ++n) {
    const float *Fn = sF + (n & 1) * N * P;
    float *Fo = sF + ((n + 1) & 1) * N * P;
    float G = 0.f;
    if (live) {
      // four independent partial sums; every term is a small integer, so the
      // sum is exact and equals the sequential one
      const float *Ji = sJ + i * ldj;
      float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
      int j = 0;
      for (; j + 3 < N; j += 4) {
        g0 = fmaf(Ji[j], Fn[j * P + k], g0);
        g1 = fmaf(Ji[j + 1], Fn[(j + 1) * P + k], g1);
        g2 = fmaf(Ji[j + 2], Fn[(j + 2) * P + k], g2);
        g3 = fmaf(Ji[j + 3], Fn[(j + 3) * P + k], g3);
      }
      for (; j < N; ++j) g0 = fmaf(Ji[j], Fn[j * P + k], g0);
      G = (g0 + g1) + (g2 + g3);
    }
    // ring neighbours (P consecutive threads of one spin hold the run's replicas)
    float xm, xp;
    if constexpr (P == 1) {
      xm = xp = x;
    } else {
      xm = __shfl_sync(0xffffffffu, x, src_l);
      xp = __shfl_sync(0xffffffffu, x, src_r);
    }
    if (live) {
      float yn = fmaf(a.kc, G + hi, y);
      yn = fmaf(-sKa[n], x, yn);
      yn = fmaf(sKj[n], xm + xp, yn);
      const float xn = fmaf(a.kx, yn, x);
      const float xc = fminf(fmaxf(xn, -1.f), 1.f);  // wall
      y = (xc != xn) ? 0.f : yn;
      x = xc;
      const float d = sDl[n + 1];
      Fo[i * P + k] = float(int(x > d) - int(x < -d));
    }
    __syncthreads();
  }
  // final state
  if (live) {
    const size_t off = size_t(i) * a.Cp + c;
    a.x[off] = x;
    a.y[off] = y;
    a.Sg[off] = x >= 0.f ? 1 : -1;
  }
  // readout: t_i = sum_j J_ij s_j in integers, then per replica
  // -(1/2) sum_i s_i (t_i + 2 h_i)
  float *sS = sF;  // reuse: spins as floats [N][P]
  if (live) sS[i * P + k] = x >= 0.f ? 1.f : -1.f;
  __syncthreads();
  long long vi = 0;
  if (live) {
    const long long si = x >= 0.f ? 1 : -1;
    long long ti = 0;
    for (int j = 0; j < N; ++j) ti += (long long)a.J_i32[size_t(i) * N + j] * (long long)sS[j * P + k];
    vi = si * (ti + 2 * a.h_i64[i]);
  }
  // fixed-order reduction over i for each replica k: thread k sums i = 0..N-1
  __syncthreads();
  long long *red = reinterpret_cast<long long *>(sJ);  // J no longer needed: [N][P] partials
  if (live) red[i * P + k] = vi;
  __syncthreads();
  if (t < P) {
    long long acc = 0;
    for (int q = 0; q < N; ++q) acc += red[q * P + t];
    const int cc = r * P + t;
    const long long e = -(acc / 2);
    a.e_int[cc] = e;
    a.e_f64[cc] = double(e);
    sRed[t] = double(e);
  }
  __syncthreads();
  if (t == 0) {
    int kb = 0;
    for (int q = 1; q < P; ++q)
      if (sRed[q] < sRed[kb]) kb = q;
    a.best_k[r] = kb;
    a.best_e[r] = sRed[kb];
    a.best_e_int[r] = (long long)sRed[kb];
    a.best_step[r] = S - 1;
    a.have_best[r] = 1;
    sRed[P] = double(kb);
  }
  __syncthreads();
  const int kb = int(sRed[P]);
  if (live && k == kb) a.best_spins[size_t(r) * N + i] = x >= 0.f ? 1 : -1;
}

size_t small_smem_bytes(int N, int P, int S) {
  return sizeof(float) * (size_t(N) * (N + 1) + 2 * size_t(N) * P + 3 * size_t(S) + 4) + sizeof(double) * (P + 1) + 16;
}

bool small_eligible(int N, int P, int S) {
  return S >= 1 && N <= 128 && N * P <= 1024 && small_smem_bytes(N, P, S) <= 200 * 1024 &&
         size_t(N) * P * sizeof(long long) <= size_t(N) * N * sizeof(float);
}

cudaError_t launch_solve_small(const SmallArgs &a, cudaStream_t st) {
  const size_t smem = small_smem_bytes(a.N, a.P, a.S);
  const int threads = ((a.N * a.P + 31) / 32) * 32;
  cudaError_t e = cudaSuccess;
#define SBQA_SMALL_CASE(PP)                                                                              \
  case PP:                                                                                               \
    e = cudaFuncSetAttribute(k_solve_small<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)); \
    if (e != cudaSuccess) return e;                                                                      \
    k_solve_small<PP><<<a.R, threads, smem, st>>>(a);                                                    \
    break;
  switch (a.P) {
    SBQA_SMALL_CASE(1)
    SBQA_SMALL_CASE(2)
    SBQA_SMALL_CASE(4)
    SBQA_SMALL_CASE(8)
    SBQA_SMALL_CASE(16)
    SBQA_SMALL_CASE(32)
    default: return cudaErrorInvalidValue;
  }
#undef SBQA_SMALL_CASE
  return cudaGetLastError();
}

}  // namespace sbqa
