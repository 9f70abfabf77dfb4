// init_readout.cu -- initial state, threshold refresh and the readout
// (s = sign(q), Ising energies, per-run best) of the SBQA hot path.
//
// Initial state ("initialized in a random state", Sec. II A): every x and y
// of element (run r, replica k, spin i) is an independent uniform draw from
// SplitMix64 (Steele, Lea & Flood 2014) -- output number
// ctr = 2 * ((r * P + k) * N + i) + w (w = 0 for x, 1 for y) of the
// generator seeded with the run seed, mapped to FP32 as
// ((top 24 bits) - 2^23) * 2^-23 * amp.
//
// Readout (Sec. II A: solution s_i = sign(q_i); Sec. II B: best over runs):
//   E(s) = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i
//        = -(1/2) sum_i (s_i t_i + 2 h_i s_i),   t_i = sum_j J_ij s_j.
// Integer instances accumulate in int64 (exact); real ones in FP64.  Row
// blocks write partial column sums that a second kernel adds in a fixed
// order, so energies are reproducible run to run.
#include <cfloat>
#include <climits>

#include "step_common.cuh"

namespace sbqa {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1ull) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float to_uniform(uint64_t z, float amp) {
  const int m = int(z >> 40) - 8388608;
  return __fmul_rn(float(m) * 0x1p-23f, amp);
}

__global__ void k_init(StateView s, uint64_t seed, float amp, float delta0) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= size_t(s.N) * s.Cp) return;
  const int i = int(e / s.Cp), c = int(e % s.Cp);
  float x = 0.f, y = 0.f;
  uint8_t f = kFZero;
  const int r = c / s.P, k = c % s.P;  // run and replica of column c (k >= Pr: padding, left at zero)
  if (c < s.C && k < s.Pr) {
    const uint64_t el = (uint64_t(r) * uint64_t(s.Pr) + uint64_t(k)) * uint64_t(s.N) + uint64_t(i);
    x = to_uniform(splitmix64_at(seed, 2ull * el), amp);
    y = to_uniform(splitmix64_at(seed, 2ull * el + 1ull), amp);
    f = uint8_t(fcode(x, delta0));
  }
  s.x[e] = x;
  s.y[e] = y;
  s.F[0][e] = f;
  s.F[1][e] = kFZero;
}

cudaError_t launch_init(const StateView &s, uint64_t seed, float amp, float delta0,
                        cudaStream_t st) {
  const size_t total = size_t(s.N) * s.Cp;
  k_init<<<unsigned((total + 255) / 256), 256, 0, st>>>(s, seed, amp, delta0);
  return cudaGetLastError();
}

__global__ void k_refresh_f(StateView s, int which, float delta) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= size_t(s.N) * s.Cp) return;
  const int c = int(e % s.Cp);
  s.f_of(which)[e] = (c < s.C) ? uint8_t(fcode(s.x[e], delta)) : kFZero;
}

cudaError_t launch_refresh_f(const StateView &s, int which, float delta, cudaStream_t st) {
  const size_t total = size_t(s.N) * s.Cp;
  k_refresh_f<<<unsigned((total + 255) / 256), 256, 0, st>>>(s, which, delta);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- signs
__global__ void k_sign(StateView s) {
  const size_t q = size_t(blockIdx.x) * blockDim.x + threadIdx.x;  // one float4 per thread
  if (q * 4 >= size_t(s.N) * s.Cp) return;
  const float4 v = reinterpret_cast<const float4 *>(s.x)[q];
  const int c = int((q * 4) % s.Cp);
  const float xs[4] = {v.x, v.y, v.z, v.w};
  int8_t o[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) o[j] = (c + j < s.C) ? (xs[j] >= 0.f ? int8_t(1) : int8_t(-1)) : int8_t(0);
  reinterpret_cast<uint32_t *>(s.Sg)[q] = pack4(o[0], o[1], o[2], o[3]);
}

static cudaError_t launch_sign(const StateView &s, cudaStream_t st) {
  const size_t quads = size_t(s.N) * s.Cp / 4;
  k_sign<<<unsigned((quads + 255) / 256), 256, 0, st>>>(s);
  return cudaGetLastError();
}

constexpr int kEnergyRows = 32;  // rows per block of the energy kernels

int energy_row_blocks(int N) { return (N + kEnergyRows - 1) / kEnergyRows; }

// Block reduction of per-warp column partials (8 warps x 128 columns) into
// part[blockIdx.y][col0 + c], in warp order.
template <typename T>
__device__ __forceinline__ void reduce_block_cols(T (*sm)[kColsPerWarp], const T v[4], T *part,
                                                  int Cp, int col0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 4; ++j) sm[warp][lane * 4 + j] = v[j];
  __syncthreads();
  if (threadIdx.x < kColsPerWarp) {
    T acc = T(0);
    for (int w = 0; w < 8; ++w) acc += sm[w][threadIdx.x];
    part[size_t(blockIdx.y) * Cp + col0 + threadIdx.x] = acc;
  }
}

// ---------------------------------------------------------------- CSR energies
template <bool INT>
__global__ void __launch_bounds__(256) k_energy_csr(StateView s, CsrView J, EnergyView E,
                                                    BestView b) {
  using T = typename std::conditional<INT, long long, double>::type;
  __shared__ T sm[8][kColsPerWarp];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col0 = blockIdx.x * kColsPerWarp;
  const int c4 = col0 + lane * 4;
  T v[4] = {T(0), T(0), T(0), T(0)};
  for (int a = 0; a < 4; ++a) {
    const int i = blockIdx.y * kEnergyRows + warp * 4 + a;
    if (i >= s.N) break;
    const uint32_t si4 = *reinterpret_cast<const uint32_t *>(s.Sg + size_t(i) * s.Cp + c4);
    T t[4] = {T(0), T(0), T(0), T(0)};
    for (int e = J.row_ptr[i]; e < J.row_ptr[i + 1]; ++e) {
      const int j = J.col[e];
      const uint32_t sj4 = *reinterpret_cast<const uint32_t *>(s.Sg + size_t(j) * s.Cp + c4);
      const T w = INT ? T(E.val_i32[e]) : T(E.val_f64[e]);
#pragma unroll
      for (int q = 0; q < 4; ++q) t[q] += w * T(int8_t(sj4 >> (8 * q)));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T si = T(int8_t(si4 >> (8 * q)));
      if constexpr (INT) v[q] += si * t[q] + 2 * T(E.h_i64[i]) * si;
      else v[q] += si * (0.5 * t[q] + E.h_f64[i]);
    }
  }
  reduce_block_cols<T>(sm, v, INT ? reinterpret_cast<T *>(b.part_int) : reinterpret_cast<T *>(b.part_f64),
                       s.Cp, col0);
}

// ---------------------------------------------------------------- dense energies
template <bool INT>
__global__ void __launch_bounds__(256) k_energy_dense(StateView s, EnergyView E, BestView b) {
  using T = typename std::conditional<INT, long long, double>::type;
  using W = typename std::conditional<INT, int, double>::type;
  __shared__ W Js[kEnergyRows][33];
  __shared__ __align__(16) int8_t Ss[32][kColsPerWarp];
  __shared__ T sm[8][kColsPerWarp];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.y * kEnergyRows, col0 = blockIdx.x * kColsPerWarp;
  const int N = s.N;
  W acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = W(0);
  for (int k0 = 0; k0 < N; k0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = threadIdx.x + q * 256, r = idx >> 5, k = idx & 31;
      const int gi = row0 + r, gk = k0 + k;
      W w = W(0);
      if (gi < N && gk < N) w = INT ? W(E.val_i32[size_t(gi) * N + gk]) : W(E.val_f64[size_t(gi) * N + gk]);
      Js[r][k] = w;
    }
    {
      const int r = threadIdx.x >> 3, seg = (threadIdx.x & 7) * 16;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (k0 + r < N) v = *reinterpret_cast<const uint4 *>(s.Sg + size_t(k0 + r) * s.Cp + col0 + seg);
      *reinterpret_cast<uint4 *>(&Ss[r][seg]) = v;
    }
    __syncthreads();
    for (int k = 0; k < 32; ++k) {
      const uint32_t s4 = *reinterpret_cast<const uint32_t *>(&Ss[k][lane * 4]);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const W w = Js[warp * 4 + a][k];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q] += w * W(int8_t(s4 >> (8 * q)));
      }
    }
    __syncthreads();
  }
  T v[4] = {T(0), T(0), T(0), T(0)};
  const int c4 = col0 + lane * 4;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = row0 + warp * 4 + a;
    if (i >= N) continue;
    const uint32_t si4 = *reinterpret_cast<const uint32_t *>(s.Sg + size_t(i) * s.Cp + c4);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T si = T(int8_t(si4 >> (8 * q)));
      if constexpr (INT) v[q] += si * T(acc[a][q]) + 2 * T(E.h_i64[i]) * si;
      else v[q] += si * (0.5 * T(acc[a][q]) + E.h_f64[i]);
    }
  }
  reduce_block_cols<T>(sm, v, INT ? reinterpret_cast<T *>(b.part_int) : reinterpret_cast<T *>(b.part_f64),
                       s.Cp, col0);
}

// Column totals in a fixed order: lanes stride over row blocks, then a
// shuffle tree.
template <bool INT>
__global__ void k_energy_final(StateView s, BestView b) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= s.C) return;
  if constexpr (INT) {
    long long acc = 0;
    for (int k = lane; k < b.nblk; k += 32) acc += b.part_int[size_t(k) * s.Cp + c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const long long e = -(acc / 2);
      b.e_int[c] = e;
      b.e_f64[c] = double(e);
    }
  } else {
    double acc = 0.0;
    for (int k = lane; k < b.nblk; k += 32) acc += b.part_f64[size_t(k) * s.Cp + c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) b.e_f64[c] = -acc;
  }
}

static cudaError_t launch_final(const StateView &s, const EnergyView &E, const BestView &b,
                                cudaStream_t st) {
  const unsigned blocks = unsigned((s.C + 7) / 8);
  if (E.is_integer) k_energy_final<true><<<blocks, 256, 0, st>>>(s, b);
  else k_energy_final<false><<<blocks, 256, 0, st>>>(s, b);
  return cudaGetLastError();
}

cudaError_t launch_energy_csr(const StateView &s, const CsrView &J, const EnergyView &E,
                              const BestView &b, cudaStream_t st) {
  cudaError_t err = launch_sign(s, st);
  if (err != cudaSuccess) return err;
  dim3 grid(s.Cp / kColsPerWarp, energy_row_blocks(s.N));
  if (E.is_integer) k_energy_csr<true><<<grid, 256, 0, st>>>(s, J, E, b);
  else k_energy_csr<false><<<grid, 256, 0, st>>>(s, J, E, b);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  return launch_final(s, E, b, st);
}

cudaError_t launch_energy_dense(const StateView &s, const EnergyView &E, const BestView &b,
                                cudaStream_t st) {
  cudaError_t err = launch_sign(s, st);
  if (err != cudaSuccess) return err;
  dim3 grid(s.Cp / kColsPerWarp, energy_row_blocks(s.N));
  if (E.is_integer) k_energy_dense<true><<<grid, 256, 0, st>>>(s, E, b);
  else k_energy_dense<false><<<grid, 256, 0, st>>>(s, E, b);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  return launch_final(s, E, b, st);
}

cudaError_t launch_energy_dense_tc(const void *plan, const StateView &s, int Kp, uint8_t *FT, int buffer, int *err,
                                   const EnergyView &E, const BestView &b, cudaStream_t st) {
  cudaError_t e = launch_sign(s, st);
  if (e != cudaSuccess) return e;
  e = launch_energy_partials_tc(plan, s, Kp, FT, buffer, err, E.h_i64, b.part_int, b.nblk, st);
  if (e != cudaSuccess) return e;
  return launch_final(s, E, b, st);
}

// ---------------------------------------------------------------- best per run
// One block per run: warp 0 takes the argmin over the Pr replicas (lowest k
// on ties; replica k of run r is column r * P + k), kept if strictly lower
// than the best so far; then all threads copy the winner's spins (a strided
// gather of N bytes).
constexpr int kBestThreads = 256;

__global__ void __launch_bounds__(kBestThreads) k_best(StateView s, EnergyView E, BestView b, int step) {
  __shared__ int s_k;  // the winning replica, or -1 when the run does not improve
  const int r = blockIdx.x;
  const int lane = threadIdx.x & 31;
  const int P = s.P;
  if (threadIdx.x < 32) {
    long long ei = LLONG_MAX;
    double ef = DBL_MAX;
    int k = lane;
    for (int q = lane; q < s.Pr; q += 32) {  // each lane: the lowest of its replicas, the first on ties
      const long long qi = E.is_integer ? b.e_int[r * P + q] : 0;
      const double qf = E.is_integer ? 0.0 : b.e_f64[r * P + q];
      if (q == lane || (E.is_integer ? qi < ei : qf < ef)) {
        ei = E.is_integer ? qi : LLONG_MAX;
        ef = E.is_integer ? DBL_MAX : qf;
        k = q;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const long long oi = __shfl_down_sync(0xffffffffu, ei, o);
      const double of = __shfl_down_sync(0xffffffffu, ef, o);
      const int ok = __shfl_down_sync(0xffffffffu, k, o);
      const bool better = E.is_integer ? (oi < ei || (oi == ei && ok < k)) : (of < ef || (of == ef && ok < k));
      if (better) { ei = oi; ef = of; k = ok; }
    }
    if (lane == 0) {
      const bool have = b.have_best[r] != 0;
      const bool improve = !have || (E.is_integer ? ei < b.best_e_int[r] : ef < b.best_e[r]);
      s_k = improve ? k : -1;
      if (improve) {
        b.best_e_int[r] = E.is_integer ? ei : 0;
        b.best_e[r] = E.is_integer ? double(ei) : ef;
        b.best_k[r] = k;
        b.best_step[r] = step;
        b.have_best[r] = 1;
      }
    }
  }
  __syncthreads();
  const int k = s_k;
  if (k < 0) return;
  const int c = r * P + k;
  for (int i = threadIdx.x; i < s.N; i += kBestThreads) b.best_spins[size_t(r) * s.N + i] = s.Sg[size_t(i) * s.Cp + c];
}

cudaError_t launch_best(const StateView &s, const EnergyView &E, const BestView &b, int step,
                        cudaStream_t st) {
  k_best<<<s.R, kBestThreads, 0, st>>>(s, E, b, step);
  return cudaGetLastError();
}

__global__ void k_reset_best(int R, BestView b) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  b.have_best[r] = 0;
  b.best_e_int[r] = LLONG_MAX;
  b.best_e[r] = DBL_MAX;
  b.best_k[r] = -1;
  b.best_step[r] = -2;
}

cudaError_t launch_reset_best(const StateView &s, const BestView &b, cudaStream_t st) {
  k_reset_best<<<(s.R + 127) / 128, 128, 0, st>>>(s.R, b);
  return cudaGetLastError();
}

}  // namespace sbqa
