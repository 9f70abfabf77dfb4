// energy_noalloc.cu -- Ising energies of caller-supplied spin configurations
// for a CSR instance, computed without allocating any device memory.
//
// Some callers cannot allocate device memory at the point where they need
// energies: code running while a CUDA graph is being captured (cudaMalloc is
// not a capturable operation), real-time loops that must not block on the
// allocator, and hosts that route every allocation through their own pool
// and forbid the library from calling cudaMalloc behind their back.  This
// entry point serves them: inputs and outputs are the caller's device
// buffers, and the only extra memory it uses is a fixed scratch array that
// is part of the library image (a file-scope __device__ array, reserved on
// every GPU that loads the library until the process exits).
//
// The computation is the readout of the hot path (same formula and the same
// fixed summation order as the per-run readout kernels):
//   E(s) = -(1/2) sum_i (s_i t_i + 2 h_i s_i),  t_i = sum_j J_ij s_j
// with int64 arithmetic for integer instances and FP64 otherwise.  Row
// blocks of 32 spins write partial column sums into the scratch array; a
// second kernel adds them in a fixed order.  Every scratch entry that is read
// is written earlier in the same call, so nothing has to be cleared between
// calls.
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/sbqa.h"
#include "internal.h"

namespace {

constexpr int kRows = 32;         // spins per row block
constexpr int kCols = 128;        // configurations per block (32 lanes x 4)
constexpr size_t kScratchBytes = size_t(4) << 20;  // 4 MiB
constexpr size_t kScratchWords = kScratchBytes / 8;

// Partial sums [row blocks][configurations padded to 128], int64 or double.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

template <bool INT>
__global__ void __launch_bounds__(256) k_energy_noalloc(int n, const int32_t *row_ptr, const int32_t *col,
                                                        const int32_t *val_i32, const double *val_f64,
                                                        const int64_t *h_i64, const double *h_f64,
                                                        const int8_t *spins, int ld, int count,
                                                        int cols_pad, void *scratch) {
  using T = typename std::conditional<INT, long long, double>::type;
  __shared__ T sm[8][kCols];
  T *part = static_cast<T *>(scratch);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col0 = blockIdx.x * kCols;
  T v[4] = {T(0), T(0), T(0), T(0)};
  for (int a = 0; a < 4; ++a) {
    const int i = blockIdx.y * kRows + warp * 4 + a;
    if (i >= n) break;
    int8_t si[4];
    for (int q = 0; q < 4; ++q) {
      const int c = col0 + lane * 4 + q;
      si[q] = c < count ? spins[size_t(i) * ld + c] : int8_t(0);
    }
    T t[4] = {T(0), T(0), T(0), T(0)};
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const int j = col[e];
      const T w = INT ? T(val_i32[e]) : T(val_f64[e]);
      for (int q = 0; q < 4; ++q) {
        const int c = col0 + lane * 4 + q;
        const int8_t sj = c < count ? spins[size_t(j) * ld + c] : int8_t(0);
        t[q] += w * T(sj);
      }
    }
    for (int q = 0; q < 4; ++q) {
      const T s = T(si[q]);
      if constexpr (INT) v[q] += s * t[q] + 2 * T(h_i64 ? h_i64[i] : 0) * s;
      else v[q] += s * (0.5 * t[q] + (h_f64 ? h_f64[i] : 0.0));
    }
  }
  for (int q = 0; q < 4; ++q) sm[warp][lane * 4 + q] = v[q];
  __syncthreads();
  if (threadIdx.x < kCols) {
    T acc = T(0);
    for (int w = 0; w < 8; ++w) acc += sm[w][threadIdx.x];
    part[size_t(blockIdx.y) * cols_pad + col0 + threadIdx.x] = acc;
  }
}

template <bool INT>
__global__ void k_energy_noalloc_final(int count, int nblk, int cols_pad, const void *scratch, int64_t *out_i64,
                                       double *out_f64) {
  using T = typename std::conditional<INT, long long, double>::type;
  const T *part = static_cast<const T *>(scratch);
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= count) return;
  T acc = T(0);
  for (int k = lane; k < nblk; k += 32) acc += part[size_t(k) * cols_pad + c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    if constexpr (INT) {
      const long long e = -(acc / 2);
      if (out_i64) out_i64[c] = e;
      if (out_f64) out_f64[c] = double(e);
    } else {
      out_f64[c] = -acc;
    }
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per
// device; cudaGetSymbolAddress must not run inside a stream capture).
int scratch_for_current_device(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return sbqa::set_error(SBQA_ERR_CUDA, "sbqa_energies_csr_noalloc: no usable current device");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return sbqa::set_error(SBQA_ERR_CUDA, std::string("sbqa_energies_csr_noalloc: cudaGetSymbolAddress: ") +
                                                cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return SBQA_OK;
}

}  // namespace

extern "C" int sbqa_energies_csr_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                         const int32_t *val_i32, const double *val_f64, const int64_t *h_i64,
                                         const double *h_f64, const int8_t *spins, int32_t ld, int32_t count,
                                         int64_t *energy_int, double *energy, void *stream) {
  const bool integer = val_i32 != nullptr;
  if (n < 1 || count < 1 || ld < count || !row_ptr || !col_idx || !spins || (integer == (val_f64 != nullptr)) ||
      (!integer && (h_i64 || !energy)) || (integer && (h_f64 || (!energy_int && !energy))))
    return sbqa::set_error(SBQA_ERR_INVALID_ARG,
                           "sbqa_energies_csr_noalloc: need n, count >= 1, ld >= count, row_ptr, col_idx, spins, "
                           "exactly one of val_i32 / val_f64 with the matching h and an output");
  // sizes in 64 bits: count near INT32_MAX must reach the limit check, not overflow before it
  const int64_t nblk64 = (int64_t(n) + kRows - 1) / kRows;
  const int64_t cols_pad64 = (int64_t(count) + kCols - 1) / kCols * kCols;
  if (nblk64 * cols_pad64 > int64_t(kScratchWords))
    return sbqa::set_error(SBQA_ERR_UNSUPPORTED,
                           "sbqa_energies_csr_noalloc: ceil(n/32) * ceil(count/128)*128 = " +
                               std::to_string(nblk64 * cols_pad64) + " exceeds the scratch limit of " +
                               std::to_string(kScratchWords) + " partial sums (4 MiB)");
  const int nblk = int(nblk64), cols_pad = int(cols_pad64);
  void *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != SBQA_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 grid(cols_pad / kCols, nblk);
  const unsigned fblocks = unsigned((count + 7) / 8);
  if (integer) {
    k_energy_noalloc<true><<<grid, 256, 0, st>>>(n, row_ptr, col_idx, val_i32, nullptr, h_i64, nullptr, spins, ld,
                                                 count, cols_pad, scratch);
    k_energy_noalloc_final<true><<<fblocks, 256, 0, st>>>(count, nblk, cols_pad, scratch, energy_int, energy);
  } else {
    k_energy_noalloc<false><<<grid, 256, 0, st>>>(n, row_ptr, col_idx, nullptr, val_f64, nullptr, h_f64, spins, ld,
                                                  count, cols_pad, scratch);
    k_energy_noalloc_final<false><<<fblocks, 256, 0, st>>>(count, nblk, cols_pad, scratch, nullptr, energy);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return sbqa::set_error(SBQA_ERR_CUDA, std::string("sbqa_energies_csr_noalloc: launch: ") + cudaGetErrorString(e));
  return SBQA_OK;
}
