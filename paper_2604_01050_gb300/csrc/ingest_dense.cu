// ingest_dense.cu -- a dense coupling matrix read by the GPU straight from
// the caller's host array, and the device forms made from the device copy.
//
// On systems where the GPU reaches pageable host memory through the host's
// page tables (cudaDevAttrPageableMemoryAccessUsesHostPageTables), the
// checks and statistics that sbqa_create_problem_dense needs -- finiteness,
// a zero diagonal, symmetry, integrality, +-1, max |J_ij|, the sum of
// squares (the scale c0 of Eq. 6) and the row degrees -- run in one pass
// over the caller's FP64 J (tile against mirror tile, every entry read
// once), and the library's copy of J stays in device
// memory: one byte per entry (integer values in [-128, 127], exactly as the
// host pass stores them) and the FP64 values.  The operand and readout forms
// (e4m3 or bfloat16 for the tensor cores, int32 / FP64 for the readout, FP32
// or bfloat16 for the CUDA-core kernel) are then converted on the device with
// the same rules as the host conversions, so both ways give the same bits.
#include <cstdint>

#include "internal.h"

namespace sbqa {

namespace {

// Row statistics, reduced in a fixed order (results do not depend on timing).
__device__ __forceinline__ void warp_reduce(double &mx, double &s2, int &nnz, unsigned &flags) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
    nnz += __shfl_down_sync(0xffffffffu, nnz, o);
    flags &= __shfl_down_sync(0xffffffffu, flags, o);
  }
}

// One pass over J (host memory), each entry read once: block (bi, bj), bi <=
// bj, takes the 32 x 32 tile (bi, bj) and its mirror (bj, bi) (the diagonal
// tile alone), compares the two for symmetry (any difference sets *asym),
// writes both tiles' byte copy d8 (int(v) for v in [-128, 127], else 0, as
// the host pass) and FP64 copy d64, and for every row of each tile the
// statistics of its 32 entries into part[tile column][row] (warp-shuffle
// sums in a fixed order).
__device__ __forceinline__ void tile_row_stats(double v, int i, int j, IngestRow *out) {
  double mx = 0.0, s2 = 0.0;
  int nnz = 0;
  unsigned flags = kIngestFinite | kIngestDiagZero | kIngestInteger | kIngestPm1;
  if (!isfinite(v)) flags &= ~kIngestFinite;
  if (v != 0.0) {
    nnz = 1;
    if (v != rint(v)) flags &= ~kIngestInteger;
    if (fabs(v) != 1.0) flags &= ~kIngestPm1;
    mx = fabs(v);
    s2 = v * v;
    if (j == i) flags &= ~kIngestDiagZero;
  }
  warp_reduce(mx, s2, nnz, flags);
  if ((threadIdx.x & 31) == 0) *out = IngestRow{mx, s2, nnz, flags};
}

__global__ void __launch_bounds__(256) k_ingest_tiles(const double *__restrict__ J, int n, int8_t *d8, double *d64,
                                                      IngestRow *part, int *asym) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj < bi) return;
  __shared__ double tb[32][33];  // the mirror tile (bj, bi), or the tile itself on the diagonal
  const int c = threadIdx.x & 31, r0 = threadIdx.x >> 5;
  const bool diag = bi == bj;
  // the mirror tile first (its entries are compared against the transposed reads below)
  for (int r = r0; r < 32; r += 8) {
    const int i = bj * 32 + r, j = bi * 32 + c;
    tb[r][c] = (i < n && j < n) ? J[size_t(i) * n + j] : 0.0;
  }
  __syncthreads();
  bool same = true;
  for (int r = r0; r < 32; r += 8) {
    const int i = bi * 32 + r, j = bj * 32 + c;
    const bool in = i < n && j < n;
    const double v = in ? (diag ? tb[r][c] : J[size_t(i) * n + j]) : 0.0;
    if (in) {
      same = same && v == tb[c][r];
      d8[size_t(i) * n + j] = int8_t(v >= -128.0 && v <= 127.0 ? int(v) : 0);
      d64[size_t(i) * n + j] = v;
    }
    if (i < n) tile_row_stats(v, i, j, part + size_t(bj) * n + i);  // padding adds nothing
    if (!diag) {  // row j' = bj * 32 + r of the mirror tile
      const int i2 = bj * 32 + r, j2 = bi * 32 + c;
      const bool in2 = i2 < n && j2 < n;
      const double w = in2 ? tb[r][c] : 0.0;
      if (in2) {
        d8[size_t(i2) * n + j2] = int8_t(w >= -128.0 && w <= 127.0 ? int(w) : 0);
        d64[size_t(i2) * n + j2] = w;
      }
      if (i2 < n) tile_row_stats(w, i2, j2, part + size_t(bi) * n + i2);
    }
  }
  if (!__all_sync(0xffffffffu, same) && c == 0) atomicOr(asym, 1);
}

// Row i's statistics from its tiles' partials, in tile-column order.
__global__ void k_ingest_rows_reduce(const IngestRow *__restrict__ part, int n, int nb, IngestRow *rows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  IngestRow r{0.0, 0.0, 0, kIngestFinite | kIngestDiagZero | kIngestInteger | kIngestPm1};
  for (int t = 0; t < nb; ++t) {
    const IngestRow q = part[size_t(t) * n + i];
    r.mx = fmax(r.mx, q.mx);
    r.s2 += q.s2;
    r.nnz += q.nnz;
    r.flags &= q.flags;
  }
  rows[i] = r;
}

// bfloat16 bits of v, round to nearest even in one step from FP64 (the host
// conversion's steps: 8 significant bits of the FP64 value, then FP32).
__device__ __forceinline__ uint16_t bf16_bits_rne_dev(double v) {
  if (v == 0.0) return signbit(v) ? 0x8000u : 0u;
  int e;
  const double m = frexp(v, &e);
  const double q = rint(ldexp(m, 8));
  const float f = float(ldexp(q, e - 8));
  return uint16_t(__float_as_uint(f) >> 16);
}

// e4m3 bits of a small integer (|v| <= 16, exact): 1.mmm x 2^e, bias 7.
__device__ __forceinline__ uint8_t e4m3_of_int_dev(int v) {
  if (v == 0) return 0;
  const uint8_t sign = v < 0 ? 0x80 : 0x00;
  const int a = v < 0 ? -v : v;
  const int e = 31 - __clz(a);
  const int mant = ((a << 3) >> e) & 7;
  return uint8_t(sign | ((e + 7) << 3) | mant);
}

// Padded operand rows [Kp][Kp] from the device copy (zeros past N).
__global__ void k_j8_from_i8(const int8_t *__restrict__ d8, int n, int Kp, uint8_t *out) {
  const size_t m = size_t(Kp) * Kp;
  for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < m; e += size_t(gridDim.x) * blockDim.x) {
    const int i = int(e / Kp), j = int(e % Kp);
    out[e] = (i < n && j < n) ? e4m3_of_int_dev(d8[size_t(i) * n + j]) : uint8_t(0);
  }
}

__global__ void k_jbf16_pad(const int8_t *__restrict__ d8, const double *__restrict__ d64, int n, int Kp,
                            uint16_t *out) {
  const size_t m = size_t(Kp) * Kp;
  for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < m; e += size_t(gridDim.x) * blockDim.x) {
    const int i = int(e / Kp), j = int(e % Kp);
    uint16_t b = 0;
    if (i < n && j < n) {
      const size_t s = size_t(i) * n + j;
      b = bf16_bits_rne_dev(d8 ? double(d8[s]) : d64[s]);
    }
    out[e] = b;
  }
}

// Flat forms [N][N]: int32 or FP64 readout values, FP32 (or bfloat16 values
// held in FP32) for the CUDA-core kernel.
__global__ void k_flat_from(const int8_t *__restrict__ d8, const double *__restrict__ d64, size_t m, int form,
                            void *out) {
  for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < m; e += size_t(gridDim.x) * blockDim.x) {
    const double v = d8 ? double(d8[e]) : d64[e];
    switch (form) {
      case kFlatI32: static_cast<int32_t *>(out)[e] = d8 ? int32_t(d8[e]) : int32_t(llrint(v)); break;
      case kFlatF64: static_cast<double *>(out)[e] = v; break;
      case kFlatF32: static_cast<float *>(out)[e] = float(v); break;
      default: static_cast<float *>(out)[e] = __uint_as_float(uint32_t(bf16_bits_rne_dev(v)) << 16); break;
    }
  }
}

int grid_for(size_t m) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (m + 255) / 256;
  return int(want < size_t(sms) * 8 ? (want > 0 ? want : 1) : size_t(sms) * 8);
}

}  // namespace

bool ingest_on_device_possible() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return v == 1;
}

size_t ingest_part_count(int n) { return size_t((n + 31) / 32) * size_t(n); }

cudaError_t launch_ingest_dense(const double *J, int n, int8_t *d8, double *d64, IngestRow *part, IngestRow *rows,
                                int *asym, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(asym, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int nb = (n + 31) / 32;
  k_ingest_tiles<<<dim3(nb, nb), 256, 0, st>>>(J, n, d8, d64, part, asym);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_ingest_rows_reduce<<<(n + 255) / 256, 256, 0, st>>>(part, n, nb, rows);
  return cudaGetLastError();
}

cudaError_t launch_tc_j8_from_device(const int8_t *d8, int n, int Kp, uint8_t *out, cudaStream_t st) {
  k_j8_from_i8<<<grid_for(size_t(Kp) * Kp), 256, 0, st>>>(d8, n, Kp, out);
  return cudaGetLastError();
}

cudaError_t launch_tc_jbf16_from_device(const int8_t *d8, const double *d64, int n, int Kp, uint16_t *out,
                                        cudaStream_t st) {
  k_jbf16_pad<<<grid_for(size_t(Kp) * Kp), 256, 0, st>>>(d8, d64, n, Kp, out);
  return cudaGetLastError();
}

cudaError_t launch_flat_from_device(const int8_t *d8, const double *d64, size_t m, int form, void *out,
                                    cudaStream_t st) {
  k_flat_from<<<grid_for(m), 256, 0, st>>>(d8, d64, m, form, out);
  return cudaGetLastError();
}

}  // namespace sbqa
