// step_dense_tc.cu -- one SBQA step for dense integer couplings on the 5th
// generation tensor cores (tcgen05), product and update fused.
//
// G = J . f(X) (Sec. II A, Eq. 7).  f(X) is in {-1, 0, +1} and J holds small
// integers (|J_ij| <= 16), all exact in FP8 e4m3, and an FP32 accumulation of
// at most 2^16 such products is exact: the product equals the CUDA-core
// result bit for bit.  (tcgen05.mma kind::i8 does not exist on sm_103a, so
// kind::f8f6f4 with e4m3 operands is the exact path.)
//
// Operands (K = spin index j, padded to Kp, a multiple of 128, with zeros):
//   A = J8   [Kp rows i][Kp cols j]   e4m3, K-major
//   B = FT8  [2][Cp][Kp]              e4m3 f(x) transposed (column c, spin j),
//                                     K-major, double-buffered by step parity
// Tile: 128 spin rows x 128 replica columns per CTA (one wave of 128 CTAs for
// N = 2000, R*P = 1024).  Three TMA stages of 128 x 128-byte tiles of A and B
// (128-byte swizzle) feed tcgen05.mma M=128 N=128 K=32 (4 per stage); the
// FP32 accumulator lives in 128 TMEM columns.  Thread 0 of warp 0 issues the
// TMA loads -- the operand stages and, behind the first stages, the x and y
// tiles of the CTA (4 boxes of 128 rows x 32 floats each) -- and thread 0 of
// warp 1 the MMAs.  The epilogue then works in shared memory: every warp
// reads its 32 TMEM lanes (= spin rows) for 64 columns, updates whole runs of
// 32 columns in place in the swizzled state boxes and stages f(x_next) as
// e4m3; finally one thread stores x, y and the transposed f tile with TMA.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "step_common.cuh"
#include "tc_common.cuh"

namespace sbqa {

constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 128, kTcStages = 3;
constexpr int kTcThreads = 256;          // 8 warps: all run the epilogue
constexpr int kTcTile = kTcBM * kTcBK;   // bytes of one operand stage (e4m3)
constexpr int kTcBox = kTcBM * 128;      // one 128-row x 32-float state box (16 KB)
constexpr int kTcStateTile = 4 * kTcBox; // x or y tile, 128 rows x 128 columns (64 KB)
constexpr int kTcSmem = 2 * kTcStages * kTcTile + 2 * kTcStateTile + 1024 + 128;
constexpr uint8_t kE4M3One = 0x38, kE4M3MinusOne = 0xB8;

struct TcArgs {
  int Kp;
  uint8_t *FT;  // [2][Cp][Kp]
  int *err;     // device error flag (0 = ok)
  const float *h;
};

struct TcMaps {
  CUtensorMap A, B;  // J8 and FT operand tiles (128 x 128 bytes, 128B swizzle)
  CUtensorMap X, Y;  // x, y state boxes (128 rows x 32 floats, 128B swizzle)
  CUtensorMap Fst;   // FT tile store (128 columns x 128 spins bytes, no swizzle)
};

__device__ __forceinline__ uint8_t f_to_e4m3(int8_t f) {
  return f == 0 ? uint8_t(0) : (f > 0 ? kE4M3One : kE4M3MinusOne);
}

// Address of the float4 (16-byte chunk u, 0..7) of row r inside a 128B-swizzled
// box of 128-byte rows: chunks are permuted by XOR with r mod 8.
__device__ __forceinline__ float4 *box_chunk(uint8_t *box, int r, int u) {
  return reinterpret_cast<float4 *>(box + r * 128 + ((u ^ (r & 7)) << 4));
}

// Update of one spin row for 32 aligned columns c0..c0+31 (whole runs,
// because P divides 32); x and y are read from and written back to one row of
// the swizzled shared-memory state boxes.  Same arithmetic, in the same
// order, as sb_update4.
template <int P>
__device__ __forceinline__ void sb_update_row32(const StateView &s, const StepTables &t, float ka, float dnext,
                                                const float *kjn, int c0, const uint32_t (&g)[32], float hi,
                                                uint8_t *xbox, uint8_t *ybox, int r, int8_t (&f)[32]) {
  float xs[32], ys[32];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const float4 a = *box_chunk(xbox, r, u), b = *box_chunk(ybox, r, u);
    xs[4 * u] = a.x; xs[4 * u + 1] = a.y; xs[4 * u + 2] = a.z; xs[4 * u + 3] = a.w;
    ys[4 * u] = b.x; ys[4 * u + 1] = b.y; ys[4 * u + 2] = b.z; ys[4 * u + 3] = b.w;
  }
  float kjv[32 / (P < 32 ? P : 32)];
#pragma unroll
  for (int q = 0; q < 32 / (P < 32 ? P : 32); ++q) kjv[q] = (c0 + q * P < s.C) ? __ldg(kjn + c0 / P + q) : 0.f;
  float xo[32], yo[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int k = j % P, base = j - k;
    const float xm = xs[base + (k + P - 1) % P], xp = xs[base + (k + 1) % P];
    f[j] = 0;
    xo[j] = xs[j];
    yo[j] = ys[j];
    if (c0 + j >= s.C) continue;
    const float kj = kjv[j / (P < 32 ? P : 32)];
    float yn = fmaf(t.kc, __uint_as_float(g[j]) + hi, ys[j]);
    yn = fmaf(-ka, xs[j], yn);
    yn = fmaf(kj, xm + xp, yn);
    float xn = fmaf(t.kx, yn, xs[j]);
    if (fabsf(xn) > 1.f) {
      xn = copysignf(1.f, xn);
      yn = 0.f;
    }
    xo[j] = xn;
    yo[j] = yn;
    f[j] = thresh(xn, dnext);
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    *box_chunk(xbox, r, u) = make_float4(xo[4 * u], xo[4 * u + 1], xo[4 * u + 2], xo[4 * u + 3]);
    *box_chunk(ybox, r, u) = make_float4(yo[4 * u], yo[4 * u + 1], yo[4 * u + 2], yo[4 * u + 3]);
  }
}

template <int P>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_step_dense_tc(const __grid_constant__ TcMaps m, StateView s, TcArgs a, StepTables t, int n) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = smem;
  uint8_t *sB = smem + kTcStages * kTcTile;
  uint8_t *sX = smem + 2 * kTcStages * kTcTile;
  uint8_t *sY = sX + kTcStateTile;
  uint64_t *full = reinterpret_cast<uint64_t *>(sY + kTcStateTile);
  uint64_t *empty = full + kTcStages;
  uint64_t *done = empty + kTcStages;
  uint64_t *xy_full = done + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(xy_full + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * kTcBN;
  const int KB = a.Kp / kTcBK;
  const int brow = (n & 1) * s.Cp + n0;  // row of F_n in the [2 Cp][Kp] map

  if (threadIdx.x == 0) {
    for (int q = 0; q < kTcStages; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&empty[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(xy_full, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&m.A);
    tc::prefetch_tmap(&m.B);
    tc::prefetch_tmap(&m.X);
    tc::prefetch_tmap(&m.Y);
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, 128);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    bool xy_issued = false;
    for (int kb = 0; kb < KB; ++kb) {
      const int st = kb % kTcStages, q = kb / kTcStages;
      if (q > 0 && !tc::mbar_wait(&empty[st], (q - 1) & 1, a.err, tc::ERR_WAIT_EMPTY)) break;
      tc::mbar_arrive_expect_tx(&full[st], 2 * kTcTile);
      tc::tma_load_2d(sA + st * kTcTile, &m.A, &full[st], kb * kTcBK, m0);
      tc::tma_load_2d(sB + st * kTcTile, &m.B, &full[st], kb * kTcBK, brow);
      if (!xy_issued && (kb == kTcStages - 1 || kb == KB - 1)) {
        // the state tile, needed only by the epilogue, loads behind the first stages
        tc::mbar_arrive_expect_tx(xy_full, 2 * kTcStateTile);
        for (int b = 0; b < 4; ++b) {
          tc::tma_load_2d(sX + b * kTcBox, &m.X, xy_full, n0 + 32 * b, m0);
          tc::tma_load_2d(sY + b * kTcBox, &m.Y, xy_full, n0 + 32 * b, m0);
        }
        xy_issued = true;
      }
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = tc::idesc_f8_e4m3(kTcBM, kTcBN);
    for (int kb = 0; kb < KB; ++kb) {
      const int st = kb % kTcStages, q = kb / kTcStages;
      if (!tc::mbar_wait(&full[st], q & 1, a.err, tc::ERR_WAIT_FULL)) break;
      tc::tc_fence_after();
      const uint32_t a0 = tc::smem_u32(sA + st * kTcTile), b0 = tc::smem_u32(sB + st * kTcTile);
#pragma unroll
      for (int kk = 0; kk < kTcBK / 32; ++kk)
        tc::mma_f8(tmem, tc::smem_desc_sw128(a0 + kk * 32), tc::smem_desc_sw128(b0 + kk * 32), idesc,
                   (kb | kk) != 0 ? 1u : 0u);
      tc::mma_commit(&empty[st]);
    }
    tc::mma_commit(done);
  }
  __syncwarp();
  const float ka = __ldg(t.ka + n), dnext = __ldg(t.dl + n + 1);
  const float *kjn = t.kj + size_t(n) * t.R;
  const int quarter = warp & 3, half = warp >> 2;
  const int rl = quarter * 32 + lane;
  const int i = m0 + rl;
  const float hi = i < s.N ? __ldg(a.h + i) : 0.f;
  tc::mbar_wait(done, 0, a.err, tc::ERR_WAIT_DONE);
  tc::mbar_wait(xy_full, 0, a.err, tc::ERR_WAIT_FULL);
  tc::tc_fence_after();

  // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (= spin rows) and
  // columns 64 (w / 4) .. + 63 in two chunks of 32 (one state box each).
  uint8_t *sF = sA;  // [128 columns][128 spins] e4m3 f(x_next); the operand stages are consumed
#pragma unroll 1
  for (int cc = 0; cc < 2; ++cc) {
    const int b = half * 2 + cc;  // state box
    const int cl = 32 * b;        // first column of the chunk inside the tile
    const int c0 = n0 + cl;
    uint32_t g[32];
    tc::tmem_ld_32x32b_x32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(cl), g);
    int8_t f[32];
    if (i < s.N && c0 < s.C) {
      sb_update_row32<P>(s, t, ka, dnext, kjn, c0, g, hi, sX + b * kTcBox, sY + b * kTcBox, rl, f);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) f[j] = 0;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) sF[(cl + j) * kTcBM + rl] = f_to_e4m3(f[j]);
  }
  tc::fence_proxy_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    // x, y boxes back (rows past N are clipped by the tensor map) and the f
    // tile into the other FT buffer: column n0 + c, spins m0 .. m0 + 127
    for (int b = 0; b < 4; ++b) {
      tc::tma_store_2d(&m.X, sX + b * kTcBox, n0 + 32 * b, m0);
      tc::tma_store_2d(&m.Y, sY + b * kTcBox, n0 + 32 * b, m0);
    }
    tc::tma_store_2d(&m.Fst, sF, m0, ((n + 1) & 1) * s.Cp + n0);
    tc::tma_store_commit_and_wait_read();
  }
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// f codes [N][Cp] -> e4m3 f [Cp][Kp] (zeros for padded spins), for buffer b.
__global__ void k_f_to_ft8(StateView s, int which, uint8_t *FT, int Kp, int b) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;  // over Cp * Kp
  if (e >= size_t(s.Cp) * Kp) return;
  const int c = int(e / Kp), j = int(e % Kp);
  const int8_t f = (j < s.N) ? int8_t(int(s.f_of(which)[size_t(j) * s.Cp + c]) - 1) : int8_t(0);
  FT[size_t(b) * s.Cp * Kp + e] = f_to_e4m3(f);
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D tensor map [rows][cols] (cols contiguous) with the given box and swizzle.
static bool make_map(CUtensorMap *m, const void *base, CUtensorMapDataType dt, size_t esize, uint64_t rows,
                     uint64_t cols, uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle sw) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * esize};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_plan_make(void **plan, const uint8_t *J8, uint8_t *FT, int Kp, int Cp, float *x, float *y, int N) {
  auto *p = new TcMaps();
  const auto U8 = CU_TENSOR_MAP_DATA_TYPE_UINT8, F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const bool ok = make_map(&p->A, J8, U8, 1, uint64_t(Kp), uint64_t(Kp), 128, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
                  make_map(&p->B, FT, U8, 1, uint64_t(2) * Cp, uint64_t(Kp), 128, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
                  make_map(&p->X, x, F32, 4, uint64_t(N), uint64_t(Cp), 32, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
                  make_map(&p->Y, y, F32, 4, uint64_t(N), uint64_t(Cp), 32, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
                  make_map(&p->Fst, FT, U8, 1, uint64_t(2) * Cp, uint64_t(Kp), 128, 128, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (!ok) {
    delete p;
    return false;
  }
  *plan = p;
  return true;
}

void tc_plan_free(void *plan) { delete static_cast<TcMaps *>(plan); }

cudaError_t tc_set_attributes() {
  const void *fns[6] = {(const void *)k_step_dense_tc<1>, (const void *)k_step_dense_tc<2>,
                        (const void *)k_step_dense_tc<4>, (const void *)k_step_dense_tc<8>,
                        (const void *)k_step_dense_tc<16>, (const void *)k_step_dense_tc<32>};
  for (const void *f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int P>
static cudaError_t launch_tc_p(const TcMaps *p, const StateView &s, const TcArgs &a, const StepTables &t, int n,
                               cudaStream_t st) {
  dim3 grid(s.Cp / kTcBN, a.Kp / kTcBM);
  k_step_dense_tc<P><<<grid, kTcThreads, kTcSmem, st>>>(*p, s, a, t, n);
  return cudaGetLastError();
}

cudaError_t launch_step_dense_tc(const void *plan, const StateView &s, int Kp, uint8_t *FT, int *err, const float *h,
                                 const StepTables &t, int n, cudaStream_t st) {
  const auto *p = static_cast<const TcMaps *>(plan);
  TcArgs a{Kp, FT, err, h};
  switch (s.P) {
    case 1: return launch_tc_p<1>(p, s, a, t, n, st);
    case 2: return launch_tc_p<2>(p, s, a, t, n, st);
    case 4: return launch_tc_p<4>(p, s, a, t, n, st);
    case 8: return launch_tc_p<8>(p, s, a, t, n, st);
    case 16: return launch_tc_p<16>(p, s, a, t, n, st);
    case 32: return launch_tc_p<32>(p, s, a, t, n, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_f_to_ft8(const StateView &s, int which, uint8_t *FT, int Kp, int buffer, cudaStream_t st) {
  const size_t total = size_t(s.Cp) * Kp;
  k_f_to_ft8<<<unsigned((total + 255) / 256), 256, 0, st>>>(s, which, FT, Kp, buffer);
  return cudaGetLastError();
}

}  // namespace sbqa
