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
// N = 2000, R*P = 1024).  Six TMA stages of 128 x 128-byte tiles of A and B
// (128-byte swizzle) feed tcgen05.mma M=128 N=128 K=32 (4 per stage); the
// FP32 accumulator lives in 128 TMEM columns.  Thread 0 of warp 0 issues the
// TMA loads, thread 0 of warp 1 the MMAs.  Afterwards the x, y tiles are
// brought into shared memory with coalesced loads, every warp reads its 32
// TMEM lanes (= spin rows) for 64 columns and runs the SBQA update on whole
// runs of 32 columns, the tiles go back with coalesced stores, and f(x_next)
// (staged in shared memory) is stored transposed into the other FT8 buffer.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "step_common.cuh"
#include "tc_common.cuh"

namespace sbqa {

constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 128, kTcStages = 6;
constexpr int kTcThreads = 256;  // 8 warps: all run the epilogue
constexpr int kTcTile = kTcBM * kTcBK;  // bytes of one operand stage (e4m3)
constexpr int kTcSmem = 2 * kTcStages * kTcTile + 1024 + 256;
constexpr uint8_t kE4M3One = 0x38, kE4M3MinusOne = 0xB8;

struct TcArgs {
  int Kp;
  uint8_t *FT;  // [2][Cp][Kp]
  int *err;     // device error flag (0 = ok)
  const float *h;
};

__device__ __forceinline__ uint8_t f_to_e4m3(int8_t f) {
  return f == 0 ? uint8_t(0) : (f > 0 ? kE4M3One : kE4M3MinusOne);
}

constexpr int kTileLd = kTcBN + 1;  // padded row of the x, y tiles in shared memory (conflict-free columns)

// Update of one spin row for 32 aligned columns c0..c0+31 (whole runs,
// because P divides 32); x and y are read from and written back to rows of
// the shared-memory tiles.  Same arithmetic, in the same order, as sb_update4.
template <int P>
__device__ __forceinline__ void sb_update_row32(const StateView &s, const StepTables &t, int n, int c0,
                                                const uint32_t (&g)[32], float hi, float *xr, float *yr,
                                                int8_t (&f)[32]) {
  float xs[32], ys[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    xs[j] = xr[j];
    ys[j] = yr[j];
  }
  const float ka = t.ka[n];
  const float dnext = t.dl[n + 1];
  const float *kjn = t.kj + size_t(n) * t.R;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int k = j % P, base = j - k;
    const float xm = xs[base + (k + P - 1) % P], xp = xs[base + (k + 1) % P];
    f[j] = 0;
    if (c0 + j >= s.C) continue;
    const float kj = kjn[(c0 + j) / P];
    float yn = fmaf(t.kc, __uint_as_float(g[j]) + hi, ys[j]);
    yn = fmaf(-ka, xs[j], yn);
    yn = fmaf(kj, xm + xp, yn);
    float xn = fmaf(t.kx, yn, xs[j]);
    if (fabsf(xn) > 1.f) {
      xn = copysignf(1.f, xn);
      yn = 0.f;
    }
    xr[j] = xn;
    yr[j] = yn;
    f[j] = thresh(xn, dnext);
  }
}

template <int P>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_step_dense_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, StateView s,
                    TcArgs a, StepTables t, int n) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = smem;
  uint8_t *sB = smem + kTcStages * kTcTile;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + 2 * kTcStages * kTcTile);
  uint64_t *empty = full + kTcStages;
  uint64_t *done = empty + kTcStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

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
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, 128);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < KB; ++kb) {
      const int st = kb % kTcStages, q = kb / kTcStages;
      if (q > 0 && !tc::mbar_wait(&empty[st], (q - 1) & 1, a.err, tc::ERR_WAIT_EMPTY)) break;
      tc::mbar_arrive_expect_tx(&full[st], 2 * kTcTile);
      tc::tma_load_2d(sA + st * kTcTile, &tmA, &full[st], kb * kTcBK, m0);
      tc::tma_load_2d(sB + st * kTcTile, &tmB, &full[st], kb * kTcBK, brow);
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

  tc::mbar_wait(done, 0, a.err, tc::ERR_WAIT_DONE);
  tc::tc_fence_after();

  // Epilogue.  The operand stages are consumed; their memory now holds the
  // x and y tiles (128 rows x 128 columns, padded rows) and the f codes of
  // the next step.  Global x, y are read and written with coalesced
  // row-contiguous accesses; each thread then works on one spin row.
  float *sx = reinterpret_cast<float *>(smem);
  float *sy = sx + kTcBM * kTileLd;
  uint8_t *sF = reinterpret_cast<uint8_t *>(sy + kTcBM * kTileLd);  // [128 columns][128 rows]
  const int cols_valid = min(kTcBN, s.C - n0);  // multiple of P, hence of 4 when P >= 4
  for (int q = threadIdx.x; q < kTcBM * (kTcBN / 4); q += kTcThreads) {
    const int r = q / (kTcBN / 4), c = (q % (kTcBN / 4)) * 4;
    if (m0 + r < s.N && c < cols_valid) {
      const size_t off = size_t(m0 + r) * s.Cp + n0 + c;
      const float4 xv = *reinterpret_cast<const float4 *>(s.x + off);
      const float4 yv = *reinterpret_cast<const float4 *>(s.y + off);
      float *px = sx + r * kTileLd + c, *py = sy + r * kTileLd + c;
      px[0] = xv.x; px[1] = xv.y; px[2] = xv.z; px[3] = xv.w;
      py[0] = yv.x; py[1] = yv.y; py[2] = yv.z; py[3] = yv.w;
    }
  }
  __syncthreads();
  // warp w: TMEM lanes 32 (w % 4) .. + 31 (= spin rows), columns 64 (w / 4) .. + 63
  const int quarter = warp & 3, half = warp >> 2;
  const int rl = quarter * 32 + lane;
  const int i = m0 + rl;
#pragma unroll 1
  for (int cc = 0; cc < 2; ++cc) {
    const int cl = half * 64 + cc * 32;  // first column of the chunk inside the tile
    const int c0 = n0 + cl;
    uint32_t g[32];
    tc::tmem_ld_32x32b_x32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(cl), g);
    int8_t f[32];
    if (i < s.N && c0 < s.C) {
      sb_update_row32<P>(s, t, n, c0, g, __ldg(a.h + i), sx + rl * kTileLd + cl, sy + rl * kTileLd + cl, f);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) f[j] = 0;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) sF[(cl + j) * kTcBM + rl] = f_to_e4m3(f[j]);
  }
  tc::tc_fence_before();
  __syncthreads();
  for (int q = threadIdx.x; q < kTcBM * (kTcBN / 4); q += kTcThreads) {
    const int r = q / (kTcBN / 4), c = (q % (kTcBN / 4)) * 4;
    if (m0 + r < s.N && c < cols_valid) {
      const size_t off = size_t(m0 + r) * s.Cp + n0 + c;
      const float *px = sx + r * kTileLd + c, *py = sy + r * kTileLd + c;
      *reinterpret_cast<float4 *>(s.x + off) = make_float4(px[0], px[1], px[2], px[3]);
      *reinterpret_cast<float4 *>(s.y + off) = make_float4(py[0], py[1], py[2], py[3]);
    }
  }
  // column n0 + c of FT_next gets rows m0 .. m0 + 127 (128 contiguous bytes);
  // two threads per column, 64 bytes each
  {
    const int c = threadIdx.x >> 1, part = threadIdx.x & 1;
    uint8_t *dst = a.FT + (size_t((n + 1) & 1) * s.Cp + n0 + c) * a.Kp + m0 + part * 64;
    const uint4 *src = reinterpret_cast<const uint4 *>(sF + c * kTcBM + part * 64);
#pragma unroll
    for (int q = 0; q < 4; ++q) reinterpret_cast<uint4 *>(dst)[q] = src[q];
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

// 2D uint8 tensor map [rows][cols] (cols contiguous), box 128 x 128, 128B swizzle.
static bool make_map(CUtensorMap *m, const void *base, uint64_t rows, uint64_t cols) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols};
  const cuuint32_t box[2] = {128, 128};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcPlanImpl {
  CUtensorMap tmA, tmB;
};

bool tc_plan_make(void **plan, const uint8_t *J8, uint8_t *FT, int Kp, int Cp) {
  auto *p = new TcPlanImpl();
  if (!make_map(&p->tmA, J8, uint64_t(Kp), uint64_t(Kp)) || !make_map(&p->tmB, FT, uint64_t(2) * Cp, uint64_t(Kp))) {
    delete p;
    return false;
  }
  *plan = p;
  return true;
}

void tc_plan_free(void *plan) { delete static_cast<TcPlanImpl *>(plan); }

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
static cudaError_t launch_tc_p(const TcPlanImpl *p, const StateView &s, const TcArgs &a, const StepTables &t, int n,
                               cudaStream_t st) {
  dim3 grid(s.Cp / kTcBN, a.Kp / kTcBM);
  k_step_dense_tc<P><<<grid, kTcThreads, kTcSmem, st>>>(p->tmA, p->tmB, s, a, t, n);
  return cudaGetLastError();
}

cudaError_t launch_step_dense_tc(const void *plan, const StateView &s, int Kp, uint8_t *FT, int *err, const float *h,
                                 const StepTables &t, int n, cudaStream_t st) {
  const auto *p = static_cast<const TcPlanImpl *>(plan);
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
