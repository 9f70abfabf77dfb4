// dense_tc_common.cuh -- pieces shared by the tcgen05 dense kernels: tile
// constants, operand forms, tensor maps, the f-tile writer and the per-row
// update of one 32-column chunk (Sec. II A, Eqs. 5-8).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "step_common.cuh"
#include "tc_common.cuh"

namespace sbqa {

constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 128, kTcStages = 3;
constexpr int kTcThreads = 512;          // 16 warps: all run the epilogue, one 32-column box each
constexpr int kTcTile = kTcBM * kTcBK;   // bytes of one operand stage (e4m3)
constexpr int kTcBox = kTcBM * 128;      // one 128-row x 32-float state box (16 KB)
constexpr int kTcStateTile = 4 * kTcBox; // x or y tile, 128 rows x 128 columns (64 KB)
constexpr int kTcSmem = 2 * kTcStages * kTcTile + 2 * kTcStateTile + 1024 + 128;
constexpr uint8_t kE4M3One = 0x38, kE4M3MinusOne = 0xB8;

// Operand forms of the product G = J . F on the tensor cores (TcMaps::op).
//   kOpF8    integer J (|J_ij| <= 16) and the f codes of Eq. 8 in e4m3: exact
//   kOpBf16  J rounded to bfloat16 (exact for integers |J_ij| <= 256) and the
//            f codes of Eq. 8 in bfloat16: exact products, FP32 sums
//   kOpBsb   the ballistic form f(x) = x: J in bfloat16, and x as the two
//            bfloat16 terms hi = bf16(x), lo = bf16(x - hi) (x to 2^-16
//            relative), two B operands sharing each A tile
constexpr int kOpF8 = kTcOpF8, kOpBf16 = kTcOpBf16, kOpBsb = kTcOpBsb;

template <int OP>
struct TcOp {
  static constexpr bool kBf = OP != kOpF8;
  static constexpr int kKE = kBf ? 64 : 128;       // K elements per 128-byte operand row (one k-block)
  static constexpr int kEB = kBf ? 2 : 1;          // bytes per operand element
  static constexpr int kNB = OP == kOpBsb ? 2 : 1;  // B operands per k-block
  static constexpr int kFTile = kTcBM * kTcBN * kEB;  // one 128 x 128 f tile (bytes)
  __host__ __device__ static constexpr uint32_t idesc(int M, int N) {
    return kBf ? tc::idesc_bf16(M, N) : tc::idesc_f8_e4m3(M, N);
  }
  __device__ __forceinline__ static void mma(uint32_t d, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
    if constexpr (kBf) tc::mma_bf16(d, ad, bd, id, acc);
    else tc::mma_f8(d, ad, bd, id, acc);
  }
};

// 2D tensor map [rows][cols] (cols contiguous) with the given box and
// swizzle (step_dense_tc.cu); false when the driver refuses it.
bool tc_make_map(CUtensorMap *m, const void *base, CUtensorMapDataType dt, size_t esize, uint64_t rows,
                 uint64_t cols, uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle sw);
// The same for `rank` dimensions (dims[0] contiguous; strides[k] in bytes
// between consecutive indices of dimension k + 1).
bool tc_make_map_nd(CUtensorMap *m, const void *base, CUtensorMapDataType dt, int rank, const uint64_t *dims,
                    const uint64_t *strides, const uint32_t *box, CUtensorMapSwizzle sw);

// k-blocks per TMA box of the single-CTA persistent e4m3 and bfloat16 solvers
constexpr int kTpGroup = 3;

struct TcArgs {
  int Kp;
  uint8_t *FT;  // [2][Cp][Kp]
  int *err;     // device error flag (0 = ok)
  const float *h;
};

struct TcMaps {
  CUtensorMap A, B;  // J8 and FT operand tiles (128 x 128 bytes, 128B swizzle)
  CUtensorMap B2;    // FT operand tiles of 256 columns (256 x 128 bytes, 128B swizzle)
  CUtensorMap B64;   // FT operand half tiles of a CTA pair (64 x 128 bytes, 128B swizzle)
  CUtensorMap X, Y;  // x, y state boxes (128 rows x 32 floats, 128B swizzle)
  CUtensorMap Fst;   // FT tile store (128 columns x 128 spins, no swizzle)
  CUtensorMap Bl, Fstl;  // kOpBsb: the lo terms of x (load and store), as B and Fst
  // kOpF8, kOpBf16: 3D views (128 bytes, rows, k-blocks; strides one row and
  // 128 bytes) of J and FT, boxes of kTpGroup consecutive k-blocks of 128 rows
  CUtensorMap A3, B3;
  int op;                // operand form (kOpF8, kOpBf16, kOpBsb)
};

__device__ __forceinline__ uint8_t f_to_e4m3(int8_t f) {
  return f == 0 ? uint8_t(0) : (f > 0 ? kE4M3One : kE4M3MinusOne);
}

// e4m3 code of f(x) for the threshold delta >= 0 (Eq. 8: 0 when |x| <= delta).
__device__ __forceinline__ uint8_t thresh_e4m3(float x, float delta) {
  return x > delta ? kE4M3One : (x < -delta ? kE4M3MinusOne : uint8_t(0));
}

// Writer of f(x_next) into the transposed f tile of one spin row: base points
// at column 0 of the thread's 32-column chunk; column j is base[j * 128]
// elements on.  kOpF8 / kOpBf16: the code of Eq. 8 (0 when |x| <= Delta);
// kOpBsb: f(x) = x as hi = bf16(x) and lo = bf16(x - hi) (exact in FP32),
// the lo tile following the hi tile.
template <int OP>
struct FOut {
  uint8_t *base;
  __device__ __forceinline__ void put(int j, float x, float delta) const {
    if constexpr (OP == kOpF8) {
      base[j * kTcBM] = thresh_e4m3(x, delta);
    } else if constexpr (OP == kOpBf16) {
      reinterpret_cast<uint16_t *>(base)[j * kTcBM] =
          x > delta ? uint16_t(0x3F80) : (x < -delta ? uint16_t(0xBF80) : uint16_t(0));
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
      reinterpret_cast<uint16_t *>(base)[j * kTcBM] = __bfloat16_as_ushort(h);
      reinterpret_cast<uint16_t *>(base + TcOp<OP>::kFTile)[j * kTcBM] = __bfloat16_as_ushort(l);
    }
  }
  __device__ __forceinline__ void zero(int j) const {
    if constexpr (OP == kOpF8) {
      base[j * kTcBM] = 0;
    } else {
      reinterpret_cast<uint16_t *>(base)[j * kTcBM] = 0;
      if constexpr (OP == kOpBsb) reinterpret_cast<uint16_t *>(base + TcOp<OP>::kFTile)[j * kTcBM] = 0;
    }
  }
};

template <int OP>
__device__ __forceinline__ FOut<OP> f_out(uint8_t *sF, int cl, int rl) {
  return FOut<OP>{sF + (cl * kTcBM + rl) * TcOp<OP>::kEB};
}

// Address of the float4 (16-byte chunk u, 0..7) of row r inside a 128B-swizzled
// box of 128-byte rows: chunks are permuted by XOR with r mod 8.
__device__ __forceinline__ float4 *box_chunk(uint8_t *box, int r, int u) {
  return reinterpret_cast<float4 *>(box + r * 128 + ((u ^ (r & 7)) << 4));
}

// J_perp of the runs of a 32-column chunk.  For P >= 4 (at most 8 runs) the
// values are read before the accumulator is ready, off the critical path; for
// P < 4 (16 or 32 runs, which would not fit beside the tile in registers) they
// are read inside the update.
template <int P>
struct KjChunk {
  static constexpr int kRuns = 32 / (P < 32 ? P : 32);
  static constexpr bool kEarly = P >= 4;
  float v[kEarly ? kRuns : 1];
  const float *kjn;
  __device__ __forceinline__ void load(const StateView &s, const float *kj_step, int c0) {
    kjn = kj_step;
    if constexpr (kEarly) {
#pragma unroll
      for (int q = 0; q < kRuns; ++q) v[q] = (c0 + q * P < s.C) ? __ldg(kjn + c0 / P + q) : 0.f;
    }
  }
  __device__ __forceinline__ float get(int c0, int q) const {
    if constexpr (kEarly) return v[q];
    else return __ldg(kjn + c0 / P + q);
  }
};

// Positions of one spin row just outside a 32-column chunk of a run that
// spans several chunks (P = 64, 128): the columns left and right of the
// chunk and the run's replicas 0 and Pr - 1, read before any chunk of the
// tile is written back.
struct RingExt {
  float left, right, first, last;
};

// Ring neighbours (k modulo Pr) of a row's 32 consecutive columns c0.. held
// by one thread: runs inside the chunk for P <= 32 (GEN = false: Pr = P,
// the form of power-of-two replica counts), else from the chunk and the four
// outside values of e.
template <int P, bool GEN>
__device__ __forceinline__ void ring32(const float (&xs)[32], int Pr, int c0, const RingExt &e, float (&xm)[32],
                                       float (&xp)[32]) {
  if constexpr (P <= 32) {
    ring_nb<P, 32, GEN>(xs, Pr, xm, xp);
  } else {
    const int part = (c0 % P) / 32;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int k = part * 32 + j;
      xm[j] = j == 0 ? (part == 0 ? e.last : e.left) : xs[j - 1];
      xp[j] = k == Pr - 1 ? e.first : (j == 31 ? e.right : xs[j + 1]);
    }
  }
}

// Column c (inside the 128-column tile) of row r in the swizzled state boxes.
__device__ __forceinline__ float box_at(uint8_t *boxes, int r, int c) {
  const uint8_t *box = boxes + (c >> 5) * kTcBox;
  const int e = c & 31;
  return reinterpret_cast<const float *>(box + r * 128 + (((e >> 2) ^ (r & 7)) << 4))[e & 3];
}

// The outside values of ring32 for the chunk at tile column cl of row r.
template <int P>
__device__ __forceinline__ RingExt ring_ext_boxes(uint8_t *xboxes, int r, int cl, int Pr) {
  RingExt e{0.f, 0.f, 0.f, 0.f};
  if constexpr (P > 32) {
    const int rb = cl - cl % P;  // first column of the run inside the tile
    e.left = cl > rb ? box_at(xboxes, r, cl - 1) : 0.f;
    e.right = cl + 32 < rb + P ? box_at(xboxes, r, cl + 32) : 0.f;
    e.first = box_at(xboxes, r, rb);
    e.last = box_at(xboxes, r, rb + Pr - 1);
  }
  return e;
}

// Update of one spin row for 32 aligned columns c0..c0+31 (whole runs,
// because P divides 32); x and y are read from and written back to one row of
// the swizzled shared-memory state boxes; the e4m3 code of f(x_next) of
// column j goes to sFcol[j * 128] of the transposed f tile.  Same arithmetic,
// in the same order, as sb_update4.  FULL: all 32 columns are below C (no
// per-column test).
template <int P, bool FULL, int OP, bool GEN = false>
__device__ __forceinline__ void sb_update_row32(const StateView &s, const StepTables &t, float ka, float dnext,
                                                const KjChunk<P> &kj, int c0, const uint32_t (&g)[32], float hi,
                                                uint8_t *xbox, uint8_t *ybox, int r, const FOut<OP> &fo,
                                                const RingExt &ext) {
  constexpr int PR = P < 32 ? P : 32;
  float xs[32], ys[32];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const float4 a = *box_chunk(xbox, r, u), b = *box_chunk(ybox, r, u);
    xs[4 * u] = a.x; xs[4 * u + 1] = a.y; xs[4 * u + 2] = a.z; xs[4 * u + 3] = a.w;
    ys[4 * u] = b.x; ys[4 * u + 1] = b.y; ys[4 * u + 2] = b.z; ys[4 * u + 3] = b.w;
  }
  float xms[32], xps[32];
  ring32<P, GEN>(xs, s.Pr, c0, ext, xms, xps);
  float xo[32], yo[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float xm = xms[j], xp = xps[j];
    xo[j] = xs[j];
    yo[j] = ys[j];
    if (!FULL && c0 + j >= s.C) {
      fo.zero(j);
      continue;
    }
    float yn = fmaf(t.kc, __uint_as_float(g[j]) + hi, ys[j]);
    yn = fmaf(-ka, xs[j], yn);
    yn = fmaf(kj.get(c0, j / PR), xm + xp, yn);
    float xn = fmaf(t.kx, yn, xs[j]);
    if (fabsf(xn) > 1.f) {
      xn = copysignf(1.f, xn);
      yn = 0.f;
    }
    xo[j] = xn;
    yo[j] = yn;
    fo.put(j, xn, dnext);
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    *box_chunk(xbox, r, u) = make_float4(xo[4 * u], xo[4 * u + 1], xo[4 * u + 2], xo[4 * u + 3]);
    *box_chunk(ybox, r, u) = make_float4(yo[4 * u], yo[4 * u + 1], yo[4 * u + 2], yo[4 * u + 3]);
  }
}

}  // namespace sbqa
