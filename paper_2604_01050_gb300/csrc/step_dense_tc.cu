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
//
// Real-valued J (and integers up to |J| = 256) take the same kernels with
// BF16 operands (tcgen05.mma kind::f16, K = 64 elements per 128-byte operand
// row); the ballistic form f(x) = x carries x as two BF16 terms (hi + lo) in
// two B operands that share each A tile.
#include "dense_tc_common.cuh"
#include "dense_tc_persistent.cuh"

namespace sbqa {

template <int P, int OP, bool GEN>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_step_dense_tc(const __grid_constant__ TcMaps m, StateView s, TcArgs a, StepTables t, int n) {
  using O = TcOp<OP>;
  // operand stages: 3 of A + B (32 KB), or 2 of A + B hi + B lo (48 KB) for kOpBsb: 96 KB either way
  constexpr int kStages = O::kNB == 2 ? 2 : kTcStages;
  constexpr int kStageB = O::kNB * kTcTile;
  static_assert(kStages * (kTcTile + kStageB) == 2 * kTcStages * kTcTile, "operand stages of the 128 x 128 kernel");
  static_assert(O::kNB * O::kFTile <= 2 * kTcStages * kTcTile, "f tile must fit the consumed operand stages");
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kTcTile;
  uint8_t *sX = smem + 2 * kTcStages * kTcTile;
  uint8_t *sY = sX + kTcStateTile;
  uint64_t *full = reinterpret_cast<uint64_t *>(sY + kTcStateTile);
  uint64_t *empty = full + kTcStages;
  uint64_t *done = empty + kTcStages;
  uint64_t *xy_full = done + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(xy_full + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * kTcBN;
  const int KB = a.Kp / O::kKE;
  const int brow = (n & 1) * s.Cp + n0;  // row of F_n in the [2 Cp][Kp] map

  if (threadIdx.x == 0) {
    for (int q = 0; q < kStages; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&empty[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(xy_full, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&m.A);
    tc::prefetch_tmap(&m.B);
    if constexpr (O::kNB == 2) tc::prefetch_tmap(&m.Bl);
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
      const int st = kb % kStages, q = kb / kStages;
      if (q > 0 && !tc::mbar_wait(&empty[st], (q - 1) & 1, a.err, tc::ERR_WAIT_EMPTY)) break;
      tc::mbar_arrive_expect_tx(&full[st], kTcTile + kStageB);
      tc::tma_load_2d(sA + st * kTcTile, &m.A, &full[st], kb * O::kKE, m0);
      tc::tma_load_2d(sB + st * kStageB, &m.B, &full[st], kb * O::kKE, brow);
      if constexpr (O::kNB == 2) tc::tma_load_2d(sB + st * kStageB + kTcTile, &m.Bl, &full[st], kb * O::kKE, brow);
      if (!xy_issued && (kb == kStages - 1 || kb == KB - 1)) {
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
    constexpr uint32_t idesc = O::idesc(kTcBM, kTcBN);
    for (int kb = 0; kb < KB; ++kb) {
      const int st = kb % kStages, q = kb / kStages;
      if (!tc::mbar_wait(&full[st], q & 1, a.err, tc::ERR_WAIT_FULL)) break;
      tc::tc_fence_after();
      const uint32_t a0 = tc::smem_u32(sA + st * kTcTile), b0 = tc::smem_u32(sB + st * kStageB);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        O::mma(tmem, tc::smem_desc_sw128(a0 + kk * 32), tc::smem_desc_sw128(b0 + kk * 32), idesc,
               (kb | kk) != 0 ? 1u : 0u);
        if constexpr (O::kNB == 2)
          O::mma(tmem, tc::smem_desc_sw128(a0 + kk * 32), tc::smem_desc_sw128(b0 + kTcTile + kk * 32), idesc, 1u);
      }
      tc::mma_commit(&empty[st]);
    }
    tc::mma_commit(done);
  }
  __syncwarp();
  const float ka = __ldg(t.ka + n), dnext = __ldg(t.dl + n + 1);
  const int quarter = warp & 3, b = warp >> 2;  // TMEM lanes 32 (w % 4).., state box w / 4
  const int rl = quarter * 32 + lane;
  const int i = m0 + rl;
  const float hi = i < s.N ? __ldg(a.h + i) : 0.f;
  KjChunk<P> kj;
  kj.load(s, t.kj + size_t(n) * t.R, n0 + 32 * b);
  tc::mbar_wait(done, 0, a.err, tc::ERR_WAIT_DONE);
  tc::mbar_wait(xy_full, 0, a.err, tc::ERR_WAIT_FULL);
  tc::tc_fence_after();

  // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (= spin rows) and
  // columns 32 (w / 4) .. + 31 (one state box).
  uint8_t *sF = sA;  // [128 columns][128 spins] f(x_next) (kOpBsb: hi, then lo); the operand stages are consumed
  {
    const int cl = 32 * b;  // first column of the chunk inside the tile
    const int c0 = n0 + cl;
    // runs over several chunks (P > 32): their outside neighbours before any chunk is written back
    const RingExt ext = ring_ext_boxes<P>(sX, rl, cl, s.Pr);
    if constexpr (P > 32) __syncthreads();
    uint32_t g[32];
    tc::tmem_ld_32x32b_x32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(cl), g);
    const FOut<OP> fo = f_out<OP>(sF, cl, rl);
    if (i < s.N && c0 + 32 <= s.C) {
      sb_update_row32<P, true, OP, GEN>(s, t, ka, dnext, kj, c0, g, hi, sX + b * kTcBox, sY + b * kTcBox, rl, fo,
                                        ext);
    } else if (i < s.N && c0 < s.C) {
      sb_update_row32<P, false, OP, GEN>(s, t, ka, dnext, kj, c0, g, hi, sX + b * kTcBox, sY + b * kTcBox, rl, fo,
                                         ext);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) fo.zero(j);
    }
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
    if constexpr (O::kNB == 2) tc::tma_store_2d(&m.Fstl, sF + O::kFTile, m0, ((n + 1) & 1) * s.Cp + n0);
    tc::tma_store_commit_and_wait_read();
  }
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// ---------------------------------------------------------------- wide per-step kernel
// The same step with 128 x 256 tiles (tcgen05.mma M=128 N=256 K=32), for
// Cp a multiple of 256.  With N = 128 the tensor core reads a 128 x 32 A
// slice and a 128 x 32 B slice from shared memory per instruction while TMA
// writes the next stages into the same memory, and the K loop runs at about
// half the MMA rate; with N = 256 one A slice serves twice the columns and
// the loop runs at the MMA rate.  Four stages of 48 KB (A 16 KB, B 32 KB)
// fill shared memory, so the state tile (x and y of 128 rows x 256 columns,
// 256 KB) goes through the freed stages after the MMAs in two rounds of 128
// columns:
//   box slots (16 KB each): [0, 64K) = A stages, [64K, 192K) = B stages
//   round 0 (columns 0-127):   x boxes 0-3 at 0-48K, y boxes 0-3 at 64K-112K
//   round 1 (columns 128-255): x boxes 4-7 at 128K-176K (loaded with round 0),
//                              y boxes 4-7 at 0-48K once round 0's x boxes
//                              have been stored
// f(x_next) of all 256 columns collects in its own 32 KB tile.
constexpr int kTwBN = 256, kTwStages = 4;
constexpr int kTwTileB = kTwBN * kTcBK;                       // 32 KB
constexpr int kTwStageBytes = kTcTile + kTwTileB;             // 48 KB
constexpr int kTwOperands = kTwStages * kTwStageBytes;        // 192 KB
constexpr int kTwSmem = kTwOperands + kTcBM * kTwBN + 1024 + 128;
static_assert(kTwSmem <= 227 * 1024, "wide tile exceeds the shared memory of one CTA");
static_assert(2 * kTcStateTile + kTcStateTile <= kTwOperands, "state boxes of a round must fit the operand stages");

template <int P>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_step_dense_tc_wide(const __grid_constant__ TcMaps m, StateView s, TcArgs a, StepTables t, int n) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = smem;                                 // [4][16 KB]
  uint8_t *sB = smem + kTwStages * kTcTile;           // [4][32 KB]
  uint8_t *sF = smem + kTwOperands;                   // [256 columns][128 spins] e4m3 f(x_next)
  uint64_t *full = reinterpret_cast<uint64_t *>(sF + kTcBM * kTwBN);
  uint64_t *empty = full + kTwStages;
  uint64_t *done = empty + kTwStages;
  uint64_t *xy0 = done + 1, *x1 = xy0 + 1, *y1 = x1 + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(y1 + 1);
  uint8_t *sX0 = smem, *sY0 = smem + kTcStateTile, *sX1 = smem + 2 * kTcStateTile, *sY1 = smem;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * kTwBN;
  const int KB = a.Kp / kTcBK;
  const int brow = (n & 1) * s.Cp + n0;  // row of F_n in the [2 Cp][Kp] map

  if (threadIdx.x == 0) {
    for (int q = 0; q < kTwStages; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&empty[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(xy0, 1);
    tc::mbar_init(x1, 1);
    tc::mbar_init(y1, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&m.A);
    tc::prefetch_tmap(&m.B2);
    tc::prefetch_tmap(&m.X);
    tc::prefetch_tmap(&m.Y);
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTwBN);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    const uint64_t keep = tc::policy_evict_last();
    for (int kb = 0; kb < KB; ++kb) {
      const int st = kb % kTwStages, q = kb / kTwStages;
      if (q > 0 && !tc::mbar_wait(&empty[st], (q - 1) & 1, a.err, tc::ERR_WAIT_EMPTY)) break;
      tc::mbar_arrive_expect_tx(&full[st], kTwStageBytes);
      tc::tma_load_2d_hint(sA + st * kTcTile, &m.A, &full[st], kb * kTcBK, m0, keep);
      tc::tma_load_2d_hint(sB + st * kTwTileB, &m.B2, &full[st], kb * kTcBK, brow, keep);
    }
    // the operand stages are free once every MMA has completed: state boxes
    // of round 0 and the x boxes of round 1 (whatever the wait's outcome, so
    // that every barrier below completes)
    tc::mbar_wait(done, 0, a.err, tc::ERR_WAIT_DONE);
    tc::mbar_arrive_expect_tx(xy0, 2 * kTcStateTile);
    tc::mbar_arrive_expect_tx(x1, kTcStateTile);
    for (int b = 0; b < 4; ++b) {
      tc::tma_load_2d(sX0 + b * kTcBox, &m.X, xy0, n0 + 32 * b, m0);
      tc::tma_load_2d(sY0 + b * kTcBox, &m.Y, xy0, n0 + 32 * b, m0);
      tc::tma_load_2d(sX1 + b * kTcBox, &m.X, x1, n0 + 128 + 32 * b, m0);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = tc::idesc_f8_e4m3(kTcBM, kTwBN);
    for (int kb = 0; kb < KB; ++kb) {
      const int st = kb % kTwStages, q = kb / kTwStages;
      if (!tc::mbar_wait(&full[st], q & 1, a.err, tc::ERR_WAIT_FULL)) break;
      tc::tc_fence_after();
      const uint32_t a0 = tc::smem_u32(sA + st * kTcTile), b0 = tc::smem_u32(sB + st * kTwTileB);
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
  const int quarter = warp & 3, b = warp >> 2;  // TMEM lanes 32 (w % 4).., box w / 4 of each round
  const int rl = quarter * 32 + lane;
  const int i = m0 + rl;
  const float hi = i < s.N ? __ldg(a.h + i) : 0.f;
  KjChunk<P> kj[2];
  kj[0].load(s, t.kj + size_t(n) * t.R, n0 + 32 * b);
  kj[1].load(s, t.kj + size_t(n) * t.R, n0 + 128 + 32 * b);
  tc::mbar_wait(done, 0, a.err, tc::ERR_WAIT_DONE);
  tc::tc_fence_after();

#pragma unroll 1
  for (int round = 0; round < 2; ++round) {
    uint8_t *xbox = (round == 0 ? sX0 : sX1) + b * kTcBox;
    uint8_t *ybox = (round == 0 ? sY0 : sY1) + b * kTcBox;
    if (round == 0) {
      tc::mbar_wait(xy0, 0, a.err, tc::ERR_WAIT_FULL);
    } else {
      tc::mbar_wait(x1, 0, a.err, tc::ERR_WAIT_FULL);
      tc::mbar_wait(y1, 0, a.err, tc::ERR_WAIT_FULL);
    }
    const int cl = 128 * round + 32 * b;  // first column of the chunk inside the tile
    const int c0 = n0 + cl;
    uint32_t g[32];
    tc::tmem_ld_32x32b_x32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(cl), g);
    const FOut<kOpF8> fo = f_out<kOpF8>(sF, cl, rl);
    if (i < s.N && c0 + 32 <= s.C) {
      sb_update_row32<P, true, kOpF8>(s, t, ka, dnext, kj[round], c0, g, hi, xbox, ybox, rl, fo, RingExt{});
    } else if (i < s.N && c0 < s.C) {
      sb_update_row32<P, false, kOpF8>(s, t, ka, dnext, kj[round], c0, g, hi, xbox, ybox, rl, fo, RingExt{});
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) fo.zero(j);
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      // the round's x, y boxes back (rows past N are clipped by the tensor map),
      // x and y as separate store groups
      for (int q = 0; q < 4; ++q)
        tc::tma_store_2d(&m.X, (round == 0 ? sX0 : sX1) + q * kTcBox, n0 + 128 * round + 32 * q, m0);
      tc::tma_store_commit();
      for (int q = 0; q < 4; ++q)
        tc::tma_store_2d(&m.Y, (round == 0 ? sY0 : sY1) + q * kTcBox, n0 + 128 * round + 32 * q, m0);
      tc::tma_store_commit();
      if (round == 0) {
        // round 1's y boxes take the place of round 0's x boxes once those are
        // read (the y group may still be reading)
        tc::tma_store_wait_read<1>();
        tc::mbar_arrive_expect_tx(y1, kTcStateTile);
        for (int q = 0; q < 4; ++q) tc::tma_load_2d(sY1 + q * kTcBox, &m.Y, y1, n0 + 128 + 32 * q, m0);
      } else {
        const uint64_t keep = tc::policy_evict_last();
        // f_{n+1} of this tile into the other FT buffer: columns n0.., spins m0..
        tc::tma_store_2d_hint(&m.Fst, sF, m0, ((n + 1) & 1) * s.Cp + n0, keep);
        tc::tma_store_2d_hint(&m.Fst, sF + kTcBM * kTcBN, m0, ((n + 1) & 1) * s.Cp + n0 + kTcBN, keep);
        tc::tma_store_commit_and_wait_read();
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTwBN);
  }
}

template <int P, int OP, bool GEN>
__global__ void __launch_bounds__(kTpThreads, 1)
    k_solve_dense_tc_persistent(const __grid_constant__ TcMaps m, StateView s, TpArgs a, StepTables t) {
  solve_dense_tc_persistent<P, false, OP, GEN>(m, s, a, t, blockIdx.y, blockIdx.x);
}

template <int P>
__global__ void __launch_bounds__(kTpThreads, 1)
    k_solve_dense_tc_pair(const __grid_constant__ TcMaps m, StateView s, TpArgs a, StepTables t) {
  solve_dense_tc_persistent<P, true, kOpF8, false>(m, s, a, t, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- split-K persistent solver
// The persistent solver for Cp and Kp multiples of 256, with the K loop at the
// MMA rate: a cluster of two CTAs owns one 128 x 256 output tile (spin rows
// m0.., replica columns n0..); CTA r of the pair runs M=128 N=256 MMAs over
// half r of the spins j (k-blocks r KB/2 ..), so both keep 256 partial sums
// per row in TMEM (columns 0-255).  CTA r then finishes columns n0 + 128 r ..
// + 127: it stages the partial sums of the other half in its freed operand
// stages and sends them with one bulk copy into the peer's shared memory
// (completing on the peer's recv_full mbarrier), adds the peer's partial sums
// of its own half, and updates x and y, which stay in TMEM (columns 256-383
// and 384-511).  The f tiles are published
// with per-(row tile, 128-column half) step counters as in the solver above,
// and a producer waits for both halves of each k-block it loads.  The sum of
// two exact integer partial sums is the same integer, so the result is bit for
// bit that of the other kernels.  Flow control: a CTA re-arms recv_full and
// then arrives on its peer's send_ok once it has read its receive buffer, and
// sends step q only after send_ok completed phase q; it arrives on its peer's
// stage_free once the peer's copy has landed, and its producer loads the
// next step's operands only after stage_free completed the phase of the step
// before.  Every wait is bounded; a CTA that gives up records an error and
// both stop at their next step boundary.
constexpr int kSkStages = 3;
constexpr int kSkThreads = 512;
constexpr int kSkStageBytes = kTcTile + kTwTileB;  // 48 KB: A 128 x 128, B 256 x 128 (e4m3)
constexpr int kSkRecv = kTcBM * kTcBN * 4;          // the peer's partial sums of this CTA's half (64 KB)
constexpr int kSkSmem = kSkStages * kSkStageBytes + kSkRecv + kTcBM * kTcBN + 1024 + 256;
static_assert(kSkSmem <= 227 * 1024, "split-K tile exceeds the shared memory of one CTA");
constexpr uint32_t kSkTmemX = 256, kSkTmemY = 384;

// Byte offset of the 16-byte chunk ch (0..31) of row r in the receive buffer
// (rows of 512 bytes; chunks permuted within each 128-byte group by r mod 8,
// so a quarter warp's 16-byte accesses to 8 consecutive rows hit distinct banks).
__device__ __forceinline__ uint32_t recv_offset(int r, int ch) {
  return uint32_t(r * 512 + (((ch & ~7) | ((ch & 7) ^ (r & 7))) << 4));
}

template <int P>
__global__ void __launch_bounds__(kSkThreads, 1)
    k_solve_dense_tc_split(const __grid_constant__ TcMaps m, StateView s, TpArgs a, StepTables t) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = smem;                                  // [3][16 KB]
  uint8_t *sB = smem + kSkStages * kTcTile;            // [3][32 KB]
  uint8_t *sR = smem + kSkStages * kSkStageBytes;      // [128 rows][512 B] partial sums from the peer
  uint8_t *sF = sR + kSkRecv;                          // [128 columns][128 spins] e4m3 f(x_next)
  uint64_t *full = reinterpret_cast<uint64_t *>(sF + kTcBM * kTcBN);
  uint64_t *empty = full + kSkStages;
  uint64_t *done = empty + kSkStages;
  uint64_t *recv_full = done + 1, *send_ok = recv_full + 1, *stage_free = send_ok + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(stage_free + 1);
  uint8_t *sS = smem;  // staging of the partial sums sent to the peer (the operand stages, after the MMAs)
  int *s_abort = reinterpret_cast<int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = tc::cluster_ctarank(), peer = rank ^ 1u;
  if (tc::cluster_nctarank() != 2 || rank != (blockIdx.x & 1u)) {
    // not launched as pairs of CTAs (every access to a peer would be invalid): report, touch nothing
    if (threadIdx.x == 0) atomicCAS(a.err, 0, tc::ERR_CLUSTER_SHAPE);
    return;
  }
  const int ct = blockIdx.x >> 1, mt = blockIdx.y;
  const int m0 = mt * kTcBM, n0 = ct * kTwBN;
  const int KB = a.Kp / kTcBK, KH = KB / 2, kb_begin = int(rank) * KH, kb_end = kb_begin + KH;
  const int quarter = warp & 3, chunk = warp >> 2;
  const int rl = quarter * 32 + lane, i = m0 + rl;
  const int cl = 32 * chunk, c0 = n0 + kTcBN * int(rank) + cl;
  const uint32_t lane_off = uint32_t(quarter * 32) << 16;
  const bool any = a.n_begin < a.n_end;

  if (threadIdx.x == 0) {
    for (int q = 0; q < kSkStages; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&empty[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(recv_full, 1);
    tc::mbar_init(send_ok, 1);
    tc::mbar_init(stage_free, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&m.A);
    tc::prefetch_tmap(&m.B2);
    tc::prefetch_tmap(&m.Fst);
    *s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  {  // this CTA's half of the state tile into TMEM (rows past N hold zeros and stay unchanged)
    uint32_t xr[32], yr[32];
    if (i < s.N) {
      const float4 *px = reinterpret_cast<const float4 *>(s.x + size_t(i) * s.Cp + c0);
      const float4 *py = reinterpret_cast<const float4 *>(s.y + size_t(i) * s.Cp + c0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 vx = px[u], vy = py[u];
        xr[4 * u] = __float_as_uint(vx.x); xr[4 * u + 1] = __float_as_uint(vx.y);
        xr[4 * u + 2] = __float_as_uint(vx.z); xr[4 * u + 3] = __float_as_uint(vx.w);
        yr[4 * u] = __float_as_uint(vy.x); yr[4 * u + 1] = __float_as_uint(vy.y);
        yr[4 * u + 2] = __float_as_uint(vy.z); yr[4 * u + 3] = __float_as_uint(vy.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) xr[j] = yr[j] = 0u;
    }
    __syncwarp();
    tc::tmem_st_32x32b_x32(tmem + lane_off + kSkTmemX + cl, xr);
    tc::tmem_st_32x32b_x32(tmem + lane_off + kSkTmemY + cl, yr);
    tc::tmem_wait_st();
  }
  const float hi = i < s.N ? __ldg(a.h + i) : 0.f;
  if (threadIdx.x == 0 && any) tc::mbar_arrive_expect_tx(recv_full, kSkRecv);  // receive step 0
  tc::tc_fence_before();
  tc::cluster_sync();  // both CTAs' barriers initialised, receive buffers armed
  tc::tc_fence_after();
  const uint32_t r_recv = tc::map_to_rank(tc::smem_u32(sR), peer);
  const uint32_t r_full = tc::map_to_rank(tc::smem_u32(recv_full), peer);
  const uint32_t r_ok = tc::map_to_rank(tc::smem_u32(send_ok), peer);
  const uint32_t r_free = tc::map_to_rank(tc::smem_u32(stage_free), peer);
  if (threadIdx.x == 0 && any) tc::mbar_arrive_remote(r_ok);  // the peer may send step 0

  constexpr uint32_t idesc = tc::idesc_f8_e4m3(kTcBM, kTwBN);
  int n = a.n_begin;
  for (; n < a.n_end; ++n) {
    const uint32_t q = uint32_t(n - a.n_begin);
    if (warp == 0) {
      // producer: k-blocks of this half as both 128-column f tiles of their row tile are published
      const int brow = (n & 1) * s.Cp + n0;
      uint64_t t0 = 0;
      uint32_t polls = 0;
      int kb = kb_begin;
      while (kb < kb_end) {
        const int kq = kb + (lane >> 1);
        const bool ok = q == 0 || kq >= kb_end ||
                        tc::ld_acquire_gpu(a.flags + kq * a.Ct + 2 * ct + (lane & 1)) >= q;
        const unsigned ball = __ballot_sync(0xffffffffu, ok);
        int nready = (ball == 0xffffffffu ? 32 : __ffs(~ball) - 1) >> 1;
        nready = nready < kb_end - kb ? nready : kb_end - kb;
        if (nready == 0) {
          int give_up = 0;
          if (lane == 0) {
            const uint64_t now = tc::globaltimer_ns();
            if (t0 == 0) t0 = now;
            if (*reinterpret_cast<volatile int *>(a.err) != 0) {
              give_up = 1;
            } else if (now - t0 > kFlagTimeoutNs || ++polls > (1u << 26)) {
              atomicCAS(a.err, 0, tc::ERR_WAIT_FLAG);
              give_up = 1;
            }
          }
          if (__shfl_sync(0xffffffffu, give_up, 0)) {
            nready = kb_end - kb;  // proceed with whatever the buffer holds; the run reports the error
          } else {
            __nanosleep(64);
            continue;
          }
        }
        if (lane == 0) {
          asm volatile("fence.acq_rel.gpu;" ::: "memory");
          tc::fence_proxy_async_global();
          // the staging of the step before must have reached the peer before the stages are reloaded
          if (kb == kb_begin && q > 0) tc::mbar_wait_cluster(stage_free, (q - 1) & 1, a.err, tc::ERR_WAIT_PEER);
          for (int j = kb; j < kb + nready; ++j) {
            const uint32_t g = q * KH + (j - kb_begin), st = g % kSkStages, use = g / kSkStages;
            if (use > 0) tc::mbar_wait(&empty[st], (use - 1) & 1, a.err, tc::ERR_WAIT_EMPTY);
            tc::mbar_arrive_expect_tx(&full[st], kSkStageBytes);
            tc::tma_load_2d(sA + st * kTcTile, &m.A, &full[st], j * kTcBK, m0);
            tc::tma_load_2d(sB + st * kTwTileB, &m.B2, &full[st], j * kTcBK, brow);
          }
        }
        __syncwarp();
        kb += nready;
      }
    } else if (warp == 1 && lane == 0) {
      for (int j = 0; j < KH; ++j) {
        const uint32_t g = q * KH + j, st = g % kSkStages, use = g / kSkStages;
        tc::mbar_wait(&full[st], use & 1, a.err, tc::ERR_WAIT_FULL);
        tc::tc_fence_after();
        const uint32_t a0 = tc::smem_u32(sA + st * kTcTile), b0 = tc::smem_u32(sB + st * kTwTileB);
#pragma unroll
        for (int kk = 0; kk < kTcBK / 32; ++kk)
          tc::mma_f8(tmem, tc::smem_desc_sw128(a0 + kk * 32), tc::smem_desc_sw128(b0 + kk * 32), idesc,
                     (j | kk) != 0 ? 1u : 0u);
        tc::mma_commit(&empty[st]);
      }
      tc::mma_commit(done);
    }
    __syncwarp();
    const float ka = __ldg(t.ka + n), dnext = __ldg(t.dl + n + 1);
    KjChunk<P> kj;
    kj.load(s, t.kj + size_t(n) * t.R, c0);
    tc::mbar_wait(done, q & 1, a.err, tc::ERR_WAIT_DONE);
    tc::tc_fence_after();
    {  // the peer's half of the partial sums, staged in the receive buffer's layout
      uint32_t gp[32];
      tc::tmem_ld_32x32b_x32_nowait(tmem + lane_off + kTcBN * peer + cl, gp);
      tc::tmem_wait_ld();
      tc::reg_fence(gp);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        *reinterpret_cast<uint4 *>(sS + recv_offset(rl, chunk * 8 + u)) =
            make_uint4(gp[4 * u], gp[4 * u + 1], gp[4 * u + 2], gp[4 * u + 3]);
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (threadIdx.x == 0 && tc::mbar_wait_cluster(send_ok, q & 1, a.err, tc::ERR_WAIT_PEER)) {
      // one bulk copy into the peer's receive buffer, completing on its recv_full
      for (int c = 0; c < 4; ++c)
        tc::bulk_copy_to_peer(r_recv + c * (kSkRecv / 4), sS + c * (kSkRecv / 4), kSkRecv / 4, r_full);
    }
    {
      uint32_t g[32], xr[32], yr[32];
      tc::tmem_ld_32x32b_x32_nowait(tmem + lane_off + kTcBN * rank + cl, g);
      tc::tmem_ld_32x32b_x32_nowait(tmem + lane_off + kSkTmemX + cl, xr);
      tc::tmem_ld_32x32b_x32_nowait(tmem + lane_off + kSkTmemY + cl, yr);
      tc::tmem_wait_ld();
      tc::reg_fence(g);
      tc::reg_fence(xr);
      tc::reg_fence(yr);
      const bool got = tc::mbar_wait_cluster(recv_full, q & 1, a.err, tc::ERR_WAIT_PEER);
      if (threadIdx.x == 32) tc::mbar_arrive_remote(r_free);  // the peer's staging has been copied
      if (got) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float4 v = *reinterpret_cast<const float4 *>(sR + recv_offset(rl, chunk * 8 + u));
          g[4 * u] = __float_as_uint(__uint_as_float(g[4 * u]) + v.x);
          g[4 * u + 1] = __float_as_uint(__uint_as_float(g[4 * u + 1]) + v.y);
          g[4 * u + 2] = __float_as_uint(__uint_as_float(g[4 * u + 2]) + v.z);
          g[4 * u + 3] = __float_as_uint(__uint_as_float(g[4 * u + 3]) + v.w);
        }
      }
      const FOut<kOpF8> fo = f_out<kOpF8>(sF, cl, rl);
      if (i < s.N && c0 < s.C) {
        if (c0 + 32 <= s.C) sb_update_regs32<P, true, kOpF8>(s, t, ka, dnext, kj, c0, g, hi, xr, yr, fo, RingExt{});
        else sb_update_regs32<P, false, kOpF8>(s, t, ka, dnext, kj, c0, g, hi, xr, yr, fo, RingExt{});
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) fo.zero(j);
      }
      __syncwarp();
      tc::tmem_st_32x32b_x32(tmem + lane_off + kSkTmemX + cl, xr);
      tc::tmem_st_32x32b_x32(tmem + lane_off + kSkTmemY + cl, yr);
      tc::tmem_wait_st();
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      // publish f_{n+1} of this half: spins m0.., columns n0 + 128 rank.. of the other FT buffer
      tc::tma_store_2d(&m.Fst, sF, m0, ((n + 1) & 1) * s.Cp + n0 + kTcBN * int(rank));
      tc::tma_store_commit_and_wait_all();
      tc::fence_proxy_async_global();
      tc::st_release_gpu(a.flags + mt * a.Ct + 2 * ct + int(rank), q + 1);
      if (n + 1 < a.n_end) {
        // the receive buffer has been read: arm it for the next step, then let the peer send
        tc::mbar_arrive_expect_tx(recv_full, kSkRecv);
        tc::mbar_arrive_remote(r_ok);
      }
      *s_abort = *reinterpret_cast<volatile int *>(a.err);
    }
    __syncthreads();
    tc::tc_fence_after();
    if (*s_abort != 0) break;
  }
  {  // this CTA's half of the state tile back to global memory
    uint32_t xr[32], yr[32];
    tc::tmem_ld_32x32b_x32_nowait(tmem + lane_off + kSkTmemX + cl, xr);
    tc::tmem_ld_32x32b_x32_nowait(tmem + lane_off + kSkTmemY + cl, yr);
    tc::tmem_wait_ld();
    tc::reg_fence(xr);
    tc::reg_fence(yr);
    if (i < s.N) {
      float4 *px = reinterpret_cast<float4 *>(s.x + size_t(i) * s.Cp + c0);
      float4 *py = reinterpret_cast<float4 *>(s.y + size_t(i) * s.Cp + c0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        px[u] = make_float4(__uint_as_float(xr[4 * u]), __uint_as_float(xr[4 * u + 1]),
                            __uint_as_float(xr[4 * u + 2]), __uint_as_float(xr[4 * u + 3]));
        py[u] = make_float4(__uint_as_float(yr[4 * u]), __uint_as_float(yr[4 * u + 1]),
                            __uint_as_float(yr[4 * u + 2]), __uint_as_float(yr[4 * u + 3]));
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::cluster_sync();  // no CTA leaves while its peer may still write into its shared memory
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// f codes [N][Cp] -> e4m3 f [Cp][Kp] (zeros for padded spins), for buffer b.
__global__ void k_f_to_ft8(StateView s, int which, uint8_t *FT, int Kp, int b) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;  // over Cp * Kp
  if (e >= size_t(s.Cp) * Kp) return;
  const int c = int(e / Kp), j = int(e % Kp);
  const int8_t f = (j < s.N) ? int8_t(int(s.f_of(which)[size_t(j) * s.Cp + c]) - 1) : int8_t(0);
  FT[size_t(b) * s.Cp * Kp + e] = f_to_e4m3(f);
}

// f codes [N][Cp] -> bfloat16 f [Cp][Kp] (zeros for padded spins), for buffer b.
__global__ void k_f_to_ft16(StateView s, int which, uint16_t *FT, int Kp, int b) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;  // over Cp * Kp
  if (e >= size_t(s.Cp) * Kp) return;
  const int c = int(e / Kp), j = int(e % Kp);
  const int f = (j < s.N) ? int(s.f_of(which)[size_t(j) * s.Cp + c]) - 1 : 0;
  FT[size_t(b) * s.Cp * Kp + e] = f == 0 ? uint16_t(0) : (f > 0 ? uint16_t(0x3F80) : uint16_t(0xBF80));
}

// Ballistic form: f(x) = x of the state [N][Cp] -> hi = bf16(x) into buffer b of
// the hi terms [2][Cp][Kp], lo = bf16(x - hi) into buffer b of the lo terms
// that follow them (zeros for padded spins and columns past C).
__global__ void k_x_to_ft_split(StateView s, uint16_t *FT, int Kp, int b) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;  // over Cp * Kp
  if (e >= size_t(s.Cp) * Kp) return;
  const int c = int(e / Kp), j = int(e % Kp);
  const float x = (j < s.N && c < s.C) ? s.x[size_t(j) * s.Cp + c] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  const size_t one = size_t(2) * s.Cp * Kp;
  FT[size_t(b) * s.Cp * Kp + e] = __bfloat16_as_ushort(h);
  FT[one + size_t(b) * s.Cp * Kp + e] = __bfloat16_as_ushort(l);
}

// ---------------------------------------------------------------- readout on the tensor cores
// Energies of the readout spins s = sign(x) for every column (Sec. II B):
// E = -(1/2) s^T J s - h^T s.  With integer J (|J| <= 16) and s in {-1, +1}
// the product G = J S is the step's GEMM with f = s, exact in FP8 and in the
// FP32 accumulator (|G_i| <= 16 N).  Each 128 x 128 tile forms, per spin row
// i and column c, the exact integer s_ic (G_ic + 2 h_i) and sums the 32 rows
// of each TMEM quarter into the row-block partial part[i / 32][c] that the
// CUDA-core energy kernel would write; the same fixed-order final kernel
// then gives E_c = -(sum over blocks) / 2.
constexpr int kEtStages = 6;
constexpr int kEtSmem = 2 * kEtStages * kTcTile + 1024 + 128;
static_assert(16 * 32 * 33 * 8 <= 2 * kEtStages * kTcTile, "row reductions must fit the operand stages");

// sign codes S [N][Cp] (+1, -1, 0 past C) -> e4m3 [Cp][Kp] in FT buffer b (zeros for padded spins)
__global__ void k_sign_to_ft8(StateView s, uint8_t *FT, int Kp, int b) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;  // over Cp * Kp
  if (e >= size_t(s.Cp) * Kp) return;
  const int c = int(e / Kp), j = int(e % Kp);
  const int8_t v = (j < s.N) ? s.Sg[size_t(j) * s.Cp + c] : int8_t(0);
  FT[size_t(b) * s.Cp * Kp + e] = f_to_e4m3(v);
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_energy_dense_tc(const __grid_constant__ TcMaps m, StateView s, int Kp, int b, int *err, const int64_t *h_i64,
                      int64_t *part, int nblk) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = smem;
  uint8_t *sB = smem + kEtStages * kTcTile;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + kEtStages * kTcTile);
  uint64_t *empty = full + kEtStages;
  uint64_t *done = empty + kEtStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * kTcBN;
  const int KB = Kp / kTcBK;
  const int brow = b * s.Cp + n0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < kEtStages; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&empty[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&m.A);
    tc::prefetch_tmap(&m.B);
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, 128);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < KB; ++kb) {
      const int st = kb % kEtStages, q = kb / kEtStages;
      if (q > 0 && !tc::mbar_wait(&empty[st], (q - 1) & 1, err, tc::ERR_WAIT_EMPTY)) break;
      tc::mbar_arrive_expect_tx(&full[st], 2 * kTcTile);
      tc::tma_load_2d(sA + st * kTcTile, &m.A, &full[st], kb * kTcBK, m0);
      tc::tma_load_2d(sB + st * kTcTile, &m.B, &full[st], kb * kTcBK, brow);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = tc::idesc_f8_e4m3(kTcBM, kTcBN);
    for (int kb = 0; kb < KB; ++kb) {
      const int st = kb % kEtStages, q = kb / kEtStages;
      if (!tc::mbar_wait(&full[st], q & 1, err, tc::ERR_WAIT_FULL)) break;
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
  const int quarter = warp & 3, chunk = warp >> 2;
  const int i = m0 + quarter * 32 + lane, c0 = n0 + 32 * chunk;
  int8_t si[32];
  int64_t h2 = 0;
  if (i < s.N) {
    const uint4 *ps = reinterpret_cast<const uint4 *>(s.Sg + size_t(i) * s.Cp + c0);
    const uint4 u0 = ps[0], u1 = ps[1];
    const uint32_t w[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
    for (int j = 0; j < 32; ++j) si[j] = int8_t(w[j >> 2] >> (8 * (j & 3)));
    h2 = 2 * h_i64[i];
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) si[j] = 0;
  }
  tc::mbar_wait(done, 0, err, tc::ERR_WAIT_DONE);
  tc::tc_fence_after();
  uint32_t g[32];
  tc::tmem_ld_32x32b_x32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(32 * chunk), g);
  // rows of this warp -> columns: [32 rows][33] int64 per warp in the freed operand stages
  int64_t *red = reinterpret_cast<int64_t *>(smem) + size_t(warp) * 32 * 33;
#pragma unroll
  for (int j = 0; j < 32; ++j)
    red[lane * 33 + j] = int64_t(si[j]) * (int64_t(__float2int_rn(__uint_as_float(g[j]))) + h2);
  __syncwarp();
  int64_t acc = 0;
#pragma unroll 8
  for (int r = 0; r < 32; ++r) acc += red[r * 33 + lane];
  const int blk = m0 / 32 + quarter;
  if (blk < nblk) part[size_t(blk) * s.Cp + c0 + lane] = acc;
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 128);
  }
}

cudaError_t launch_energy_partials_tc(const void *plan, const StateView &s, int Kp, uint8_t *FT, int b, int *err,
                                      const int64_t *h_i64, int64_t *part, int nblk, cudaStream_t st) {
  const size_t total = size_t(s.Cp) * Kp;
  k_sign_to_ft8<<<unsigned((total + 255) / 256), 256, 0, st>>>(s, FT, Kp, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid(s.Cp / kTcBN, Kp / kTcBM);
  k_energy_dense_tc<<<grid, kTcThreads, kEtSmem, st>>>(*static_cast<const TcMaps *>(plan), s, Kp, b, err, h_i64, part,
                                                     nblk);
  return cudaGetLastError();
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
bool tc_make_map(CUtensorMap *m, const void *base, CUtensorMapDataType dt, size_t esize, uint64_t rows,
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

bool tc_make_map_nd(CUtensorMap *m, const void *base, CUtensorMapDataType dt, int rank, const uint64_t *dims,
                    const uint64_t *strides, const uint32_t *box, CUtensorMapSwizzle sw) {
  auto fn = encode_fn();
  if (!fn || rank < 1 || rank > 5) return false;
  cuuint64_t d[5], st[4];
  cuuint32_t b[5], estr[5];
  for (int k = 0; k < rank; ++k) {
    d[k] = dims[k];
    b[k] = box[k];
    estr[k] = 1;
    if (k + 1 < rank) st[k] = strides[k];
  }
  return fn(m, dt, cuuint32_t(rank), const_cast<void *>(base), d, st, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tc_ft_bytes(int Kp, int Cp, int op) {
  const size_t one = size_t(2) * Cp * Kp;  // [2][Cp][Kp] elements
  return op == kOpF8 ? one : (op == kOpBf16 ? 2 * one : 4 * one);
}

size_t tc_j_bytes(int Kp, int op) { return size_t(Kp) * Kp * (op == kOpF8 ? 1 : 2); }

int tc_op_of(const void *plan) { return static_cast<const TcMaps *>(plan)->op; }

bool tc_plan_make(void **plan, const void *J, void *FT, int Kp, int Cp, float *x, float *y, int N, int op) {
  auto *p = new TcMaps();
  p->op = op;
  const auto F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const auto OT = op == kOpF8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const size_t eb = op == kOpF8 ? 1 : 2;
  const uint32_t ke = uint32_t(128 / eb);  // K elements of one 128-byte operand row
  const uint64_t rows_ft = uint64_t(2) * Cp;
  uint8_t *ftl = static_cast<uint8_t *>(FT) + rows_ft * Kp * eb;  // kOpBsb: the lo terms after the hi terms
  bool ok = tc_make_map(&p->A, J, OT, eb, uint64_t(Kp), uint64_t(Kp), ke, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
            tc_make_map(&p->B, FT, OT, eb, rows_ft, uint64_t(Kp), ke, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
            tc_make_map(&p->X, x, F32, 4, uint64_t(N), uint64_t(Cp), 32, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
            tc_make_map(&p->Y, y, F32, 4, uint64_t(N), uint64_t(Cp), 32, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
            tc_make_map(&p->Fst, FT, OT, eb, rows_ft, uint64_t(Kp), 128, 128, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (ok && op == kOpF8)  // the wide, split-K and paired kernels run the e4m3 product only
    ok = tc_make_map(&p->B2, FT, OT, 1, rows_ft, uint64_t(Kp), 128, 256, CU_TENSOR_MAP_SWIZZLE_128B) &&
         tc_make_map(&p->B64, FT, OT, 1, rows_ft, uint64_t(Kp), 128, 64, CU_TENSOR_MAP_SWIZZLE_128B);
  if (ok && op != kOpBsb) {  // two k-blocks per box: the same buffers seen as [rows][k-block][128 bytes]
    const uint64_t kbs = uint64_t(Kp) / ke;
    const uint64_t dims_a[3] = {ke, uint64_t(Kp), kbs}, dims_b[3] = {ke, rows_ft, kbs};
    const uint64_t strides[2] = {uint64_t(Kp) * eb, 128};
    const uint32_t box[3] = {ke, 128, uint32_t(kTpGroup)};
    ok = tc_make_map_nd(&p->A3, J, OT, 3, dims_a, strides, box, CU_TENSOR_MAP_SWIZZLE_128B) &&
         tc_make_map_nd(&p->B3, FT, OT, 3, dims_b, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
  }
  if (ok && op == kOpBsb)
    ok = tc_make_map(&p->Bl, ftl, OT, 2, rows_ft, uint64_t(Kp), ke, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
         tc_make_map(&p->Fstl, ftl, OT, 2, rows_ft, uint64_t(Kp), 128, 128, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (!ok) {
    delete p;
    return false;
  }
  *plan = p;
  return true;
}

void tc_plan_free(void *plan) { delete static_cast<TcMaps *>(plan); }

// [operand form][P index: log2 of the run width 1 .. 128][GEN] of the
// per-step 128 x 128 kernel and the persistent solver.  GEN (replicas fewer
// than the run width) exists for widths 4 .. 32; widths 1, 2 never have
// padding and widths 64, 128 handle any replica count in one form.
#define SBQA_TC_PS(K, OP)                                                                                       \
  {{(const void *)K<1, OP, false>, (const void *)K<1, OP, false>},                                            \
   {(const void *)K<2, OP, false>, (const void *)K<2, OP, false>},                                            \
   {(const void *)K<4, OP, false>, (const void *)K<4, OP, true>},                                             \
   {(const void *)K<8, OP, false>, (const void *)K<8, OP, true>},                                             \
   {(const void *)K<16, OP, false>, (const void *)K<16, OP, true>},                                           \
   {(const void *)K<32, OP, false>, (const void *)K<32, OP, true>},                                           \
   {(const void *)K<64, OP, true>, (const void *)K<64, OP, true>},                                            \
   {(const void *)K<128, OP, true>, (const void *)K<128, OP, true>}}
static const void *const kTcFns[3][8][2] = {SBQA_TC_PS(k_step_dense_tc, kOpF8),
                                            SBQA_TC_PS(k_step_dense_tc, kOpBf16),
                                            SBQA_TC_PS(k_step_dense_tc, kOpBsb)};
static const void *const kTpFnsOp[3][8][2] = {SBQA_TC_PS(k_solve_dense_tc_persistent, kOpF8),
                                              SBQA_TC_PS(k_solve_dense_tc_persistent, kOpBf16),
                                              SBQA_TC_PS(k_solve_dense_tc_persistent, kOpBsb)};
#undef SBQA_TC_PS

// index of a run width P (a power of two, 1 .. kMaxP) in the tables above; -1 otherwise
static int p_index(int P, int max_p = 128) {
  for (int q = 0; (1 << q) <= max_p; ++q)
    if ((1 << q) == P) return q;
  return -1;
}
static const int kTpSmemOp[3] = {TpShape<false, kOpF8>::kSmem, TpShape<false, kOpBf16>::kSmem,
                                 TpShape<false, kOpBsb>::kSmem};

static const void *const kPrFns[6] = {
    (const void *)k_solve_dense_tc_pair<1>, (const void *)k_solve_dense_tc_pair<2>,
    (const void *)k_solve_dense_tc_pair<4>, (const void *)k_solve_dense_tc_pair<8>,
    (const void *)k_solve_dense_tc_pair<16>, (const void *)k_solve_dense_tc_pair<32>};

static const void *const kSkFns[6] = {
    (const void *)k_solve_dense_tc_split<1>, (const void *)k_solve_dense_tc_split<2>,
    (const void *)k_solve_dense_tc_split<4>, (const void *)k_solve_dense_tc_split<8>,
    (const void *)k_solve_dense_tc_split<16>, (const void *)k_solve_dense_tc_split<32>};

cudaError_t tc_set_attributes() {
  for (int op = 0; op < 3; ++op)
    for (int q = 0; q < 8; ++q)
      for (const void *f : kTcFns[op][q]) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
        if (e != cudaSuccess) return e;
      }
  const void *wide[6] = {(const void *)k_step_dense_tc_wide<1>, (const void *)k_step_dense_tc_wide<2>,
                         (const void *)k_step_dense_tc_wide<4>, (const void *)k_step_dense_tc_wide<8>,
                         (const void *)k_step_dense_tc_wide<16>, (const void *)k_step_dense_tc_wide<32>};
  for (const void *f : wide) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTwSmem);
    if (e != cudaSuccess) return e;
  }
  for (int op = 0; op < 3; ++op)
    for (int q = 0; q < 8; ++q)
      for (const void *f : kTpFnsOp[op][q]) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTpSmemOp[op]);
        if (e != cudaSuccess) return e;
      }
  for (const void *f : kPrFns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, TpShape<true>::kSmem);
    if (e != cudaSuccess) return e;
  }
  for (const void *f : kSkFns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kSkSmem);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute((const void *)k_energy_dense_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kEtSmem);
}

// Launch configuration of a cooperative grid of 2 x 1 x 1 clusters.
static void cluster_config(cudaLaunchConfig_t *cfg, cudaLaunchAttribute *attr, dim3 grid, int threads, int smem,
                           cudaStream_t st, bool cooperative) {
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = grid;
  cfg->blockDim = dim3(threads);
  cfg->dynamicSmemBytes = smem;
  cfg->stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg->attrs = attr;
  cfg->numAttrs = cooperative ? 2 : 1;
}

int tc_split_blocks() {
  int best = 1 << 30;
  for (const void *f : kSkFns) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    cluster_config(&cfg, attr, dim3(2, 1), kSkThreads, kSkSmem, 0, false);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, f, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    best = clusters < best ? clusters : best;
  }
  return 2 * best;
}

bool tc_split_eligible(int Kp, int Cp, int blocks) {
  return blocks > 0 && Kp % (2 * kTcBM) == 0 && Cp % kTwBN == 0 && (Kp / kTcBM) * (Cp / kTcBN) <= blocks;
}

cudaError_t launch_solve_dense_tc_split(const void *plan, const StateView &s, int Kp, int *err, const float *h,
                                        const StepTables &t, int n_begin, int n_end, uint32_t *flags,
                                        cudaStream_t st) {
  const int idx = s.P == 1 ? 0 : s.P == 2 ? 1 : s.P == 4 ? 2 : s.P == 8 ? 3 : s.P == 16 ? 4 : s.P == 32 ? 5 : -1;
  if (idx < 0 || Kp % (2 * kTcBM) != 0 || s.Cp % kTwBN != 0) return cudaErrorInvalidValue;
  const int Ct = s.Cp / kTcBN;
  cudaError_t e = cudaMemsetAsync(flags, 0, tc_persistent_flag_count(Kp, s.Cp) * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  TpArgs a{Kp, Ct, n_begin, n_end, err, h, flags, -1};
  TcMaps maps = *static_cast<const TcMaps *>(plan);
  StateView sv = s;
  StepTables tv = t;
  void *args[] = {&maps, &sv, &a, &tv};
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[2];
  cluster_config(&cfg, attr, dim3(2 * (s.Cp / kTwBN), Kp / kTcBM), kSkThreads, kSkSmem, st, true);
  return cudaLaunchKernelExC(&cfg, kSkFns[idx], args);
}

int tc_persistent_blocks() {
  int dev = 0, sms = 0, best = 1 << 30;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int op = 0; op < 3; ++op)
    for (int q = 0; q < 8; ++q)
      for (const void *f : kTpFnsOp[op][q]) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kTpThreads, kTpSmemOp[op]) != cudaSuccess)
          return 0;
        best = per_sm < best ? per_sm : best;
      }
  return sms * best;
}

bool tc_persistent_eligible(int Kp, int Cp, int blocks) {
  return blocks > 0 && Kp % kTcBM == 0 && Cp % kTcBN == 0 && (Kp / kTcBM) * (Cp / kTcBN) <= blocks;
}

size_t tc_persistent_flag_count(int Kp, int Cp) { return size_t(Kp / kTcBM) * (Cp / kTcBN); }

cudaError_t launch_solve_dense_tc_persistent(const void *plan, const StateView &s, int Kp, int *err, const float *h,
                                             const StepTables &t, int n_begin, int n_end, uint32_t *flags,
                                             cudaStream_t st) {
  const int idx = p_index(s.P);
  const int op = tc_op_of(plan);
  if (idx < 0 || op < 0 || op > 2 || Kp % kTcBM != 0 || s.Cp % kTcBN != 0) return cudaErrorInvalidValue;
  const int Ct = s.Cp / kTcBN;
  cudaError_t e = cudaMemsetAsync(flags, 0, tc_persistent_flag_count(Kp, s.Cp) * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  TpArgs a{Kp, Ct, n_begin, n_end, err, h, flags, -1};
  TcMaps maps = *static_cast<const TcMaps *>(plan);
  StateView sv = s;
  StepTables tv = t;
  void *args[] = {&maps, &sv, &a, &tv};
  return cudaLaunchCooperativeKernel(kTpFnsOp[op][idx][s.Pr != s.P ? 1 : 0], dim3(Ct, Kp / kTcBM),
                                     dim3(kTpThreads), args, kTpSmemOp[op], st);
}

int tc_pair_blocks() {
  int best = 1 << 30;
  for (const void *f : kPrFns) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    cluster_config(&cfg, attr, dim3(2, 1), kTpThreads, TpShape<true>::kSmem, 0, false);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, f, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    best = clusters < best ? clusters : best;
  }
  return 2 * best;
}

bool tc_pair_eligible(int Kp, int Cp, int blocks) {
  return blocks > 0 && Kp % (2 * kTcBM) == 0 && Cp % kTcBN == 0 && (Kp / kTcBM) * (Cp / kTcBN) <= blocks;
}

cudaError_t launch_solve_dense_tc_pair(const void *plan, const StateView &s, int Kp, int *err, const float *h,
                                       const StepTables &t, int n_begin, int n_end, uint32_t *flags,
                                       cudaStream_t st) {
  const int idx = s.P == 1 ? 0 : s.P == 2 ? 1 : s.P == 4 ? 2 : s.P == 8 ? 3 : s.P == 16 ? 4 : s.P == 32 ? 5 : -1;
  if (idx < 0 || Kp % (2 * kTcBM) != 0 || s.Cp % kTcBN != 0) return cudaErrorInvalidValue;
  const int Ct = s.Cp / kTcBN;
  cudaError_t e = cudaMemsetAsync(flags, 0, tc_persistent_flag_count(Kp, s.Cp) * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  TpArgs a{Kp, Ct, n_begin, n_end, err, h, flags, -1};
  TcMaps maps = *static_cast<const TcMaps *>(plan);
  StateView sv = s;
  StepTables tv = t;
  void *args[] = {&maps, &sv, &a, &tv};
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[2];
  // row tiles along x (cluster pairs 2p, 2p+1), column tiles along y
  cluster_config(&cfg, attr, dim3(Kp / kTcBM, Ct), kTpThreads, TpShape<true>::kSmem, st, true);
  return cudaLaunchKernelExC(&cfg, kPrFns[idx], args);
}

template <int P>
static cudaError_t launch_tc_p(const TcMaps *p, const StateView &s, const TcArgs &a, const StepTables &t, int n,
                               cudaStream_t st) {
  if constexpr (P <= 32) {  // e4m3 with whole power-of-two runs: 128 x 256 tiles where the columns allow
    if (p->op == kOpF8 && s.Pr == s.P && s.Cp % kTwBN == 0) {
      k_step_dense_tc_wide<P><<<dim3(s.Cp / kTwBN, a.Kp / kTcBM), kTcThreads, kTwSmem, st>>>(*p, s, a, t, n);
      return cudaGetLastError();
    }
  }
  TcMaps maps = *p;
  StateView sv = s;
  TcArgs av = a;
  StepTables tv = t;
  int nv = n;
  void *args[] = {&maps, &sv, &av, &tv, &nv};
  const void *fn = kTcFns[p->op][p_index(P)][s.Pr != s.P ? 1 : 0];
  return cudaLaunchKernel(fn, dim3(s.Cp / kTcBN, a.Kp / kTcBM), dim3(kTcThreads), args, kTcSmem, st);
}

cudaError_t launch_step_dense_tc(const void *plan, const StateView &s, int Kp, uint8_t *FT, int *err, const float *h,
                                 const StepTables &t, int n, cudaStream_t st) {
  const auto *p = static_cast<const TcMaps *>(plan);
  TcArgs a{Kp, FT, err, h};
  if (s.Cp % kTcBN != 0 || Kp % kTcBM != 0) return cudaErrorInvalidValue;
  switch (s.P) {
    case 1: return launch_tc_p<1>(p, s, a, t, n, st);
    case 2: return launch_tc_p<2>(p, s, a, t, n, st);
    case 4: return launch_tc_p<4>(p, s, a, t, n, st);
    case 8: return launch_tc_p<8>(p, s, a, t, n, st);
    case 16: return launch_tc_p<16>(p, s, a, t, n, st);
    case 32: return launch_tc_p<32>(p, s, a, t, n, st);
    case 64: return launch_tc_p<64>(p, s, a, t, n, st);
    case 128: return launch_tc_p<128>(p, s, a, t, n, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_f_to_ft(const StateView &s, int which, uint8_t *FT, int Kp, int buffer, int op, cudaStream_t st) {
  const size_t total = size_t(s.Cp) * Kp;
  const unsigned blocks = unsigned((total + 255) / 256);
  if (op == kOpF8) k_f_to_ft8<<<blocks, 256, 0, st>>>(s, which, FT, Kp, buffer);
  else if (op == kOpBf16) k_f_to_ft16<<<blocks, 256, 0, st>>>(s, which, reinterpret_cast<uint16_t *>(FT), Kp, buffer);
  else if (op == kOpBsb) k_x_to_ft_split<<<blocks, 256, 0, st>>>(s, reinterpret_cast<uint16_t *>(FT), Kp, buffer);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace sbqa
