// solve_dense_tc_f4.cu -- the persistent dense solver with the coupling
// product G = J . f in packed 4-bit floats (e2m1) on the block-scaled
// tensor-core path, tcgen05.mma kind::mxf4 (Sec. II A, Eqs. 5-8).
//
// Integer couplings |J_ij| <= 4 and the codes f in {-1, 0, 1} of Eq. 8 are
// exact in e2m1 (0, 1, 2, 3, 4 and their negatives are e2m1 values).  Every
// scale factor is 2^0: the two scale-factor regions of tensor memory are
// filled with the ue8m0 code 127 before the first MMA, whatever part of them
// an MMA reads.  The products are summed in FP32 in TMEM, so G_ic is the same
// integer as in the e4m3 solver and the states agree bit for bit.
//
// Two values share a byte, so a step moves half the operand bytes of the e4m3
// form, and the 128 rows of J of a CTA (Kh bytes each, at most 144 KB for
// Kp <= 2304) stay in shared memory for the whole launch: per step only the
// f tiles stream in (16 KB per 256 spins).  That removes most of the traffic
// that bounds the e4m3 solver's K loop, where the MMAs' shared-memory reads
// and the TMA writes of both operands into the same memory serialise.
//
// Layout: J4 [Kp][Kh] bytes with Kh = 128 ceil(Kp / 256) (zeros past Kp), and
// FT4 [2][Kh / 128][Cp][128] bytes, k-block-major, so that one 4D TMA box
// brings several k-blocks of a column tile: the number of boxes a CTA keeps
// in flight, not their size, is what bounds the f loads (about one box per
// 300 ns per SM measured with one 16 KB box per k-block).  Spin 2t in the
// low nibble of byte t (within its k-block of 256 spins), 2t + 1 in the high
// nibble.  The MMA pairs element k of A with element k of B, so any nibble
// order that both operands share gives the same sums.
//
// Step counters, bounded waits, the epilogue (sb_update_regs32) and the stop
// protocol are those of the e4m3 persistent solver (dense_tc_persistent.cuh);
// a k-block of 256 spins waits for the counters of its two row tiles.
#include "dense_tc_persistent.cuh"

#include <cstdlib>
#include <cstring>

namespace sbqa {

constexpr int kOpF4 = 3;
constexpr int kF4MaxKB = 9;                 // resident J boxes of 256 spins: Kp <= 2304
constexpr int kF4Box = kTcBM * 128;         // 128 rows x 128 bytes (256 e2m1 values per row)
constexpr int kF4FTile = kTcBN * 64;        // packed f tile: 128 columns x 64 bytes (128 spins)
// f staging: two slots of 32 KB beside the resident J, each filled by one
// box of kG k-blocks.  A single CTA stages whole 128-column k-blocks (16 KB,
// two per box); a CTA of a pair stages its 64 of the pair's 128 columns
// (8 KB, four per box), so both slots hold every k-block of a step at once.
template <bool PAIR>
struct F4Shape {
  static constexpr int kG = PAIR ? 4 : 2;                         // k-blocks per box
  static constexpr int kKbBytes = PAIR ? kF4Box / 2 : kF4Box;     // one k-block of this CTA's columns
  static constexpr int kSlotBytes = kG * kKbBytes;
  static constexpr int kSlots = 2;
};
constexpr int kF4Stages = 4;  // staging bytes in 16 KB units: 2 slots x 32 KB
constexpr uint32_t kTmemSfa = 384, kTmemSfb = 416;  // scale factors of A and B, 32 columns each
constexpr uint32_t kUnitScales = 0x7F7F7F7Fu;       // four ue8m0 codes of 2^0
constexpr int kF4Smem = (kF4MaxKB + kF4Stages) * kF4Box + kF4FTile + 1024 + 256;
static_assert(kF4Smem <= 227 * 1024, "resident J, stages and f tile exceed the shared memory of one CTA");
static_assert(F4Shape<true>::kSlots * F4Shape<true>::kSlotBytes == kF4Stages * kF4Box &&
                  F4Shape<false>::kSlots * F4Shape<false>::kSlotBytes == kF4Stages * kF4Box,
              "both forms fit the same shared-memory layout");
static_assert(kTmemSfb + 32 <= kTmemCols, "scale-factor regions outside the allocated tensor memory");

// Instruction descriptor of tcgen05.mma kind::mxf4 (block-scaled): A = B =
// e2m1, both K-major, ue8m0 scale factors (ids 0), shape M x N.
__host__ __device__ constexpr uint32_t idesc_mxf4(int M, int N) {
  return (1u << 7) | (1u << 10)        // A, B format: e2m1
         | (uint32_t(N >> 3) << 17)    // N / 8
         | (1u << 23)                  // scale-factor type: ue8m0
         | (uint32_t(M >> 7) << 27);   // M / 128
}

// D (+)= (A . scale A) (B . scale B) with packed e2m1 operands (K = 64 per
// instruction: 32 bytes of a 128-byte swizzled row), two scale factors per
// row and instruction (blocks of 32 along K), FP32 accumulator in TMEM.
__device__ __forceinline__ void mma_mxf4(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t tmem_sfa, uint32_t tmem_sfb, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
      " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(tmem_sfa), "r"(tmem_sfb), "r"(accumulate)
      : "memory");
}

// The same MMA for a CTA pair, issued by the even CTA: A (M = 256) is the two
// CTAs' 128-row tiles at the same shared-memory address, B the two CTAs'
// 64-column halves; each CTA's TMEM receives its own 128 rows.
__device__ __forceinline__ void mma_mxf4_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t tmem_sfa, uint32_t tmem_sfb, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
      " tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(tmem_sfa), "r"(tmem_sfb), "r"(accumulate)
      : "memory");
}

// f codes of one spin row's 32 columns as e2m1 nibbles in registers: column
// j at bits 4 (j % 8) of word j / 8 (+1 = 0x2, -1 = 0xA, 0 = 0); the warp
// pairs rows 2t and 2t + 1 into bytes afterwards.
template <>
struct FOut<kOpF4> {
  uint32_t *nib;
  __device__ __forceinline__ void put(int j, float x, float delta) const {
    const uint32_t c = x > delta ? 0x2u : (x < -delta ? 0xAu : 0u);
    nib[j >> 3] |= c << (4 * (j & 7));
  }
  __device__ __forceinline__ void zero(int) const {}
};

struct Tc4Maps {
  CUtensorMap A;    // J4 [Kp][Kh]: 128 rows x 128 bytes, 128B swizzle
  CUtensorMap B;    // FT4 [2][KB][Cp][128]: boxes of 2 k-blocks x 128 columns x 128 bytes, 128B swizzle
  CUtensorMap B64;  // FT4 boxes of a CTA of a pair: 4 k-blocks x 64 columns x 128 bytes, 128B swizzle
  CUtensorMap Fst;  // FT4 tile store: 128 columns x 64 bytes of one k-block, no swizzle
  int Kh;           // bytes per row of J4 and FT4 (a multiple of 128)
};

// Steps [a.n_begin, a.n_end) of tile (mt, ct): 128 spin rows x 128 replica
// columns, x and y resident in TMEM (columns 128-383, the accumulator in
// 0-127, the scale factors in 384-447).
//
// Paired form (PAIR): the CTAs of row tiles 2p and 2p + 1 of one column tile
// form a 2-CTA cluster sharing one M=256 N=128 MMA per K slice (tcgen05
// cta_group::2, issued by the even CTA).  Each CTA keeps its own 128 J rows
// resident and stages 64 of the 128 f columns of every k-block, so a step's
// f tiles fit the eight stages at once and the K loop waits for one round
// trip to L2 instead of two.  The loads of both CTAs complete on the even
// CTA's barriers; MMA completion is multicast to both CTAs' empty and done
// barriers; a cluster barrier closes every step (ordering the odd CTA's
// accumulator reads before the next step's MMAs) and carries the abort
// decision, so both CTAs stop at the same step.
template <int P, bool GEN, bool PAIR>
__device__ __forceinline__ void solve_dense_tc_f4(const Tc4Maps &m, const StateView &s, const TpArgs &a,
                                                  const StepTables &t, int mt, int ct) {
  using Sh = F4Shape<PAIR>;
  constexpr int kSlots = Sh::kSlots, kSlotB = Sh::kSlotBytes, kG = Sh::kG, kKbB = Sh::kKbBytes;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int KB = m.Kh / 128;     // k-blocks of 256 spins
  const int NG = (KB + kG - 1) / kG;  // f boxes per step (the last one may reach past KB: zeros)
  const int Mt = a.Kp / kTcBM;   // row tiles: step counters per column tile
  uint8_t *sA = smem;                          // this tile's J rows, KB boxes, loaded once
  uint8_t *sB = sA + KB * kF4Box;              // f stages
  uint8_t *sF = sB + kF4Stages * kF4Box;       // packed f(x_next) tile [128 columns][64 bytes]
  uint64_t *full = reinterpret_cast<uint64_t *>(sF + kF4FTile);
  uint64_t *empty = full + kSlots;
  uint64_t *done = empty + kSlots;
  uint64_t *jfull = done + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(jfull + 1);
  int *s_abort = reinterpret_cast<int *>(tmem_slot + 1);  // PAIR: [step parity][rank]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t rank = 0;
  if constexpr (PAIR) {
    // both CTAs of a cluster read the same cluster shape, so both return here or neither does
    if (tc::cluster_nctarank() != 2 || tc::cluster_nctaid_x() != 2) {
      if (threadIdx.x == 0) atomicCAS(a.err, 0, tc::ERR_CLUSTER_SHAPE);
      return;
    }
    rank = tc::cluster_ctarank();
  }
  const bool leader = rank == 0;
  const int m0 = mt * kTcBM, n0 = ct * kTcBN;
  const int quarter = warp & 3, chunk = warp >> 2;
  const int rl = quarter * 32 + lane, i = m0 + rl;
  const int cl = 32 * chunk, c0 = n0 + cl;
  const uint32_t lane_off = uint32_t(quarter * 32) << 16;
  const CUtensorMap *mapB = PAIR ? &m.B64 : &m.B;
  const int bcol = n0 + (PAIR ? 64 * int(rank) : 0);  // first f column this CTA stages
  // loads completing on the (even CTA's) barrier bar
  auto load_j = [&](uint8_t *dst, uint64_t *bar, int c0_, int c1_) {
    if constexpr (PAIR)
      tc::tma_load_2d_pair(dst, &m.A, tc::map_to_rank(tc::smem_u32(bar), 0), c0_, c1_);
    else
      tc::tma_load_2d(dst, &m.A, bar, c0_, c1_);
  };
  auto load_f = [&](uint8_t *dst, uint64_t *bar, int gi, int buf) {
    if constexpr (PAIR)
      tc::tma_load_4d_pair(dst, mapB, tc::map_to_rank(tc::smem_u32(bar), 0), 0, bcol, gi * kG, buf);
    else
      tc::tma_load_4d(dst, mapB, bar, 0, bcol, gi * kG, buf);
  };

  if (threadIdx.x == 0) {
    for (int q = 0; q < kSlots; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&empty[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(jfull, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&m.A);
    tc::prefetch_tmap(mapB);
    tc::prefetch_tmap(&m.Fst);
    for (int q = 0; q < 4; ++q) s_abort[q] = 0;
  }
  if (warp == 0) {
    if constexpr (PAIR) tc::tmem_alloc_pair(tmem_slot, kTmemCols);
    else tc::tmem_alloc(tmem_slot, kTmemCols);
  }
  tc::tc_fence_before();
  if constexpr (PAIR) tc::cluster_sync();  // the pair's barriers and TMEM exist before either CTA uses them
  else __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  {  // the state tile (rows past N hold zeros and stay unchanged) and the unit scale factors into TMEM
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
    tc::tmem_st_32x32b_x32(tmem + lane_off + kTmemX + cl, xr);
    tc::tmem_st_32x32b_x32(tmem + lane_off + kTmemY + cl, yr);
    if (chunk < 2) {  // warps 0-3: scale factors of A, warps 4-7: of B (all 128 lanes, 32 columns each)
      uint32_t sf[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) sf[j] = kUnitScales;
      tc::tmem_st_32x32b_x32(tmem + lane_off + (chunk == 0 ? kTmemSfa : kTmemSfb), sf);
    }
    tc::tmem_wait_st();
  }
  const float hi = i < s.N ? __ldg(a.h + i) : 0.f;
  if (warp == 0 && lane == 0 && a.n_begin < a.n_end) {  // this tile's J rows, resident for the launch
    if (leader) tc::mbar_arrive_expect_tx(jfull, uint32_t((PAIR ? 2 : 1) * KB * kF4Box));
    for (int kb = 0; kb < KB; ++kb) load_j(sA + kb * kF4Box, jfull, kb * 128, m0);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();

  constexpr uint32_t idesc = idesc_mxf4(PAIR ? 2 * kTcBM : kTcBM, kTcBN);
  constexpr uint32_t kExpect = (PAIR ? 2 : 1) * kSlotB;  // bytes completing on one full barrier
  int n = a.n_begin;
  for (; n < a.n_end; ++n) {
    const uint32_t q = uint32_t(n - a.n_begin);
    if (warp == 0) {
      // producer: box gi (k-blocks kG gi ..) once row tiles 2 kb and 2 kb + 1 of each of its
      // k-blocks have published step q
      uint64_t t0 = 0;
      uint32_t polls = 0;
      int kb = 0;
      while (kb < KB) {
        const int kq = kb + lane;
        bool ok = q == 0 || kq >= KB;
        if (!ok) {
          const int r1 = 2 * kq + 1;
          ok = tc::ld_acquire_gpu(a.flags + (2 * kq) * a.Ct + ct) >= q &&
               (r1 >= Mt || tc::ld_acquire_gpu(a.flags + r1 * a.Ct + ct) >= q);
        }
        const unsigned ball = __ballot_sync(0xffffffffu, ok);
        int nready = ball == 0xffffffffu ? 32 : __ffs(~ball) - 1;
        nready = nready < KB - kb ? nready : KB - kb;
        int ng = kb + nready >= KB ? NG - kb / kG : nready / kG;  // whole boxes ready (kb is a box start)
        if (ng == 0) {
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
            ng = NG - kb / kG;  // proceed with whatever the buffer holds; the run reports the error
          } else {
            __nanosleep(64);
            continue;
          }
        }
        if (lane == 0) {
          asm volatile("fence.acq_rel.gpu;" ::: "memory");
          tc::fence_proxy_async_global();
          for (int gi = kb / kG; gi < kb / kG + ng; ++gi) {
            const uint32_t g = q * NG + gi, sl = g % kSlots, use = g / kSlots;
            if (use > 0) tc::mbar_wait(&empty[sl], (use - 1) & 1, a.err, tc::ERR_WAIT_EMPTY);
            if (leader) tc::mbar_arrive_expect_tx(&full[sl], kExpect);
            load_f(sB + sl * kSlotB, &full[sl], gi, n & 1);
          }
        }
        __syncwarp();
        kb += ng * kG;
      }
    } else if (warp == 1 && lane == 0 && leader) {
      if (q == 0) tc::mbar_wait(jfull, 0, a.err, tc::ERR_WAIT_FULL);
      for (int gi = 0; gi < NG; ++gi) {
        const uint32_t g = q * NG + gi, sl = g % kSlots, use = g / kSlots;
        tc::mbar_wait(&full[sl], use & 1, a.err, tc::ERR_WAIT_FULL);
        tc::tc_fence_after();
        for (int u = 0; u < kG && gi * kG + u < KB; ++u) {
          const int kb = gi * kG + u;
          const uint32_t a0 = tc::smem_u32(sA + kb * kF4Box), b0 = tc::smem_u32(sB + sl * kSlotB + u * kKbB);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = tc::smem_desc_sw128(a0 + kk * 32), bd = tc::smem_desc_sw128(b0 + kk * 32);
            const uint32_t acc = (kb | kk) != 0 ? 1u : 0u;
            if constexpr (PAIR) mma_mxf4_pair(tmem, ad, bd, idesc, tmem + kTmemSfa, tmem + kTmemSfb, acc);
            else mma_mxf4(tmem, ad, bd, idesc, tmem + kTmemSfa, tmem + kTmemSfb, acc);
          }
        }
        if constexpr (PAIR) tc::mma_commit_pair(&empty[sl]);
        else tc::mma_commit(&empty[sl]);
      }
      if constexpr (PAIR) tc::mma_commit_pair(done);
      else tc::mma_commit(done);
    }
    __syncwarp();
    const float ka = __ldg(t.ka + n), dnext = __ldg(t.dl + n + 1);
    KjChunk<P> kj;
    kj.load(s, t.kj + size_t(n) * t.R, c0);
    tc::mbar_wait(done, q & 1, a.err, tc::ERR_WAIT_DONE);
    tc::tc_fence_after();
    {
      uint32_t g[32], xr[32], yr[32];
      tc::tmem_ld_32x32b_x32_nowait(tmem + lane_off + cl, g);
      tc::tmem_ld_32x32b_x32_nowait(tmem + lane_off + kTmemX + cl, xr);
      tc::tmem_ld_32x32b_x32_nowait(tmem + lane_off + kTmemY + cl, yr);
      RingExt ext{0.f, 0.f, 0.f, 0.f};
      if constexpr (P > 32) {
        // runs over several chunks: their outside neighbours, read before any warp stores its new x
        const int rb = cl - cl % P;
        const uint32_t xb = tmem + lane_off + kTmemX;
        const uint32_t u0 = tc::tmem_ld_32x32b_x1_nowait(xb + uint32_t(cl > rb ? cl - 1 : cl));
        const uint32_t u1 = tc::tmem_ld_32x32b_x1_nowait(xb + uint32_t(cl + 32 < rb + P ? cl + 32 : cl));
        const uint32_t u2 = tc::tmem_ld_32x32b_x1_nowait(xb + uint32_t(rb));
        const uint32_t u3 = tc::tmem_ld_32x32b_x1_nowait(xb + uint32_t(rb + s.Pr - 1));
        tc::tmem_wait_ld();
        ext = RingExt{__uint_as_float(u0), __uint_as_float(u1), __uint_as_float(u2), __uint_as_float(u3)};
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
      }
      tc::tmem_wait_ld();
      tc::reg_fence(g);
      tc::reg_fence(xr);
      tc::reg_fence(yr);
      uint32_t nib[4] = {0u, 0u, 0u, 0u};
      const FOut<kOpF4> fo{nib};
      if (i < s.N && c0 < s.C) {
        if (c0 + 32 <= s.C) sb_update_regs32<P, true, kOpF4, GEN>(s, t, ka, dnext, kj, c0, g, hi, xr, yr, fo, ext);
        else sb_update_regs32<P, false, kOpF4, GEN>(s, t, ka, dnext, kj, c0, g, hi, xr, yr, fo, ext);
      }
      // rows 2t (even lane) and 2t + 1 (the next lane) share byte t of each column of the f tile;
      // both lanes of a pair hold both rows' nibbles and store alternate columns (the two rows of
      // one store instruction lie 64 bytes apart: no bank conflict)
      const int par = lane & 1;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const uint32_t o = __shfl_xor_sync(0xffffffffu, nib[w], 1);
        const uint32_t lo = par ? o : nib[w], hi = par ? nib[w] : o;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = 2 * i + par;
          sF[(cl + 8 * w + c) * 64 + (rl >> 1)] = uint8_t(((lo >> (4 * c)) & 0xFu) | (((hi >> (4 * c)) & 0xFu) << 4));
        }
      }
      __syncwarp();
      tc::tmem_st_32x32b_x32(tmem + lane_off + kTmemX + cl, xr);
      tc::tmem_st_32x32b_x32(tmem + lane_off + kTmemY + cl, yr);
      tc::tmem_wait_st();
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      // publish f_{n+1} of this tile: spins m0.. (half mt & 1 of k-block mt / 2), columns n0.., of the
      // other FT4 buffer
      tc::tma_store_4d(&m.Fst, sF, 64 * (mt & 1), n0, mt >> 1, (n + 1) & 1);
      tc::tma_store_commit_and_wait_all();
      tc::fence_proxy_async_global();
      if (n != a.hold_step || mt != 0 || ct != 0) tc::st_release_gpu(a.flags + mt * a.Ct + ct, q + 1);
      const int v = *reinterpret_cast<volatile int *>(a.err);
      if constexpr (PAIR) {
        int *slot = s_abort + 2 * (q & 1) + rank;  // double-buffered by step parity
        *slot = v;
        tc::st_cluster_u32(tc::map_to_rank(tc::smem_u32(slot), rank ^ 1u), uint32_t(v));
      } else {
        *s_abort = v;
      }
    }
    if constexpr (PAIR) tc::cluster_sync();  // also orders the odd CTA's accumulator reads before the next MMAs
    else __syncthreads();
    tc::tc_fence_after();
    const int stop = PAIR ? (s_abort[2 * (q & 1)] | s_abort[2 * (q & 1) + 1]) : *s_abort;
    if (stop != 0) break;
  }
  __syncwarp();
  {  // the state tile back to global memory
    uint32_t xr[32], yr[32];
    tc::tmem_ld_32x32b_x32_nowait(tmem + lane_off + kTmemX + cl, xr);
    tc::tmem_ld_32x32b_x32_nowait(tmem + lane_off + kTmemY + cl, yr);
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
  // PAIR: neither CTA leaves (or frees its TMEM) while the other's MMAs, loads or reads may still use it
  if constexpr (PAIR) tc::cluster_sync();
  else __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    if constexpr (PAIR) tc::tmem_dealloc_pair(tmem, kTmemCols);
    else tc::tmem_dealloc(tmem, kTmemCols);
  }
}

template <int P, bool GEN>
__global__ void __launch_bounds__(kTpThreads, 1)
    k_solve_dense_tc_f4(const __grid_constant__ Tc4Maps m, StateView s, TpArgs a, StepTables t) {
  solve_dense_tc_f4<P, GEN, false>(m, s, a, t, blockIdx.y, blockIdx.x);
}

// Row tiles along x (cluster pairs 2p, 2p + 1), column tiles along y.
template <int P, bool GEN>
__global__ void __launch_bounds__(kTpThreads, 1)
    k_solve_dense_tc_f4_pair(const __grid_constant__ Tc4Maps m, StateView s, TpArgs a, StepTables t) {
  solve_dense_tc_f4<P, GEN, true>(m, s, a, t, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- batched form
// The chunks of several small problems in one cooperative launch (as the
// batched e4m3 solver, solve_dense_tc_batched.cu): CTAs tile0 .. tile0 + Mt *
// Ct - 1 run problem r's tiles, row-tile major; the problem's tensor maps are
// read from the descriptor table in device memory (fenced into the tensormap
// proxy by the thread that issues the TMA copies), its step counters sit in
// the batch's flag array at tile0, and its error flag and step range are its
// own.  All problems of a launch share the run width P and the ring form.
struct Tb4Req {
  Tc4Maps m;  // first, so that every map of every entry is 64-byte aligned
  StateView s;
  TpArgs a;
  StepTables t;
  int tile0;
};

template <int P, bool GEN>
__global__ void __launch_bounds__(kTpThreads, 1) k_solve_dense_tc_f4_batched(const Tb4Req *__restrict__ q, int nq) {
  int r = 0;
  for (int k = 1; k < nq; ++k)
    if (int(blockIdx.x) >= q[k].tile0) r = k;
  const Tb4Req &d = q[r];
  if (threadIdx.x == 0) {  // the one thread that issues this CTA's TMA loads and stores
    tc::fence_tmap_acquire_sys(&d.m.A);
    tc::fence_tmap_acquire_sys(&d.m.B);
    tc::fence_tmap_acquire_sys(&d.m.Fst);
  }
  const StateView s = d.s;
  const TpArgs a = d.a;
  const StepTables t = d.t;
  const int local = int(blockIdx.x) - d.tile0;
  solve_dense_tc_f4<P, GEN, false>(d.m, s, a, t, local / a.Ct, local % a.Ct);
}

// e2m1 nibble of an e4m3 byte holding an integer |v| <= 4 (the only values
// an eligible instance has): 1, 2, 3, 4 -> 0x2, 0x4, 0x5, 0x6, sign in bit 3.
__device__ __forceinline__ uint32_t e2m1_of_e4m3_int(uint8_t e) {
  const uint32_t mag = e & 0x7Fu;
  const uint32_t m = mag == 0x38u ? 0x2u : mag == 0x40u ? 0x4u : mag == 0x44u ? 0x5u : mag == 0x48u ? 0x6u : 0u;
  return m == 0u ? 0u : (m | ((e & 0x80u) >> 4));
}

// J8 (e4m3 [Kp][Kp]) -> J4 ([Kp][Kh] bytes, two spins per byte, zeros past Kp).
__global__ void k_j4_from_j8(const uint8_t *J8, int Kp, int Kh, uint8_t *J4) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;  // over Kp * Kh
  if (e >= size_t(Kp) * Kh) return;
  const int r = int(e / Kh), j = 2 * int(e % Kh);
  uint32_t v = 0;
  if (j < Kp) v = e2m1_of_e4m3_int(J8[size_t(r) * Kp + j]);
  if (j + 1 < Kp) v |= e2m1_of_e4m3_int(J8[size_t(r) * Kp + j + 1]) << 4;
  J4[e] = uint8_t(v);
}

// f codes of F buffer `which` ([N][Cp], f + 1) -> FT4 buffer b ([KB][Cp][128]:
// byte t of k-block kb holds spins 256 kb + 2t and + 2t + 1; zeros for
// padded spins).
__global__ void k_f_to_ft4(StateView s, int which, uint8_t *FT4, int Kh, int b) {
  const size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x;  // over KB * Cp * 128
  if (e >= size_t(s.Cp) * Kh) return;
  const size_t per_kb = size_t(s.Cp) * 128;
  const int kb = int(e / per_kb), r = int(e % per_kb);
  const int c = r / 128, j = 256 * kb + 2 * (r % 128);
  uint32_t v = 0;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    if (j + u < s.N) {
      const int f = int(s.f_of(which)[size_t(j + u) * s.Cp + c]) - 1;
      v |= (f == 0 ? 0u : (f > 0 ? 0x2u : 0xAu)) << (4 * u);
    }
  }
  FT4[size_t(b) * s.Cp * Kh + e] = uint8_t(v);
}

// ---------------------------------------------------------------- host side
#define SBQA_F4_PS(K)                                                                                        \
  {{(const void *)K<1, false>, (const void *)K<1, false>},                                                   \
   {(const void *)K<2, false>, (const void *)K<2, false>},                                                   \
   {(const void *)K<4, false>, (const void *)K<4, true>},                                                    \
   {(const void *)K<8, false>, (const void *)K<8, true>},                                                    \
   {(const void *)K<16, false>, (const void *)K<16, true>},                                                  \
   {(const void *)K<32, false>, (const void *)K<32, true>},                                                  \
   {(const void *)K<64, true>, (const void *)K<64, true>},                                                   \
   {(const void *)K<128, true>, (const void *)K<128, true>}}
static const void *const kF4Fns[8][2] = SBQA_F4_PS(k_solve_dense_tc_f4);
static const void *const kF4PairFns[8][2] = SBQA_F4_PS(k_solve_dense_tc_f4_pair);
static const void *const kF4BatchFns[8][2] = SBQA_F4_PS(k_solve_dense_tc_f4_batched);
#undef SBQA_F4_PS

static int f4_p_index(int P) {
  for (int q = 0; q < 8; ++q)
    if ((1 << q) == P) return q;
  return -1;
}

int tc_f4_row_bytes(int Kp) { return (Kp + 255) / 256 * 128; }

static int f4_smem(int Kp) { return (tc_f4_row_bytes(Kp) / 128 + kF4Stages) * kF4Box + kF4FTile + 1024 + 256; }

cudaError_t tc_f4_set_attributes() {
  for (int q = 0; q < 8; ++q)
    for (int form = 0; form < 3; ++form)
      for (const void *f : (form == 2 ? kF4BatchFns : form == 1 ? kF4PairFns : kF4Fns)[q]) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kF4Smem);
        if (e != cudaSuccess) return e;
      }
  return cudaSuccess;
}

// Launch configuration of a cooperative grid of 2 x 1 x 1 clusters.
static void f4_cluster_config(cudaLaunchConfig_t *cfg, cudaLaunchAttribute *attr, dim3 grid, int smem,
                              cudaStream_t st, bool cooperative) {
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = grid;
  cfg->blockDim = dim3(kTpThreads);
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

int tc_f4_pair_blocks() {
  if (tc_f4_set_attributes() != cudaSuccess) return 0;
  int best = 1 << 30;
  for (int q = 0; q < 8; ++q)
    for (const void *f : kF4PairFns[q]) {
      cudaLaunchConfig_t cfg;
      cudaLaunchAttribute attr[2];
      f4_cluster_config(&cfg, attr, dim3(2, 1), kF4Smem, 0, false);
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, f, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      best = clusters < best ? clusters : best;
    }
  return 2 * best;
}

bool tc_f4_pair_eligible(int Kp, int Cp, int blocks) {
  return tc_f4_eligible(Kp, Cp, blocks) && Kp % (2 * kTcBM) == 0;
}

int tc_f4_blocks() {
  int dev = 0, sms = 0, best = 1 << 30;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (tc_f4_set_attributes() != cudaSuccess) return 0;
  for (int q = 0; q < 8; ++q)
    for (int form = 0; form < 2; ++form)
      for (const void *f : (form ? kF4BatchFns : kF4Fns)[q]) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kTpThreads, kF4Smem) != cudaSuccess) return 0;
        best = per_sm < best ? per_sm : best;
      }
  return sms * best;
}

bool tc_f4_eligible(int Kp, int Cp, int blocks) {
  return blocks > 0 && Kp % kTcBM == 0 && Cp % kTcBN == 0 && tc_f4_row_bytes(Kp) / 128 <= kF4MaxKB &&
         (Kp / kTcBM) * (Cp / kTcBN) <= blocks;
}

bool tc4_plan_make(void **plan, const void *J4, void *FT4, int Kp, int Cp) {
  auto *p = new Tc4Maps();
  const auto U8 = CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const int Kh = tc_f4_row_bytes(Kp);
  p->Kh = Kh;
  const uint64_t KB = uint64_t(Kh / 128);
  const uint64_t dims[4] = {128, uint64_t(Cp), KB, 2};  // FT4 [2][KB][Cp][128]
  const uint64_t strides[3] = {128, uint64_t(Cp) * 128, KB * Cp * 128};
  const uint32_t box_b[4] = {128, 128, uint32_t(F4Shape<false>::kG), 1};
  const uint32_t box_b64[4] = {128, 64, uint32_t(F4Shape<true>::kG), 1};
  const uint32_t box_st[4] = {64, 128, 1, 1};
  const bool ok =
      tc_make_map(&p->A, J4, U8, 1, uint64_t(Kp), uint64_t(Kh), 128, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
      tc_make_map_nd(&p->B, FT4, U8, 4, dims, strides, box_b, CU_TENSOR_MAP_SWIZZLE_128B) &&
      tc_make_map_nd(&p->B64, FT4, U8, 4, dims, strides, box_b64, CU_TENSOR_MAP_SWIZZLE_128B) &&
      tc_make_map_nd(&p->Fst, FT4, U8, 4, dims, strides, box_st, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (!ok) {
    delete p;
    return false;
  }
  *plan = p;
  return true;
}

void tc4_plan_free(void *plan) { delete static_cast<Tc4Maps *>(plan); }

cudaError_t launch_j4_from_j8(const uint8_t *J8, int Kp, uint8_t *J4, cudaStream_t st) {
  const int Kh = tc_f4_row_bytes(Kp);
  const size_t total = size_t(Kp) * Kh;
  k_j4_from_j8<<<unsigned((total + 255) / 256), 256, 0, st>>>(J8, Kp, Kh, J4);
  return cudaGetLastError();
}

cudaError_t launch_f_to_ft4(const StateView &s, int which, uint8_t *FT4, int Kp, int buffer, cudaStream_t st) {
  const int Kh = tc_f4_row_bytes(Kp);
  const size_t total = size_t(s.Cp) * Kh;
  k_f_to_ft4<<<unsigned((total + 255) / 256), 256, 0, st>>>(s, which, FT4, Kh, buffer);
  return cudaGetLastError();
}

cudaError_t launch_solve_dense_tc_f4(const void *plan, const StateView &s, int Kp, int *err, const float *h,
                                     const StepTables &t, int n_begin, int n_end, uint32_t *flags, cudaStream_t st) {
  const int idx = f4_p_index(s.P);
  const auto *m = static_cast<const Tc4Maps *>(plan);
  if (idx < 0 || Kp % kTcBM != 0 || s.Cp % kTcBN != 0 || m->Kh != tc_f4_row_bytes(Kp) ||
      m->Kh / 128 > kF4MaxKB)
    return cudaErrorInvalidValue;
  const int Ct = s.Cp / kTcBN;
  cudaError_t e = cudaMemsetAsync(flags, 0, tc_persistent_flag_count(Kp, s.Cp) * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  TpArgs a{Kp, Ct, n_begin, n_end, err, h, flags, -1};
  Tc4Maps maps = *m;
  StateView sv = s;
  StepTables tv = t;
  void *args[] = {&maps, &sv, &a, &tv};
  return cudaLaunchCooperativeKernel(kF4Fns[idx][s.Pr != s.P ? 1 : 0], dim3(Ct, Kp / kTcBM), dim3(kTpThreads), args,
                                     f4_smem(Kp), st);
}

cudaError_t launch_solve_dense_tc_f4_pair(const void *plan, const StateView &s, int Kp, int *err, const float *h,
                                          const StepTables &t, int n_begin, int n_end, uint32_t *flags,
                                          cudaStream_t st) {
  const int idx = f4_p_index(s.P);
  const auto *m = static_cast<const Tc4Maps *>(plan);
  if (idx < 0 || Kp % (2 * kTcBM) != 0 || s.Cp % kTcBN != 0 || m->Kh != tc_f4_row_bytes(Kp) ||
      m->Kh / 128 > kF4MaxKB)
    return cudaErrorInvalidValue;
  const int Ct = s.Cp / kTcBN;
  cudaError_t e = cudaMemsetAsync(flags, 0, tc_persistent_flag_count(Kp, s.Cp) * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  TpArgs a{Kp, Ct, n_begin, n_end, err, h, flags, -1};
  Tc4Maps maps = *m;
  StateView sv = s;
  StepTables tv = t;
  void *args[] = {&maps, &sv, &a, &tv};
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[2];
  // row tiles along x (cluster pairs 2p, 2p + 1), column tiles along y
  f4_cluster_config(&cfg, attr, dim3(Kp / kTcBM, Ct), f4_smem(Kp), st, true);
  return cudaLaunchKernelExC(&cfg, kF4PairFns[idx][s.Pr != s.P ? 1 : 0], args);
}


struct Tc4Batch {
  int cap_reqs = 0, cap_tiles = 0;
  Tb4Req *host = nullptr;     // staging, 64-byte aligned
  Tb4Req *dev = nullptr;      // descriptor table
  uint32_t *flags = nullptr;  // step counters of all tiles of a launch
  int n = 0, tiles = 0, P = 0, gen = 0;
};

cudaError_t tc4_batch_create(Tc4Batch **out, int cap_reqs, int cap_tiles) {
  *out = nullptr;
  if (cap_reqs < 1 || cap_tiles < 1) return cudaErrorInvalidValue;
  Tc4Batch *b = new Tc4Batch;
  b->cap_reqs = cap_reqs;
  b->cap_tiles = cap_tiles;
  const size_t hb = (sizeof(Tb4Req) * size_t(cap_reqs) + 63) / 64 * 64;
  b->host = static_cast<Tb4Req *>(std::aligned_alloc(64, hb));
  cudaError_t e = b->host ? cudaSuccess : cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = cudaMalloc(&b->dev, sizeof(Tb4Req) * size_t(cap_reqs));
  if (e == cudaSuccess) e = cudaMalloc(&b->flags, sizeof(uint32_t) * size_t(cap_tiles));
  if (e != cudaSuccess) {
    tc4_batch_destroy(b);
    return e;
  }
  *out = b;
  return cudaSuccess;
}

void tc4_batch_destroy(Tc4Batch *b) {
  if (!b) return;
  std::free(b->host);
  if (b->dev) cudaFree(b->dev);
  if (b->flags) cudaFree(b->flags);
  delete b;
}

void tc4_batch_clear(Tc4Batch *b) { b->n = b->tiles = 0; }

int tc4_batch_size(const Tc4Batch *b) { return b->n; }

bool tc4_batch_fits(const Tc4Batch *b, const StateView &s, int Kp) {
  const int tiles = (Kp / kTcBM) * (s.Cp / kTcBN);
  if (b->n >= b->cap_reqs || b->tiles + tiles > b->cap_tiles) return false;
  return b->n == 0 || (b->P == s.P && b->gen == (s.Pr != s.P ? 1 : 0));
}

cudaError_t tc4_batch_add(Tc4Batch *b, const void *plan4, const StateView &s, int Kp, int *err, const float *h,
                          const StepTables &t, int n_begin, int n_end, int hold_step) {
  const auto *m = static_cast<const Tc4Maps *>(plan4);
  if (f4_p_index(s.P) < 0 || Kp % kTcBM != 0 || s.Cp % kTcBN != 0 || n_end < n_begin ||
      m->Kh != tc_f4_row_bytes(Kp) || m->Kh / 128 > kF4MaxKB || !tc4_batch_fits(b, s, Kp))
    return cudaErrorInvalidValue;
  Tb4Req &d = b->host[b->n];
  std::memcpy(&d.m, m, sizeof(Tc4Maps));
  d.s = s;
  d.a = TpArgs{Kp, s.Cp / kTcBN, n_begin, n_end, err, h, b->flags + b->tiles, hold_step};
  d.t = t;
  d.tile0 = b->tiles;
  b->P = s.P;
  b->gen = s.Pr != s.P ? 1 : 0;
  b->tiles += (Kp / kTcBM) * (s.Cp / kTcBN);
  ++b->n;
  return cudaSuccess;
}

// Copies the descriptors (pageable staging: the call returns once the host
// buffer has been read), zeroes the flags and launches, all ordered on st.
cudaError_t tc4_batch_launch(Tc4Batch *b, cudaStream_t st) {
  if (b->n == 0) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(b->dev, b->host, sizeof(Tb4Req) * size_t(b->n), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->flags, 0, sizeof(uint32_t) * size_t(b->tiles), st);
  if (e != cudaSuccess) return e;
  const Tb4Req *q = b->dev;
  int nq = b->n;
  void *args[] = {&q, &nq};
  return cudaLaunchCooperativeKernel(kF4BatchFns[f4_p_index(b->P)][b->gen], dim3(b->tiles), dim3(kTpThreads), args,
                                     kF4Smem, st);
}

}  // namespace sbqa
