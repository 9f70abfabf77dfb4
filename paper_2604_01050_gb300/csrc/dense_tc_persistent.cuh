// dense_tc_persistent.cuh -- the body of the persistent tcgen05 dense solver
// (one CTA per 128 x 128 output tile for a whole stretch of steps, Sec. II A,
// Eqs. 5-8), shared by the single-problem solvers and the batched solver.
#pragma once
#include "dense_tc_common.cuh"

namespace sbqa {

// ---------------------------------------------------------------- persistent solver
// All steps of a stretch in one cooperative launch.  Each CTA owns one 128 x
// 128 tile (spin rows x replica columns) for the whole stretch and keeps its x
// and y in tensor memory next to the accumulator (TMEM columns 0-127: G,
// 128-255: x, 256-383: y), so shared memory holds six operand stages and a
// step moves only J and f through the memory system.  A step of tile (mt, ct)
// needs f_n of the 128 spins of every row tile kb for its columns, which CTA
// (kb, ct) wrote at the end of its previous step; instead of a grid barrier
// every CTA publishes a per-tile step counter (release, after its f tile's
// TMA store has completed) and the producer warp polls the counters of its
// column group (acquire, then a proxy fence before the TMA loads of those
// tiles), issuing k-blocks in order as their tiles become ready (kTpGroup
// consecutive k-blocks of J and of f per TMA box in the single-CTA e4m3 and
// bfloat16 forms, one per box otherwise).  The J tiles of the next step's
// first stages are loaded while the epilogue runs.  A wait
// that gives up (2 s, or at once when another CTA has already failed)
// records an error; every CTA then stops at its next step boundary.
//
// Paired form (PAIR): the CTAs of row tiles 2p and 2p+1 (same column tile)
// form a 2-CTA cluster that shares one M=256 N=128 MMA per K slice
// (tcgen05 cta_group::2, issued by the even CTA): each CTA stages its own 128
// J rows and 64 of the 128 fT rows of the column tile, and each keeps the
// accumulator rows, x and y of its own 128 spins in its own TMEM.  Per CTA the
// operands of an MMA are then 24 KB per k-block instead of 32 KB, which is
// what lets the K loop run at the full MMA rate where 128 x 128 tiles fed by
// TMA run at half of it.  The even CTA's full barrier collects the bytes of
// both CTAs' loads; MMA completion is multicast to both CTAs' empty and done
// barriers; a cluster barrier closes every step (so the next step's MMAs do
// not overwrite an accumulator the odd CTA still reads) and carries the
// abort decision, so that both CTAs stop at the same step.
constexpr int kTpThreads = 512;  // 16 warps: warp w updates TMEM lanes 32 (w % 4).. and columns 32 (w / 4)..
constexpr uint32_t kTmemX = 128, kTmemY = 256, kTmemCols = 512;
constexpr uint64_t kFlagTimeoutNs = 2000000000ull;

template <bool PAIR, int OP = kOpF8>
struct TpShape {
  static constexpr int kNB = TcOp<OP>::kNB;
  static constexpr int kStages = PAIR ? 8 : (kNB == 2 ? 3 : 6);
  // k-blocks per TMA box: the single-CTA e4m3 and bfloat16 forms bring
  // kTpGroup consecutive k-blocks of J and of f per box (3D views of the same
  // buffers), because the loads are bound by the boxes a CTA keeps in flight
  // more than by their bytes; slots of kG stages
  static constexpr int kG = (PAIR || kNB == 2) ? 1 : kTpGroup;
  static constexpr int kSlots = kStages / kG;
  static constexpr int kTileB = PAIR ? 64 * kTcBK : kTcTile;  // fT rows staged by this CTA: 64 of the pair's 128, or 128
  static constexpr int kStageBytes = kTcTile + kNB * kTileB;
  static constexpr uint32_t kExpect = PAIR ? 2 * kStageBytes : kStageBytes;  // bytes completing on one full barrier
  static constexpr int kFBytes = kNB * TcOp<OP>::kFTile;                 // f tile(s) of the epilogue
  static constexpr int kSmem = kStages * kStageBytes + kFBytes + 1024 + 256;
};
static_assert(TpShape<false>::kSmem <= 227 * 1024 && TpShape<true>::kSmem <= 227 * 1024 &&
                  TpShape<false, kOpBf16>::kSmem <= 227 * 1024 && TpShape<false, kOpBsb>::kSmem <= 227 * 1024,
              "persistent tile exceeds the shared memory of one CTA");

struct TpArgs {
  int Kp, Ct, n_begin, n_end;
  int *err;
  const float *h;
  uint32_t *flags;  // [Kp / 128][Ct] steps completed in this launch, zeroed by the host
  int hold_step;    // test hook: tile (0, 0) leaves its counter unpublished after this step (-1: never)
};

// One run-aligned chunk of 32 columns of spin row i, in registers (bit
// patterns of FP32 x, y and the accumulated G).  Same arithmetic, in the same
// order, as sb_update_row32: all momenta first (they read the old positions of
// the ring neighbours), then positions, wall and f, whose e4m3 code goes to
// column j of the transposed f tile (sFcol[j * 128]).  FULL: all 32 columns
// are below C.
template <int P, bool FULL, int OP, bool GEN = false>
__device__ __forceinline__ void sb_update_regs32(const StateView &s, const StepTables &t, float ka, float dnext,
                                                 const KjChunk<P> &kj, int c0, const uint32_t (&g)[32], float hi,
                                                 uint32_t (&xr)[32], uint32_t (&yr)[32], const FOut<OP> &fo,
                                                 const RingExt &ext) {
  constexpr int PR = P < 32 ? P : 32;
  float xs[32], xms[32], xps[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) xs[j] = __uint_as_float(xr[j]);
  ring32<P, GEN>(xs, s.Pr, c0, ext, xms, xps);
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    if (!FULL && c0 + j >= s.C) continue;
    const float xm = xms[j], xp = xps[j];
    const float xj = xs[j];
    float yn = fmaf(t.kc, __uint_as_float(g[j]) + hi, __uint_as_float(yr[j]));
    yn = fmaf(-ka, xj, yn);
    yn = fmaf(kj.get(c0, j / PR), xm + xp, yn);
    yr[j] = __float_as_uint(yn);
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    if (FULL || c0 + j < s.C) {
      float xn = fmaf(t.kx, __uint_as_float(yr[j]), __uint_as_float(xr[j]));
      if (fabsf(xn) > 1.f) {
        xn = copysignf(1.f, xn);
        yr[j] = __float_as_uint(0.f);
      }
      xr[j] = __float_as_uint(xn);
      fo.put(j, xn, dnext);
    } else {
      fo.zero(j);
    }
  }
}

template <int P, bool PAIR, int OP, bool GEN>
__device__ __forceinline__ void solve_dense_tc_persistent(const TcMaps &m, const StateView &s, const TpArgs &a,
                                                          const StepTables &t, int mt, int ct) {
  static_assert(!PAIR || OP == kOpF8, "CTA pairs run the e4m3 product only");
  using Sh = TpShape<PAIR, OP>;
  using O = TcOp<OP>;
  constexpr int kStages = Sh::kStages, kG = Sh::kG, kSlots = Sh::kSlots;
  constexpr int kStageB = O::kNB * Sh::kTileB;  // B bytes of one stage (hi and lo for kOpBsb)
  static_assert(kSlots * kG == kStages, "slots of whole stages");
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kTcTile;
  uint8_t *sF = sB + kStages * kStageB;  // [128 columns][128 spins] f(x_next) (kOpBsb: hi, then lo)
  uint64_t *full = reinterpret_cast<uint64_t *>(sF + Sh::kFBytes);
  uint64_t *empty = full + kStages;
  uint64_t *done = empty + kStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  int *s_abort = reinterpret_cast<int *>(tmem_slot + 1);  // PAIR: [step parity][rank]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t rank = 0;
  if constexpr (PAIR) {
    // both CTAs of a cluster read the same cluster shape, so both return here or neither does
    if (tc::cluster_nctarank() != 2 || tc::cluster_nctaid_x() != 2) {
      if (threadIdx.x == 0) atomicCAS(a.err, 0, tc::ERR_CLUSTER_SHAPE);
      return;
    }
    rank = tc::cluster_ctarank();  // = blockIdx.x & 1
  }
  const bool leader = rank == 0;
  const int m0 = mt * kTcBM, n0 = ct * kTcBN;
  const int KB = a.Kp / O::kKE;
  const int NS = (KB + kG - 1) / kG;             // slot loads per step (a last box past KB reads zeros)
  const int npre = NS < kSlots ? NS : kSlots;    // slot loads whose J box is loaded ahead
  // this CTA's operand loads: fT rows (B box) and the full barrier they complete on
  const CUtensorMap *mapB = PAIR ? &m.B64 : &m.B;
  const int b_off = PAIR ? 64 * int(rank) : 0;
  auto load_tile = [&](uint8_t *dst, const CUtensorMap *map, int st, int c0_, int c1_) {
    if constexpr (PAIR)
      tc::tma_load_2d_pair(dst, map, tc::map_to_rank(tc::smem_u32(&full[st]), 0), c0_, c1_);
    else
      tc::tma_load_2d(dst, map, &full[st], c0_, c1_);
  };
  // J box of slot load js (k-blocks kG js ..) into slot sl, and its f box(es) at f row brow
  auto load_a = [&](int sl, int js) {
    if constexpr (kG == 1) load_tile(sA + sl * kTcTile, &m.A, sl, js * O::kKE, m0);
    else tc::tma_load_3d(sA + sl * kG * kTcTile, &m.A3, &full[sl], 0, m0, js * kG);
  };
  auto load_b = [&](int sl, int js, int brow) {
    if constexpr (kG == 1) {
      load_tile(sB + sl * kStageB, mapB, sl, js * O::kKE, brow + b_off);
      if constexpr (O::kNB == 2) load_tile(sB + sl * kStageB + Sh::kTileB, &m.Bl, sl, js * O::kKE, brow);
    } else {
      tc::tma_load_3d(sB + sl * kG * kStageB, &m.B3, &full[sl], 0, brow, js * kG);
    }
  };
  constexpr uint32_t kSlotExpect = kG * Sh::kExpect;  // bytes completing on one full barrier
  const int quarter = warp & 3, chunk = warp >> 2;
  const int rl = quarter * 32 + lane, i = m0 + rl;
  const int cl = 32 * chunk, c0 = n0 + cl;
  const uint32_t lane_off = uint32_t(quarter * 32) << 16;

  if (threadIdx.x == 0) {
    for (int q = 0; q < kStages; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&empty[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&m.A);
    tc::prefetch_tmap(mapB);
    if constexpr (kG > 1) {
      tc::prefetch_tmap(&m.A3);
      tc::prefetch_tmap(&m.B3);
    }
    tc::prefetch_tmap(&m.Fst);
    if constexpr (O::kNB == 2) {
      tc::prefetch_tmap(&m.Bl);
      tc::prefetch_tmap(&m.Fstl);
    }
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

  {  // the state tile into TMEM (rows past N hold zeros and stay unchanged)
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
    tc::tmem_wait_st();
  }
  const float hi = i < s.N ? __ldg(a.h + i) : 0.f;
  if (warp == 0 && lane == 0 && a.n_begin < a.n_end) {  // J tiles of the first step's first stages
    for (int js = 0; js < npre; ++js) {
      if (leader) tc::mbar_arrive_expect_tx(&full[js], kSlotExpect);
      load_a(js, js);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();

  constexpr uint32_t idesc = O::idesc(PAIR ? 2 * kTcBM : kTcBM, kTcBN);
  constexpr int kFlagShift = OP == kOpF8 ? 0 : 1;  // k-blocks per 128-spin row tile: 1 (e4m3) or 2 (bf16)
  int n = a.n_begin;
  bool prefetched = a.n_begin < a.n_end;
  for (; n < a.n_end; ++n) {
    const uint32_t q = uint32_t(n - a.n_begin);
    if (warp == 0) {
      // producer: f tiles as their row tiles publish step q, J tiles beyond the prefetched ones
      const int brow = (n & 1) * s.Cp + n0;
      uint64_t t0 = 0;
      uint32_t polls = 0;
      int kb = 0;
      while (kb < KB) {
        const int kq = kb + lane;
        const bool ok = q == 0 || kq >= KB || tc::ld_acquire_gpu(a.flags + (kq >> kFlagShift) * a.Ct + ct) >= q;
        const unsigned ball = __ballot_sync(0xffffffffu, ok);
        int nready = ball == 0xffffffffu ? 32 : __ffs(~ball) - 1;
        nready = nready < KB - kb ? nready : KB - kb;
        int ns = kb + nready >= KB ? NS - kb / kG : nready / kG;  // whole slot loads ready (kb starts one)
        if (ns == 0) {
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
            ns = NS - kb / kG;  // proceed with whatever the buffer holds; the run reports the error
          } else {
            __nanosleep(64);
            continue;
          }
        }
        if (lane == 0) {
          asm volatile("fence.acq_rel.gpu;" ::: "memory");
          tc::fence_proxy_async_global();
          for (int js = kb / kG; js < kb / kG + ns; ++js) {
            const uint32_t g = q * NS + js, sl = g % kSlots, use = g / kSlots;
            if (js >= npre) {
              if (use > 0) tc::mbar_wait(&empty[sl], (use - 1) & 1, a.err, tc::ERR_WAIT_EMPTY);
              if (leader) tc::mbar_arrive_expect_tx(&full[sl], kSlotExpect);
              load_a(int(sl), js);
            }
            load_b(int(sl), js, brow);
          }
        }
        __syncwarp();
        kb += ns * kG;
      }
      // J boxes of the next step's first slot loads, behind this step's MMAs
      prefetched = n + 1 < a.n_end;
      if (lane == 0 && prefetched) {
        for (int js = 0; js < npre; ++js) {
          const uint32_t g = (q + 1) * NS + js, sl = g % kSlots, use = g / kSlots;
          if (use > 0) tc::mbar_wait(&empty[sl], (use - 1) & 1, a.err, tc::ERR_WAIT_EMPTY);
          if (leader) tc::mbar_arrive_expect_tx(&full[sl], kSlotExpect);
          load_a(int(sl), js);
        }
      }
    } else if (warp == 1 && lane == 0 && leader) {
      for (int kb = 0; kb < KB; ++kb) {
        const int js = kb / kG, u = kb - js * kG;
        const uint32_t g = q * NS + js, sl = g % kSlots, use = g / kSlots;
        if (u == 0) {
          tc::mbar_wait(&full[sl], use & 1, a.err, tc::ERR_WAIT_FULL);
          tc::tc_fence_after();
        }
        const int st = int(sl) * kG + u;  // the stage (memory) of k-block kb
        const uint32_t a0 = tc::smem_u32(sA + st * kTcTile), b0 = tc::smem_u32(sB + st * kStageB);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t ad = tc::smem_desc_sw128(a0 + kk * 32), bd = tc::smem_desc_sw128(b0 + kk * 32);
          if constexpr (PAIR) {
            tc::mma_f8_pair(tmem, ad, bd, idesc, (kb | kk) != 0 ? 1u : 0u);
          } else {
            O::mma(tmem, ad, bd, idesc, (kb | kk) != 0 ? 1u : 0u);
            if constexpr (O::kNB == 2)
              O::mma(tmem, ad, tc::smem_desc_sw128(b0 + Sh::kTileB + kk * 32), idesc, 1u);
          }
        }
        if (u == kG - 1 || kb == KB - 1) {
          if constexpr (PAIR) tc::mma_commit_pair(&empty[sl]);
          else tc::mma_commit(&empty[sl]);
        }
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
      const FOut<OP> fo = f_out<OP>(sF, cl, rl);
      if (i < s.N && c0 < s.C) {
        if (c0 + 32 <= s.C) sb_update_regs32<P, true, OP, GEN>(s, t, ka, dnext, kj, c0, g, hi, xr, yr, fo, ext);
        else sb_update_regs32<P, false, OP, GEN>(s, t, ka, dnext, kj, c0, g, hi, xr, yr, fo, ext);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) fo.zero(j);
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
      // publish f_{n+1} of this tile: spins m0.., columns n0.. of the other FT buffer
      tc::tma_store_2d(&m.Fst, sF, m0, ((n + 1) & 1) * s.Cp + n0);
      if constexpr (O::kNB == 2) tc::tma_store_2d(&m.Fstl, sF + O::kFTile, m0, ((n + 1) & 1) * s.Cp + n0);
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
  if (n < a.n_end && prefetched && warp == 0 && lane == 0) {
    // stopped early with J tiles of step n + 1 in flight: complete those stages
    // (with any f tile) and wait for them, so no copy outlives the block
    const uint32_t q = uint32_t(n + 1 - a.n_begin);
    const int brow = ((n + 1) & 1) * s.Cp + n0;
    for (int js = 0; js < npre; ++js) {
      const uint32_t g = q * NS + js, sl = g % kSlots, use = g / kSlots;
      load_b(int(sl), js, brow);
      if (leader) tc::mbar_wait(&full[sl], use & 1, a.err, tc::ERR_WAIT_FULL);
    }
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

}  // namespace sbqa
