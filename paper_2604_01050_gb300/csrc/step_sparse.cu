// step_sparse.cu -- one SBQA step for CSR couplings (Sec. II A, Eq. 7 with a
// sparse J), the coupling product and the update fused in one kernel.
//
// A warp owns one spin row i and walks all its replica columns in chunks of
// 32 W (W = 4, 8 or 16 consecutive columns per lane, picked per problem shape
// by the autotuner).  The row's (col, J) entries are read 32 at a time, one
// per lane, and broadcast by shuffle; the lane gathers W bytes of F (the f
// codes of the neighbour spin for its columns) for several entries at once,
// so the gathers overlap.  The x, y loads are issued before the product.
// Accumulation:
//   VAL_PM1   J = +-1: plain 32-bit adds of packed f + 1 codes, one sum per
//             sign (rows are stored +1 entries first), exact while the row
//             degree is <= 127 (checked on the host)
//   VAL_F32   FP32 J, FP32 accumulation (exact for small-integer J)
//   VAL_BF16  bfloat16 J, FP32 accumulation
// Memory per update: x, y read + write (16 B) + F write (1 B); F gathers and
// the CSR arrays are shared by all columns of a row and mostly hit in cache.
#include <algorithm>

#include "step_common.cuh"

namespace sbqa {

template <int KIND>
__device__ __forceinline__ float load_val(const void *val, int e) {
  if constexpr (KIND == VAL_F32) return __ldg(static_cast<const float *>(val) + e);
  else return __bfloat162float(static_cast<const __nv_bfloat16 *>(val)[e]);
}

// F codes of W consecutive columns (one 4, 8 or 16 byte load).
template <int W>
struct FVec;
template <>
struct FVec<4> {
  uint32_t w[1];
  __device__ __forceinline__ void load(const uint8_t *p) { w[0] = __ldg(reinterpret_cast<const uint32_t *>(p)); }
  __device__ __forceinline__ void zero(uint32_t z) { w[0] = z; }
};
template <>
struct FVec<8> {
  uint32_t w[2];
  __device__ __forceinline__ void load(const uint8_t *p) {
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
    w[0] = v.x; w[1] = v.y;
  }
  __device__ __forceinline__ void zero(uint32_t z) { w[0] = w[1] = z; }
};
template <>
struct FVec<16> {
  uint32_t w[4];
  __device__ __forceinline__ void load(const uint8_t *p) {
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  }
  __device__ __forceinline__ void zero(uint32_t z) { w[0] = w[1] = w[2] = w[3] = z; }
};

// One warp per (spin row, chunk of 32 W replica columns), W consecutive
// columns per lane.  The lane issues its x, y loads, then gathers W bytes of
// f codes per neighbour (U neighbours at a time), accumulates and runs the
// update.  The row's (col, J) entries are read 32 at a time, one per lane,
// and broadcast by shuffle.
// GS = false: grid (ceil(N / 8), Cp / 32 W), one item per warp.  GS = true:
// one wave of resident blocks; warp g takes items g, g + warps, ... in
// row-major (row, chunk) order, so no block is launched per item.
template <int P, int KIND, int W, bool GS>
__global__ void __launch_bounds__(256, W == 16 ? 2 : (W == 8 ? 3 : 4))
    k_step_csr(StateView s, CsrView J, StepTables t, int n) {
  constexpr int U = W == 16 ? 4 : 8;  // gathers in flight per lane
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float ka = __ldg(t.ka + n), dnext = __ldg(t.dl + n + 1);
  const uint8_t *Fin = s.f_of(n);
  uint8_t *Fout = s.f_of(n + 1);
  const int chunks = s.Cp / (32 * W);
  const long long n_items = GS ? (long long)s.N * chunks : 1;
  const long long stride = GS ? (long long)gridDim.x * 8 : 1;
  for (long long item = GS ? (long long)blockIdx.x * 8 + warp : 0; item < n_items; item += stride) {
    const int i = GS ? int(item / chunks) : blockIdx.x * 8 + warp;
    const int chunk = GS ? int(item - (long long)i * chunks) : blockIdx.y;
    if (i >= s.N) return;  // whole warp (per-item grid only)
    const float hi = __ldg(J.h + i);
    const int e0 = __ldg(J.row_ptr + i), e1 = __ldg(J.row_ptr + i + 1);
    const int ep = (KIND == VAL_PM1) ? e0 + __ldg(J.npos + i) : e1;
    const int cw = chunk * 32 * W;
    const int c0 = cw + lane * W;
    float xs[W], ys[W];
    {
      const size_t off = size_t(i) * s.Cp + c0;
#pragma unroll
      for (int q = 0; q < W / 4; ++q) {
        const float4 a = *reinterpret_cast<const float4 *>(s.x + off + 4 * q);
        const float4 b = *reinterpret_cast<const float4 *>(s.y + off + 4 * q);
        xs[4 * q] = a.x; xs[4 * q + 1] = a.y; xs[4 * q + 2] = a.z; xs[4 * q + 3] = a.w;
        ys[4 * q] = b.x; ys[4 * q + 1] = b.y; ys[4 * q + 2] = b.z; ys[4 * q + 3] = b.w;
      }
    }
    uint32_t ap[W / 4], am[W / 4];
    float g[W];
#pragma unroll
    for (int q = 0; q < W / 4; ++q) ap[q] = am[q] = 0;
#pragma unroll
    for (int q = 0; q < W; ++q) g[q] = 0.f;
    const uint8_t *Fc = Fin + c0;
    for (int base = e0; base < e1; base += 32) {
      const int cnt = min(32, e1 - base);
      int my_col = 0;
      float my_w = 0.f;
      if (lane < cnt) {
        my_col = __ldg(J.col + base + lane);
        if constexpr (KIND != VAL_PM1) my_w = load_val<KIND>(J.val, base + lane);
      }
      for (int q = 0; q < cnt; q += U) {
        FVec<W> f[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = __shfl_sync(0xffffffffu, my_col, q + u);
          if (q + u < cnt) f[u].load(Fc + size_t(j) * s.Cp);
          else f[u].zero(KIND == VAL_PM1 ? 0u : kFZero4);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if constexpr (KIND == VAL_PM1) {
            if (base + q + u < ep) {  // warp-uniform
#pragma unroll
              for (int w = 0; w < W / 4; ++w) ap[w] += f[u].w[w];
            } else {
#pragma unroll
              for (int w = 0; w < W / 4; ++w) am[w] += f[u].w[w];
            }
          } else {
            const float wt = __shfl_sync(0xffffffffu, my_w, q + u);  // 0 past the row end
            acc_codes<W>(g, wt, f[u].w);
          }
        }
      }
    }
    float G[W];
    if constexpr (KIND == VAL_PM1) {
      const int bias = (e1 - ep) - (ep - e0);  // codes carry f + 1
#pragma unroll
      for (int c = 0; c < W; ++c)
        G[c] = float(int((ap[c / 4] >> (8 * (c % 4))) & 0xffu) - int((am[c / 4] >> (8 * (c % 4))) & 0xffu) + bias);
    } else {
#pragma unroll
      for (int c = 0; c < W; ++c) G[c] = g[c];
    }
    if (P > 2 && s.Pr != P) sb_updateW<P, W, true>(s, t, ka, dnext, n, i, c0, G, hi, xs, ys, Fout);
    else sb_updateW<P, W, false>(s, t, ka, dnext, n, i, c0, G, hi, xs, ys, Fout);
  }
}

// ELL form for rows of degree <= 8 (variants 6, 7): each row's entries sit
// in 8 slots (column, value; +1 entries first for +-1 J) with (degree, +1
// count), so one load gives a row's neighbours.  One wave of blocks loops over
// the (row, chunk) items; while a warp gathers and updates one item it has
// already issued the next item's slots and x, y, so each item waits for one
// round of gathers only.  Entries are summed in the CSR kernel's order.
// LPI = 16: a half warp per item of 16 W columns, the warp on two items at a
// time (lanes 16-31 on the odd one): twice the items in flight per warp and
// half the per-item instructions; the same sums and update per column.
// (The half-warp form loads each pass's rows when it starts it, without the
// one-pass-ahead prefetch: two items per warp are in flight already, and four
// blocks per SM fit its registers.)
template <int P, int KIND, int W, int LPI = 32>
__global__ void __launch_bounds__(256, (W == 8 && LPI == 32) ? 3 : 4)
    k_step_ell(StateView s, CsrView J, StepTables t, int n) {
  constexpr int IPW = 32 / LPI;  // items per warp at a time
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / LPI, sl = lane % LPI;  // the lane's item of the pass, its place in the item
  const float ka = __ldg(t.ka + n), dnext = __ldg(t.dl + n + 1);
  const uint8_t *Fin = s.f_of(n);
  uint8_t *Fout = s.f_of(n + 1);
  const int chunks = s.Cp / (LPI * W);
  const long long n_items = (long long)s.N * chunks;
  const long long n_passes = (n_items + IPW - 1) / IPW;
  const long long stride = (long long)gridDim.x * 8;
  long long pass = (long long)blockIdx.x * 8 + warp;
  if (pass >= n_passes) return;  // whole warp
  // the item of this lane's group in a pass; a group past the last item repeats the pass's first
  // item for its loads and stores nothing
  auto item_of = [&](long long ps, bool &act) {
    const long long it = ps * IPW + sub;
    act = it < n_items;
    return act ? it : ps * IPW;
  };
  bool nact;
  long long nit = item_of(pass, nact);
  int ni = int(nit / chunks), nch = int(nit - (long long)ni * chunks);
  int ncol = 0;
  float nval = 0.f;
  int2 nmeta;
  float nxs[W], nys[W];
  auto fetch = [&](int row, int ch) {
    if (sl < kEllSlots) {
      ncol = __ldg(J.ell_col + size_t(row) * kEllSlots + sl);
      if constexpr (KIND != VAL_PM1) nval = __ldg(J.ell_val + size_t(row) * kEllSlots + sl);
    }
    nmeta = __ldg(reinterpret_cast<const int2 *>(J.ell_meta) + row);
    const size_t off = size_t(row) * s.Cp + ch * LPI * W + sl * W;
#pragma unroll
    for (int q = 0; q < W / 4; ++q) {
      const float4 a = *reinterpret_cast<const float4 *>(s.x + off + 4 * q);
      const float4 b = *reinterpret_cast<const float4 *>(s.y + off + 4 * q);
      nxs[4 * q] = a.x; nxs[4 * q + 1] = a.y; nxs[4 * q + 2] = a.z; nxs[4 * q + 3] = a.w;
      nys[4 * q] = b.x; nys[4 * q + 1] = b.y; nys[4 * q + 2] = b.z; nys[4 * q + 3] = b.w;
    }
  };
  if constexpr (LPI == 32) fetch(ni, nch);
  for (; pass < n_passes; pass += stride) {
    if constexpr (LPI != 32) {
      nit = item_of(pass, nact);
      ni = int(nit / chunks);
      nch = int(nit - (long long)ni * chunks);
      fetch(ni, nch);
    }
    const int i = ni, ch = nch;
    const bool act = nact;
    const int my_col = ncol;
    const float my_w = nval;
    const int deg = act ? nmeta.x : 0, npos = nmeta.y;
    float xs[W], ys[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
      xs[q] = nxs[q];
      ys[q] = nys[q];
    }
    const long long next = pass + stride;
    if (LPI == 32 && next < n_passes) {  // warp-uniform
      nit = item_of(next, nact);
      ni = int(nit / chunks);
      nch = int(nit - (long long)ni * chunks);
      fetch(ni, nch);
    }
    const int c0 = ch * LPI * W + sl * W;
    const uint8_t *Fc = Fin + c0;
    const int src0 = sub * LPI;  // lane holding slot 0 of this group's row
    FVec<W> f[kEllSlots];
#pragma unroll
    for (int e = 0; e < kEllSlots; ++e) {
      const int j = __shfl_sync(0xffffffffu, my_col, src0 + e);
      if (e < deg) f[e].load(Fc + size_t(j) * s.Cp);
      else f[e].zero(KIND == VAL_PM1 ? 0u : kFZero4);
    }
    float G[W];
    if constexpr (KIND == VAL_PM1) {
      uint32_t ap[W / 4], am[W / 4];
#pragma unroll
      for (int q = 0; q < W / 4; ++q) ap[q] = am[q] = 0;
#pragma unroll
      for (int e = 0; e < kEllSlots; ++e) {
        if (e < npos) {
#pragma unroll
          for (int q = 0; q < W / 4; ++q) ap[q] += f[e].w[q];
        } else {
#pragma unroll
          for (int q = 0; q < W / 4; ++q) am[q] += f[e].w[q];
        }
      }
      const int bias = (deg - npos) - npos;  // codes carry f + 1; padding slots hold 0
#pragma unroll
      for (int c = 0; c < W; ++c)
        G[c] = float(int((ap[c / 4] >> (8 * (c % 4))) & 0xffu) - int((am[c / 4] >> (8 * (c % 4))) & 0xffu) + bias);
    } else {
      float g[W];
#pragma unroll
      for (int c = 0; c < W; ++c) g[c] = 0.f;
#pragma unroll
      for (int e = 0; e < kEllSlots; ++e) {
        const float wt = __shfl_sync(0xffffffffu, my_w, src0 + e);
        if (e < deg) {  // the CSR kernel's entries, in its order
          acc_codes<W>(g, wt, f[e].w);
        }
      }
#pragma unroll
      for (int c = 0; c < W; ++c) G[c] = g[c];
    }
    // an idle group takes part in the ring shuffles only (a column past C stores nothing)
    const int cs = act ? c0 : s.C;
    if (P > 2 && s.Pr != P) sb_updateW<P, W, true>(s, t, ka, dnext, n, i, cs, G, __ldg(J.h + i), xs, ys, Fout);
    else sb_updateW<P, W, false>(s, t, ka, dnext, n, i, cs, G, __ldg(J.h + i), xs, ys, Fout);
  }
}

// One wave of resident blocks of kernel fn (cached per kernel).
static unsigned wave_blocks(const void *fn) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
  return unsigned(sms * per_sm);
}

// W = 4 (128-column items) runs as W = 8 on half warps, two items per warp.
template <int P, int KIND, int W>
static cudaError_t launch_ell(const StateView &s, const CsrView &J, const StepTables &t, int n, cudaStream_t st) {
  constexpr bool HALF = W == 4;
  constexpr int WK = HALF ? 8 : W, LPI = HALF ? 16 : 32;
  static const unsigned wave = wave_blocks((const void *)k_step_ell<P, KIND, WK, LPI>);
  const long long passes = (long long)s.N * (s.Cp / (32 * W)) / (HALF ? 2 : 1) + 1;
  const unsigned blocks = unsigned(std::min<long long>(wave, (passes + 7) / 8));
  k_step_ell<P, KIND, WK, LPI><<<blocks, 256, 0, st>>>(s, J, t, n);
  return cudaGetLastError();
}

template <int P, int W>
static cudaError_t launch_pw_ell(const StateView &s, const CsrView &J, const StepTables &t, int n, cudaStream_t st) {
  switch (J.kind) {
    case VAL_PM1: return launch_ell<P, VAL_PM1, W>(s, J, t, n, st);
    case VAL_F32: return launch_ell<P, VAL_F32, W>(s, J, t, n, st);
    default: return launch_ell<P, VAL_BF16, W>(s, J, t, n, st);
  }
}

template <int P, int KIND, int W, bool GS>
static cudaError_t launch_k(const StateView &s, const CsrView &J, const StepTables &t, int n, cudaStream_t st) {
  if constexpr (GS) {
    static const unsigned wave = wave_blocks((const void *)k_step_csr<P, KIND, W, true>);
    const long long items = (long long)s.N * (s.Cp / (32 * W));
    const unsigned blocks = unsigned(std::min<long long>(wave, (items + 7) / 8));
    k_step_csr<P, KIND, W, true><<<blocks, 256, 0, st>>>(s, J, t, n);
  } else {
    const dim3 blocks(unsigned((s.N + 7) / 8), unsigned(s.Cp / (32 * W)));
    k_step_csr<P, KIND, W, false><<<blocks, 256, 0, st>>>(s, J, t, n);
  }
  return cudaGetLastError();
}

template <int P, int W, bool GS>
static cudaError_t launch_pw(const StateView &s, const CsrView &J, const StepTables &t, int n, cudaStream_t st) {
  switch (J.kind) {
    case VAL_PM1: return launch_k<P, VAL_PM1, W, GS>(s, J, t, n, st);
    case VAL_F32: return launch_k<P, VAL_F32, W, GS>(s, J, t, n, st);
    default: return launch_k<P, VAL_BF16, W, GS>(s, J, t, n, st);
  }
}

template <int P>
static cudaError_t launch_p(const StateView &s, const CsrView &J, const StepTables &t, int n, int variant,
                            cudaStream_t st) {
  switch (variant) {
    case 7: return launch_pw_ell<P, 8>(s, J, t, n, st);
    case 6: return launch_pw_ell<P, 4>(s, J, t, n, st);
    case 5: return launch_pw<P, 16, true>(s, J, t, n, st);
    case 4: return launch_pw<P, 8, true>(s, J, t, n, st);
    case 3: return launch_pw<P, 4, true>(s, J, t, n, st);
    case 2: return launch_pw<P, 16, false>(s, J, t, n, st);
    case 1: return launch_pw<P, 8, false>(s, J, t, n, st);
    default: return launch_pw<P, 4, false>(s, J, t, n, st);
  }
}

// Variants 0-2: W = 4, 8, 16 columns per lane, one item per warp; 3-5: the
// same widths with one wave of blocks looping over the items; 6, 7: the ELL
// form (W = 4, 8), when the problem has one (degree <= 8).  W needs Cp to be a
// multiple of 32 W.
int csr_step_variants() { return 8; }

bool csr_step_variant_ok(int variant, int Cp, bool has_ell) {
  if (variant >= 6) return has_ell && Cp % (32 * (4 << (variant - 6))) == 0;
  return Cp % (32 * (4 << (variant % 3))) == 0;
}

cudaError_t launch_step_csr(const StateView &s, const CsrView &J, const StepTables &t, int n, int variant,
                            cudaStream_t st) {
  if (!csr_step_variant_ok(variant, s.Cp, J.ell_col != nullptr)) variant = 0;
  switch (s.P) {
    case 1: return launch_p<1>(s, J, t, n, variant, st);
    case 2: return launch_p<2>(s, J, t, n, variant, st);
    case 4: return launch_p<4>(s, J, t, n, variant, st);
    case 8: return launch_p<8>(s, J, t, n, variant, st);
    case 16: return launch_p<16>(s, J, t, n, variant, st);
    case 32: return launch_p<32>(s, J, t, n, variant, st);
    case 64: return launch_p<64>(s, J, t, n, variant, st);
    case 128: return launch_p<128>(s, J, t, n, variant, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sbqa
