// step_common.cuh -- the per-element part of one SBQA step, shared by the
// sparse and dense step kernels.
//
// One lane owns 4 (or W) consecutive columns of one spin row i.  A run of Pr
// replicas occupies P columns, P the power of two >= Pr (up to 128), and a
// warp owns 128 (32 W) aligned columns, so the replica ring of every run
// (k - 1, k + 1 modulo Pr; periodic imaginary time, Supplement Eq. S3) lies
// inside the warp: the neighbour positions come from registers and warp
// shuffles, and x can be updated in place.
//
// Update of Sec. II A, Eqs. 6-7 (symplectic Euler, momentum first) with the
// wall rule stated after Eq. 3 and the threshold f of Eq. 8 for the next step:
//   y <- y + dt [ -(a0 - a_n)/P x + (c0/P)(G + h) + J_perp (x_{k-1} + x_{k+1}) ]
//   x <- x + dt (a0/P) y
//   |x| > 1  ->  x = sign(x), y = 0
//   F_next = 0 if |x| <= Delta_{n+1} else sign(x)   (stored as the code f + 1)
#pragma once
#include "internal.h"

namespace sbqa {

// Ring neighbours x_{k-1}, x_{k+1} (k modulo Pr, periodic imaginary time) of
// the W consecutive columns c0 .. c0 + W - 1 of one lane.  Runs occupy P
// columns (a power of two dividing the warp's 32 W columns, so a run never
// leaves the warp); the first Pr of them are the run's replicas (P / 2 < Pr
// <= P) and the rest padding that no replica reads.  P <= W: whole runs
// inside the lane; P > W: a run spans P / W lanes and the neighbours across
// lanes come by shuffle.  GEN = false takes Pr = P (no padding); GEN = true
// handles any Pr without branches, and gives the same values when Pr = P.
// Every lane takes part (Pr is the same in the whole warp).
template <int P, int W, bool GEN = true>
__device__ __forceinline__ void ring_nb(const float (&xs)[W], int Pr, float (&xm)[W], float (&xp)[W]) {
  if constexpr (P <= 2 || !GEN) {
    Pr = P;  // a run of 1 or 2 columns has no padding (P = run_width(Pr))
  }
  if constexpr (P <= W) {
#pragma unroll
    for (int base = 0; base < W; base += P) {
      // replica Pr - 1 of the run (Pr - 1 >= P / 2 when P >= 2)
      float last = xs[base + P - 1];
      if constexpr (P > 2 && GEN) {
#pragma unroll
        for (int k = P / 2; k < P - 1; ++k) last = (k == Pr - 1) ? xs[base + k] : last;
      }
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int j = base + k;
        xm[j] = k == 0 ? last : xs[j - 1];
        xp[j] = (k == P - 1 || k == Pr - 1) ? xs[base] : xs[j + 1];
      }
    }
  } else {
    constexpr int L = P / W;  // lanes per run
    const int lane = threadIdx.x & 31, part = lane % L, base_lane = lane - part;
    const float left = __shfl_sync(0xffffffffu, xs[W - 1], part == 0 ? lane : lane - 1);
    const float right = __shfl_sync(0xffffffffu, xs[0], part == L - 1 ? lane : lane + 1);
    // replica Pr - 1 sits in lane base_lane + (Pr - 1) / W, slot (Pr - 1) % W
    float mine = xs[W - 1];
    if constexpr (GEN) {
      const int slot = (Pr - 1) % W;
#pragma unroll
      for (int u = 0; u < W - 1; ++u) mine = (u == slot) ? xs[u] : mine;
    }
    const float last = __shfl_sync(0xffffffffu, mine, base_lane + (Pr - 1) / W);
    const float first = __shfl_sync(0xffffffffu, xs[0], base_lane);
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const int k = part * W + j;
      xm[j] = j == 0 ? (part == 0 ? last : left) : xs[j - 1];
      xp[j] = k == Pr - 1 ? first : (j == W - 1 ? right : xs[j + 1]);
    }
  }
}

// Neighbour positions of the lane's 4 columns (c4 = first column, a multiple
// of 4; a warp owns 128 aligned columns, so with P <= 128 every run lies
// inside the warp).
template <int P, bool GEN = true>
__device__ __forceinline__ void ring_neighbours(const float (&xs)[4], int Pr, float (&xm)[4], float (&xp)[4]) {
  ring_nb<P, 4, GEN>(xs, Pr, xm, xp);
}

__device__ __forceinline__ int8_t thresh(float x, float delta) {
  return fabsf(x) > delta ? (x > 0.f ? int8_t(1) : int8_t(-1)) : int8_t(0);
}

// F buffers hold f(x) + 1 in one byte: 0 = -1, 1 = 0, 2 = +1 (padding = 1).
// The offset keeps every byte non-negative, so four of them can be summed in
// one 32-bit add without carries between bytes (up to 127 terms).
constexpr uint8_t kFZero = 1;
constexpr uint32_t kFZero4 = 0x01010101u;

__device__ __forceinline__ uint32_t fcode(float x, float delta) {
  return fabsf(x) > delta ? (x > 0.f ? 2u : 0u) : 1u;
}

__device__ __forceinline__ uint32_t pack4(int8_t a, int8_t b, int8_t c, int8_t d) {
  return uint32_t(uint8_t(a)) | (uint32_t(uint8_t(b)) << 8) | (uint32_t(uint8_t(c)) << 16) |
         (uint32_t(uint8_t(d)) << 24);
}

// Applies the step to the lane's 4 columns of row i.  G = coupling sums,
// hi = h_i, xv / yv = x, y of (i, c4..c4+3) loaded by the caller (so the
// loads can be issued before the coupling product).  Writes x, y and the f
// codes of the next step.  The FP32 arithmetic runs on column pairs with the
// packed Blackwell instructions (each lane of __ffma2_rn / __fadd2_rn is an
// ordinary round-to-nearest fma / add, so results equal the scalar form).
template <int P, bool GEN = true>
__device__ __forceinline__ void sb_update4(const StateView &s, const StepTables &t, int n,
                                           int i, int c4, const float G[4], float hi,
                                           float4 xv, float4 yv, uint8_t *Fout) {
  const size_t off = size_t(i) * s.Cp + c4;
  float xs[4] = {xv.x, xv.y, xv.z, xv.w};
  float ys[4] = {yv.x, yv.y, yv.z, yv.w};
  float xm[4], xp[4];
  ring_neighbours<P, GEN>(xs, s.Pr, xm, xp);  // all lanes take part (shuffles)
  if (c4 >= s.C) return;                 // padding columns past R * P
  const float ka = t.ka[n];
  const float dnext = t.dl[n + 1];
  const float *kjn = t.kj + size_t(n) * t.R;
  float kj[4];
  if constexpr (P >= 4) {
    const float k = kjn[c4 / P];
    kj[0] = kj[1] = kj[2] = kj[3] = k;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) kj[j] = (c4 + j < s.C) ? kjn[(c4 + j) / P] : 0.f;
  }
  const float2 kc2 = make_float2(t.kc, t.kc), mka2 = make_float2(-ka, -ka);
  const float2 kx2 = make_float2(t.kx, t.kx), h2 = make_float2(hi, hi);
  float xo[4], yo[4];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int a = 2 * q, b = 2 * q + 1;
    const float2 x2 = make_float2(xs[a], xs[b]);
    float2 y2 = make_float2(ys[a], ys[b]);
    y2 = __ffma2_rn(kc2, __fadd2_rn(make_float2(G[a], G[b]), h2), y2);
    y2 = __ffma2_rn(mka2, x2, y2);
    y2 = __ffma2_rn(make_float2(kj[a], kj[b]), __fadd2_rn(make_float2(xm[a], xm[b]), make_float2(xp[a], xp[b])), y2);
    const float2 xn2 = __ffma2_rn(kx2, y2, x2);
    xo[a] = xn2.x; xo[b] = xn2.y;
    yo[a] = y2.x; yo[b] = y2.y;
  }
  uint32_t code = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    // wall: |x| > 1 exactly when clamping to [-1, 1] changes x
    const float xc = fminf(fmaxf(xo[j], -1.f), 1.f);
    float yn = (xc != xo[j]) ? 0.f : yo[j];
    float xn = xc;
    // code f + 1: 2 if x > Delta, 0 if x < -Delta, else 1
    uint32_t cj = 1u + uint32_t(xn > dnext) - uint32_t(xn < -dnext);
    if (P < 4 && c4 + j >= s.C) {  // ragged tail: leave the padding column alone
      xn = xs[j];
      yn = ys[j];
      cj = kFZero;
    }
    xo[j] = xn;
    yo[j] = yn;
    code |= cj << (8 * j);
  }
  *reinterpret_cast<float4 *>(s.x + off) = make_float4(xo[0], xo[1], xo[2], xo[3]);
  *reinterpret_cast<float4 *>(s.y + off) = make_float4(yo[0], yo[1], yo[2], yo[3]);
  *reinterpret_cast<uint32_t *>(Fout + off) = code;
}

template <int P>
__device__ __forceinline__ void sb_update4(const StateView &s, const StepTables &t, int n,
                                           int i, int c4, const float G[4], float hi, uint8_t *Fout) {
  const size_t off = size_t(i) * s.Cp + c4;
  const float4 xv = *reinterpret_cast<const float4 *>(s.x + off);
  const float4 yv = *reinterpret_cast<const float4 *>(s.y + off);
  sb_update4<P>(s, t, n, i, c4, G, hi, xv, yv, Fout);
}

// Per-step, per-lane constants of the update (independent of the spin row),
// loaded once before a warp's loop over rows.
template <int P>
struct LaneConsts {
  float2 kc2, mka2, kx2;
  float kj[4];
  float dnext;
  int Pr;            // replicas of a run
  bool active;       // the lane's first column is inside R * P

  __device__ __forceinline__ void load(const StateView &s, const StepTables &t, int n, int c4) {
    Pr = s.Pr;
    const float ka = __ldg(t.ka + n);
    dnext = __ldg(t.dl + n + 1);
    kc2 = make_float2(t.kc, t.kc);
    mka2 = make_float2(-ka, -ka);
    kx2 = make_float2(t.kx, t.kx);
    const float *kjn = t.kj + size_t(n) * t.R;
    active = c4 < s.C;
    if constexpr (P >= 4) {
      const float k = active ? __ldg(kjn + c4 / P) : 0.f;
      kj[0] = kj[1] = kj[2] = kj[3] = k;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) kj[j] = (c4 + j < s.C) ? __ldg(kjn + (c4 + j) / P) : 0.f;
    }
  }
};

// sb_update4 with the per-lane constants already loaded (same arithmetic).
template <int P, bool GEN = true>
__device__ __forceinline__ void sb_update4c(const StateView &s, const LaneConsts<P> &L, int i, int c4,
                                            const float G[4], float hi, float4 xv, float4 yv, uint8_t *Fout) {
  const size_t off = size_t(i) * s.Cp + c4;
  float xs[4] = {xv.x, xv.y, xv.z, xv.w};
  float ys[4] = {yv.x, yv.y, yv.z, yv.w};
  float xm[4], xp[4];
  if constexpr (P == 1) {
#pragma unroll
    for (int j = 0; j < 4; ++j) { xm[j] = xs[j]; xp[j] = xs[j]; }
  } else if constexpr (P == 2) {
    xm[0] = xp[0] = xs[1]; xm[1] = xp[1] = xs[0];
    xm[2] = xp[2] = xs[3]; xm[3] = xp[3] = xs[2];
  } else {
    ring_nb<P, 4, GEN>(xs, L.Pr, xm, xp);
  }
  if (!L.active) return;
  const float2 h2 = make_float2(hi, hi);
  float xo[4], yo[4];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int a = 2 * q, b = 2 * q + 1;
    const float2 x2 = make_float2(xs[a], xs[b]);
    float2 y2 = make_float2(ys[a], ys[b]);
    y2 = __ffma2_rn(L.kc2, __fadd2_rn(make_float2(G[a], G[b]), h2), y2);
    y2 = __ffma2_rn(L.mka2, x2, y2);
    y2 = __ffma2_rn(make_float2(L.kj[a], L.kj[b]), __fadd2_rn(make_float2(xm[a], xm[b]), make_float2(xp[a], xp[b])), y2);
    const float2 xn2 = __ffma2_rn(L.kx2, y2, x2);
    xo[a] = xn2.x; xo[b] = xn2.y;
    yo[a] = y2.x; yo[b] = y2.y;
  }
  uint32_t code = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float xc = fminf(fmaxf(xo[j], -1.f), 1.f);  // wall: clamping changes x iff |x| > 1
    float yn = (xc != xo[j]) ? 0.f : yo[j];
    float xn = xc;
    uint32_t cj = 1u + uint32_t(xn > L.dnext) - uint32_t(xn < -L.dnext);
    if (P < 4 && c4 + j >= s.C) {
      xn = xs[j];
      yn = ys[j];
      cj = kFZero;
    }
    xo[j] = xn;
    yo[j] = yn;
    code |= cj << (8 * j);
  }
  *reinterpret_cast<float4 *>(s.x + off) = make_float4(xo[0], xo[1], xo[2], xo[3]);
  *reinterpret_cast<float4 *>(s.y + off) = make_float4(yo[0], yo[1], yo[2], yo[3]);
  *reinterpret_cast<uint32_t *>(Fout + off) = code;
}

// Generalisation of sb_update4c to W consecutive columns per lane (W = 4,
// 8 or 16; W >= P or P divides W).  Ring neighbours inside the lane's
// columns are registers; across lanes (P > W) they come by shuffle from the
// neighbouring lane of the same run.  Same arithmetic as sb_update4.
template <int P, int W, bool GEN = true>
__device__ __forceinline__ void sb_updateW(const StateView &s, const StepTables &t, float ka, float dnext, int n,
                                           int i, int c0, const float (&G)[W], float hi, float (&xs)[W],
                                           float (&ys)[W], uint8_t *Fout) {
  float xm[W], xp[W];
  ring_nb<P, W, GEN>(xs, s.Pr, xm, xp);  // all lanes take part (shuffles)
  if (c0 >= s.C) return;
  const float *kjn = t.kj + size_t(n) * t.R;
  const float2 kc2 = make_float2(t.kc, t.kc), mka2 = make_float2(-ka, -ka), kx2 = make_float2(t.kx, t.kx);
  const float2 h2 = make_float2(hi, hi);
  uint32_t code[W / 4];
#pragma unroll
  for (int q = 0; q < W / 4; ++q) code[q] = 0;
  // dt * J_perp of the run of each column (one load per run in the lane)
  float kjv[W];
  if constexpr (P >= W) {
    const float k = (c0 < s.C) ? __ldg(kjn + c0 / P) : 0.f;
#pragma unroll
    for (int j = 0; j < W; ++j) kjv[j] = k;
  } else {
#pragma unroll
    for (int r = 0; r < W / P; ++r) {
      const float k = (c0 + r * P < s.C) ? __ldg(kjn + c0 / P + r) : 0.f;
#pragma unroll
      for (int u = 0; u < P; ++u) kjv[r * P + u] = k;
    }
  }
#pragma unroll
  for (int pr = 0; pr < W / 2; ++pr) {
    const int a = 2 * pr, b = a + 1;
    const float kja = kjv[a], kjb = kjv[b];
    const float2 x2 = make_float2(xs[a], xs[b]);
    float2 y2 = make_float2(ys[a], ys[b]);
    y2 = __ffma2_rn(kc2, __fadd2_rn(make_float2(G[a], G[b]), h2), y2);
    y2 = __ffma2_rn(mka2, x2, y2);
    y2 = __ffma2_rn(make_float2(kja, kjb), __fadd2_rn(make_float2(xm[a], xm[b]), make_float2(xp[a], xp[b])), y2);
    const float2 xn2 = __ffma2_rn(kx2, y2, x2);
    const float xo[2] = {xn2.x, xn2.y}, yo[2] = {y2.x, y2.y};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int j = a + u;
      const float xc = fminf(fmaxf(xo[u], -1.f), 1.f);  // wall
      const float yn = (xc != xo[u]) ? 0.f : yo[u];
      uint32_t cj = 1u + uint32_t(xc > dnext) - uint32_t(xc < -dnext);
      if (c0 + j >= s.C) {  // ragged tail (P < 4): padding column untouched
        cj = kFZero;
      } else {
        xs[j] = xc;
        ys[j] = yn;
      }
      code[j / 4] |= cj << (8 * (j % 4));
    }
  }
  const size_t off = size_t(i) * s.Cp + c0;
#pragma unroll
  for (int q = 0; q < W / 4; ++q) {
    *reinterpret_cast<float4 *>(s.x + off + 4 * q) = make_float4(xs[4 * q], xs[4 * q + 1], xs[4 * q + 2], xs[4 * q + 3]);
    *reinterpret_cast<float4 *>(s.y + off + 4 * q) = make_float4(ys[4 * q], ys[4 * q + 1], ys[4 * q + 2], ys[4 * q + 3]);
  }
  if constexpr (W == 4) {
    *reinterpret_cast<uint32_t *>(Fout + off) = code[0];
  } else if constexpr (W == 8) {
    *reinterpret_cast<uint2 *>(Fout + off) = make_uint2(code[0], code[1]);
  } else {
    *reinterpret_cast<uint4 *>(Fout + off) = make_uint4(code[0], code[1], code[2], code[3]);
  }
}

// Value of f encoded in byte q of a packed word of f codes.
__device__ __forceinline__ float fdec(uint32_t w, int q) {
  return float(int((w >> (8 * q)) & 0xffu) - 1);
}

// g[c] += w * f_c for the W f codes of one neighbour (W / 4 packed words),
// two columns per packed FMA.  One byte permute puts code byte b into the low
// mantissa bits of 2^23 (0x4B0000cc = 2^23 + code, exact), one packed add of
// -(2^23 + 1) gives f = code - 1 in {-1, 0, 1} exactly, and each lane of
// __ffma2_rn is the ordinary round-to-nearest fma: the sums equal
// fmaf(w, fdec(...), g) term by term, in the same order.
template <int W>
__device__ __forceinline__ void acc_codes(float (&g)[W], float w, const uint32_t *cw) {
  const float2 w2 = make_float2(w, w);
  const float2 off = make_float2(-8388609.f, -8388609.f);
#pragma unroll
  for (int q = 0; q < W / 4; ++q) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t m0 = __byte_perm(cw[q], 0x4B000000u, 0x7540u | uint32_t(2 * h));
      const uint32_t m1 = __byte_perm(cw[q], 0x4B000000u, 0x7540u | uint32_t(2 * h + 1));
      const float2 f2 = __fadd2_rn(make_float2(__uint_as_float(m0), __uint_as_float(m1)), off);
      const int c = 4 * q + 2 * h;
      const float2 r = __ffma2_rn(w2, f2, make_float2(g[c], g[c + 1]));
      g[c] = r.x;
      g[c + 1] = r.y;
    }
  }
}

// sb_update4 with f(x) = x: same momentum, position and wall arithmetic,
// writes the new x into the f buffer of the next step.
template <int P>
__device__ __forceinline__ void sb_update4_bsb(const StateView &s, const StepTables &t, int n, int i, int c4,
                                               const float G[4], float hi, float4 xv, float4 yv, float *Fout) {
  const size_t off = size_t(i) * s.Cp + c4;
  float xs[4] = {xv.x, xv.y, xv.z, xv.w};
  float ys[4] = {yv.x, yv.y, yv.z, yv.w};
  float xm[4], xp[4];
  ring_neighbours<P>(xs, s.Pr, xm, xp);  // all lanes take part (shuffles)
  if (c4 >= s.C) return;                 // padding columns past R * P
  const float ka = __ldg(t.ka + n);
  const float *kjn = t.kj + size_t(n) * t.R;
  float kj[4];
  if constexpr (P >= 4) {
    const float k = __ldg(kjn + c4 / P);
    kj[0] = kj[1] = kj[2] = kj[3] = k;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) kj[j] = (c4 + j < s.C) ? __ldg(kjn + (c4 + j) / P) : 0.f;
  }
  const float2 kc2 = make_float2(t.kc, t.kc), mka2 = make_float2(-ka, -ka);
  const float2 kx2 = make_float2(t.kx, t.kx), h2 = make_float2(hi, hi);
  float xo[4], yo[4];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int a = 2 * q, b = 2 * q + 1;
    const float2 x2 = make_float2(xs[a], xs[b]);
    float2 y2 = make_float2(ys[a], ys[b]);
    y2 = __ffma2_rn(kc2, __fadd2_rn(make_float2(G[a], G[b]), h2), y2);
    y2 = __ffma2_rn(mka2, x2, y2);
    y2 = __ffma2_rn(make_float2(kj[a], kj[b]), __fadd2_rn(make_float2(xm[a], xm[b]), make_float2(xp[a], xp[b])), y2);
    const float2 xn2 = __ffma2_rn(kx2, y2, x2);
    xo[a] = xn2.x; xo[b] = xn2.y;
    yo[a] = y2.x; yo[b] = y2.y;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float xc = fminf(fmaxf(xo[j], -1.f), 1.f);  // wall: clamping changes x iff |x| > 1
    float yn = (xc != xo[j]) ? 0.f : yo[j];
    float xn = xc;
    if (P < 4 && c4 + j >= s.C) {  // ragged tail: leave the padding column alone
      xn = xs[j];
      yn = ys[j];
    }
    xo[j] = xn;
    yo[j] = yn;
  }
  const float4 xnew = make_float4(xo[0], xo[1], xo[2], xo[3]);
  *reinterpret_cast<float4 *>(s.x + off) = xnew;
  *reinterpret_cast<float4 *>(s.y + off) = make_float4(yo[0], yo[1], yo[2], yo[3]);
  *reinterpret_cast<float4 *>(Fout + off) = xnew;
}

}  // namespace sbqa
