// step_common.cuh -- the per-element part of one SBQA step, shared by the
// sparse and dense step kernels.
//
// One lane owns 4 consecutive columns (replicas) of one spin row i.  Because
// P divides 32 and a warp owns 128 aligned columns, the replica ring of every
// run (k - 1, k + 1 modulo P; periodic imaginary time, Supplement Eq. S3)
// lies inside the warp, so the neighbour positions come from warp shuffles
// and x can be updated in place.
//
// Update of Sec. II A, Eqs. 6-7 (symplectic Euler, momentum first) with the
// wall rule stated after Eq. 3 and the threshold f of Eq. 8 for the next step:
//   y <- y + dt [ -(a0 - a_n)/P x + (c0/P)(G + h) + J_perp (x_{k-1} + x_{k+1}) ]
//   x <- x + dt (a0/P) y
//   |x| > 1  ->  x = sign(x), y = 0
//   F_next = 0 if |x| <= Delta_{n+1} else sign(x)
#pragma once
#include "internal.h"

namespace sbqa {

// Neighbour positions of the lane's 4 columns.  c4 = first column (multiple
// of 4); xs = the lane's positions.  All shuffle sources stay inside the warp
// because lane 0 starts a run and lane 31 ends one.
template <int P>
__device__ __forceinline__ void ring_neighbours(const float xs[4], int c4, float xm[4],
                                                float xp[4]) {
  const int lane = threadIdx.x & 31;
  if constexpr (P == 1) {
#pragma unroll
    for (int j = 0; j < 4; ++j) { xm[j] = xs[j]; xp[j] = xs[j]; }
  } else if constexpr (P == 2) {
    xm[0] = xp[0] = xs[1];
    xm[1] = xp[1] = xs[0];
    xm[2] = xp[2] = xs[3];
    xm[3] = xp[3] = xs[2];
  } else {
    const int k0 = c4 % P;        // replica index of the lane's first column
    const int k3 = k0 + 3;        // and of its last column (same run)
    const int src_l = (k0 == 0) ? lane + P / 4 - 1 : lane - 1;
    const int src_r = (k3 == P - 1) ? lane - P / 4 + 1 : lane + 1;
    const float left = __shfl_sync(0xffffffffu, xs[3], src_l);
    const float right = __shfl_sync(0xffffffffu, xs[0], src_r);
    xm[0] = left;  xp[0] = xs[1];
    xm[1] = xs[0]; xp[1] = xs[2];
    xm[2] = xs[1]; xp[2] = xs[3];
    xm[3] = xs[2]; xp[3] = right;
  }
}

__device__ __forceinline__ int8_t thresh(float x, float delta) {
  return fabsf(x) > delta ? (x > 0.f ? int8_t(1) : int8_t(-1)) : int8_t(0);
}

__device__ __forceinline__ uint32_t pack4(int8_t a, int8_t b, int8_t c, int8_t d) {
  return uint32_t(uint8_t(a)) | (uint32_t(uint8_t(b)) << 8) | (uint32_t(uint8_t(c)) << 16) |
         (uint32_t(uint8_t(d)) << 24);
}

// Applies the step to the lane's 4 columns of row i.  G = coupling sums,
// hi = h_i, xv / yv = x, y of (i, c4..c4+3) loaded by the caller (so the
// loads can be issued before the coupling product).  Writes x, y, F_next.
template <int P>
__device__ __forceinline__ void sb_update4(const StateView &s, const StepTables &t, int n,
                                           int i, int c4, const float G[4], float hi,
                                           float4 xv, float4 yv, int8_t *Fout) {
  const size_t off = size_t(i) * s.Cp + c4;
  float xs[4] = {xv.x, xv.y, xv.z, xv.w};
  float ys[4] = {yv.x, yv.y, yv.z, yv.w};
  float xm[4], xp[4];
  ring_neighbours<P>(xs, c4, xm, xp);  // all lanes take part (shuffles)
  if (c4 >= s.C) return;               // padding columns past R * P
  const float ka = t.ka[n];
  const float dnext = t.dl[n + 1];
  const float *kjn = t.kj + size_t(n) * t.R;
  int8_t f[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    f[j] = 0;
    if (c4 + j >= s.C) continue;  // ragged tail when P < 4
    const int r = (c4 + j) / P;
    const float kj = kjn[r];
    float yn = fmaf(t.kc, G[j] + hi, ys[j]);
    yn = fmaf(-ka, xs[j], yn);
    yn = fmaf(kj, xm[j] + xp[j], yn);
    float xn = fmaf(t.kx, yn, xs[j]);
    if (fabsf(xn) > 1.f) {
      xn = copysignf(1.f, xn);
      yn = 0.f;
    }
    xs[j] = xn;
    ys[j] = yn;
    f[j] = thresh(xn, dnext);
  }
  *reinterpret_cast<float4 *>(s.x + off) = make_float4(xs[0], xs[1], xs[2], xs[3]);
  *reinterpret_cast<float4 *>(s.y + off) = make_float4(ys[0], ys[1], ys[2], ys[3]);
  *reinterpret_cast<uint32_t *>(Fout + off) = pack4(f[0], f[1], f[2], f[3]);
}

template <int P>
__device__ __forceinline__ void sb_update4(const StateView &s, const StepTables &t, int n,
                                           int i, int c4, const float G[4], float hi, int8_t *Fout) {
  const size_t off = size_t(i) * s.Cp + c4;
  const float4 xv = *reinterpret_cast<const float4 *>(s.x + off);
  const float4 yv = *reinterpret_cast<const float4 *>(s.y + off);
  sb_update4<P>(s, t, n, i, c4, G, hi, xv, yv, Fout);
}

__device__ __forceinline__ float sbyte(uint32_t w, int j) {
  return float(int8_t((w >> (8 * j)) & 0xffu));
}

}  // namespace sbqa
