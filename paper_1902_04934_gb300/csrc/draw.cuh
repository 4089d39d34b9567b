// Monte Carlo draws of the extrinsic parameters (Eq. (lnLmarg)): sample i of a point's round
// from its Philox stream, under the prior (optionally stratified), the adapted histograms, or
// the learned proposal.  Shared by the cell kernel and the sample export, which re-draws the
// samples of a round from their indices.
#pragma once
#include <cmath>

#include "rift_device.cuh"
#include "rift_internal.h"

namespace {

// Piecewise-constant inverse CDF of one adapted coordinate at a double-float uniform U in
// (0, 1): returns the fraction of the range (double-float) and the bin, the largest b with
// cdf[b] <= U (exact comparison: cdf values are float32, U = hi + lo with |lo| <= ulp(hi)/2).
__device__ __forceinline__ df inv_cdf_df(const float *cdf, int nb, df U, int &b) {
  int lo = 0, hi = nb;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    const float c = cdf[mid];
    if (c < U.hi || (c == U.hi && U.lo >= 0.f)) lo = mid; else hi = mid;
  }
  b = lo;
  const float c0 = cdf[lo], c1 = cdf[lo + 1];
  const df num = two_sum(U.hi, -c0);
  const df den = two_sum(c1, -c0);
  const float f = __fdiv_rn(num.hi + (num.lo + U.lo), den.hi + den.lo);
  const df bf = two_sum((float)b, f);
  const float fnb = (float)nb;
  const float qh = __fdiv_rn(bf.hi, fnb);
  const float r = __fmaf_rn(-qh, fnb, bf.hi);
  const float ql = __fdiv_rn(r + bf.lo, fnb);
  return fast_two_sum(qh, ql);
}

struct Drawn {
  df x0, x1, x2;   // fractions of the ra, sin dec, t ranges
  float u_psi;     // 2 psi = 2 pi u_psi
  float u_phi;     // phi = 2 pi u_phi
  float c_frac;    // (1 + cos incl) / 2
  float dist;      // D (Mpc)
  float xd;        // D_ref / D
  float lpq;       // ln p - ln q (+ stratification weight)
  uint32_t bins;   // adapted bins, 8 bits each
};

// cos dec of a draw from its sin dec fraction x1 = (1 + sin dec) / 2 (double-float):
// 2 sqrt(x1 (1 - x1)), with 1 - x1 formed from both words of x1.  Near the north pole, where
// 1 - x1 ~ (pi/2 - dec)^2 / 4 is tiny, the high word alone would leave 1 - x1 with only a few
// correct bits (a relative error in cos dec of several per cent within 1e-3 rad of the pole).
__device__ __forceinline__ float cos_dec_of(df x1) {
  return 2.f * sqrtf(x1.hi * __fsub_rn(__fsub_rn(1.f, x1.hi), x1.lo));
}

// Sample i (index in the point's round) of cell `cell`: Philox uniforms, stratified
// (ra, sin dec, t) uniforms U_d = (c_d + u_d) / S_d (exact: S_d is a power of two),
// prior or tabulated proposal.
__device__ __forceinline__ Drawn draw_cell_sample(unsigned long long seed, const RoundPt &R, uint32_t i,
                                                  uint32_t cell, const float *tab, const float *lnw, float dref,
                                                  float d_lo3, float d_span3) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint4 a = philox4x32_10(make_uint4(i, R.round, 0u, R.point_id), key);
  const uint4 b = philox4x32_10(make_uint4(i, R.round, 1u, R.point_id), key);
  const uint32_t c0 = cell & ((1u << R.ls0) - 1u);
  const uint32_t c1 = (cell >> R.ls0) & ((1u << R.ls1) - 1u);
  const uint32_t c2 = cell >> (R.ls0 + R.ls1);
  df U0 = two_sum((float)c0, bits_to_u(a.x));
  df U1 = two_sum((float)c1, bits_to_u(a.y));
  df U2 = two_sum((float)c2, bits_to_u(a.z));
  const float s0 = __int_as_float((127 - (int)R.ls0) << 23);   // 2^-ls
  const float s1 = __int_as_float((127 - (int)R.ls1) << 23);
  const float s2 = __int_as_float((127 - (int)R.ls2) << 23);
  U0 = df{U0.hi * s0, U0.lo * s0};
  U1 = df{U1.hi * s1, U1.lo * s1};
  U2 = df{U2.hi * s2, U2.lo * s2};
  Drawn d;
  d.u_psi = bits_to_u(a.w);
  d.u_phi = bits_to_u(b.x);
  d.c_frac = bits_to_u(b.y);
  const float D3 = fmaf(bits_to_u(b.z), d_span3, d_lo3);
  d.dist = cbrtf(D3);
  d.xd = dref * rcbrtf(D3);
  d.lpq = (cell < R.rem) ? R.lcorr0 : R.lcorr1;
  if (R.proposal == 0) {
    d.x0 = U0; d.x1 = U1; d.x2 = U2;
    d.bins = 0u;
  } else {
    const int nb = R.nb;
    int b0, b1, b2;
    d.x0 = inv_cdf_df(tab, nb, U0, b0);
    d.x1 = inv_cdf_df(tab + (nb + 1), nb, U1, b1);
    d.x2 = inv_cdf_df(tab + 2 * (nb + 1), nb, U2, b2);
    d.lpq += lnw[b0] + lnw[nb + b1] + lnw[2 * nb + b2];
    d.bins = (uint32_t)b0 | ((uint32_t)b1 << 8) | ((uint32_t)b2 << 16);
  }
  return d;
}

// Sample i from the learned proposal G (layout RIFT_GMM_FLOATS): Box-Muller normals from
// (u0,u1), (u2,u3), (u4,u5); component = first j with u6 < cumulative pi_j; u7 < 0.9 takes the
// network, otherwise the prior transforms of u0..u4; u8 -> psi, u9 -> phi.  ln q is the
// defensive mixture 0.9 q_MDN + 0.1 p5 with the logit change of variables.
template <int TM>
__device__ __forceinline__ Drawn draw_learned(unsigned long long seed, const RoundPt &R, uint32_t i, const float *G,
                                              float dref, float d_lo3, float d_span3) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint4 a = philox4x32_10(make_uint4(i, R.round, 0u, R.point_id), key);
  const uint4 b = philox4x32_10(make_uint4(i, R.round, 1u, R.point_id), key);
  const uint4 c = philox4x32_10(make_uint4(i, R.round, 2u, R.point_id), key);
  const float u0 = bits_to_u(a.x), u1 = bits_to_u(a.y), u2 = bits_to_u(a.z), u3 = bits_to_u(a.w);
  const float u4 = bits_to_u(b.x), u5 = bits_to_u(b.y), u6 = bits_to_u(b.z), u7 = bits_to_u(b.w);
  const float lnDlo = G[138], lnDspan = G[139];
  float x[5], z[5];
  if (u7 < 0.9f) {
    float n[6];
    const float uu[6] = {u0, u1, u2, u3, u4, u5};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float r = sqrtf(-2.f * logf(uu[2 * q]));
      float sn, cs;
      sincospif(2.f * uu[2 * q + 1], &sn, &cs);
      n[2 * q] = r * cs;
      n[2 * q + 1] = r * sn;
    }
    int j = 7;
#pragma unroll
    for (int q = 6; q >= 0; --q) if (u6 < G[8 + q]) j = q;
#pragma unroll
    for (int dd = 0; dd < 5; ++dd) {
      z[dd] = fmaf(expf(G[56 + 5 * j + dd]), n[dd], G[16 + 5 * j + dd]);
      x[dd] = 1.f / (1.f + expf(-z[dd]));
    }
  } else {
    const float D = cbrtf(fmaf(u4, d_span3, d_lo3));
    x[0] = u0; x[1] = u1; x[2] = u2; x[3] = u3;
    x[4] = fminf(fmaxf((logf(D) - lnDlo) / lnDspan, 1e-7f), 1.f - 6e-8f);
#pragma unroll
    for (int dd = 0; dd < 5; ++dd) z[dd] = logf(x[dd]) - log1pf(-x[dd]);
  }
  // ln q_MDN: mixture in z plus the logit Jacobian, ln x + ln(1 - x) = -softplus(-z) - softplus(z)
  float comp[8];
  float mx = -INFINITY;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float acc = G[j];
#pragma unroll
    for (int dd = 0; dd < 5; ++dd) {
      if (TM && dd == 2) continue;   // time integrated by quadrature: the diagonal mixture drops it exactly
      const float t = (z[dd] - G[16 + 5 * j + dd]) * G[96 + 5 * j + dd];
      acc -= 0.5f * t * t + G[56 + 5 * j + dd] + 0.91893853320467274f;
    }
    comp[j] = acc;
    mx = fmaxf(mx, acc);
  }
  float se = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) se += expf(comp[j] - mx);
  float jac = G[136];
#pragma unroll
  for (int dd = 0; dd < 5; ++dd) {
    if (TM && dd == 2) continue;
    const float az = fabsf(z[dd]);
    jac -= az + 2.f * log1pf(expf(-az));   // softplus(z) + softplus(-z) = |z| + 2 log(1 + e^{-|z|})
  }
  const float lq_mdn = mx + logf(se) - jac;
  const float lnD = fmaf(x[4], lnDspan, lnDlo);
  const float lp5 = G[137] + 3.f * lnD;
  const float A = -0.10536051565782628f + lq_mdn;   // ln 0.9
  const float B = -2.3025850929940457f + lp5;       // ln 0.1
  const float M = fmaxf(A, B);
  const float lnq = M + logf(expf(A - M) + expf(B - M));
  Drawn d;
  d.x0 = df{x[0], 0.f};
  d.x1 = df{x[1], 0.f};
  d.x2 = df{x[2], 0.f};
  d.c_frac = x[3];
  d.dist = expf(lnD);
  d.xd = dref * expf(-lnD);
  d.u_psi = bits_to_u(c.x);
  d.u_phi = bits_to_u(c.y);
  d.lpq = lp5 - lnq;
  d.bins = 0u;
  return d;
}

// LEARNED: the launch's points use learned proposals; each point's round says which proposal it
// draws from (R.proposal 2, or 1 after a fallback to the adaptive tables).
template <int LEARNED, int TM = 0>
__device__ __forceinline__ Drawn draw_any(unsigned long long seed, const RoundPt &R, uint32_t i, uint32_t cell,
                                          const float *tab, const float *lnw, const float *G, float dref, float d_lo3,
                                          float d_span3) {
  if (LEARNED && R.proposal == 2) return draw_learned<TM>(seed, R, i, G, dref, d_lo3, d_span3);
  return draw_cell_sample(seed, R, i, cell, tab, lnw, dref, d_lo3, d_span3);
}

}  // namespace
