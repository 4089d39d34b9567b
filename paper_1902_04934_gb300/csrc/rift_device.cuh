// Device-side data layout and per-sample arithmetic of the extrinsic likelihood.
//
// Eq. (def:lnL:Decomposed), evaluated per sample in FP32 with the time index,
// the sidereal angle offset and the time of flight kept in double-float (pairs of
// FP32, error-free transformations), which the sample-to-sample precision needs:
// Q oscillates at ~100 Hz, so 1e-9 s of time error is ~1e-4 in lnL at SNR 30.
#pragma once
#include <cstdint>
#include <type_traits>
#include <utility>
#include <cuda_runtime.h>

#define RIFT_MAXK 4
#define RIFT_MAXM 21
#define RIFT_MAXPAIR (RIFT_MAXM * (RIFT_MAXM + 1) / 2)
#define RIFT_MAXMH 12   // modes with m >= 0 among 2 <= l <= 4
#define RIFT_MAXTERM 5
#define RIFT_MAXBINS 256

// status bits written by kernels
#define RIFT_FLAG_WINDOW 1u
#define RIFT_FLAG_NONFINITE 2u

struct DetC {
  float d[6];         // response tensor xx xy xz yy yz zz
  float P[3], Plo[3]; // fs * x_k / c, samples (double-float)
  float c0, c0lo;     // (t_lo - tau0_k) fs: Q index of the prior's lower edge (double-float)
  float ct, ctlo;     // -tau0_k fs: Q index of t = 0 (double-float)
};

struct ModeC {
  int l, m, nterm, pad;
  float coef[RIFT_MAXTERM]; // -2Y_lm = e^{i m phi} sum_j coef_j c^{kc_j} s^{2l-kc_j}
  int kc[RIFT_MAXTERM];
};

// One intrinsic point.  Lives in device memory (array over points); kernels copy
// it into shared memory.
struct PointC {
  int K, M, T, Mp;    // detectors, modes, Q samples, Q row stride (M rounded up to even)
  int npair, interp;
  int J, pad1;        // J: points of the time quadrature, floor((t_hi - t_lo) fs)
  long long q_off;    // offset of this point's Q in the Q arena (float2 units), 16-byte aligned
  long long uv_off;   // offset of this point's pair coefficients (float4 units)
  long long coef_off; // offset of the coefficients the quadratic form reads (uv_off, or the
                      // grouped canonical array of a point with all 21 modes)
  float fs, dref;     // Q rate (Hz), D_ref (Mpc)
  float g_hi, g_lo;   // GMST / 2pi (turns), double-float
  float A, Alo;       // (t_hi - t_lo) fs, samples (double-float)
  float t_lo, t_span; // time prior (s)
  float tmin_idx, tmax_idx; // first/last admissible interpolation base index (window check)
  DetC det[RIFT_MAXK];
  ModeC mode[RIFT_MAXM];
  // the same harmonics by canonical index j (l = 2..4, m = -l..l in order): bit j of canon_mask
  // is set when mode j is present; its terms r = r_min(j).. have coefficients ccoef[j][r - r_min(j)]
  uint32_t canon_mask;
  int ncoef;          // float4 entries at coef_off (staged into shared memory by the kernels)
  int grouped;        // grouped quadratic form (quad_canon) over the 21 canonical modes, absent
                      // modes with zero coefficients (kCanonPath kernels, at least kCanonMinModes)
  int canon_sparse;   // and U vanishes exactly between modes of opposite-sign m, V between modes of
                      // same-sign m (each h_lm on one sign of frequency): those pairs are skipped
  int mirror;         // the modes satisfy the reflection symmetry checked on the host (every mode's
                      // mirror (l, -m) present, V_ab = sigma_a U_{mirror(a) b}, U zero between
                      // opposite-sign m): the quadratic form is the positive form of quad_mirror and
                      // coef_off holds its coefficients [kMirrorPairs][K] float2 (grouped is set too)
  uint32_t sigma_neg; // bit j: sigma = -1 for canonical mode j (mirror points)
  float ccoef[RIFT_MAXM][RIFT_MAXTERM];
  // merged rows for the time quadrature: with real data and the reflection symmetry of the modes,
  // Eq. (QUV) gives Q_abar(t) = sigma_a conj(Q_a(t)) (checked per pair on the host), so a pair
  // (a, abar) is read from the row of a alone.  [K][T][Mhp] complex64 at q_off + qh_rel, Mhp = Mh
  // rounded up to even: slot h holds the row of stored mode h_a[h], whose merged mirror is stored
  // mode h_b[h] (h_a[h] when it has none), with sigma = -1 where bit h of h_neg is set
  int qhalf, Mh, Mhp, pad2;
  long long qh_rel;
  unsigned char h_a[RIFT_MAXMH], h_b[RIFT_MAXMH];
  uint32_t h_neg, pad3;
};

// FP64 constants of one point for the refinement of heavy samples (refine.cu): the same quantities
// as PointC, unrounded, and the offset of the point's U, V in the FP64 pair arena.
struct PointD {
  int K, M, T, Mp, interp, pad;
  long long q_off;           // the point's FP32 Q block (float2 units)
  long long uv_off;          // U [K][M][M] then V [K][M][M] complex128 in the FP64 arena (double2 units)
  double g;                  // GMST / 2pi (turns)
  double A;                  // (t_hi - t_lo) fs
  double t_lo, t_span, fs, dref;
  double d[RIFT_MAXK][6];    // response tensors xx xy xz yy yz zz
  double P[RIFT_MAXK][3];    // fs x_k / c (samples)
  double c0[RIFT_MAXK];      // (t_lo - tau0_k) fs
  int ml[RIFT_MAXM], mm[RIFT_MAXM], nterm[RIFT_MAXM];
  int kc[RIFT_MAXM][RIFT_MAXTERM];
  double coef[RIFT_MAXM][RIFT_MAXTERM];
};

// Canonical mode index j <-> (l, m) and the Goldberg terms of -2Y_lm present for it:
// r from max(0, m + 2) to min(l + 2, l + m), exponent of cos(theta/2) k = 2 r - 2 - m.
__host__ __device__ constexpr int canon_l(int j) { return j < 5 ? 2 : (j < 12 ? 3 : 4); }
__host__ __device__ constexpr int canon_m(int j) { return j < 5 ? j - 2 : (j < 12 ? j - 8 : j - 16); }
__host__ __device__ constexpr int canon_rmin(int j) { return canon_m(j) + 2 > 0 ? canon_m(j) + 2 : 0; }
__host__ __device__ constexpr int canon_rmax(int j) {
  return canon_l(j) + canon_m(j) < canon_l(j) + 2 ? canon_l(j) + canon_m(j) : canon_l(j) + 2;
}
__host__ __device__ constexpr int canon_index(int l, int m) { return l * l - 4 + (m + l); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), written from the published round function.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// u = ((x >> 9) + 1/2) 2^-23: 24 significant bits, exact in FP32 and FP64, in (0, 1).
__device__ __forceinline__ float bits_to_u(uint32_t x) {
  return ((float)(x >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

// ---------------------------------------------------------------------------
// Double-float helpers (Knuth two-sum, FMA two-product).
// ---------------------------------------------------------------------------
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return fast_two_sum(p, e);
}

// Split a double-float index into integer base and fraction in [0, 1).
__device__ __forceinline__ void df_floor(df s, int &i, float &f) {
  float fl = floorf(s.hi);
  f = __fadd_rn(__fsub_rn(s.hi, fl), s.lo);
  i = (int)fl;
  if (f < 0.f) { f += 1.f; i -= 1; }
  else if (f >= 1.f) { f -= 1.f; i += 1; }
}

// ---------------------------------------------------------------------------
// Per-sample geometry: everything but the Q gather and quadratic forms.
// ---------------------------------------------------------------------------
struct SampleGeo {
  float2 F[RIFT_MAXK];  // F_k = F_+ - i F_x
  df s[RIFT_MAXK];      // Q index of t + delay_k (double-float, samples)
  float x;              // D_ref / D
};

// Antenna pattern at psi = 0 and the delay from the source direction.
// e_ra = (-sin a, cos a, 0), e_dec = (-sd cos a, -sd sin a, cd); at psi = 0 the axes are
// X0 = -e_ra, Y0 = e_dec and F(psi) = e^{2 i psi} F(0) for F = F_+ - i F_x.
template <int K>
__device__ __forceinline__ void response_delay(const PointC &P, float ca, float sa, df sd, float cd,
                                               float c2p, float s2p, SampleGeo &g, const df base_rel[]) {
  const float ex = -sa, ey = ca;                   // e_ra (z = 0)
  const float fx = -sd.hi * ca, fy = -sd.hi * sa, fz = cd; // e_dec
  const float nx = cd * ca, ny = cd * sa;                // source direction (z = sin dec)
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float *d = P.det[k].d;
    // e_ra^T d e_ra, e_dec^T d e_dec, e_ra^T d e_dec
    const float dex = d[0] * ex + d[1] * ey;
    const float dey = d[1] * ex + d[3] * ey;
    const float dez = d[2] * ex + d[4] * ey;
    const float ee = ex * dex + ey * dey;
    const float ff = fx * (d[0] * fx + d[1] * fy + d[2] * fz) + fy * (d[1] * fx + d[3] * fy + d[4] * fz) +
                     fz * (d[2] * fx + d[4] * fy + d[5] * fz);
    const float ef = fx * dex + fy * dey + fz * dez;
    // X0 = -e_ra, Y0 = e_dec: F+0 = ee - ff, Fx0 = -2 ef; F0 = F+0 - i Fx0 = (ee - ff) + 2 i ef
    const float fr = ee - ff, fi = 2.f * ef;
    g.F[k] = make_float2(c2p * fr - s2p * fi, s2p * fr + c2p * fi);
    // delay_k fs = -(P . n) fs-scaled; double-float accumulation of the three products
    const DetC &D = P.det[k];
    df acc = df_mul_f(df{D.P[0], D.Plo[0]}, nx);
    acc = df_add(acc, df_mul_f(df{D.P[1], D.Plo[1]}, ny));
    acc = df_add(acc, df_mul(df{D.P[2], D.Plo[2]}, sd));
    g.s[k] = df_add(base_rel[k], df{-acc.hi, -acc.lo});
  }
}

// Real factor d_j(iota) of -2Y_lm = e^{i m phi} d_j for canonical mode j, from the powers
// cp[k] = cos(iota/2)^k, sp[k] = sin(iota/2)^k (j compile-time after unrolling).
__device__ __forceinline__ float canon_dval(const PointC &P, int j, const float (&cp)[9], const float (&sp)[9]) {
  float v = 0.f;
#pragma unroll
  for (int r = canon_rmin(j); r <= canon_rmax(j); ++r) {
    const int kc = 2 * r - 2 - canon_m(j);
    v = fmaf(P.ccoef[j][r - canon_rmin(j)], cp[kc] * sp[2 * canon_l(j) - kc], v);
  }
  return v;
}

// -2Y_lm of the present modes, unrolled over the canonical table so every power index is a
// compile-time constant; stored mode a = number of present canonical modes before j.
// WITH_D: also d[j] = d_j(iota) for every canonical j (0 for absent modes), the real factors the
// grouped quadratic form needs.
// e^{i m phi}, m = 0..4, from (cos phi, sin phi): the factors the harmonics take.
__device__ __forceinline__ void eiphi_powers(float cphi, float sphi, float2 (&e)[5]) {
  e[0] = make_float2(1.f, 0.f);
  e[1] = make_float2(cphi, sphi);
  e[2] = make_float2(cphi * cphi - sphi * sphi, 2.f * cphi * sphi);
  e[3] = make_float2(e[2].x * cphi - e[2].y * sphi, e[2].x * sphi + e[2].y * cphi);
  e[4] = make_float2(e[2].x * e[2].x - e[2].y * e[2].y, 2.f * e[2].x * e[2].y);
}

// -2Y_lm of canonical mode j from its real factor d_j and the phase factors e (j compile-time).
__device__ __forceinline__ float2 canon_y(int j, float dj, const float2 (&e)[5]) {
  const int am = canon_m(j) < 0 ? -canon_m(j) : canon_m(j);
  const float2 em = e[am];
  return make_float2(dj * em.x, canon_m(j) < 0 ? -(dj * em.y) : dj * em.y);
}

// The real factors d_j(iota) of all 21 canonical modes (c, s = cos, sin(iota/2)).
__device__ __forceinline__ void canon_d_all(const PointC &P, float c, float s, float (&d)[RIFT_MAXM]) {
  float cp[9], sp[9];
  cp[0] = 1.f; sp[0] = 1.f;
#pragma unroll
  for (int j = 1; j < 9; ++j) { cp[j] = cp[j - 1] * c; sp[j] = sp[j - 1] * s; }
#pragma unroll
  for (int j = 0; j < RIFT_MAXM; ++j) d[j] = canon_dval(P, j, cp, sp);
}

template <bool WITH_D>
__device__ __forceinline__ void swsh_canonical_t(const PointC &P, float c, float s, float cphi, float sphi,
                                                 float2 *Ys, int stride, float *d) {
  float cp[9], sp[9];
  cp[0] = 1.f; sp[0] = 1.f;
#pragma unroll
  for (int j = 1; j < 9; ++j) { cp[j] = cp[j - 1] * c; sp[j] = sp[j - 1] * s; }
  float2 e[5];
  eiphi_powers(cphi, sphi, e);
  const uint32_t mask = P.canon_mask;
#pragma unroll
  for (int j = 0; j < RIFT_MAXM; ++j) {
    if (WITH_D) d[j] = 0.f;
    if (mask & (1u << j)) {
      const float v = canon_dval(P, j, cp, sp);
      if (WITH_D) d[j] = v;
      const int a = __popc(mask & ((1u << j) - 1u));
      Ys[a * stride] = canon_y(j, v, e);
    }
  }
}

__device__ __forceinline__ void swsh_canonical(const PointC &P, float c, float s, float cphi, float sphi,
                                               float2 *Ys, int stride) {
  swsh_canonical_t<false>(P, c, s, cphi, sphi, Ys, stride, nullptr);
}

// Lagrange interpolation weights on NT taps: i-1..i+2 (cubic), i..i+1 (linear), i (nearest).
template <int NT>
__device__ __forceinline__ void interp_weights(float mu, float w[NT]) {
  if (NT == 4) {
    const float a = mu + 1.f, b = mu - 1.f, c = mu - 2.f;
    w[0] = -mu * b * c * (1.f / 6.f);
    w[1] = a * b * c * 0.5f;
    w[2 % NT] = -a * mu * c * 0.5f;
    w[3 % NT] = a * mu * b * (1.f / 6.f);
  } else if (NT == 2) {
    w[0] = 1.f - mu;
    w[1 % NT] = mu;
  } else {
    w[0] = 1.f;
  }
}

// Linear term: Re sum_k F_k sum_lm conj(Y_lm) Q_{k,lm}(t_k), taps gathered from the point's
// Q rows [K][T][Mp] (modes contiguous: the taps of one detector are one contiguous block of
// NT * Mp complex values).  Per mode the taps are combined first (qbar = sum_r w_r Q_r),
// then Z_k = sum_lm conj(Y_lm) qbar_lm, and the detector factor is applied once: Re(F_k Z_k).
template <int K, int NT>
__device__ __forceinline__ float linear_term(const PointC &P, const float2 *__restrict__ Q, const SampleGeo &g,
                                             const float2 *Ys, int ystride, uint32_t &flags) {
  constexpr int first = (NT == 4) ? -1 : 0;
  float lin = 0.f;
  const int rs = P.Mp >> 1;          // row stride in float4 (two modes per float4)
  const int npairs = (P.M + 1) >> 1;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int i; float mu;
    df s = g.s[k];
    if (NT == 1) s = df_add_f(s, 0.5f);
    df_floor(s, i, mu);
    float w[NT];
    interp_weights<NT>(mu, w);
    int i0 = i + first;
    if (i0 < 0 || i0 + NT > P.T) {
      flags |= RIFT_FLAG_WINDOW;
      i0 = min(max(i0, 0), P.T - NT);
    }
    const float4 *row = reinterpret_cast<const float4 *>(Q + ((long long)k * P.T + i0) * P.Mp);
    float zr = 0.f, zi = 0.f;
#pragma unroll 2
    for (int a2 = 0; a2 < npairs; ++a2) {
      float4 q[NT];
#pragma unroll
      for (int r = 0; r < NT; ++r) q[r] = __ldg(row + r * rs + a2);
      float q0r = 0.f, q0i = 0.f, q1r = 0.f, q1i = 0.f;
#pragma unroll
      for (int r = 0; r < NT; ++r) {
        q0r = fmaf(w[r], q[r].x, q0r); q0i = fmaf(w[r], q[r].y, q0i);
        q1r = fmaf(w[r], q[r].z, q1r); q1i = fmaf(w[r], q[r].w, q1i);
      }
      const float2 y0 = Ys[(2 * a2) * ystride];
      // the pad column of an odd M is zero in Q, so y1 may be anything finite there
      const float2 y1 = (2 * a2 + 1 < P.M) ? Ys[(2 * a2 + 1) * ystride] : make_float2(0.f, 0.f);
      // conj(y) qbar
      zr = fmaf(y0.x, q0r, fmaf(y0.y, q0i, zr));
      zi = fmaf(y0.x, q0i, fmaf(-y0.y, q0r, zi));
      zr = fmaf(y1.x, q1r, fmaf(y1.y, q1i, zr));
      zi = fmaf(y1.x, q1i, fmaf(-y1.y, q1r, zi));
    }
    const float2 Fk = g.F[k];
    lin += Fk.x * zr - Fk.y * zi;
  }
  return lin;
}

// Slot of the mode pair (a, b), a <= b, in the pair-coefficient layout of quad_term: rows in
// blocks of two (a0 = 2 j, a0 + 1), each block ordered (a0,a0), (a0,a0+1), (a0+1,a0+1), then
// (a0,b), (a0+1,b) for b = a0+2 .. M-1; a block of one row (odd M) holds (a0,a0) only.  Blocks
// before block j hold sum_{i<j} (2M - 4i - 1) = j (2M - 1) - 2 j (j - 1) pairs.
__host__ __device__ inline int pair_slot(int a, int b, int M) {
  const int j = a >> 1, a0 = 2 * j;
  const int base = j * (2 * M - 1) - 2 * j * (j - 1);
  if (b == a) return base + (a == a0 ? 0 : 2);
  if (b == a0 + 1) return base + 1;   // (a0, a0 + 1)
  return base + 3 + 2 * (b - a0 - 2) + (a - a0);
}

// Quadratic term: sum_k |F_k|^2 conj(Y)^T U_k Y + Re(conj(F_k)^2 Y^T V_k Y), using the
// upper triangle a <= b (U Hermitian, V symmetric); coefficients C[pair_slot][k] = (U, V) with
// the factor 2 of the off-diagonal pairs folded in.  Rows go in blocks of two so that one load
// of Y_b serves two pairs; each row keeps its own partial sums (pairs in order b = a..M-1),
// added to the totals row by row.
template <int K>
__device__ __forceinline__ void quad_pair(float2 ya, float2 yb, const float4 *__restrict__ c, float (&rA)[K],
                                          float (&rBr)[K], float (&rBi)[K]) {
  const float pr = ya.x * yb.x + ya.y * yb.y;   // conj(ya) yb
  const float pi = ya.x * yb.y - ya.y * yb.x;
  const float qr = ya.x * yb.x - ya.y * yb.y;   // ya yb
  const float qi = ya.x * yb.y + ya.y * yb.x;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float4 ck = c[k];
    rA[k] = fmaf(pr, ck.x, fmaf(-pi, ck.y, rA[k]));
    rBr[k] = fmaf(qr, ck.z, fmaf(-qi, ck.w, rBr[k]));
    rBi[k] = fmaf(qr, ck.w, fmaf(qi, ck.z, rBi[k]));
  }
}

template <int K>
__device__ __forceinline__ float quad_term(const PointC &P, const float4 *__restrict__ C, const SampleGeo &g,
                                           const float2 *Ys, int ystride) {
  float A[K], Br[K], Bi[K];
#pragma unroll
  for (int k = 0; k < K; ++k) { A[k] = 0.f; Br[k] = 0.f; Bi[k] = 0.f; }
  const int M = P.M;
  const float4 *c = C;
  for (int a0 = 0; a0 < M; a0 += 2) {
    float rA[K], rBr[K], rBi[K], sA[K], sBr[K], sBi[K];   // rows a0 and a0 + 1
#pragma unroll
    for (int k = 0; k < K; ++k) { rA[k] = 0.f; rBr[k] = 0.f; rBi[k] = 0.f; sA[k] = 0.f; sBr[k] = 0.f; sBi[k] = 0.f; }
    const float2 y0 = Ys[a0 * ystride];
    quad_pair<K>(y0, y0, c, rA, rBr, rBi);
    c += K;
    if (a0 + 1 < M) {
      const float2 y1 = Ys[(a0 + 1) * ystride];
      quad_pair<K>(y0, y1, c, rA, rBr, rBi);
      quad_pair<K>(y1, y1, c + K, sA, sBr, sBi);
      c += 2 * K;
      for (int b = a0 + 2; b < M; ++b, c += 2 * K) {
        const float2 yb = Ys[b * ystride];
        quad_pair<K>(y0, yb, c, rA, rBr, rBi);
        quad_pair<K>(y1, yb, c + K, sA, sBr, sBi);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) { A[k] += rA[k]; Br[k] += rBr[k]; Bi[k] += rBi[k]; }
    if (a0 + 1 < M) {
#pragma unroll
      for (int k = 0; k < K; ++k) { A[k] += sA[k]; Br[k] += sBr[k]; Bi[k] += sBi[k]; }
    }
  }
  float quad = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float2 F = g.F[k];
    const float f2 = F.x * F.x + F.y * F.y;
    // conj(F)^2 = (Fr^2 - Fi^2) - 2 i Fr Fi
    const float gr = F.x * F.x - F.y * F.y, gi = -2.f * F.x * F.y;
    quad += f2 * A[k] + (gr * Br[k] - gi * Bi[k]);
  }
  return quad;
}

// ---------------------------------------------------------------------------
// Quadratic term over the 21 canonical modes (absent ones with zero coefficients).  With
// -2Y_lm(i, phi) = e^{i m phi} d_lm(i)
// (d real), conj(Y_a) Y_b = d_a d_b e^{i (m_b - m_a) phi} and Y_a Y_b = d_a d_b e^{i (m_a + m_b) phi}, so
//   A_k = sum_{D=0..8} Re(e^{i D phi} S_kD),   S_kD = sum_{a<=b, |m_b - m_a| = D} d_a d_b c_ab
//   B_k = sum_{s=-8..8} e^{i s phi} T_ks,       T_ks = sum_{a<=b, m_a + m_b = s}  d_a d_b v_ab
// with c_ab, v_ab the pair coefficients of quad_term (c_ab conjugated where m_b < m_a).  Each pair
// costs one real product and two FMAs per detector and part instead of complex products.  The
// pairs are enumerated at compile time in group order (canon_pair_A / canon_pair_B: group << 10 |
// a << 5 | b); the grouped coefficients hold two pairs per float4 per detector: [slot][k] =
// (c_{2s}, c_{2s+1}), the U part first, then the V part.
// ---------------------------------------------------------------------------
constexpr int kCanonPairs = RIFT_MAXM * (RIFT_MAXM + 1) / 2;
constexpr int kCanonSlots = (kCanonPairs + 1) / 2;

// Pair tables, built once at compile time: A[i], B[i] = group << 10 | a << 5 | b.
struct CanonPairs {
  int A[kCanonPairs];
  int B[kCanonPairs];
};

__host__ __device__ constexpr CanonPairs make_canon_pairs() {
  CanonPairs t{};
  int n = 0;
  for (int D = 0; D <= 8; ++D)
    for (int a = 0; a < RIFT_MAXM; ++a)
      for (int b = a; b < RIFT_MAXM; ++b) {
        const int dm = canon_m(b) - canon_m(a);
        if ((dm < 0 ? -dm : dm) == D) t.A[n++] = (D << 10) | (a << 5) | b;
      }
  n = 0;
  for (int S = -8; S <= 8; ++S)
    for (int a = 0; a < RIFT_MAXM; ++a)
      for (int b = a; b < RIFT_MAXM; ++b)
        if (canon_m(a) + canon_m(b) == S) t.B[n++] = ((S + 8) << 10) | (a << 5) | b;
  return t;
}

// host copies (the coefficient layout is built on the host)
constexpr CanonPairs kCanonPairTab = make_canon_pairs();
constexpr int canon_pair_A(int i) { return kCanonPairTab.A[i]; }
constexpr int canon_pair_B(int i) { return kCanonPairTab.B[i]; }

// the pair tables as constant data (folded into immediates once the loops below are unrolled)
__constant__ const CanonPairs kCanonPairDev = make_canon_pairs();

__device__ __forceinline__ float2 eiphi_n(const float2 (&e)[9], int n) {
  const float2 r = e[n < 0 ? -n : n];
  return n < 0 ? make_float2(r.x, -r.y) : r;
}

// One part (U: B = false, V: B = true) over the 231 pairs in group order.
// SP: skip the pairs whose coefficient the host found to be exactly zero (canon_sparse); adding
// p * 0 would leave the sums unchanged, so both variants give the same bits.
template <int K, bool B, bool SP>
__device__ __forceinline__ void canon_part(const float4 *__restrict__ G, const float (&d)[RIFT_MAXM],
                                           const float2 (&e)[9], float (&acc)[K][2]) {
  float S[K][2];
#pragma unroll
  for (int k = 0; k < K; ++k) { S[k][0] = 0.f; S[k][1] = 0.f; }
  bool any = false;   // the group has a pair that is not skipped (folded at compile time)
#pragma unroll
  for (int i = 0; i < kCanonPairs; ++i) {
    const int code = B ? kCanonPairDev.B[i] : kCanonPairDev.A[i];
    const int grp = code >> 10;
    const int a = (code >> 5) & 31, b = code & 31;
    const int mm = canon_m(a) * canon_m(b);
    const bool skip = SP && (B ? mm > 0 : mm < 0);
    if (!skip) {
      any = true;
      const float4 *c = G + (B ? kCanonSlots * K : 0) + (i >> 1) * K;
      // d_a d_b; the V part forms it as an FMA with zero (the same value) so that the compiler does
      // not keep the U part's products alive for reuse
      const float p = B ? __fmaf_rn(d[a], d[b], 0.f) : d[a] * d[b];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float4 ck = c[k];
        S[k][0] = fmaf(p, (i & 1) ? ck.z : ck.x, S[k][0]);
        if (B || grp != 0) S[k][1] = fmaf(p, (i & 1) ? ck.w : ck.y, S[k][1]);   // D = 0: only Re S counts
      }
    }
    const bool last = (i + 1 == kCanonPairs) || ((B ? kCanonPairDev.B[i + 1] : kCanonPairDev.A[i + 1]) >> 10) != grp;
    if (last && any) {
      any = false;
      // the group ends: rotate its sum by e^{i n phi} into the part's total
      const float2 r = eiphi_n(e, B ? grp - 8 : grp);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        acc[k][0] = fmaf(r.x, S[k][0], fmaf(-r.y, S[k][1], acc[k][0]));
        if (B) acc[k][1] = fmaf(r.x, S[k][1], fmaf(r.y, S[k][0], acc[k][1]));
        S[k][0] = 0.f;
        S[k][1] = 0.f;
      }
    }
  }
}

// quad_canon is not inlined: one copy per translation unit instead of one per kernel keeps the
// build short (the kernel that reads G from its parameters inlines the body instead).
// c, s = cos, sin(iota/2): the d_j are evaluated here from the same sums as swsh_canonical.
// phi = 2 pi n1 2^-24 with n1 odd (the sampler's lattice): e^{i D phi} = sincospi(D n1 2^-23),
// reduced modulo 2 exactly in integers, so every rotation is good to an ulp (a product chain
// from e^{i phi} would carry D times its rounding into whole group sums).
template <int K, bool SP>
__device__ __forceinline__ float quad_canon_from_d(const float4 *__restrict__ G, const SampleGeo &g,
                                                   const float (&d)[RIFT_MAXM], uint32_t n1) {
  float2 e[9];
  e[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int D = 1; D <= 8; ++D) {
    const uint32_t r = ((uint32_t)D * n1) & 0xFFFFFFu;
    sincospif((float)r * 1.1920928955078125e-07f, &e[D].y, &e[D].x);
  }
  float A[K][2], Bc[K][2];
#pragma unroll
  for (int k = 0; k < K; ++k) { A[k][0] = 0.f; A[k][1] = 0.f; Bc[k][0] = 0.f; Bc[k][1] = 0.f; }
  canon_part<K, false, SP>(G, d, e, A);
  canon_part<K, true, SP>(G, d, e, Bc);
  float quad = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float2 F = g.F[k];
    const float f2 = F.x * F.x + F.y * F.y;
    const float gr = F.x * F.x - F.y * F.y, gi = -2.f * F.x * F.y;
    quad += f2 * A[k][0] + (gr * Bc[k][0] - gi * Bc[k][1]);
  }
  return quad;
}

template <int K, bool SP>
__device__ __forceinline__ float quad_canon_body(const PointC &P, const float4 *__restrict__ G, const SampleGeo &g,
                                                 float c, float s, uint32_t n1) {
  float cp[9], sp[9];
  cp[0] = 1.f; sp[0] = 1.f;
#pragma unroll
  for (int j = 1; j < 9; ++j) { cp[j] = cp[j - 1] * c; sp[j] = sp[j - 1] * s; }
  float d[RIFT_MAXM];
#pragma unroll
  for (int j = 0; j < RIFT_MAXM; ++j) d[j] = canon_dval(P, j, cp, sp);
  return quad_canon_from_d<K, SP>(G, g, d, n1);
}

template <int K, bool SP>
__device__ __noinline__ float quad_canon(const PointC &P, const float4 *__restrict__ G, const SampleGeo &g, float c,
                                         float s, uint32_t n1) {
  return quad_canon_body<K, SP>(P, G, g, c, s, n1);
}

// ---------------------------------------------------------------------------
// Quadratic term of a point with the reflection symmetry of non-precessing modes.  When each mode's
// mirror (l, -m) is present and the mirror of h_lm is a signed mode of the point,
// conj(h_a(-f)) = sigma_a h_abar(f) with sigma_a = +-1 (which the host reads off V: V_ab =
// sigma_a U_{abar b} for every b), the detector strain
//   h_k = (x/2) sum_a [conj(F) Y_a h_a + F conj(Y_a) conj(h_a(-f))] = x sum_a beta_a h_a,
//   beta_a = (conj(F) Y_a + sigma_a F conj(Y_abar)) / 2,
// is a combination of the mode waveforms alone, and <h_k|h_k> = x^2 beta^H U beta, so the
// |F|^2 conj(Y) U Y + Re(conj(F)^2 Y V Y) of Eq. (def:lnL:Decomposed) equals 2 beta^H U beta: a
// positive form whose terms do not cancel.  The general form cancels where h_k is small against
// |F|^2 conj(Y) U Y (nearly edge-on sources, whose strain is nearly linearly polarised): its FP32
// sums then carry errors of a few ulp of the large terms into a small result.  Here the
// cancellation happens in the two-term coefficients beta_a, each exact to an ulp of its terms.
// With Y_a = d_a e^{i m_a phi} and sigma_abar = sigma_a, beta_a = e^{i m_a phi} (Fr p_a + i Fi q_a),
// p_a = (d_a + sigma_a d_abar) / 2, q_a = (sigma_a d_abar - d_a) / 2, and beta_abar =
// sigma_a conj(beta_a); with U zero between opposite-sign m and U_{abar bbar} = sigma_a sigma_b
// conj(U_ab), the negative-m block of beta^H U beta is the conjugate of the positive-m block and
// the (negative m, m = 0) block that of the (positive m, m = 0) block, so
//   2 beta^H U beta = sum over pairs a <= b with m_a, m_b >= 0 (78 of them) of
//                     w_ab Re( e^{i (m_b - m_a) phi} U_ab conj(g_a) g_b ),   g_a = Fr p_a + i Fi q_a,
//   conj(g_a) g_b = Fr^2 p_a p_b + Fi^2 q_a q_b + i Fr Fi (p_a q_b - q_a p_b),
// w_ab = 4 (a = b, m > 0), 8 (a < b, both m > 0, or one m = 0), 2 (a = b, m = 0), 4 (a < b, m = 0).
// Coefficients c_ab = w_ab U_ab per detector: [pair][k] float2, pairs in group order of
// D = m_b - m_a (-4..4); per group and detector three complex sums X = sum pp c, Y = sum qq c,
// Z = sum (pq - qp) c, combined once: Re(e^{i D phi} (Fr^2 X + Fi^2 Y + i Fr Fi Z)).
// ---------------------------------------------------------------------------
constexpr int kMirrorModes = 12;   // canonical modes with m >= 0
constexpr int kMirrorPairs = kMirrorModes * (kMirrorModes + 1) / 2;

struct MirrorPairs {
  int code[kMirrorPairs];   // (D + 4) << 10 | a << 5 | b, canonical a <= b
};

__host__ __device__ constexpr MirrorPairs make_mirror_pairs() {
  MirrorPairs t{};
  int n = 0;
  for (int D = -4; D <= 4; ++D)
    for (int a = 0; a < RIFT_MAXM; ++a)
      for (int b = a; b < RIFT_MAXM; ++b)
        if (canon_m(a) >= 0 && canon_m(b) >= 0 && canon_m(b) - canon_m(a) == D) t.code[n++] = ((D + 4) << 10) | (a << 5) | b;
  return t;
}

constexpr MirrorPairs kMirrorPairTab = make_mirror_pairs();
constexpr int mirror_pair(int i) { return kMirrorPairTab.code[i]; }
// weight w_ab of canonical pair (a, b), a <= b, both m >= 0
constexpr float mirror_weight(int a, int b) {
  return (canon_m(a) > 0 && canon_m(b) > 0) ? (a == b ? 4.f : 8.f)
                                            : ((canon_m(a) == 0 && canon_m(b) == 0) ? (a == b ? 2.f : 4.f) : 8.f);
}
__constant__ const MirrorPairs kMirrorPairDev = make_mirror_pairs();

// e[D] = e^{i D phi}, D = 0..4.
template <int K>
__device__ __forceinline__ float quad_mirror_from_e(const float2 *__restrict__ G, const SampleGeo &g,
                                                    const float (&d)[RIFT_MAXM], uint32_t sigma_neg,
                                                    const float2 (&e)[5]) {
  float p[RIFT_MAXM], q[RIFT_MAXM];
#pragma unroll
  for (int j = 0; j < RIFT_MAXM; ++j) {
    if (canon_m(j) >= 0) {
      const int jb = canon_index(canon_l(j), -canon_m(j));
      const float sd = ((sigma_neg >> j) & 1u) ? -d[jb] : d[jb];
      p[j] = 0.5f * (d[j] + sd);
      q[j] = 0.5f * (sd - d[j]);
    } else {
      p[j] = 0.f;
      q[j] = 0.f;
    }
  }
  float fr2[K], fi2[K], fri[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    fr2[k] = g.F[k].x * g.F[k].x;
    fi2[k] = g.F[k].y * g.F[k].y;
    fri[k] = g.F[k].x * g.F[k].y;
  }
  float X[K][2], Y[K][2], Z[K][2];
#pragma unroll
  for (int k = 0; k < K; ++k) { X[k][0] = X[k][1] = Y[k][0] = Y[k][1] = Z[k][0] = Z[k][1] = 0.f; }
  float quad = 0.f;
#pragma unroll
  for (int i = 0; i < kMirrorPairs; ++i) {
    const int code = kMirrorPairDev.code[i];
    const int D = (code >> 10) - 4;
    const int a = (code >> 5) & 31, b = code & 31;
    const float pp = p[a] * p[b], qq = q[a] * q[b];
    const float r = (a == b) ? 0.f : fmaf(p[a], q[b], -(q[a] * p[b]));
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float2 c = G[i * K + k];
      X[k][0] = fmaf(pp, c.x, X[k][0]);
      Y[k][0] = fmaf(qq, c.x, Y[k][0]);
      if (D != 0) {
        X[k][1] = fmaf(pp, c.y, X[k][1]);
        Y[k][1] = fmaf(qq, c.y, Y[k][1]);
        Z[k][0] = fmaf(r, c.x, Z[k][0]);
      }
      if (a != b) Z[k][1] = fmaf(r, c.y, Z[k][1]);   // U_aa is real: diagonal pairs add no Im c
    }
    const bool last = (i + 1 == kMirrorPairs) || ((kMirrorPairDev.code[i + 1] >> 10) - 4 != D);
    if (last) {
      const float2 ed = e[D < 0 ? -D : D];
      const float er = ed.x, ei = D < 0 ? -ed.y : ed.y;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float wr = fmaf(fr2[k], X[k][0], fmaf(fi2[k], Y[k][0], -fri[k] * Z[k][1]));
        if (D == 0) {
          quad += wr;
        } else {
          const float wi = fmaf(fr2[k], X[k][1], fmaf(fi2[k], Y[k][1], fri[k] * Z[k][0]));
          quad += fmaf(er, wr, -ei * wi);
        }
        X[k][0] = X[k][1] = Y[k][0] = Y[k][1] = Z[k][0] = Z[k][1] = 0.f;
      }
    }
  }
  return quad;
}

// phi = 2 pi n1 2^-24 on the sampler's lattice: e^{i D phi} = sincospi(D n1 2^-23) reduced exactly.
template <int K>
__device__ __forceinline__ float quad_mirror_from_d(const float2 *__restrict__ G, const SampleGeo &g,
                                                    const float (&d)[RIFT_MAXM], uint32_t sigma_neg, uint32_t n1) {
  float2 e[5];
  e[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int D = 1; D <= 4; ++D) {
    const uint32_t r = ((uint32_t)D * n1) & 0xFFFFFFu;
    sincospif((float)r * 1.1920928955078125e-07f, &e[D].y, &e[D].x);
  }
  return quad_mirror_from_e<K>(G, g, d, sigma_neg, e);
}

// Any phi (caller draws).
template <int K>
__device__ __forceinline__ float quad_mirror_at(const float2 *__restrict__ G, const SampleGeo &g,
                                                const float (&d)[RIFT_MAXM], uint32_t sigma_neg, float phi) {
  float2 e[5];
  e[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int D = 1; D <= 4; ++D) sincosf((float)D * phi, &e[D].y, &e[D].x);
  return quad_mirror_from_e<K>(G, g, d, sigma_neg, e);
}

template <int K>
__device__ __forceinline__ float quad_mirror_body(const PointC &P, const float2 *__restrict__ G, const SampleGeo &g,
                                                  float c, float s, uint32_t n1) {
  float cp[9], sp[9];
  cp[0] = 1.f; sp[0] = 1.f;
#pragma unroll
  for (int j = 1; j < 9; ++j) { cp[j] = cp[j - 1] * c; sp[j] = sp[j - 1] * s; }
  float d[RIFT_MAXM];
#pragma unroll
  for (int j = 0; j < RIFT_MAXM; ++j) d[j] = canon_dval(P, j, cp, sp);
  return quad_mirror_from_d<K>(G, g, d, P.sigma_neg, n1);
}

template <int K>
__device__ __noinline__ float quad_mirror(const PointC &P, const float2 *__restrict__ G, const SampleGeo &g, float c,
                                          float s, uint32_t n1) {
  return quad_mirror_body<K>(P, G, g, c, s, n1);
}

// The mirror coefficients of one three-detector point as a kernel parameter (single-point launches).
struct MirrorCoefParam {
  float2 g[kMirrorPairs * 3];
};

// Cell kernels compiled with the grouped form: three detectors and cubic taps (the full-size
// workload); the host marks a point grouped only for these, so that compile time stays short.
// The other kernels read the pair layout (uv_off) and use quad_term for every point.
template <int K, int NT>
constexpr bool kCanonPath = (K == 3 && NT == 4);

// The grouped form runs over all 21 canonical modes whatever the point holds (291 pair-parts with
// the one-sign pairs skipped, about 3.9 kflop at K = 3); the pair form costs about 22 flop per
// pair-part, M (M + 1) of them, so the grouped form pays from 13 modes on.
constexpr int kCanonMinModes = 13;

// The grouped coefficients of one three-detector point as a kernel parameter: single-point launches
// pass them by value, so the quadratic form reads them from the parameter (constant) bank instead of
// shared memory.
struct CanonCoefParam {
  float4 g[2 * kCanonSlots * 3];
};

// ---------------------------------------------------------------------------
// Time-marginalised likelihood, Eq. (lnL:tmarg): ln (1/J) sum_j exp(lnL(theta, t_j)) over the
// midpoints t_j = t_lo + (j + 1/2)/fs, j < J.  For detector k the Q index of t_j + delay_k is
// s0_k + j with s0_k = (t_lo - tau0_k) fs + 1/2 + delay_k fs, so the interpolation weights are
// the same for every j and consecutive j use consecutive rows: Z_k[i] = sum_lm conj(Y_lm)
// Q_{k,lm}[i] is formed once per row and the NT taps slide along.  lnL_j = x (Re sum_k F_k
// Zbar_k(j) - x quad / 4).  tgrid_scan walks the grid and hands each lnL_j to a visitor;
// tmarg_term takes their log-sum-exp with a running maximum.
// Y: the point's harmonics in registers (pairs of modes, zero beyond M).
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ float2 z_row(const float4 *__restrict__ row, const float2 (&y)[RIFT_MAXM + 1], int npairs) {
  float zr = 0.f, zi = 0.f;
#pragma unroll
  for (int a2 = 0; a2 < (RIFT_MAXM + 1) / 2; ++a2) {
    if (a2 < npairs) {
      const float4 q = row[a2];
      const float2 y0 = y[2 * a2], y1 = y[2 * a2 + 1];
      // conj(y) q
      zr = fmaf(y0.x, q.x, fmaf(y0.y, q.y, zr));
      zi = fmaf(y0.x, q.y, fmaf(-y0.y, q.x, zi));
      zr = fmaf(y1.x, q.z, fmaf(y1.y, q.w, zr));
      zi = fmaf(y1.x, q.w, fmaf(-y1.y, q.z, zi));
    }
  }
  return make_float2(zr, zi);
}

// Merged rows (P.qhalf): lin_j = sum_k sum_r w_kr s_k[r0_k + j + r] with the real row sums
// s_k[i] = Re sum_h gamma_kh Qh_k,h[i] over the slots, where F_k is taken into the coefficients,
// gamma_kh = F_k conj(Y_a) + sigma_a conj(F_k) Y_abar (F_k conj(Y_a) for a mode without a merged
// mirror): the pair (a, abar) contributes Re[F_k (conj(Y_a) Q_a + conj(Y_abar) sigma_a conj(Q_a))],
// which is Re[gamma_kh Q_a].  Each row costs 2 Mh FMAs on 8 Mh bytes instead of 4 M on 8 M (all 21
// modes: Mh = 12).
__device__ __forceinline__ float s_row(const float4 *__restrict__ row, const float4 (&g)[RIFT_MAXMH / 2], int npairs) {
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int a2 = 0; a2 < RIFT_MAXMH / 2; ++a2) {
    if (a2 < npairs) {
      const float4 q = row[a2];
      s0 = fmaf(g[a2].x, q.x, fmaf(g[a2].y, q.y, s0));
      s1 = fmaf(g[a2].z, q.z, fmaf(g[a2].w, q.w, s1));
    }
  }
  return s0 + s1;
}

// The draw's part of the merged-row scan: (Re gamma, -Im gamma) of slots 2 h2 and 2 h2 + 1 of
// each detector (so that Re(gamma q) is a dot product with the row), the interpolation weights and
// the first row r0_k (clamped into the window, with the flag set, as the full-row scan does).
template <int K, int NT>
__device__ __forceinline__ void tmarg_prep(const PointC &P, const df s0[K], const float2 F[K], const float2 *Ys,
                                           int ystride, float4 (&g)[K][RIFT_MAXMH / 2], float (&w)[K][NT],
                                           int (&r0)[K], uint32_t &flags) {
  constexpr int first = (NT == 4) ? -1 : 0;
#pragma unroll
  for (int h2 = 0; h2 < RIFT_MAXMH / 2; ++h2) {
    float2 ya[2], yb[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int h = 2 * h2 + e;
      ya[e] = make_float2(0.f, 0.f);
      yb[e] = make_float2(0.f, 0.f);
      if (h < P.Mh) {
        ya[e] = Ys[P.h_a[h] * ystride];
        if (P.h_b[h] != P.h_a[h]) {
          yb[e] = Ys[P.h_b[h] * ystride];
          if (P.h_neg >> h & 1u) yb[e] = make_float2(-yb[e].x, -yb[e].y);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float c[4];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        // F conj(ya) + conj(F) yb
        const float gr = F[k].x * ya[e].x + F[k].y * ya[e].y + F[k].x * yb[e].x + F[k].y * yb[e].y;
        const float gi = F[k].y * ya[e].x - F[k].x * ya[e].y + F[k].x * yb[e].y - F[k].y * yb[e].x;
        c[2 * e] = gr;
        c[2 * e + 1] = -gi;
      }
      g[k][h2] = make_float4(c[0], c[1], c[2], c[3]);
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int i; float mu;
    df sk = s0[k];
    if (NT == 1) sk = df_add_f(sk, 0.5f);
    df_floor(sk, i, mu);
    interp_weights<NT>(mu, w[k]);
    r0[k] = i + first;
    if (r0[k] < 0 || r0[k] + P.J - 1 + NT > P.T) {
      flags |= RIFT_FLAG_WINDOW;
      r0[k] = min(max(r0[k], 0), P.T - NT - (P.J - 1));
      if (r0[k] < 0) r0[k] = 0;
    }
  }
}

// The scan of one draw over its own merged rows (read from Qh = Q + P.qh_rel through the cache).
template <int K, int NT, class Visit>
__device__ __forceinline__ void tgrid_rows(const PointC &P, const float2 *__restrict__ Qh,
                                           const float4 (&g)[K][RIFT_MAXMH / 2], const float (&w)[K][NT],
                                           const int (&r0)[K], float x, float quad, Visit &&visit) {
  const int rs = P.Mhp >> 1, npairs = (P.Mh + 1) >> 1;
  float z[K][NT];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float4 *base = reinterpret_cast<const float4 *>(Qh + ((long long)k * P.T + r0[k]) * P.Mhp);
#pragma unroll
    for (int r = 0; r < NT - 1; ++r) z[k][r] = s_row(base + (size_t)r * rs, g[k], npairs);
  }
  const float c = -0.25f * x * quad;
  const int J = P.J;
  for (int j = 0; j < J; ++j) {
    float lin = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int row = min(r0[k] + j + NT - 1, P.T - 1);
      z[k][NT - 1] = s_row(reinterpret_cast<const float4 *>(Qh + ((long long)k * P.T + row) * P.Mhp), g[k], npairs);
#pragma unroll
      for (int r = 0; r < NT; ++r) lin = fmaf(w[k][r], z[k][r], lin);
#pragma unroll
      for (int r = 0; r < NT - 1; ++r) z[k][r] = z[k][r + 1];
    }
    visit(j, x * (lin + c));
  }
}

template <int K, int NT, class Visit>
__device__ __forceinline__ void tgrid_scan_half(const PointC &P, const float2 *__restrict__ Q, const df s0[K],
                                                const float2 F[K], const float2 *Ys, int ystride, float x, float quad,
                                                uint32_t &flags, Visit &&visit) {
  float4 g[K][RIFT_MAXMH / 2];
  float w[K][NT];
  int r0[K];
  tmarg_prep<K, NT>(P, s0, F, Ys, ystride, g, w, r0, flags);
  tgrid_rows<K, NT>(P, Q + P.qh_rel, g, w, r0, x, quad, visit);
}

// HALF: 1 the half rows (the point must have them), 0 the full rows, -1 chosen by P.qhalf
template <int K, int NT, int HALF = -1, class Visit>
__device__ __forceinline__ void tgrid_scan(const PointC &P, const float2 *__restrict__ Q, const df s0[K],
                                           const float2 F[K], const float2 *Ys, int ystride, float x, float quad,
                                           uint32_t &flags, Visit &&visit) {
  if constexpr (HALF != 0) {
    if (HALF == 1 || P.qhalf) {
      tgrid_scan_half<K, NT>(P, Q, s0, F, Ys, ystride, x, quad, flags, visit);
      return;
    }
  }
  if constexpr (HALF == 1) return;
  constexpr int first = (NT == 4) ? -1 : 0;
  float2 y[RIFT_MAXM + 1];
#pragma unroll
  for (int a = 0; a < RIFT_MAXM + 1; ++a) y[a] = (a < P.M) ? Ys[a * ystride] : make_float2(0.f, 0.f);
  const int rs = P.Mp >> 1, npairs = (P.M + 1) >> 1;
  const int J = P.J;
  float w[K][NT];
  int r0[K];
  float2 z[K][NT];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int i; float mu;
    df sk = s0[k];
    if (NT == 1) sk = df_add_f(sk, 0.5f);
    df_floor(sk, i, mu);
    interp_weights<NT>(mu, w[k]);
    r0[k] = i + first;
    if (r0[k] < 0 || r0[k] + J - 1 + NT > P.T) {
      flags |= RIFT_FLAG_WINDOW;
      r0[k] = min(max(r0[k], 0), P.T - NT - (J - 1));
      if (r0[k] < 0) r0[k] = 0;
    }
    const float4 *base = reinterpret_cast<const float4 *>(Q + ((long long)k * P.T + r0[k]) * P.Mp);
#pragma unroll
    for (int r = 0; r < NT - 1; ++r) z[k][r] = z_row<NT>(base + (size_t)r * rs, y, npairs);
  }
  const float c = -0.25f * x * quad;
  for (int j = 0; j < J; ++j) {
    float lin = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int row = min(r0[k] + j + NT - 1, P.T - 1);
      z[k][NT - 1] = z_row<NT>(reinterpret_cast<const float4 *>(Q + ((long long)k * P.T + row) * P.Mp), y, npairs);
      float zr = 0.f, zi = 0.f;
#pragma unroll
      for (int r = 0; r < NT; ++r) { zr = fmaf(w[k][r], z[k][r].x, zr); zi = fmaf(w[k][r], z[k][r].y, zi); }
      lin += F[k].x * zr - F[k].y * zi;
#pragma unroll
      for (int r = 0; r < NT - 1; ++r) z[k][r] = z[k][r + 1];
    }
    visit(j, x * (lin + c));
  }
}

template <int K, int NT, int HALF = -1>
__device__ __forceinline__ float tmarg_term(const PointC &P, const float2 *__restrict__ Q, const df s0[K],
                                            const float2 F[K], const float2 *Ys, int ystride, float x, float quad,
                                            uint32_t &flags) {
  float m = -INFINITY, s = 0.f;
  tgrid_scan<K, NT, HALF>(P, Q, s0, F, Ys, ystride, x, quad, flags, [&](int, float l) {
    if (l > m) { s = fmaf(s, expf(m - l), 1.f); m = l; }
    else s += expf(l - m);
  });
  return m + logf(s) - logf((float)P.J);
}

// Event time of a draw from its conditional on the same grid, P(t_j | rest) proportional to
// exp(lnL_j): the first j with sum_{i<=j} e^{lnL_i - m} > u sum_i e^{lnL_i - m} (m the maximum), or
// the last j of positive weight when rounding leaves the cumulative sum short of the target.
// Returns j (-1 if no j has a finite positive weight) and lnL_j.
template <int K, int NT>
__device__ __forceinline__ int tmarg_pick(const PointC &P, const float2 *__restrict__ Q, const df s0[K],
                                          const float2 F[K], const float2 *Ys, int ystride, float x, float quad,
                                          float u, float &l_out, uint32_t &flags) {
  float m = -INFINITY, s = 0.f;
  tgrid_scan<K, NT>(P, Q, s0, F, Ys, ystride, x, quad, flags, [&](int, float l) {
    if (l > m) { s = fmaf(s, expf(m - l), 1.f); m = l; }
    else s += expf(l - m);
  });
  const float target = u * s;
  float c = 0.f, lp = NAN, ll = NAN;
  int jp = -1, jl = -1;
  tgrid_scan<K, NT>(P, Q, s0, F, Ys, ystride, x, quad, flags, [&](int j, float l) {
    const float e = expf(l - m);
    c += e;
    if (e > 0.f) { jl = j; ll = l; }
    if (jp < 0 && c > target) { jp = j; lp = l; }
  });
  if (jp < 0) { jp = jl; lp = ll; }
  l_out = lp;
  return jp;
}
