// Cell kernel: the Monte Carlo round of Eq. (lnLmarg) organised by stratification cells.
//
// A round of n samples of a point is split into C = S_ra S_sd S_t cells of the unit cube of
// the (ra, sin dec, t) uniforms; the samples of one cell share a small box of sky and time,
// so the Q rows their time-of-flight-shifted taps need (Sec. II.A: Q_{k,lm}(t + n.x_k)) form a
// short contiguous window per detector.  One CTA takes one cell at a time (a dynamic work
// queue over the cells of every active point, so the same kernel runs one point or a batch):
//
//   A. every thread draws its samples of the cell and computes only their Q indices;
//      a block min/max gives the window of each detector;
//   B. one thread stages the windows (contiguous rows of the [K][T][Mp] arena) into shared
//      memory with bulk asynchronous copies completing on an mbarrier;
//   C. every thread re-draws its samples and evaluates Eq. (def:lnL:Decomposed) with the taps
//      read from the staged window (taps outside it, if the window did not fit, come from
//      global memory: same values);
//   D. log weights -> per-thread log-sum-exp -> warp shuffles -> one partial per cell.
#include <cfloat>
#include <cmath>

#include "draw.cuh"
#include "rift_device.cuh"
#include "rift_internal.h"

namespace {

constexpr float kTwoPi = 6.283185307179586f;
constexpr float kNegInf = -INFINITY;
constexpr long long kWaitCycles = 2000000000ll;   // bounded mbarrier wait (~1 s)

__device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity`; false if the bound expired.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void copy_words(const void *src, void *dst, int nbytes) {
  const int *s = reinterpret_cast<const int *>(src);
  int *d = reinterpret_cast<int *>(dst);
  for (int i = threadIdx.x; i < nbytes / 4; i += blockDim.x) d[i] = s[i];
}

// Quadratic term of a drawn sample: for points in the canonical layout (the kernels compiled with
// it) the positive form of a mirror-symmetric point or the grouped form, the pair form otherwise.
// CP: coefficients from the shared copy C (0) or the kernel parameters cpg: grouped dense (1),
// grouped sparse (2), mirror (3).  u_phi = n1 2^-24, n1 odd.
template <int K, int NT, int CP>
__device__ __forceinline__ float quad_cell(const PointC &P, const float4 *__restrict__ C,
                                           const void *__restrict__ cpg, const SampleGeo &g, const float2 *Ys,
                                           int ystride, float ch, float sh, float u_phi) {
  const uint32_t n1 = (uint32_t)(u_phi * 16777216.f);
  if constexpr (CP == 3) return quad_mirror_body<K>(P, static_cast<const float2 *>(cpg), g, ch, sh, n1);
  if constexpr (CP) return quad_canon_body<K, CP == 2>(P, static_cast<const float4 *>(cpg), g, ch, sh, n1);
  if constexpr (kCanonPath<K, NT>) {
    if (P.grouped) {
      if (P.mirror) return quad_mirror<K>(P, reinterpret_cast<const float2 *>(C), g, ch, sh, n1);
      return P.canon_sparse ? quad_canon<K, true>(P, C, g, ch, sh, n1) : quad_canon<K, false>(P, C, g, ch, sh, n1);
    }
  }
  return quad_term<K>(P, C, g, Ys, ystride);
}

// Sky and time geometry of a drawn sample: cos/sin of (ra - GMST) and sin/cos dec.
struct Sky { float ca, sa, cd; df sd; };

__device__ __forceinline__ Sky sky_of(const PointC &P, const Drawn &d) {
  const df v = df_add(d.x0, df{-P.g_hi, -P.g_lo});   // ra/2pi - GMST/2pi (turns)
  float s0, c0;
  sincospif(2.f * v.hi, &s0, &c0);
  const float ares = kTwoPi * v.lo;
  Sky s;
  s.ca = c0 - s0 * ares;
  s.sa = s0 + c0 * ares;
  s.sd = df_add_f(df{2.f * d.x1.hi, 2.f * d.x1.lo}, -1.f);
  s.cd = cos_dec_of(d.x1);
  return s;
}

// Q index of t + delay_k for every detector (double-float samples).
template <int K>
__device__ __forceinline__ void time_index(const PointC &P, const Drawn &d, const Sky &s, df out[K]) {
  const df tf = df_mul(df{P.A, P.Alo}, d.x2);   // (t - t_lo) fs
  const float nx = s.cd * s.ca, ny = s.cd * s.sa;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const DetC &D = P.det[k];
    df acc = df_mul_f(df{D.P[0], D.Plo[0]}, nx);
    acc = df_add(acc, df_mul_f(df{D.P[1], D.Plo[1]}, ny));
    acc = df_add(acc, df_mul(df{D.P[2], D.Plo[2]}, s.sd));
    out[k] = df_add(df_add(df{D.c0, D.c0lo}, tf), df{-acc.hi, -acc.lo});
  }
}

// Global sample index of the j-th sample of a cell.
__device__ __forceinline__ uint32_t sample_index(const RoundPt &R, uint32_t cell, uint32_t j) {
  return (cell < R.rem) ? cell * (R.base + 1u) + j : R.rem * (R.base + 1u) + (cell - R.rem) * R.base + j;
}

// Cell of global sample i (i < R.n, so R.base >= 1 whenever cells hold samples).
__device__ __forceinline__ uint32_t cell_of(const RoundPt &R, uint32_t i) {
  const uint32_t big = R.rem * (R.base + 1u);
  return (i < big) ? i / (R.base + 1u) : R.rem + (i - big) / R.base;
}

__device__ __forceinline__ void lse_push(float l, float &m, float &s1, float &s2) {
  if (l > m) {
    const float e = expf(m - l);
    s1 = fmaf(s1, e, 1.f);
    s2 = fmaf(s2, e * e, 1.f);
    m = l;
  } else {
    const float e = expf(l - m);
    s1 += e;
    s2 = fmaf(e, e, s2);
  }
}

__device__ __forceinline__ void lse_merge(float &m, float &s1, float &s2, float m2, float t1, float t2) {
  if (m2 > m) {
    float tm = m, a = s1, b = s2;
    m = m2; s1 = t1; s2 = t2; m2 = tm; t1 = a; t2 = b;
  }
  if (m2 == kNegInf) return;
  const float e = expf(m2 - m);
  s1 = fmaf(t1, e, s1);
  s2 = fmaf(t2, e * e, s2);
}

// Linear term with taps from a staged window when they lie inside it.
template <int K, int NT>
__device__ __forceinline__ float linear_term_staged(const PointC &P, const float2 *__restrict__ Q, const df s_idx[K],
                                                    const float2 F[K], const float2 *Ys, int ystride,
                                                    const float4 *const win[K], const int wlo[K],
                                                    const int whi[K], uint32_t &flags) {
  constexpr int first = (NT == 4) ? -1 : 0;
  const int rs = P.Mp >> 1;
  const int npairs = (P.M + 1) >> 1;
  // per detector: interpolation weights and the first tap row (staged window or global)
  float w[K][NT];
  const float4 *row[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int i; float mu;
    df s = s_idx[k];
    if (NT == 1) s = df_add_f(s, 0.5f);
    df_floor(s, i, mu);
    interp_weights<NT>(mu, w[k]);
    int i0 = i + first;
    if (i0 < 0 || i0 + NT > P.T) {
      flags |= RIFT_FLAG_WINDOW;
      i0 = min(max(i0, 0), P.T - NT);
    }
    const bool in_win = win[k] != nullptr && i0 >= wlo[k] && i0 + NT - 1 <= whi[k];
    row[k] = in_win ? win[k] + (size_t)(i0 - wlo[k]) * rs
                    : reinterpret_cast<const float4 *>(Q + ((long long)k * P.T + i0) * P.Mp);
  }
  // modes outside, detectors inside: each Y_lm is read from shared memory once
  float zr[K], zi[K];
#pragma unroll
  for (int k = 0; k < K; ++k) { zr[k] = 0.f; zi[k] = 0.f; }
  for (int a2 = 0; a2 < npairs; ++a2) {
    const float2 y0 = Ys[(2 * a2) * ystride];
    const float2 y1 = (2 * a2 + 1 < P.M) ? Ys[(2 * a2 + 1) * ystride] : make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float4 q[NT];
#pragma unroll
      for (int r = 0; r < NT; ++r) q[r] = row[k][r * rs + a2];
      float q0r = 0.f, q0i = 0.f, q1r = 0.f, q1i = 0.f;
#pragma unroll
      for (int r = 0; r < NT; ++r) {
        q0r = fmaf(w[k][r], q[r].x, q0r); q0i = fmaf(w[k][r], q[r].y, q0i);
        q1r = fmaf(w[k][r], q[r].z, q1r); q1i = fmaf(w[k][r], q[r].w, q1i);
      }
      zr[k] = fmaf(y0.x, q0r, fmaf(y0.y, q0i, zr[k]));
      zi[k] = fmaf(y0.x, q0i, fmaf(-y0.y, q0r, zi[k]));
      zr[k] = fmaf(y1.x, q1r, fmaf(y1.y, q1i, zr[k]));
      zi[k] = fmaf(y1.x, q1i, fmaf(-y1.y, q1r, zi[k]));
    }
  }
  float lin = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) lin += F[k].x * zr[k] - F[k].y * zi[k];
  return lin;
}

// The same linear term for a point holding all 21 canonical modes (stored order = canonical order),
// with the harmonics formed in registers from their real factors d_j and e^{i m phi} instead of read
// from a per-thread shared buffer; every operation is the one linear_term_staged performs on the
// same values, so the results are the same bits.
template <int K, int NT>
__device__ __forceinline__ float linear_term_yreg(const PointC &P, const float2 *__restrict__ Q, const df s_idx[K],
                                                  const float2 F[K], const float (&dj)[RIFT_MAXM],
                                                  const float2 (&e)[5], const float4 *const win[K], const int wlo[K],
                                                  const int whi[K], uint32_t &flags) {
  constexpr int first = (NT == 4) ? -1 : 0;
  constexpr int rs = (RIFT_MAXM + 1) / 2;   // row stride in float4 (Mp = 22)
  float w[K][NT];
  const float4 *row[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int i; float mu;
    df s = s_idx[k];
    if (NT == 1) s = df_add_f(s, 0.5f);
    df_floor(s, i, mu);
    interp_weights<NT>(mu, w[k]);
    int i0 = i + first;
    if (i0 < 0 || i0 + NT > P.T) {
      flags |= RIFT_FLAG_WINDOW;
      i0 = min(max(i0, 0), P.T - NT);
    }
    const bool in_win = win[k] != nullptr && i0 >= wlo[k] && i0 + NT - 1 <= whi[k];
    row[k] = in_win ? win[k] + (size_t)(i0 - wlo[k]) * rs
                    : reinterpret_cast<const float4 *>(Q + ((long long)k * P.T + i0) * (2 * rs));
  }
  float zr[K], zi[K];
#pragma unroll
  for (int k = 0; k < K; ++k) { zr[k] = 0.f; zi[k] = 0.f; }
#pragma unroll
  for (int a2 = 0; a2 < rs; ++a2) {
    const float2 y0 = canon_y(2 * a2, dj[2 * a2], e);
    const float2 y1 = (2 * a2 + 1 < RIFT_MAXM) ? canon_y(2 * a2 + 1, dj[(2 * a2 + 1) % RIFT_MAXM], e)
                                               : make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float4 q[NT];
#pragma unroll
      for (int r = 0; r < NT; ++r) q[r] = row[k][r * rs + a2];
      float q0r = 0.f, q0i = 0.f, q1r = 0.f, q1i = 0.f;
#pragma unroll
      for (int r = 0; r < NT; ++r) {
        q0r = fmaf(w[k][r], q[r].x, q0r); q0i = fmaf(w[k][r], q[r].y, q0i);
        q1r = fmaf(w[k][r], q[r].z, q1r); q1i = fmaf(w[k][r], q[r].w, q1i);
      }
      zr[k] = fmaf(y0.x, q0r, fmaf(y0.y, q0i, zr[k]));
      zi[k] = fmaf(y0.x, q0i, fmaf(-y0.y, q0r, zi[k]));
      zr[k] = fmaf(y1.x, q1r, fmaf(y1.y, q1i, zr[k]));
      zi[k] = fmaf(y1.x, q1i, fmaf(-y1.y, q1r, zi[k]));
    }
  }
  float lin = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) lin += F[k].x * zr[k] - F[k].y * zi[k];
  return lin;
}

// The linear term of a point with all 21 modes whose 9 mirror pairs all merge (P.qhalf, P.Mh = 12):
// rows of the 12 modes with m >= 0 (merged rows, Mhp = 12), in the canonical order, slot h holding
// canonical mode kMergedA[h] and its mirror kMergedB[h] (itself for m = 0).  With Y_a = d_a e^{i m
// phi} and Y_abar = d_abar e^{-i m phi}, the coefficient of the pair's row is
// gamma_k = F_k conj(Y_a) + sigma conj(F_k) Y_abar = (fr p c + fi q s, fi q c - fr p s), where
// p = d_a + sigma d_abar, q = d_a - sigma d_abar, (c, s) = (cos m phi, sin m phi) and F_k = fr + i fi;
// for m = 0, gamma_k = F_k d_a.  lin = sum_k sum_r w_kr sum_h Re(gamma_kh Q_kh[i_k + r]): each tap
// row is dotted with (Re gamma, -Im gamma) and the NT row sums are interpolated.
__device__ constexpr int kMergedA[RIFT_MAXMH] = {2, 3, 4, 8, 9, 10, 11, 16, 17, 18, 19, 20};
__device__ constexpr int kMergedB[RIFT_MAXMH] = {2, 1, 0, 8, 7, 6, 5, 16, 15, 14, 13, 12};

template <int K, int NT>
__device__ __forceinline__ float linear_term_merged(const PointC &P, const float2 *__restrict__ Qh, const df s_idx[K],
                                                    const float2 F[K], const float (&dj)[RIFT_MAXM],
                                                    const float2 (&e)[5], const float4 *const win[K],
                                                    const int wlo[K], const int whi[K], uint32_t &flags) {
  constexpr int first = (NT == 4) ? -1 : 0;
  constexpr int rs = RIFT_MAXMH / 2;   // merged row stride in float4
  float w[K][NT];
  const float4 *row[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int i; float mu;
    df s = s_idx[k];
    if (NT == 1) s = df_add_f(s, 0.5f);
    df_floor(s, i, mu);
    interp_weights<NT>(mu, w[k]);
    int i0 = i + first;
    if (i0 < 0 || i0 + NT > P.T) {
      flags |= RIFT_FLAG_WINDOW;
      i0 = min(max(i0, 0), P.T - NT);
    }
    const bool in_win = win[k] != nullptr && i0 >= wlo[k] && i0 + NT - 1 <= whi[k];
    row[k] = in_win ? win[k] + (size_t)(i0 - wlo[k]) * rs
                    : reinterpret_cast<const float4 *>(Qh + ((long long)k * P.T + i0) * (2 * rs));
  }
  float sr[K][NT];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int r = 0; r < NT; ++r) sr[k][r] = 0.f;
#pragma unroll
  for (int h2 = 0; h2 < rs; ++h2) {
    // per slot of the pair: (fr, fi) -> (Re gamma, -Im gamma) = (fr A + fi B, fr C + fi D)
    float A[2], Bc[2], Cc[2], D[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int h = 2 * h2 + u;
      const int ja = kMergedA[h], jb = kMergedB[h];
      const int m = canon_m(ja);
      const float da = dj[ja];
      if (m == 0) {
        A[u] = da; Bc[u] = 0.f; Cc[u] = 0.f; D[u] = -da;
      } else {
        const float db = (P.h_neg >> h & 1u) ? -dj[jb] : dj[jb];
        const float pp = da + db, qq = da - db;
        const float c = e[m].x, sn = e[m].y;
        A[u] = pp * c; Bc[u] = qq * sn; Cc[u] = pp * sn; D[u] = -qq * c;
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float fr = F[k].x, fi = F[k].y;
      const float4 gk = make_float4(fmaf(fr, A[0], fi * Bc[0]), fmaf(fr, Cc[0], fi * D[0]),
                                    fmaf(fr, A[1], fi * Bc[1]), fmaf(fr, Cc[1], fi * D[1]));
#pragma unroll
      for (int r = 0; r < NT; ++r) {
        const float4 q = row[k][r * rs + h2];
        sr[k][r] = fmaf(gk.x, q.x, fmaf(gk.y, q.y, fmaf(gk.z, q.z, fmaf(gk.w, q.w, sr[k][r]))));
      }
    }
  }
  float lin = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int r = 0; r < NT; ++r) lin = fmaf(w[k][r], sr[k][r], lin);
  return lin;
}

// Q index of t_0 + delay_k for the time quadrature: (t_lo - tau0_k) fs + 1/2 - fs x_k . n.
template <int K>
__device__ __forceinline__ void delay_index(const PointC &P, const Sky &s, df out[K]) {
  const float nx = s.cd * s.ca, ny = s.cd * s.sa;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const DetC &D = P.det[k];
    df acc = df_mul_f(df{D.P[0], D.Plo[0]}, nx);
    acc = df_add(acc, df_mul_f(df{D.P[1], D.Plo[1]}, ny));
    acc = df_add(acc, df_mul(df{D.P[2], D.Plo[2]}, s.sd));
    out[k] = df_add(df_add_f(df{D.c0, D.c0lo}, 0.5f), df{-acc.hi, -acc.lo});
  }
}

// Antenna patterns F_k = F+ - i Fx of a draw: the pattern at psi = 0 rotated by e^{2 i psi},
// 2 psi = 2 pi u_psi.
template <int K>
__device__ __forceinline__ void antenna_of(const PointC &P, const Sky &s, float u_psi, SampleGeo &g) {
  float s2p, c2p;
  sincospif(2.f * u_psi, &s2p, &c2p);
  const float ex = -s.sa, ey = s.ca;
  const float fx = -s.sd.hi * s.ca, fy = -s.sd.hi * s.sa, fz = s.cd;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float *dd = P.det[k].d;
    const float dex = dd[0] * ex + dd[1] * ey;
    const float dey = dd[1] * ex + dd[3] * ey;
    const float dez = dd[2] * ex + dd[4] * ey;
    const float ee = ex * dex + ey * dey;
    const float ff = fx * (dd[0] * fx + dd[1] * fy + dd[2] * fz) + fy * (dd[1] * fx + dd[3] * fy + dd[4] * fz) +
                     fz * (dd[2] * fx + dd[4] * fy + dd[5] * fz);
    const float ef = fx * dex + fy * dey + fz * dez;
    const float fr = ee - ff, fi = 2.f * ef;
    g.F[k] = make_float2(c2p * fr - s2p * fi, s2p * fr + c2p * fi);
  }
}

// ---------------------------------------------------------------------------
// Time quadrature of an item as a GEMM (Eq. (lnL:tmarg)).  The item's draws (one per thread) are
// set up first: harmonics, quadratic form, merged-row coefficients G (tmarg_prep), weights and
// first rows.  They are sorted by a key of their first rows, so that each group of 32 consecutive
// slots comes from a small patch of sky, and each group is scanned in chunks of the time grid: for
// every detector the union of the group's rows of the chunk is staged in shared memory
// (cp.async.bulk, double buffered), the row sums S[row][draw] = sum_e Q[row][e] G[e][draw] are
// formed by all threads in tiles of 8 rows x 4 draws (each row and coefficient loaded once per
// tile), and each draw then interpolates its own rows of S into lin_j.  A Q row is thus read once
// per group instead of once per draw.  Items whose groups spread over more rows than the block
// holds take the per-draw scan (tgrid_rows) instead.
// ---------------------------------------------------------------------------
constexpr int kTgLin = 32;   // time points per epilogue thread per chunk (chunks of at most 8 kTgLin)

__device__ __forceinline__ uint32_t spread_bits16(uint32_t v) {
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

template <int K, int NT, int LEARNED>
__device__ __forceinline__ void tmarg_gemm_item(const CellLaunch &L, const PointC &P, const RoundPt &R,
                                                const float4 *C, const float *tab, const float *lnw,
                                                const float *s_gmm, unsigned char *wbuf, uint64_t *tbar,
                                                uint32_t &tph, uint32_t j0, uint32_t j_end, float &m, float &s1,
                                                float &s2, float &cnt, uint32_t &flags, bool &ok) {
  constexpr int B = RIFT_CELL_BLOCK;
  constexpr int HP = RIFT_MAXMH / 2;
  const TgLayout T = tg_layout(K, NT, RIFT_MAXMH, (unsigned)L.win_budget);
  float4 *G = reinterpret_cast<float4 *>(wbuf + T.G);   // [K][HP][B]
  float *W = reinterpret_cast<float *>(wbuf + T.W);       // [K][NT][B]
  int *R0 = reinterpret_cast<int *>(wbuf + T.R0);         // [K][B]
  float *CX = reinterpret_cast<float *>(wbuf + T.CX);
  float *XX = reinterpret_cast<float *>(wbuf + T.XX);
  uint2 *KEY = reinterpret_cast<uint2 *>(wbuf + T.KEY);
  int *POS = reinterpret_cast<int *>(wbuf + T.POS);
  float2 *LT = reinterpret_cast<float2 *>(wbuf + T.LT);
  float *LN = reinterpret_cast<float *>(wbuf + T.LN);
  int *GM = reinterpret_cast<int *>(wbuf + T.GM);         // [2][K][B / 32]: min, max of r0 per group
  float *S = reinterpret_cast<float *>(wbuf + T.S);       // [rmax][RIFT_TG_SROW]
  float2 *QS = reinterpret_cast<float2 *>(wbuf + T.QS);   // [2][rmax][RIFT_MAXMH]
  float2 *Ys = reinterpret_cast<float2 *>(wbuf + T.S) + threadIdx.x;   // harmonics, setup only
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int n_it = (int)(j_end - j0);
  const int J = P.J;
  const float2 *Qh = L.qa + P.q_off + P.qh_rel;

  // 1. setup of draw j0 + t
  float4 g[K][HP];
  float w[K][NT];
  int r0[K];
  float x = 0.f, quad = 0.f, lpq = 0.f;
  uint32_t bins = 0u, i = 0u, key = 0xFFFFFFFFu;
  const bool valid = t < n_it;
  if (valid) {
    i = j0 + (uint32_t)t;
    const Drawn d = draw_any<LEARNED, 1>(L.seed, R, i, cell_of(R, i), tab, lnw, s_gmm, P.dref, L.d_lo3, L.d_span3);
    const Sky s = sky_of(P, d);
    SampleGeo gg;
    {
      df si[K];
      delay_index<K>(P, s, si);
#pragma unroll
      for (int k = 0; k < K; ++k) gg.s[k] = si[k];
    }
    antenna_of<K>(P, s, d.u_psi, gg);
    gg.x = d.xd;
    float sphi, cphi;
    sincospif(2.f * d.u_phi, &sphi, &cphi);
    const float ch = sqrtf(d.c_frac), sh = sqrtf(1.f - d.c_frac);
    swsh_canonical(P, ch, sh, cphi, sphi, Ys, B);
    quad = quad_cell<K, NT, 0>(P, C, nullptr, gg, Ys, B, ch, sh, d.u_phi);
    tmarg_prep<K, NT>(P, gg.s, gg.F, Ys, B, g, w, r0, flags);
    x = gg.x;
    lpq = d.lpq;
    bins = d.bins;
    const uint32_t k0 = (uint32_t)min(r0[0], 0xFFFF), k1 = (K > 1) ? (uint32_t)min(r0[K > 1 ? 1 : 0], 0xFFFF) : 0u;
    key = min(spread_bits16(k0) | (spread_bits16(k1) << 1), 0xFFFFFFFEu);
  }
  // 2. sort the draws by key (bitonic, ties by thread): slot POS[t] of thread t
  KEY[t] = make_uint2(key, (uint32_t)t);
  __syncthreads();
  for (int size = 2; size <= B; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int b = t ^ stride;
      if (b > t) {
        const uint2 ka = KEY[t], kb = KEY[b];
        const bool gt = ka.x > kb.x || (ka.x == kb.x && ka.y > kb.y);
        if (gt == ((t & size) == 0)) { KEY[t] = kb; KEY[b] = ka; }
      }
      __syncthreads();
    }
  POS[KEY[t].y] = t;
  __syncthreads();
  const int slot = POS[t];
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int h2 = 0; h2 < HP; ++h2) G[(k * HP + h2) * B + slot] = valid ? g[k][h2] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < NT; ++r) W[(k * NT + r) * B + slot] = valid ? w[k][r] : 0.f;
    R0[k * B + slot] = valid ? r0[k] : 0;
  }
  CX[slot] = valid ? -0.25f * x * quad : 0.f;
  XX[slot] = valid ? x : 0.f;
  __syncthreads();
  // 3. row span of each group of 32 slots (invalid slots sort last and are left out)
  const int ngroups = (n_it + 31) >> 5;
  if (wid < ngroups) {
    const bool v = 32 * wid + lane < n_it;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int r = R0[k * B + 32 * wid + lane];
      const int mn = __reduce_min_sync(0xffffffffu, v ? r : INT_MAX);
      const int mx = __reduce_max_sync(0xffffffffu, v ? r : INT_MIN);
      if (lane == 0) { GM[k * (B / 32) + wid] = mn; GM[(K + k) * (B / 32) + wid] = mx; }
    }
  }
  __syncthreads();
  // chunk of the time grid of group wg: the union of its rows for a chunk of cj points, cj + NT - 1
  // + (spread of its first rows), fits the block, and preferably B rows (one tile per thread); at
  // most 8 kTgLin, a multiple of 8
  auto chunk_of = [&](int wg) {
    int sp = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) sp = max(sp, GM[(K + k) * (B / 32) + wg] - GM[k * (B / 32) + wg]);
    const int one = (min(T.rmax, B) - (NT - 1) - sp) & ~7;
    return min(one >= 64 ? one : ((T.rmax - (NT - 1) - sp) & ~7), 8 * kTgLin);
  };
  bool gemm = T.rmax >= 64;
  for (int wg = 0; wg < ngroups && gemm; ++wg) gemm = chunk_of(wg) >= 32;

  float lnL = NAN;
  if (!gemm) {
    // 4a. per-draw scan over the cached rows
    if (valid) {
      float em = -INFINITY, es = 0.f;
      tgrid_rows<K, NT>(P, Qh, g, w, r0, x, quad, [&](int, float l) {
        if (l > em) { es = fmaf(es, expf(em - l), 1.f); em = l; }
        else es += expf(l - em);
      });
      lnL = em + logf(es) - logf((float)J);
    }
  } else {
    // 4b. stages (group, chunk, detector) in order; stage q fills buffer q & 1, issued two ahead by
    // thread 0 once the buffer is free
    const int rs = P.Mhp >> 1, npairs = (P.Mh + 1) >> 1;
    int iw = 0, ijc = 0, ik = 0;   // next stage to issue (thread 0)
    int issued = 0, consumed = 0;
    auto issue_next = [&]() {
      if (iw >= ngroups) return;
      const int buf = issued & 1;
      const int cj = min(chunk_of(iw), J - ijc);
      const int gmn = GM[ik * (B / 32) + iw];
      const int nrows = cj + NT - 1 + (GM[(K + ik) * (B / 32) + iw] - gmn);
      const uint32_t bytes = (uint32_t)nrows * (uint32_t)P.Mhp * 8u;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&tbar[buf], bytes);
      bulk_g2s(QS + (size_t)buf * T.rmax * RIFT_MAXMH, Qh + ((long long)ik * P.T + gmn + ijc) * P.Mhp, bytes,
               &tbar[buf]);
      ++issued;
      if (++ik == K) {
        ik = 0;
        ijc += chunk_of(iw);
        if (ijc >= J) { ijc = 0; ++iw; }
      }
    };
    if (t == 0) { issue_next(); issue_next(); }
    const int dl = lane, jq = wid;
    for (int wg = 0; wg < ngroups && ok; ++wg) {
      const int cjg = chunk_of(wg);
      const int pslot = 32 * wg + dl;
      const bool pv = pslot < n_it;
      float em = -INFINITY, es = 0.f;
      for (int jc = 0; jc < J && ok; jc += cjg) {
        const int cj = min(cjg, J - jc);
        const int jlo = (jq * cj) >> 3, nj = (((jq + 1) * cj) >> 3) - jlo;
        float lin[kTgLin];
#pragma unroll
        for (int jj = 0; jj < kTgLin; ++jj) lin[jj] = 0.f;
        for (int k = 0; k < K; ++k) {
          const int buf = consumed & 1;
          const uint32_t par = (tph >> buf) & 1u;
          ok = __syncthreads_and(mbar_wait(&tbar[buf], par) ? 1 : 0) != 0;
          if (!ok) { flags |= RIFT_FLAG_TIMEOUT_BIT; break; }
          tph ^= 1u << buf;
          ++consumed;
          const int gmn = GM[k * (B / 32) + wg];
          const int nrows = cj + NT - 1 + (GM[(K + k) * (B / 32) + wg] - gmn);
          const int ntask = ((nrows + 7) >> 3) * 8;
          const float4 *Qb = reinterpret_cast<const float4 *>(QS + (size_t)buf * T.rmax * RIFT_MAXMH);
          const float4 *Gk = G + (size_t)k * HP * B + 32 * wg;
          for (int task = t; task < ntask; task += B) {
            const int rt = task >> 3, td = task & 7;
            float acc[8][4];
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[q][c] = 0.f;
#pragma unroll
            for (int e4 = 0; e4 < HP; ++e4) {
              if (e4 < npairs) {
                // all operands of the step first, then four passes of 32 independent FMAs
                float4 gv[4], qv[8];
#pragma unroll
                for (int c = 0; c < 4; ++c) gv[c] = Gk[e4 * B + td + 8 * c];
#pragma unroll
                for (int q = 0; q < 8; ++q) qv[q] = Qb[(8 * rt + q) * rs + e4];
#pragma unroll
                for (int q = 0; q < 8; ++q)
#pragma unroll
                  for (int c = 0; c < 4; ++c) acc[q][c] = fmaf(qv[q].x, gv[c].x, acc[q][c]);
#pragma unroll
                for (int q = 0; q < 8; ++q)
#pragma unroll
                  for (int c = 0; c < 4; ++c) acc[q][c] = fmaf(qv[q].y, gv[c].y, acc[q][c]);
#pragma unroll
                for (int q = 0; q < 8; ++q)
#pragma unroll
                  for (int c = 0; c < 4; ++c) acc[q][c] = fmaf(qv[q].z, gv[c].z, acc[q][c]);
#pragma unroll
                for (int q = 0; q < 8; ++q)
#pragma unroll
                  for (int c = 0; c < 4; ++c) acc[q][c] = fmaf(qv[q].w, gv[c].w, acc[q][c]);
              }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
              for (int c = 0; c < 4; ++c) S[(8 * rt + q) * RIFT_TG_SROW + td + 8 * c] = acc[q][c];
          }
          __syncthreads();
          if (t == 0) issue_next();   // buffer `buf` is free again
          if (pv) {
            // the draw's rows of S for its time points, loaded before use (rows past the chunk are
            // clamped into the block and not used)
            const int off = R0[k * B + pslot] - gmn + jlo;
            float wk[NT], rowv[kTgLin + NT - 1];
#pragma unroll
            for (int r = 0; r < NT; ++r) wk[r] = W[(k * NT + r) * B + pslot];
#pragma unroll
            for (int e = 0; e < kTgLin + NT - 1; ++e) rowv[e] = S[min(off + e, T.rmax - 1) * RIFT_TG_SROW + dl];
#pragma unroll
            for (int jj = 0; jj < kTgLin; ++jj) {
              float v = 0.f;
#pragma unroll
              for (int r = 0; r < NT; ++r) v = fmaf(wk[r], rowv[jj + r], v);
              if (jj < nj) lin[jj] += v;
            }
          }
          // S is rewritten by the next stage's GEMM, which every thread reaches only through that
          // stage's barrier on the staged rows (and a group's end passes two more barriers)
        }
        if (ok && pv) {
          // the chunk's log-sum-exp against its own maximum (no per-point branch; four partial
          // sums), then merged into the draw's running (max, sum)
          const float xx = XX[pslot], cc = CX[pslot];
          float mc = kNegInf;
#pragma unroll
          for (int jj = 0; jj < kTgLin; ++jj) {
            lin[jj] = jj < nj ? xx * (lin[jj] + cc) : kNegInf;
            mc = fmaxf(mc, lin[jj]);
          }
          if (mc > kNegInf) {
            float sc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int jj = 0; jj < kTgLin; ++jj) sc[jj & 3] += expf(lin[jj] - mc);
            const float sum = (sc[0] + sc[1]) + (sc[2] + sc[3]);
            if (mc > em) { es = fmaf(es, expf(em - mc), sum); em = mc; }
            else es = fmaf(sum, expf(mc - em), es);
          }
        }
      }
      if (!ok) break;
      LT[t] = make_float2(em, es);
      __syncthreads();
      if (t < 32 && 32 * wg + t < n_it) {
        float M = -INFINITY;
        for (int q = 0; q < B / 32; ++q) M = fmaxf(M, LT[q * 32 + t].x);
        float sum = 0.f;
        for (int q = 0; q < B / 32; ++q) {
          const float2 e = LT[q * 32 + t];
          if (e.y != 0.f) sum += e.y * expf(e.x - M);
        }
        LN[32 * wg + t] = M + logf(sum) - logf((float)J);
      }
      __syncthreads();
    }
    if (!ok) {
      // copies still in flight into this CTA's shared memory: wait for them (bounded) before the
      // caller stops
      for (; consumed < issued; ++consumed) {
        const int buf = consumed & 1;
        mbar_wait(&tbar[buf], (tph >> buf) & 1u);
        tph ^= 1u << buf;
      }
      return;
    }
    if (valid) lnL = LN[slot];
  }
  // 5. the draw's log weight
  if (valid) {
    float ell = lnL + lpq;
    if (L.fault_nan && i == 0u && R.round == 0u) ell = __int_as_float(0x7fc00000);   // injected (host-requested) fault
    if (L.dbg_ell && R.dbg_off >= 0) L.dbg_ell[R.dbg_off + i] = ell;
    if (L.ell_buf && R.ell_off >= 0) { L.ell_buf[R.ell_off + i] = ell; L.bin_buf[R.ell_off + i] = bins; }
    if (isfinite(ell)) { lse_push(ell, m, s1, s2); cnt += 1.f; }
    else flags |= RIFT_FLAG_NONFINITE;
  }
}

// Rows of the Q window of each detector for the samples of a stratified cell, from the cell's box
// alone: the box in (ra, sin dec, t) (its uniforms' bounds through the round's tables when the
// proposal is adaptive), the time-of-flight term of the index on a 5 x 5 grid over the sky patch
// (one grid point per lane of the calling warp) and the time range at its ends.  Between grid
// points the term x_k . n / c (times fs) departs from the grid's range by at most
// |x_k| fs / c (h_ra^2 + h_dec^2) / 8 (its second derivative along the sky is at most |x_k|), which
// is added with one row more.  A sample whose taps still fall outside reads them from global
// memory, so the bounds decide only what is staged.  Called by whole warps; every lane returns the
// warp's bounds.
template <int K, int NT>
__device__ __forceinline__ void cell_window_rows(const PointC &P, const RoundPt &R, uint32_t cell, const float *tab,
                                                 int (&rmin)[K], int (&rmax)[K]) {
  constexpr int first = (NT == 4) ? -1 : 0;
  const int lane = threadIdx.x & 31;
  const uint32_t ls[3] = {R.ls0, R.ls1, R.ls2};
  const uint32_t cc[3] = {cell & ((1u << R.ls0) - 1u), (cell >> R.ls0) & ((1u << R.ls1) - 1u), cell >> (R.ls0 + R.ls1)};
  float xa[3], xb[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float sc = __int_as_float((127 - (int)ls[d]) << 23);   // 2^-ls
    const float ua = (float)cc[d] * sc, ub = (float)(cc[d] + 1u) * sc;
    if (R.proposal == 1) {
      int b;
      xa[d] = inv_cdf_df(tab + d * (R.nb + 1), R.nb, df{ua, 0.f}, b).hi;
      xb[d] = inv_cdf_df(tab + d * (R.nb + 1), R.nb, df{ub, 0.f}, b).hi;
    } else {
      xa[d] = ua;
      xb[d] = ub;
    }
  }
  const int g = lane < 25 ? lane : 0;
  const float fr = 0.25f * (float)(g % 5), fs = 0.25f * (float)(g / 5);
  const float v = fmaf(xb[0] - xa[0], fr, xa[0]) - P.g_hi;   // ra/2pi - GMST/2pi (turns)
  float sa, ca;
  sincospif(2.f * v, &sa, &ca);
  const float sd = fmaf(2.f, fmaf(xb[1] - xa[1], fs, xa[1]), -1.f);
  const float cd = sqrtf(fmaxf(0.f, fmaf(-sd, sd, 1.f)));
  const float nx = cd * ca, ny = cd * sa;
  const float ta = P.A * xa[2], tb = P.A * xb[2];   // (t - t_lo) fs at the ends of the time range
  const float half = (NT == 1) ? 0.5f : 0.f;
  // grid spacings (radians) in ra and dec
  const float h_ra = 0.25f * kTwoPi * (xb[0] - xa[0]);
  const float h_dec = 0.25f * (asinf(fminf(1.f, fmaf(2.f, xb[1], -1.f))) - asinf(fmaxf(-1.f, fmaf(2.f, xa[1], -1.f))));
  const float curv = 0.125f * fmaf(h_ra, h_ra, h_dec * h_dec);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const DetC &D = P.det[k];
    const float acc = fmaf(D.P[0], nx, fmaf(D.P[1], ny, D.P[2] * sd));
    const float rk = sqrtf(fmaf(D.P[0], D.P[0], fmaf(D.P[1], D.P[1], D.P[2] * D.P[2])));   // |x_k| fs / c
    const int margin = (int)ceilf(rk * curv) + 1;
    const int lo = __reduce_min_sync(0xffffffffu, (int)floorf(D.c0 + ta - acc + half));
    const int hi = __reduce_max_sync(0xffffffffu, (int)floorf(D.c0 + tb - acc + half));
    rmin[k] = lo + first - margin;
    rmax[k] = hi + first + NT - 1 + margin;
  }
}

// TMARG: the event time is marginalised by quadrature (Eq. lnL:tmarg) instead of sampled; the
// sample's t uniform is unused, its Q rows span the whole time window (no staging), and the
// likelihood is tmarg_term: each point reads its half rows (tgrid_scan_half) when it has them, and
// TMARG 2, for launches whose points all have them, compiles only that path (fewer registers).
// YR: a mirror-symmetric point with all 21 modes in the parameter bank (CP 3), harmonics in
// registers (linear_term_yreg): no per-thread harmonics buffer in shared memory (L.max_M = 0), so
// the room goes to the Q windows; YR 2: the same with all 9 mirror pairs of Q merged
// (linear_term_merged), the windows staged from the merged rows.
template <int K, int NT, int LEARNED, int TMARG, int CP, int YR = 0>
__device__ __forceinline__ void cells_body(const CellLaunch &L, const void *__restrict__ cpg) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ __align__(8) uint64_t tbar[2];   // staged Q rows of the time-quadrature GEMM (TMARG 2)
  __shared__ int s_item, s_point;
  __shared__ RoundPt sR;
  __shared__ float s_gmm[RIFT_GMM_FLOATS];
  __shared__ int s_wlo[K], s_whi[K], s_woff[K];
  __shared__ int s_red[2 * K][RIFT_CELL_BLOCK / 32];
  __shared__ float4 s_wpart[RIFT_CELL_BLOCK / 32];
  __shared__ uint32_t s_wflag[RIFT_CELL_BLOCK / 32];
  __shared__ float s_tmax[RIFT_CELL_BLOCK];
  __shared__ uint32_t s_timax[RIFT_CELL_BLOCK];

  PointC &P = *reinterpret_cast<PointC *>(smem);
  size_t off = al16(sizeof(PointC));
  float4 *C = reinterpret_cast<float4 *>(smem + off);
  off = al16(off + sizeof(float4) * (size_t)L.max_pairK);
  float *tab = reinterpret_cast<float *>(smem + off);
  float *lnw = tab + 3 * (L.max_nb + 1);
  if (L.max_nb > 0) off = al16(off + sizeof(float) * (size_t)(3 * (L.max_nb + 1) + 3 * L.max_nb));
  float2 *Ys = reinterpret_cast<float2 *>(smem + off) + threadIdx.x;
  const int ystride = blockDim.x;
  off = al16(off + sizeof(float2) * (size_t)L.max_M * blockDim.x);
  unsigned char *wbuf = smem + off;

  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    if (TMARG == 2) { mbar_init(&tbar[0], 1); mbar_init(&tbar[1], 1); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_point = -1;
  }
  __syncthreads();
  uint32_t phase = 0, tph = 0;
  int cur = -1;
  uint32_t flags = 0u;
  const uint32_t n_items = *L.n_items;

  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t it = atomicAdd(L.queue, 1u);
      int p = -1;
      if (it < n_items) {
        // point of this item: last p with item0 <= it
        int lo = 0, hi = L.n_points - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (L.rp[mid].item0 <= it) lo = mid; else hi = mid - 1;
        }
        p = lo;   // item0 is non-decreasing and inactive points own no items, so p owns `it`
      }
      s_item = (int)it;
      s_point = p;
    }
    __syncthreads();
    const uint32_t item = (uint32_t)s_item;
    const int p = s_point;
    if (item >= n_items || p < 0) break;
    const RoundPt &R = sR;
    if (p != cur) {
      copy_words(L.pts + p, &P, sizeof(PointC));
      copy_words(L.rp + p, &sR, sizeof(RoundPt));
      __syncthreads();
      if (!CP) {
        const float4 *cg = L.ca + P.coef_off;
        for (int j = threadIdx.x; j < P.ncoef; j += blockDim.x) C[j] = cg[j];
      }
      if (R.proposal == 1) {
        for (int j = threadIdx.x; j < 3 * (R.nb + 1); j += blockDim.x) tab[j] = R.tab[j];
        for (int j = threadIdx.x; j < 3 * R.nb; j += blockDim.x) lnw[j] = R.lnw[j];
      } else if (R.proposal == 2) {
        for (int j = threadIdx.x; j < RIFT_GMM_FLOATS; j += blockDim.x) s_gmm[j] = R.gmm[j];
      }
      __syncthreads();
      cur = p;
    }
    const uint32_t local = item - R.item0;
    uint32_t cell, j0, j_end;
    if constexpr (TMARG) {
      // a run of at most RIFT_TMARG_CHUNK consecutive draws of the point, one per thread (a draw
      // costs about J samples, so every item is one full pass); each draw takes its own cell
      cell = 0u;
      j0 = local * RIFT_TMARG_CHUNK;
      j_end = min(R.n, j0 + RIFT_TMARG_CHUNK);
    } else {
      cell = local / R.chunks;
      j0 = (local - cell * R.chunks) * RIFT_CHUNK;
      const uint32_t n_cell = R.base + (cell < R.rem ? 1u : 0u);
      j_end = min(n_cell, j0 + RIFT_CHUNK);
    }
    const float2 *Q = L.qa + P.q_off;
    constexpr int first = (NT == 4) ? -1 : 0;

    const float4 *win[K];
    int wlo[K], whi[K];
    bool ok = true;
    if (TMARG) {
#pragma unroll
      for (int k = 0; k < K; ++k) { win[k] = nullptr; wlo[k] = 0; whi[k] = -1; }
    } else {
    // A. window of every detector: from the cell's box for stratified prior and adaptive rounds,
    // else from the cell's samples
    int rmin[K], rmax[K];
#pragma unroll
    for (int k = 0; k < K; ++k) { rmin[k] = INT_MAX; rmax[k] = INT_MIN; }
    const bool boxed = !LEARNED && R.proposal <= 1 && (R.ls0 + R.ls1 + R.ls2) > 0u;
    if (boxed) cell_window_rows<K, NT>(P, R, cell, tab, rmin, rmax);
    for (uint32_t j = j0 + threadIdx.x; j < j_end && !boxed; j += blockDim.x) {
      const Drawn d = draw_any<LEARNED>(L.seed, R, sample_index(R, cell, j), cell, tab, lnw, s_gmm, P.dref, L.d_lo3,
                                        L.d_span3);
      const Sky s = sky_of(P, d);
      df si[K];
      time_index<K>(P, d, s, si);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        int i; float mu;
        df sk = si[k];
        if (NT == 1) sk = df_add_f(sk, 0.5f);
        df_floor(sk, i, mu);
        rmin[k] = min(rmin[k], i + first);
        rmax[k] = max(rmax[k], i + first + NT - 1);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int a = __reduce_min_sync(0xffffffffu, rmin[k]);
      const int b = __reduce_max_sync(0xffffffffu, rmax[k]);
      if (lane == 0) { s_red[2 * k][wid] = a; s_red[2 * k + 1][wid] = b; }
    }
    __syncthreads();
    // B. stage the windows that fit
    if (threadIdx.x == 0) {
      uint32_t bytes = 0;
      const int rowb = (YR == 2 ? P.Mhp : P.Mp) * 8;   // staged rows: merged rows for YR 2
      for (int k = 0; k < K; ++k) {
        int a = INT_MAX, b = INT_MIN;
        for (int w = 0; w < nw; ++w) { a = min(a, s_red[2 * k][w]); b = max(b, s_red[2 * k + 1][w]); }
        a = max(a, 0);
        b = min(b, P.T - 1);
        s_woff[k] = -1;
        s_wlo[k] = a;
        s_whi[k] = b;
        if (b >= a) {
          const uint32_t nbytes = (uint32_t)(b - a + 1) * rowb;
          if (bytes + nbytes <= (uint32_t)L.win_budget) {
            s_woff[k] = (int)bytes;
            bytes += nbytes;
          }
        }
      }
      if (bytes) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar, bytes);
        for (int k = 0; k < K; ++k)
          if (s_woff[k] >= 0 && !L.fault_stall) {   // (an injected fault leaves the announced bytes unissued)
            const float2 *src = (YR == 2) ? Q + P.qh_rel + ((long long)k * P.T + s_wlo[k]) * P.Mhp
                                          : Q + ((long long)k * P.T + s_wlo[k]) * P.Mp;
            bulk_g2s(wbuf + s_woff[k], src, (uint32_t)(s_whi[k] - s_wlo[k] + 1) * rowb, &bar);
          }
      }
      s_item = bytes ? 1 : 0;   // reused as "staged" flag for this item
    }
    __syncthreads();
    const bool staged = s_item != 0;
    if (staged) {
      ok = __syncthreads_and(mbar_wait(&bar, phase) ? 1 : 0) != 0;   // uniform across the CTA
      if (ok) phase ^= 1u;
      else flags |= RIFT_FLAG_TIMEOUT_BIT;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      win[k] = (ok && s_woff[k] >= 0) ? reinterpret_cast<const float4 *>(wbuf + s_woff[k]) : nullptr;
      wlo[k] = s_wlo[k];
      whi[k] = s_whi[k];
    }
    }

    // C. evaluate
    float m = kNegInf, s1 = 0.f, s2 = 0.f, cnt = 0.f;
    // this thread's largest log weight of the item and its sample (candidates), kept in shared
    // memory so that the sample loop holds no more registers
    s_tmax[threadIdx.x] = kNegInf;
    s_timax[threadIdx.x] = 0u;
    if constexpr (TMARG == 2) {
      tmarg_gemm_item<K, NT, LEARNED>(L, P, R, C, tab, lnw, s_gmm, wbuf, tbar, tph, j0, j_end, m, s1, s2, cnt, flags,
                                      ok);
    } else {
    for (uint32_t j = j0 + threadIdx.x; j < j_end; j += blockDim.x) {
      const uint32_t i = TMARG ? j : sample_index(R, cell, j);
      const Drawn d = draw_any<LEARNED, TMARG>(L.seed, R, i, TMARG ? cell_of(R, i) : cell, tab, lnw, s_gmm, P.dref,
                                               L.d_lo3, L.d_span3);
      const Sky s = sky_of(P, d);
      df si[K];
      if (TMARG) delay_index<K>(P, s, si);
      else time_index<K>(P, d, s, si);
      SampleGeo g;
#pragma unroll
      for (int k = 0; k < K; ++k) g.s[k] = si[k];
      antenna_of<K>(P, s, d.u_psi, g);
      g.x = d.xd;
      float sphi, cphi;
      sincospif(2.f * d.u_phi, &sphi, &cphi);
      const float ch = sqrtf(d.c_frac), sh = sqrtf(1.f - d.c_frac);   // cos, sin(incl/2)
      float dj[RIFT_MAXM];   // d_lm(incl) for the grouped quadratic form (parameter-bank kernels)
      if constexpr (YR) canon_d_all(P, ch, sh, dj);
      else if constexpr (CP != 0) swsh_canonical_t<true>(P, ch, sh, cphi, sphi, Ys, ystride, dj);
      else swsh_canonical(P, ch, sh, cphi, sphi, Ys, ystride);
      float lnL;
      if (TMARG) {
        const float quad = quad_cell<K, NT, CP>(P, C, cpg, g, Ys, ystride, ch, sh, d.u_phi);
        lnL = tmarg_term<K, NT, TMARG == 2 ? 1 : -1>(P, Q, g.s, g.F, Ys, ystride, g.x, quad, flags);
      } else {
        // merged rows (YR 2): the linear term first, so its tap rows, weights and indices are dead
        // before the quadratic form (about a third of the register spills of the other order);
        // otherwise the quadratic form first, so the d_lm it takes from the harmonics are dead
        // before the linear term's taps are loaded.  The same operations either way.
        float lin = 0.f;
        if constexpr (YR == 2) {
          float2 e[5];
          eiphi_powers(cphi, sphi, e);
          lin = linear_term_merged<K, NT>(P, Q + P.qh_rel, g.s, g.F, dj, e, win, wlo, whi, flags);
        }
        float quad;
        if constexpr (CP == 3)
          quad = quad_mirror_from_d<K>(static_cast<const float2 *>(cpg), g, dj, P.sigma_neg,
                                       (uint32_t)(d.u_phi * 16777216.f));
        else if constexpr (CP != 0)
          quad = quad_canon_from_d<K, CP == 2>(static_cast<const float4 *>(cpg), g, dj, (uint32_t)(d.u_phi * 16777216.f));
        else quad = quad_cell<K, NT, CP>(P, C, cpg, g, Ys, ystride, ch, sh, d.u_phi);
        if constexpr (YR == 1) {
          float2 e[5];
          eiphi_powers(cphi, sphi, e);
          lin = linear_term_yreg<K, NT>(P, Q, g.s, g.F, dj, e, win, wlo, whi, flags);
        } else if constexpr (YR == 0) {
          lin = linear_term_staged<K, NT>(P, Q, g.s, g.F, Ys, ystride, win, wlo, whi, flags);
        }
        lnL = g.x * fmaf(-0.25f * g.x, quad, lin);
      }
      float ell = lnL + d.lpq;
      if (L.fault_nan && i == 0u && R.round == 0u) ell = __int_as_float(0x7fc00000);   // injected (host-requested) fault
      if (L.dbg_ell && R.dbg_off >= 0) L.dbg_ell[R.dbg_off + i] = ell;
      if (L.ell_buf && R.ell_off >= 0) { L.ell_buf[R.ell_off + i] = ell; L.bin_buf[R.ell_off + i] = d.bins; }
      if (isfinite(ell)) { lse_push(ell, m, s1, s2); cnt += 1.f; }
      else flags |= RIFT_FLAG_NONFINITE;
      if (L.cand && ell > s_tmax[threadIdx.x]) { s_tmax[threadIdx.x] = ell; s_timax[threadIdx.x] = i; }
    }
    }
    // D. one partial per cell; the two largest log weights of each warp as candidates
    if (L.cand) {
      float v = s_tmax[threadIdx.x];
      uint32_t ix = s_timax[threadIdx.x];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float bv = v;
        uint32_t bi = ix;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
          const uint32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) L.cand[(size_t)item * RIFT_CAND_PER_ITEM + 2 * wid + r] = make_float2(bv, __uint_as_float(bi));
        if (v == bv && ix == bi) v = kNegInf;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float m2 = __shfl_xor_sync(0xffffffffu, m, o);
      const float a2 = __shfl_xor_sync(0xffffffffu, s1, o);
      const float b2 = __shfl_xor_sync(0xffffffffu, s2, o);
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      lse_merge(m, s1, s2, m2, a2, b2);
    }
    const uint32_t fw = __reduce_or_sync(0xffffffffu, flags);
    if (lane == 0) { s_wpart[wid] = make_float4(m, s1, s2, cnt); s_wflag[wid] = fw; }
    __syncthreads();
    if (threadIdx.x == 0) {
      float M = kNegInf, S1 = 0.f, S2 = 0.f, N = 0.f;
      uint32_t F = 0u;
      for (int w = 0; w < nw; ++w) {
        lse_merge(M, S1, S2, s_wpart[w].x, s_wpart[w].y, s_wpart[w].z);
        N += s_wpart[w].w;
        F |= s_wflag[w];
      }
      L.partials[item] = Part{(double)M, (double)S1, (double)S2, (double)N};
      if (L.cand) L.cmax[item] = M;
      if (F) atomicOr(L.flags, F);
    }
    flags = 0u;
    __syncthreads();   // windows, partial slots and the point cache are reused by the next item
    if (!ok) {
      // the copies did not complete in time: wait once more (bounded) so none is left in
      // flight into this CTA's shared memory, then stop; the flag reports the failure (the
      // time-quadrature GEMM has waited for its own copies)
      if (TMARG != 2) mbar_wait(&bar, phase);
      break;
    }
  }
}

__device__ __forceinline__ void neumaier(double &s, double &c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
  s = t;
}

// One CTA per point: the point's cell partials merged into its running compensated accumulator.
// Pass 1 takes the largest partial maximum M; pass 2 sums s1 e^{m - M} and s2 e^{2(m - M)} in FP64
// (the factors in FP32: relative 6e-8 on terms that are FP32 sums themselves), both reduced in a
// fixed order, so the result is deterministic.
constexpr int kMergeThreads = 1024;
__global__ void __launch_bounds__(kMergeThreads) merge_points_kernel(const Part *__restrict__ part,
                                                                     const RoundPt *__restrict__ rp,
                                                                     AccState *__restrict__ acc) {
  __shared__ double sm[3][kMergeThreads / 32];
  __shared__ double sM;
  const RoundPt &R = rp[blockIdx.x];
  AccState &A = acc[blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double mx = -INFINITY;
  for (uint32_t j = threadIdx.x; j < R.nitem; j += blockDim.x) {
    mx = fmax(mx, part[R.item0 + j].m);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) sm[0][wid] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = -INFINITY;
    for (int w = 0; w < nw; ++w) v = fmax(v, sm[0][w]);
    sM = v;
  }
  __syncthreads();
  const double M = sM;
  double s1 = 0.0, s2 = 0.0, n = 0.0;
  for (uint32_t j = threadIdx.x; j < R.nitem; j += blockDim.x) {
    const Part p = part[R.item0 + j];
    n += p.n;
    if (p.m != -INFINITY) {
      const double e = (double)expf((float)(p.m - M));
      s1 += p.s1 * e;
      s2 += p.s2 * e * e;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  __syncthreads();
  if (lane == 0) { sm[0][wid] = s1; sm[1][wid] = s2; sm[2][wid] = n; }
  __syncthreads();
  if (threadIdx.x == 0 && R.ncell > 0) {
    double S1 = 0.0, S2 = 0.0, N = 0.0;
    for (int w = 0; w < nw; ++w) { S1 += sm[0][w]; S2 += sm[1][w]; N += sm[2][w]; }
    A.round_max = M;
    A.round_neff = (N > 0.0 && M != -INFINITY) ? S1 : 0.0;   // the round's own sum w / max w
    if (N > 0.0 && M != -INFINITY) {
      if (M > A.m) {
        const double f = (A.m == -INFINITY) ? 0.0 : exp(A.m - M);
        A.s1 *= f; A.c1 *= f; A.s2 *= f * f; A.c2 *= f * f;
        A.m = M;
      }
      const double e = exp(M - A.m);
      neumaier(A.s1, A.c1, S1 * e);
      neumaier(A.s2, A.c2, S2 * e * e);
    }
    A.n += (unsigned long long)N;
  }
}

// Adaptive histograms of every point (grid: hblocks x points), 32.32 fixed point.
__global__ void hist_points_kernel(const float *__restrict__ ell, const uint32_t *__restrict__ bins,
                                   const RoundPt *__restrict__ rp, const AccState *__restrict__ acc, float beta, int nb,
                                   unsigned long long *__restrict__ part, const RoundCtl *ctl) {
  extern __shared__ unsigned long long h[];
  if (ctl && !ctl->adapt_now) return;
  const int p = blockIdx.y;
  const RoundPt &R = rp[p];
  for (int j = threadIdx.x; j < 3 * nb; j += blockDim.x) h[j] = 0ull;
  __syncthreads();
  if (R.ncell > 0 && R.ell_off >= 0 && R.proposal == 1) {
    const float mx = (float)acc[p].round_max;
    const uint32_t lane = threadIdx.x & 31u;
    // warp-uniform loop; adapted proposals put many samples of a warp in the same bin, so the
    // lanes of one bin are summed first (exactly: the 2^32 fixed point in 1 + 24 + 8 bit parts,
    // each part's warp sum fits 32 bits) and one atomic per distinct bin is issued
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < R.n; base += gridDim.x * blockDim.x) {
      const uint32_t i = base + lane;
      bool ok = false;
      unsigned long long q = 0ull;
      uint32_t b = 0u;
      if (i < R.n) {
        const float l = ell[R.ell_off + i];
        if (isfinite(l)) {
          ok = true;
          q = __float2ull_rn(expf(beta * (l - mx)) * 4294967296.0f);
          b = bins[R.ell_off + i];
        }
      }
      const uint32_t qhi = (uint32_t)(q >> 32), qmid = (uint32_t)(q >> 8) & 0xFFFFFFu, qlo = (uint32_t)q & 0xFFu;
#pragma unroll
      for (int dd = 0; dd < 3; ++dd) {
        const uint32_t key = ok ? ((b >> (8 * dd)) & 255u) : 0xFFFFFFFFu;
        const unsigned grp = __match_any_sync(0xFFFFFFFFu, key);
        const uint32_t shi = __reduce_add_sync(grp, qhi), smid = __reduce_add_sync(grp, qmid),
                       slo = __reduce_add_sync(grp, qlo);
        if (ok && lane == (uint32_t)(__ffs(grp) - 1))
          atomicAdd(&h[dd * nb + key], ((unsigned long long)shi << 32) + ((unsigned long long)smid << 8) + slo);
      }
    }
  }
  __syncthreads();
  unsigned long long *out = part + ((size_t)p * gridDim.x + blockIdx.x) * 3 * nb;
  for (int j = threadIdx.x; j < 3 * nb; j += blockDim.x) out[j] = h[j];
}

// New tables of every adapting point (grid: points): p_b = (1 - eps) h_b / sum h + eps / nb,
// cdf = cumsum in FP64 rounded to float32 (cdf[0] = 0, cdf[nb] = 1), lnw_b = -ln(nb (cdf[b+1] - cdf[b])).
// With part == nullptr only lnw is recomputed from the current tables.
__global__ void tables_points_kernel(const unsigned long long *__restrict__ part, int hblocks,
                                     const RoundPt *__restrict__ rp, int nb, double eps, float *tables, float *lnw,
                                     const RoundCtl *ctl, int np) {
  __shared__ double hs[3 * RIFT_MAXBINS];
  const int p = blockIdx.x;
  if (ctl) {
    // batched run: write the buffer the next round reads
    if (!ctl->adapt_now) return;
    const int nbuf = ctl->tabbuf ^ 1;
    tables += (size_t)nbuf * np * 3 * (nb + 1);
    lnw += (size_t)nbuf * np * 3 * nb;
  }
  if (part && (rp[p].ncell == 0 || rp[p].proposal != 1)) return;
  float *tb = tables + (size_t)p * 3 * (nb + 1);
  float *lw = lnw + (size_t)p * 3 * nb;
  if (part) {
    for (int j = threadIdx.x; j < 3 * nb; j += blockDim.x) {
      unsigned long long t = 0ull;
      for (int b = 0; b < hblocks; ++b) t += part[((size_t)p * hblocks + b) * 3 * nb + j];
      hs[j] = (double)t;
    }
    __syncthreads();
  }
  if (threadIdx.x < 3) {
    const int d = threadIdx.x;
    float *cdf = tb + d * (nb + 1);
    if (part) {
      double S = 0.0;
      if (!(d == 2 && rp[p].tmarg))   // the time table of a time-marginalised run stays uniform
        for (int b = 0; b < nb; ++b) S += hs[d * nb + b];
      double tot = 0.0;
      for (int b = 0; b < nb; ++b) tot += (S > 0.0 ? (1.0 - eps) * hs[d * nb + b] / S + eps / nb : 1.0 / nb);
      double c = 0.0;
      cdf[0] = 0.f;
      for (int b = 0; b < nb; ++b) {
        c += (S > 0.0 ? (1.0 - eps) * hs[d * nb + b] / S + eps / nb : 1.0 / nb);
        cdf[b + 1] = (float)(c / tot);
      }
      cdf[nb] = 1.f;
    }
    for (int b = 0; b < nb; ++b) lw[d * nb + b] = (float)(-log((double)nb * ((double)cdf[b + 1] - (double)cdf[b])));
  }
}

template <int K, int NT, int LEARNED, int TMARG>
__global__ void __launch_bounds__(RIFT_CELL_BLOCK, TMARG ? 1 : 2) cells_kernel(CellLaunch L) {
  cells_body<K, NT, LEARNED, TMARG, 0>(L, nullptr);
}

// One three-detector point in the grouped layout: its grouped coefficients come in the parameters
// (SP: the pairs that vanish for modes on one sign of frequency are skipped).
template <int K, int NT, int SP>
__global__ void __launch_bounds__(RIFT_CELL_BLOCK, 2) cells_kernel_cp(CellLaunch L, const __grid_constant__ CanonCoefParam cc) {
  cells_body<K, NT, 0, 0, SP ? 2 : 1>(L, cc.g);
}

// One mirror-symmetric three-detector point: the coefficients of its positive quadratic form come
// in the parameters.
template <int K, int NT, int YR>
__global__ void __launch_bounds__(RIFT_CELL_BLOCK, 2) cells_kernel_mp(CellLaunch L, const __grid_constant__ MirrorCoefParam mc) {
  cells_body<K, NT, 0, 0, 3, YR>(L, mc.g);
}

// The samples of one round of point 0 in cell order (no evaluation).
__global__ void draw_cells_kernel(CellLaunch L, DrawOut o, uint32_t n) {
  __shared__ __align__(16) PointC P;
  extern __shared__ float dtab[];
  const RoundPt &R = L.rp[0];
  copy_words(L.pts, &P, sizeof(PointC));
  float *tab = dtab;
  float *lnw = dtab + 3 * (R.nb + 1);
  if (R.proposal == 1) {
    for (int j = threadIdx.x; j < 3 * (R.nb + 1); j += blockDim.x) tab[j] = R.tab[j];
    for (int j = threadIdx.x; j < 3 * R.nb; j += blockDim.x) lnw[j] = R.lnw[j];
  }
  __syncthreads();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // cell of sample i
  const uint32_t big = R.rem * (R.base + 1u);
  const uint32_t cell = (i < big) ? i / (R.base + 1u) : R.rem + (i - big) / R.base;
  const Drawn d = (R.proposal == 2) ? draw_learned<0>(L.seed, R, i, R.gmm, P.dref, L.d_lo3, L.d_span3)
                                    : draw_cell_sample(L.seed, R, i, cell, tab, lnw, P.dref, L.d_lo3, L.d_span3);
  o.theta[0 * (size_t)n + i] = kTwoPi * (d.x0.hi + d.x0.lo);
  o.theta[1 * (size_t)n + i] = (2.f * d.x1.hi - 1.f) + 2.f * d.x1.lo;
  o.theta[2 * (size_t)n + i] = P.t_lo + P.t_span * (d.x2.hi + d.x2.lo);
  o.theta[3 * (size_t)n + i] = 3.14159265358979f * d.u_psi;
  o.theta[4 * (size_t)n + i] = kTwoPi * d.u_phi;
  o.theta[5 * (size_t)n + i] = 2.f * d.c_frac - 1.f;
  o.theta[6 * (size_t)n + i] = d.dist;
  o.lpq[i] = d.lpq;
  if (o.bins) {
    o.bins[0 * (size_t)n + i] = (int)(d.bins & 255u);
    o.bins[1 * (size_t)n + i] = (int)((d.bins >> 8) & 255u);
    o.bins[2 * (size_t)n + i] = (int)((d.bins >> 16) & 255u);
  }
}

// Device-side round update of a batched run (one CTA): accounts the round that just ran
// (evaluations, rounds, the n_eff / max_evals / max_rounds stopping rule of Sec. II.C per
// point), prepares the next round of every active point (cells, chunks, stratified weights,
// table buffer) and lays the points' work items out contiguously (block prefix sum).
__global__ void __launch_bounds__(1024) round_update_kernel(BatchCtl B, PtState *__restrict__ S,
                                                            const AccState *__restrict__ acc,
                                                            RoundPt *__restrict__ rp, RoundCtl *ctl) {
  __shared__ uint32_t sc[1024];
  __shared__ uint32_t sa[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int prev_adapt = ctl->adapt_now;
  const int r = ctl->round + 1;
  const int tabbuf = ctl->tabbuf ^ (prev_adapt ? 1 : 0);
  const int adapt_now = B.adaptive && (B.adapt_rounds < 0 || r < B.adapt_rounds);
  const int per = (B.np + nt - 1) / nt;
  const int p0 = min(B.np, tid * per), p1 = min(B.np, p0 + per);
  const size_t tstride = (size_t)3 * (B.nb + 1), wstride = (size_t)3 * B.nb;
  uint32_t items = 0, active = 0;
  for (int p = p0; p < p1; ++p) {
    RoundPt &R = rp[p];
    PtState &st = S[p];
    if (R.n > 0) {
      if (B.last) B.last[p] = R;
      st.evals += R.n;
      st.rounds += 1;
      const double n_eff = acc[p].s1 + acc[p].c1;
      if (n_eff >= B.n_eff_target || st.evals >= B.max_evals || (B.max_rounds > 0 && st.rounds >= B.max_rounds))
        st.done = 1;
      // fallback of the learned proposal: a learned round whose own draws have n_eff below the
      // threshold (degenerate weights) hands the point to the adaptive sampler for its remaining rounds
      if (!st.done && st.prop == 2 && B.fallback_neff > 0.0 && acc[p].round_neff < B.fallback_neff) {
        st.prop = 1;
        st.fb_round = st.rounds;
      }
    }
    RoundPt N;
    memset(&N, 0, sizeof(N));
    N.ell_off = -1;
    N.dbg_off = -1;
    if (!st.done) {
      const uint32_t n = (uint32_t)min((unsigned long long)B.npr, B.max_evals - st.evals);
      int l0 = st.ls[0], l1 = st.ls[1], l2 = st.ls[2];
      if (st.prop == 2) l0 = l1 = l2 = 0;   // learned rounds are not stratified
      if ((unsigned long long)n < (1ull << (l0 + l1 + l2))) l0 = l1 = l2 = 0;
      const uint32_t C = 1u << (l0 + l1 + l2);
      N.n = n;
      N.ncell = C;
      N.base = n / C;
      N.rem = n % C;
      if (B.tmarg) {   // runs of consecutive draws across cells (chunks unused)
        N.chunks = 0;
        N.nitem = (n + RIFT_TMARG_CHUNK - 1) / RIFT_TMARG_CHUNK;
      } else {
        N.chunks = (N.base + (N.rem ? 1u : 0u) + RIFT_CHUNK - 1) / RIFT_CHUNK;
        N.nitem = C * N.chunks;
      }
      N.round = (uint32_t)st.rounds;
      N.point_id = (B.np == 1) ? B.point_id1 : (uint32_t)p;
      N.ls0 = l0; N.ls1 = l1; N.ls2 = l2;
      N.proposal = st.prop;
      N.nb = B.nb;
      N.lcorr0 = (float)log((double)n / ((double)C * (N.base + 1.0)));
      N.lcorr1 = N.base ? (float)log((double)n / ((double)C * N.base)) : 0.f;
      N.ell_off = (B.adaptive || B.keep_ell) ? (long long)p * B.npr : -1;
      if (N.proposal == 2) N.gmm = B.gmm + (size_t)p * RIFT_GMM_FLOATS;
      N.tmarg = B.tmarg;
      if (B.adaptive) {
        N.tab = B.tables + ((size_t)tabbuf * B.np + p) * tstride;
        N.lnw = B.lnw + ((size_t)tabbuf * B.np + p) * wstride;
      }
      items += N.nitem;
      active += 1;
    }
    R = N;
  }
  sc[tid] = items;
  sa[tid] = active;
  __syncthreads();
  // inclusive scan of the per-thread item counts, total of the active counts
  for (int o = 1; o < nt; o <<= 1) {
    const uint32_t a = (tid >= o) ? sc[tid - o] : 0u;
    const uint32_t b = (tid >= o) ? sa[tid - o] : 0u;
    __syncthreads();
    sc[tid] += a;
    sa[tid] += b;
    __syncthreads();
  }
  uint32_t base = sc[tid] - items;
  for (int p = p0; p < p1; ++p) {
    rp[p].item0 = base;
    base += rp[p].nitem;
  }
  if (tid == nt - 1) {
    ctl->n_items = sc[tid];
    ctl->queue = 0u;
    ctl->active = sa[tid];
    ctl->round = r;
    ctl->adapt_now = adapt_now;
    ctl->tabbuf = tabbuf;
  }
}

// theta5 of harvested samples: for (point p, slot h) re-draw sample idx[p][h] of the point's
// last round and write (ra, sin dec, t, cos incl, ln D) into theta[p][h][0..4].
__global__ void harvest_theta_kernel(CellLaunch L, const RoundPt *__restrict__ last, const int *__restrict__ idx, int H,
                                     float *__restrict__ theta) {
  const int p = blockIdx.y;
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  const RoundPt R = last[p];
  const int i = idx[(size_t)p * H + h];
  float *o = theta + ((size_t)p * H + h) * 5;
  if (i < 0 || R.n == 0) {
    for (int q = 0; q < 5; ++q) o[q] = NAN;
    return;
  }
  const uint32_t big = R.rem * (R.base + 1u);
  const uint32_t cell = ((uint32_t)i < big) ? (uint32_t)i / (R.base + 1u) : R.rem + ((uint32_t)i - big) / R.base;
  const PointC *P = L.pts + p;
  const Drawn d = (R.proposal == 2)
                      ? draw_learned<0>(L.seed, R, (uint32_t)i, R.gmm, P->dref, L.d_lo3, L.d_span3)
                      : draw_cell_sample(L.seed, R, (uint32_t)i, cell, R.tab, R.lnw, P->dref, L.d_lo3, L.d_span3);
  o[0] = kTwoPi * (d.x0.hi + d.x0.lo);
  o[1] = (2.f * d.x1.hi - 1.f) + 2.f * d.x1.lo;
  o[2] = P->t_lo + P->t_span * (d.x2.hi + d.x2.lo);
  o[3] = 2.f * d.c_frac - 1.f;
  o[4] = logf(d.dist);
}

template <int K, int NT, int LEARNED, int TMARG>
cudaError_t cells_kl(const CellLaunch &L, int grid, int block, size_t smem, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(cells_kernel<K, NT, LEARNED, TMARG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, RIFT_CELLS_MAX_DYN_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cells_kernel<K, NT, LEARNED, TMARG><<<grid, block, smem, st>>>(L);
  return cudaGetLastError();
}

template <int K, int NT>
cudaError_t cells_k(const CellLaunch &L, int grid, int block, size_t smem, cudaStream_t st,
                    const CanonCoefParam *cc, int cc_sparse, const MirrorCoefParam *mp) {
  if constexpr (kCanonPath<K, NT>) {
    if (mp && !L.tmarg && !L.learned) {
      static bool attr = false;
      if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(cells_kernel_mp<K, NT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, RIFT_CELLS_MAX_DYN_SMEM);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(cells_kernel_mp<K, NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, RIFT_CELLS_MAX_DYN_SMEM);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(cells_kernel_mp<K, NT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, RIFT_CELLS_MAX_DYN_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
      }
      // all 21 modes: harmonics in registers, and the launch reserves no harmonics buffer (max_M 0);
      // merged rows when all 9 mirror pairs of Q merge
      if (L.max_M == 0 && L.merged) cells_kernel_mp<K, NT, 2><<<grid, block, smem, st>>>(L, *mp);
      else if (L.max_M == 0) cells_kernel_mp<K, NT, 1><<<grid, block, smem, st>>>(L, *mp);
      else cells_kernel_mp<K, NT, 0><<<grid, block, smem, st>>>(L, *mp);
      return cudaGetLastError();
    }
    if (cc && !L.tmarg && !L.learned) {
      static bool attr = false;
      if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(cells_kernel_cp<K, NT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, RIFT_CELLS_MAX_DYN_SMEM);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(cells_kernel_cp<K, NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, RIFT_CELLS_MAX_DYN_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
      }
      if (cc_sparse) cells_kernel_cp<K, NT, 1><<<grid, block, smem, st>>>(L, *cc);
      else cells_kernel_cp<K, NT, 0><<<grid, block, smem, st>>>(L, *cc);
      return cudaGetLastError();
    }
  }
  (void)cc;
  (void)cc_sparse;
  (void)mp;
  if (L.tmarg == 2)
    return L.learned ? cells_kl<K, NT, 1, 2>(L, grid, block, smem, st) : cells_kl<K, NT, 0, 2>(L, grid, block, smem, st);
  if (L.tmarg) return L.learned ? cells_kl<K, NT, 1, 1>(L, grid, block, smem, st) : cells_kl<K, NT, 0, 1>(L, grid, block, smem, st);
  return L.learned ? cells_kl<K, NT, 1, 0>(L, grid, block, smem, st) : cells_kl<K, NT, 0, 0>(L, grid, block, smem, st);
}

template <int K, int NT, int LEARNED, int TMARG>
int cells_occ1(size_t smem, int block) {
  int nb = 0;
  cudaFuncSetAttribute(cells_kernel<K, NT, LEARNED, TMARG>, cudaFuncAttributeMaxDynamicSharedMemorySize, RIFT_CELLS_MAX_DYN_SMEM);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cells_kernel<K, NT, LEARNED, TMARG>, block, smem);
  return nb;
}

template <int K, int NT>
int cells_occ(size_t smem, int block, int tmarg) {
  if (tmarg == 2) return std::min(cells_occ1<K, NT, 0, 2>(smem, block), cells_occ1<K, NT, 1, 2>(smem, block));
  if (tmarg) return std::min(cells_occ1<K, NT, 0, 1>(smem, block), cells_occ1<K, NT, 1, 1>(smem, block));
  const int a = cells_occ1<K, NT, 0, 0>(smem, block), b = cells_occ1<K, NT, 1, 0>(smem, block);
  return a < b ? a : b;
}

}  // namespace

size_t cells_smem_fixed(int K, int max_M, int max_pairK, int max_nb, int block) {
  (void)K;
  size_t off = (sizeof(PointC) + 15) & ~size_t(15);
  off = (off + sizeof(float4) * (size_t)max_pairK + 15) & ~size_t(15);
  if (max_nb > 0) off = (off + sizeof(float) * (size_t)(3 * (max_nb + 1) + 3 * max_nb) + 15) & ~size_t(15);
  off = (off + sizeof(float2) * (size_t)max_M * block + 15) & ~size_t(15);
  return off;
}

#define RIFT_CELLS_DISPATCH(K, NT, CALL)                                        \
  switch ((K) * 8 + (NT)) {                                                     \
    case 1 * 8 + 1: return CALL(1, 1); case 1 * 8 + 2: return CALL(1, 2); case 1 * 8 + 4: return CALL(1, 4); \
    case 2 * 8 + 1: return CALL(2, 1); case 2 * 8 + 2: return CALL(2, 2); case 2 * 8 + 4: return CALL(2, 4); \
    case 3 * 8 + 1: return CALL(3, 1); case 3 * 8 + 2: return CALL(3, 2); case 3 * 8 + 4: return CALL(3, 4); \
    case 4 * 8 + 1: return CALL(4, 1); case 4 * 8 + 2: return CALL(4, 2); case 4 * 8 + 4: return CALL(4, 4); \
    default: break;                                                             \
  }

cudaError_t launch_cells(int K, int ntap, const CellLaunch &L, int grid, int block, size_t smem, cudaStream_t st,
                         const CanonCoefParam *cc, int cc_sparse, const MirrorCoefParam *mp) {
#define RIFT_C(KK, TT) cells_k<KK, TT>(L, grid, block, smem, st, cc, cc_sparse, mp)
  RIFT_CELLS_DISPATCH(K, ntap, RIFT_C)
#undef RIFT_C
  return cudaErrorInvalidValue;
}

int cells_blocks_per_sm(int K, int ntap, size_t smem, int block, int tmarg) {
#define RIFT_O(KK, TT) cells_occ<KK, TT>(smem, block, tmarg)
  RIFT_CELLS_DISPATCH(K, ntap, RIFT_O)
#undef RIFT_O
  return 0;
}

cudaError_t launch_merge_points(const Part *partials, const RoundPt *rp, int n_points, AccState *acc,
                                cudaStream_t st) {
  merge_points_kernel<<<n_points, kMergeThreads, 0, st>>>(partials, rp, acc);
  return cudaGetLastError();
}

cudaError_t launch_hist_points(const float *ell, const uint32_t *bins, const RoundPt *rp, int n_points,
                               const AccState *acc, float beta, int nb, unsigned long long *part, int hblocks,
                               cudaStream_t st) {
  dim3 g(hblocks, n_points);
  hist_points_kernel<<<g, 256, sizeof(unsigned long long) * 3 * nb, st>>>(ell, bins, rp, acc, beta, nb, part,
                                                                           nullptr);
  return cudaGetLastError();
}

cudaError_t launch_tables_points(const unsigned long long *part, int hblocks, const RoundPt *rp, int n_points,
                                 int nb, double floor_eps, float *tables, float *lnw, cudaStream_t st) {
  tables_points_kernel<<<n_points, 256, 0, st>>>(part, hblocks, rp, nb, floor_eps, tables, lnw, nullptr, n_points);
  return cudaGetLastError();
}

cudaError_t launch_round_update(const BatchCtl &B, PtState *st_dev, const AccState *acc, RoundPt *rp, RoundCtl *ctl,
                                cudaStream_t st) {
  round_update_kernel<<<1, 1024, 0, st>>>(B, st_dev, acc, rp, ctl);
  return cudaGetLastError();
}

cudaError_t launch_hist_ctl(const float *ell, const uint32_t *bins, const RoundPt *rp, int n_points,
                            const AccState *acc, float beta, int nb, unsigned long long *part, int hblocks,
                            const RoundCtl *ctl, cudaStream_t st) {
  dim3 g(hblocks, n_points);
  hist_points_kernel<<<g, 256, sizeof(unsigned long long) * 3 * nb, st>>>(ell, bins, rp, acc, beta, nb, part, ctl);
  return cudaGetLastError();
}

cudaError_t launch_tables_ctl(const unsigned long long *part, int hblocks, const RoundPt *rp, int n_points, int nb,
                              double floor_eps, const BatchCtl &B, const RoundCtl *ctl, cudaStream_t st) {
  tables_points_kernel<<<n_points, 256, 0, st>>>(part, hblocks, rp, nb, floor_eps, B.tables, B.lnw, ctl, n_points);
  return cudaGetLastError();
}

cudaError_t launch_harvest_theta(const CellLaunch &L, const RoundPt *last, const int *idx, int H, float *theta,
                                 cudaStream_t st) {
  dim3 g((H + 127) / 128, L.n_points);
  harvest_theta_kernel<<<g, 128, 0, st>>>(L, last, idx, H, theta);
  return cudaGetLastError();
}

cudaError_t launch_draw_cells(const CellLaunch &L, DrawOut o, uint32_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int block = 128;
  const size_t smem = sizeof(float) * (3 * (L.max_nb + 1) + 3 * L.max_nb);
  draw_cells_kernel<<<(n + block - 1) / block, block, smem, st>>>(L, o, n);
  return cudaGetLastError();
}
