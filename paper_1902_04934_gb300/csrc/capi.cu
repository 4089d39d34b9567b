// C ABI of the extrinsic-likelihood library: validation, per-point constants (FP64
// on the host, once per point), device arenas, and the Monte Carlo round loop.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rift_ile.h"
#include "rift_device.cuh"
#include "rift_internal.h"
#include "host_par.h"

namespace {

constexpr double kC = 299792458.0;
constexpr double kPi = 3.14159265358979323846;

// IAU-1982 Greenwich mean sidereal time (radians) at GPS time gps, UT1 ~ UTC = GPS - 18 s.
// GMST[s] = 67310.54841 + (876600 h + 8640184.812866 s) T + 0.093104 T^2 - 6.2e-6 T^3 with
// T = d / 36525, d = JD(UT1) - 2451545.0; the 876600 h term is 86400 s per day exactly.
double gmst_rad(double gps) {
  const double d = (gps - 18.0) / 86400.0 + (2444244.5 - 2451545.0);
  const double T = d / 36525.0;
  double sec = 67310.54841 + 8640184.812866 * T + 0.093104 * T * T - 6.2e-6 * T * T * T;
  sec += 86400.0 * (d - std::floor(d));
  sec = std::fmod(sec, 86400.0);
  if (sec < 0) sec += 86400.0;
  return sec / 86400.0 * 2.0 * kPi;
}

// |x| as the integer bit pattern of an IEEE 754 double: magnitudes compare like their patterns,
// and patterns at or above kInfBits are infinities and NaNs.
constexpr uint64_t kInfBits = 0x7FF0000000000000ull;
inline uint64_t abs_bits(double x) {
  uint64_t u;
  std::memcpy(&u, &x, sizeof u);
  return u & 0x7FFFFFFFFFFFFFFFull;
}
inline double bits_double(uint64_t u) {
  double x;
  std::memcpy(&x, &u, sizeof x);
  return x;
}

void split(double v, float &hi, float &lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

double fact(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}
double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  return fact(n) / (fact(k) * fact(n - k));
}

// -2Y_lm(theta, phi) = e^{i m phi} sum_r coef_r cos(theta/2)^{k_r} sin(theta/2)^{2l-k_r}
// (Goldberg et al. 1967 with spin s = -2, Condon-Shortley phase).
void swsh_terms(int l, int m, ModeC &out) {
  const int s = -2;
  const double pref = ((m & 1) ? -1.0 : 1.0) *
                      std::sqrt(fact(l + m) * fact(l - m) * (2 * l + 1) / (4.0 * kPi * fact(l + s) * fact(l - s)));
  out.l = l; out.m = m; out.nterm = 0; out.pad = 0;
  for (int r = 0; r <= l - s; ++r) {
    const int j = r + s - m;
    if (j < 0 || j > l + s) continue;
    const int k = 2 * r + s - m;
    const double sign = ((l - r - s) & 1) ? -1.0 : 1.0;
    const double c = pref * binom(l - s, r) * binom(l + s, j) * sign;
    if (out.nterm < RIFT_MAXTERM) {
      out.coef[out.nterm] = (float)c;
      out.kc[out.nterm] = k;
      out.nterm++;
    }
  }
}

// The same terms in FP64 (refinement of heavy samples).
void swsh_terms_d(int l, int m, PointD &pd, int a) {
  const int s = -2;
  const double pref = ((m & 1) ? -1.0 : 1.0) *
                      std::sqrt(fact(l + m) * fact(l - m) * (2 * l + 1) / (4.0 * kPi * fact(l + s) * fact(l - s)));
  pd.ml[a] = l; pd.mm[a] = m; pd.nterm[a] = 0;
  for (int r = 0; r <= l - s; ++r) {
    const int j = r + s - m;
    if (j < 0 || j > l + s) continue;
    const double sign = ((l - r - s) & 1) ? -1.0 : 1.0;
    if (pd.nterm[a] < RIFT_MAXTERM) {
      pd.coef[a][pd.nterm[a]] = pref * binom(l - s, r) * binom(l + s, j) * sign;
      pd.kc[a][pd.nterm[a]] = 2 * r + s - m;
      pd.nterm[a]++;
    }
  }
}

// Host-side fault injection for tests of the error paths: RIFT_FAULT names one fault.
//   alloc       device allocation in rift_ile_create fails (before any CUDA call)      -> RIFT_ENOMEM
//   h2d         the host-to-device upload in rift_ile_create fails                     -> RIFT_ECUDA
//   nan_sample  sample 0 of round 0 of every point gets a NaN log weight (excluded from
//               the sums and reported through the status word)                        -> RIFT_ENONFINITE
//   stage_timeout  the cell kernel announces its window copies on the mbarrier but never
//               issues them, so its bounded wait (about 1 s) runs out; the CTA records the
//               timeout, waits once more (bounded), and stops                          -> RIFT_ETIMEOUT
// Nothing here touches device memory out of bounds or traps, and every wait is bounded.
bool fault_is(const char *name) {
  const char *f = std::getenv("RIFT_FAULT");
  return f && std::strcmp(f, name) == 0;
}

struct Point {
  PointC c;
  PointD d;   // FP64 constants (refinement of heavy samples)
  double t_lo, t_hi;
};

}  // namespace

struct rift_ile {
  int n_points = 0;
  int K = 0;
  std::vector<Point> pts;
  PointC *pts_dev = nullptr;
  float2 *q_arena = nullptr;
  float4 *c_arena = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  std::string err;
  // scratch (owned; grown on demand)
  uint32_t *flags = nullptr;
  McScratch sc{};
  size_t cap_items = 0, cap_ebuf = 0, cap_bins = 0, cap_hist = 0, cap_tab = 0, cap_lnw = 0;
  int cap_np = 0;
  float *stage = nullptr;   // lnL_host staging [8][n]
  size_t stage_n = 0;
  int max_M = 0, max_pairK = 0;
  int all_qhalf = 0;        // every point has the half rows of the time quadrature
  // refinement of heavy samples: FP64 point constants and U, V; candidates, scratch, state
  PointD *pd_dev = nullptr;
  double2 *uv64 = nullptr;
  float2 *cand = nullptr;
  size_t cap_cand = 0;
  float *cmax = nullptr;
  size_t cap_cmax = 0;
  unsigned char *rscratch = nullptr;
  size_t cap_rscratch = 0;
  RefineState *rstate = nullptr, *rstate_host = nullptr;
  int cap_rstate = 0;
  int interp = 3;
  int cell_target = 640;    // samples per stratification cell (autotuned)
  int smem_split = 3;       // shared-memory split of the cell kernel (sets the window budget; autotuned)
  // batched runs (graph replays)
  PtState *pst = nullptr;
  RoundCtl *ctl = nullptr;
  RoundCtl *ctl_host = nullptr;
  PtState *pst_host = nullptr;
  int cap_pst = 0;
  cudaStream_t gstream = nullptr;
  int graph_rounds = 4;   // rounds per captured graph
  // the instantiated graph of the last batched run and the launch arguments it was captured with:
  // a call with the same arguments replays it without capturing again
  cudaGraphExec_t gexec = nullptr;
  std::vector<unsigned char> gkey;
  // learned proposal
  double *tau0 = nullptr;     // [np][RIFT_MAXK] Q index origins (s), for the summary
  float *head = nullptr;      // [np][88] network heads (given or computed)
  float *summ = nullptr;      // [np][64]
  float *gmm = nullptr;       // [np][RIFT_GMM_FLOATS]
  float *gcst = nullptr;      // [np][4]
  bool head_given = false;
  RoundPt *last = nullptr;    // [np]
  int *hidx = nullptr;        // harvest indices
  size_t cap_hidx = 0;
  // single-point handle of a three-detector point in the grouped layout: its grouped coefficients,
  // passed to the cell kernel as a parameter
  CanonCoefParam *canon0 = nullptr;
  // or, for a mirror-symmetric point, the coefficients of its positive quadratic form
  MirrorCoefParam *mirror0 = nullptr;
};

namespace {

rift_status fail(rift_ile *h, rift_status s, const std::string &msg) {
  if (h) h->err = msg;
  return s;
}

rift_status cuda_fail(rift_ile *h, cudaError_t e, const char *where) {
  return fail(h, RIFT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RIFT_CK(h, call)                                  \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

// Build the device constants of one point from its descriptor (FP64 on the host).
// Q block of a point in the arena layout [K][T][Mp]: n_det x n_t x (n_modes rounded up to even)
// complex64, or 0 for sizes that the point's validation refuses.
size_t q_block_size(const rift_ile_desc &d) {
  if (d.n_det < 1 || d.n_det > RIFT_MAX_DET || d.n_modes < 1 || d.n_modes > RIFT_MAX_MODES || d.n_t < 4) return 0;
  return (size_t)d.n_det * d.n_t * ((d.n_modes + 1) & ~1);
}

// One point's constants; its Q block is written to qb (q_block_size(*d) entries), which sits at
// entry q_off of the arena.
rift_status build_point(rift_ile *h, const rift_ile_desc *d, Point &P, float2 *qb, long long q_off,
                        std::vector<float4> &cv, std::vector<double2> &uv64) {
  if (!d) return fail(h, RIFT_EINVAL, "null descriptor");
  const int K = d->n_det, M = d->n_modes, T = d->n_t;
  if (K < 1 || K > RIFT_MAX_DET) return fail(h, RIFT_EINVAL, "n_det out of range");
  if (M < 1 || M > RIFT_MAX_MODES) return fail(h, RIFT_EINVAL, "n_modes out of range");
  if (T < 4) return fail(h, RIFT_EINVAL, "n_t < 4");
  if (!d->det_tensor || !d->det_pos || !d->lm || !d->Q || !d->q_t0_gps || !d->U || !d->V)
    return fail(h, RIFT_EINVAL, "null array in descriptor");
  if (!(d->fs > 0) || !(d->d_ref_mpc > 0) || !(d->t_hi > d->t_lo) || !std::isfinite(d->t_ref_gps))
    return fail(h, RIFT_EINVAL, "bad fs, d_ref, t range or t_ref");
  if (d->interp != 0 && d->interp != 1 && d->interp != 3) return fail(h, RIFT_EINVAL, "interp must be 0, 1 or 3");
  PointC &c = P.c;
  std::memset(&c, 0, sizeof(c));
  c.K = K; c.M = M; c.T = T; c.Mp = (M + 1) & ~1; c.npair = M * (M + 1) / 2; c.interp = d->interp;
  c.J = std::max(1, (int)std::floor((d->t_hi - d->t_lo) * d->fs + 1e-9));
  c.fs = (float)d->fs;
  if ((double)c.fs != d->fs) return fail(h, RIFT_EINVAL, "fs must be exactly representable in float32");
  c.dref = (float)d->d_ref_mpc;
  const double g = gmst_rad(d->t_ref_gps) / (2.0 * kPi);
  split(g, c.g_hi, c.g_lo);
  split((d->t_hi - d->t_lo) * d->fs, c.A, c.Alo);
  c.t_lo = (float)d->t_lo;
  c.t_span = (float)(d->t_hi - d->t_lo);
  P.t_lo = d->t_lo; P.t_hi = d->t_hi;
  // modes, stored in canonical (l, m) order: the likelihood is a sum over modes, so the order
  // is free; a fixed order lets the full 2 <= l <= 4 set use compile-time mode tables
  int perm[RIFT_MAX_MODES];   // perm[stored] = index in the caller's arrays
  for (int a = 0; a < M; ++a) {
    const int l = d->lm[2 * a], m = d->lm[2 * a + 1];
    if (l < 2 || l > 4 || m < -l || m > l) return fail(h, RIFT_EINVAL, "mode (l,m) outside 2<=l<=4, |m|<=l");
    for (int b = 0; b < a; ++b)
      if (d->lm[2 * b] == l && d->lm[2 * b + 1] == m) return fail(h, RIFT_EINVAL, "duplicate mode");
    perm[a] = a;
  }
  std::sort(perm, perm + M, [&](int x, int y) {
    const int lx = d->lm[2 * x], ly = d->lm[2 * y];
    return lx != ly ? lx < ly : d->lm[2 * x + 1] < d->lm[2 * y + 1];
  });
  for (int a = 0; a < M; ++a) {
    swsh_terms(d->lm[2 * perm[a]], d->lm[2 * perm[a] + 1], c.mode[a]);
    c.canon_mask |= 1u << canon_index(c.mode[a].l, c.mode[a].m);
  }
  for (int j = 0; j < RIFT_MAXM; ++j) {
    ModeC t;
    swsh_terms(canon_l(j), canon_m(j), t);
    if (t.nterm != canon_rmax(j) - canon_rmin(j) + 1) return fail(h, RIFT_EINVAL, "internal: harmonic table");
    for (int r = 0; r < t.nterm; ++r) c.ccoef[j][r] = t.coef[r];
  }
  // detectors; taps of the interpolation rule around floor(s)
  const int lo_tap = (d->interp == 3) ? 1 : 0, hi_tap = (d->interp == 3) ? 2 : (d->interp == 1 ? 1 : 0);
  for (int k = 0; k < K; ++k) {
    const double *t = d->det_tensor + 9 * k;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        if (std::fabs(t[3 * i + j] - t[3 * j + i]) > 1e-12 * (1.0 + std::fabs(t[3 * i + j])))
          return fail(h, RIFT_EINVAL, "detector tensor not symmetric");
    DetC &D = c.det[k];
    D.d[0] = (float)t[0]; D.d[1] = (float)t[1]; D.d[2] = (float)t[2];
    D.d[3] = (float)t[4]; D.d[4] = (float)t[5]; D.d[5] = (float)t[8];
    const double *x = d->det_pos + 3 * k;
    for (int i = 0; i < 3; ++i) split(d->fs * x[i] / kC, D.P[i], D.Plo[i]);
    const double tau0 = d->q_t0_gps[k] - d->t_ref_gps;
    if (!std::isfinite(tau0)) return fail(h, RIFT_EINVAL, "non-finite q_t0_gps");
    split((d->t_lo - tau0) * d->fs, D.c0, D.c0lo);
    split(-tau0 * d->fs, D.ct, D.ctlo);
    // window coverage: the index s = (t + delay - tau0) fs over the prior and the sky
    const double dmax = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]) / kC;
    const double smin = (d->t_lo - dmax - tau0) * d->fs, smax = (d->t_hi + dmax - tau0) * d->fs;
    const double guard = 1e-3;
    if (d->interp == 0) {
      if (smin - 0.5 < -guard || smax + 0.5 > T - 1 + 0.5 - guard)
        return fail(h, RIFT_EWINDOW, "Q window does not cover t range + time of flight (detector " +
                                         std::to_string(k) + ")");
    } else if (std::floor(smin - guard) - lo_tap < 0 || std::floor(smax + guard) + hi_tap > T - 1) {
      return fail(h, RIFT_EWINDOW, "Q window does not cover t range + time of flight + taps (detector " +
                                       std::to_string(k) + ")");
    }
  }
  // U Hermitian, V symmetric
  double umax = 0.0, vmax = 0.0;
  for (int i = 0; i < K * M * M * 2; ++i) {
    umax = std::max(umax, std::fabs(d->U[i]));
    vmax = std::max(vmax, std::fabs(d->V[i]));
  }
  for (int k = 0; k < K; ++k)
    for (int a = 0; a < M; ++a)
      for (int b = 0; b < M; ++b) {
        const double *u1 = d->U + 2 * ((k * M + a) * M + b), *u2 = d->U + 2 * ((k * M + b) * M + a);
        const double *v1 = d->V + 2 * ((k * M + a) * M + b), *v2 = d->V + 2 * ((k * M + b) * M + a);
        if (std::fabs(u1[0] - u2[0]) > 1e-10 * umax || std::fabs(u1[1] + u2[1]) > 1e-10 * umax)
          return fail(h, RIFT_EINVAL, "U is not Hermitian");
        if (std::fabs(v1[0] - v2[0]) > 1e-10 * vmax || std::fabs(v1[1] - v2[1]) > 1e-10 * vmax)
          return fail(h, RIFT_EINVAL, "V is not symmetric");
      }
  // mirror pairs (a, b) of stored modes, m_a > 0 and b = (l_a, -m_a), for the merged rows below:
  // their largest deviations from Q_b = conj(Q_a) (dev_p) and from Q_b = -conj(Q_a) (dev_m) over
  // every detector and time are taken in the conversion pass
  int pa[RIFT_MAXM], pb[RIFT_MAXM], npr = 0;
  for (int a = 0; a < M; ++a) {
    if (c.mode[a].m <= 0) continue;
    for (int e = 0; e < M; ++e)
      if (c.mode[e].l == c.mode[a].l && c.mode[e].m == -c.mode[a].m) { pa[npr] = a; pb[npr] = e; ++npr; }
  }
  // Q arena block: [K][T][Mp] complex64, the pad column (odd M) zero; converted in tasks of 64
  // times of one detector, in parallel over host threads, so that the rows written stay in cache.
  // Magnitudes are compared as the integer bit patterns of |x| (ordered like |x|; at or above
  // kInfBits for an infinity or a NaN), so the largest |Q| and the finiteness check are one maximum
  c.q_off = q_off;
  constexpr int kParts = 8;
  struct QPart {
    uint64_t mx = 0, dp[RIFT_MAXM] = {}, dm[RIFT_MAXM] = {};
  };
  QPart qp[kParts];
  const int nblk = (T + 63) / 64;
  parallel_parts(K * nblk, 8, kParts, [&](int part, int task0, int task1) {
    QPart &r = qp[part];
    for (int task = task0; task < task1; ++task) {
      const int k = task / nblk, j0 = (task % nblk) * 64, j1 = std::min(T, j0 + 64);
      uint64_t mx = r.mx;
      for (int a = 0; a < M; ++a) {
        const double *q = d->Q + 2 * (((size_t)k * M + perm[a]) * T);
        float2 *outq = qb + (size_t)k * T * c.Mp + a;
        for (int j = j0; j < j1; ++j) {
          const double re = q[2 * j], im = q[2 * j + 1];
          mx = std::max(mx, std::max(abs_bits(re), abs_bits(im)));
          outq[(size_t)j * c.Mp] = make_float2((float)re, (float)im);
        }
      }
      r.mx = mx;
      if (c.Mp > M)
        for (int j = j0; j < j1; ++j) qb[((size_t)k * T + j) * c.Mp + M] = make_float2(0.f, 0.f);
      for (int p = 0; p < npr; ++p) {
        const double *qa = d->Q + 2 * (((size_t)k * M + perm[pa[p]]) * T);
        const double *qm = d->Q + 2 * (((size_t)k * M + perm[pb[p]]) * T);
        uint64_t dp = r.dp[p], dm = r.dm[p];
        for (int j = j0; j < j1; ++j) {
          const double ar = qa[2 * j], ai = qa[2 * j + 1], br = qm[2 * j], bi = qm[2 * j + 1];
          dp = std::max(dp, std::max(abs_bits(br - ar), abs_bits(bi + ai)));
          dm = std::max(dm, std::max(abs_bits(br + ar), abs_bits(bi - ai)));
        }
        r.dp[p] = dp;
        r.dm[p] = dm;
      }
    }
  });
  uint64_t qmax_bits = 0, dpb[RIFT_MAXM] = {}, dmb[RIFT_MAXM] = {};
  for (int t = 0; t < kParts; ++t) {
    qmax_bits = std::max(qmax_bits, qp[t].mx);
    for (int p = 0; p < npr; ++p) {
      dpb[p] = std::max(dpb[p], qp[t].dp[p]);
      dmb[p] = std::max(dmb[p], qp[t].dm[p]);
    }
  }
  if (qmax_bits >= kInfBits) return fail(h, RIFT_EINVAL, "non-finite Q");
  const double qmax = bits_double(qmax_bits);
  // FP64 constants and U, V (stored mode order) for the refinement of heavy samples
  {
    PointD &D = P.d;
    std::memset(&D, 0, sizeof(D));
    D.K = K; D.M = M; D.T = T; D.Mp = c.Mp; D.interp = d->interp;
    D.q_off = c.q_off;
    D.g = gmst_rad(d->t_ref_gps) / (2.0 * kPi);
    D.A = (d->t_hi - d->t_lo) * d->fs;
    D.t_lo = d->t_lo; D.t_span = d->t_hi - d->t_lo; D.fs = d->fs; D.dref = d->d_ref_mpc;
    for (int k = 0; k < K; ++k) {
      const double *t = d->det_tensor + 9 * k;
      D.d[k][0] = t[0]; D.d[k][1] = t[1]; D.d[k][2] = t[2]; D.d[k][3] = t[4]; D.d[k][4] = t[5]; D.d[k][5] = t[8];
      for (int i = 0; i < 3; ++i) D.P[k][i] = d->fs * d->det_pos[3 * k + i] / kC;
      D.c0[k] = (d->t_lo - (d->q_t0_gps[k] - d->t_ref_gps)) * d->fs;
    }
    for (int a = 0; a < M; ++a) swsh_terms_d(d->lm[2 * perm[a]], d->lm[2 * perm[a] + 1], D, a);
    D.uv_off = (long long)uv64.size();
    uv64.resize(uv64.size() + (size_t)2 * K * M * M);
    double2 *u = uv64.data() + D.uv_off;
    for (int w = 0; w < 2; ++w)
      for (int k = 0; k < K; ++k)
        for (int a = 0; a < M; ++a)
          for (int b = 0; b < M; ++b) {
            const double *x = (w ? d->V : d->U) + 2 * ((k * M + perm[a]) * M + perm[b]);
            u[(((size_t)w * K + k) * M + a) * M + b] = make_double2(x[0], x[1]);
          }
  }
  // merged rows for the time quadrature (tgrid_scan_half): for real data and modes with
  // conj(h_a(-f)) = sigma_a h_abar(f), Eq. (QUV) gives Q_abar(t) = sigma_a conj(Q_a(t)); each pair
  // (a, abar), m > 0, present with that relation at every sample (checked on the FP64 inputs to
  // 1e-10 of the largest |Q|) is read from the row of a alone.  The slots are the stored modes
  // but the merged m < 0 ones, in stored order; taken when at least one pair merges
  {
    const double tol = 1e-10 * qmax;
    int mate[RIFT_MAXM], sg[RIFT_MAXM];   // mate[a]: the merged partner's stored index, else a
    int merged = 0;
    for (int a = 0; a < M; ++a) { mate[a] = a; sg[a] = 1; }
    for (int p = 0; p < npr; ++p) {
      const int sv = bits_double(dpb[p]) <= tol ? 1 : (bits_double(dmb[p]) <= tol ? -1 : 0);
      if (!sv) continue;
      mate[pa[p]] = pb[p];
      mate[pb[p]] = pa[p];
      sg[pa[p]] = sv;
      ++merged;
    }
    int Mh = 0;
    for (int a = 0; a < M; ++a)
      if (!(c.mode[a].m < 0 && mate[a] != a)) ++Mh;
    if (merged > 0 && Mh <= RIFT_MAXMH) {
      Mh = 0;
      for (int a = 0; a < M; ++a) {
        if (c.mode[a].m < 0 && mate[a] != a) continue;
        c.h_a[Mh] = (unsigned char)a;
        c.h_b[Mh] = (unsigned char)mate[a];
        if (sg[a] < 0) c.h_neg |= 1u << Mh;
        ++Mh;
      }
      // the rows themselves are gathered on the device from the uploaded Q block (create_impl
      // places the merged blocks after all points' Q blocks and sets qh_rel)
      c.qhalf = 1;
      c.Mh = Mh;
      c.Mhp = (Mh + 1) & ~1;
    }
  }
  // pair coefficients [pair_slot(a, b)][K] = (U, V) upper triangle, off-diagonal doubled
  c.uv_off = (long long)cv.size();
  cv.resize(cv.size() + (size_t)c.npair * K);
  for (int a = 0; a < M; ++a)
    for (int b = a; b < M; ++b)
      for (int k = 0; k < K; ++k) {
        const double f = (a == b) ? 1.0 : 2.0;
        const int ua = perm[a], ub = perm[b];
        const double *u = d->U + 2 * ((k * M + ua) * M + ub), *v = d->V + 2 * ((k * M + ua) * M + ub);
        cv[c.uv_off + (size_t)pair_slot(a, b, M) * K + k] =
            make_float4((float)(f * u[0]), (float)(f * u[1]), (float)(f * v[0]), (float)(f * v[1]));
      }
  c.coef_off = c.uv_off;
  c.ncoef = c.npair * K;
  // the grouped quadratic form (compiled for three detectors with cubic taps, kCanonPath) over the
  // 21 canonical modes, absent modes with zero coefficients; it pays from kCanonMinModes on
  c.grouped = (K == 3 && d->interp == 3 && M >= kCanonMinModes) ? 1 : 0;
  if (c.grouped) {
    // grouped layout of quad_canon: [U part | V part][slot][k], two pairs per float4; modes are
    // stored in canonical order, so a present canonical mode j is stored at the number of present
    // modes before it
    int stored[RIFT_MAXM];
    for (int j = 0; j < RIFT_MAXM; ++j)
      stored[j] = (c.canon_mask >> j & 1u) ? __builtin_popcount(c.canon_mask & ((1u << j) - 1u)) : -1;
    c.coef_off = (long long)cv.size();
    c.ncoef = 2 * kCanonSlots * K;
    cv.resize(cv.size() + (size_t)c.ncoef, make_float4(0.f, 0.f, 0.f, 0.f));
    float *g = reinterpret_cast<float *>(cv.data() + c.coef_off);
    for (int part = 0; part < 2; ++part)
      for (int i = 0; i < kCanonPairs; ++i) {
        const int code = part ? canon_pair_B(i) : canon_pair_A(i);
        const int ja = (code >> 5) & 31, jb = code & 31;
        const int a = stored[ja], b = stored[jb];
        if (a < 0 || b < 0) continue;   // an absent mode: zero coefficient
        const bool conj = !part && canon_m(jb) < canon_m(ja);
        for (int k = 0; k < K; ++k) {
          const float4 pc = cv[c.uv_off + (size_t)pair_slot(a, b, M) * K + k];
          float *o = g + 4 * ((size_t)(part * kCanonSlots + i / 2) * K + k) + 2 * (i & 1);
          o[0] = part ? pc.z : pc.x;
          o[1] = part ? pc.w : (conj ? -pc.y : pc.y);
        }
      }
    // modes on one sign of frequency each (non-precessing): U vanishes between opposite-sign m,
    // V between same-sign m; checked exactly, so skipping those pairs changes no bit
    c.canon_sparse = 1;
    for (int a = 0; a < M && c.canon_sparse; ++a)
      for (int b = a; b < M; ++b) {
        const int mm = c.mode[a].m * c.mode[b].m;
        if (mm == 0) continue;
        for (int k = 0; k < K; ++k) {
          const float4 pc = cv[c.uv_off + (size_t)pair_slot(a, b, M) * K + k];
          if ((mm < 0 && (pc.x != 0.f || pc.y != 0.f)) || (mm > 0 && (pc.z != 0.f || pc.w != 0.f))) c.canon_sparse = 0;
        }
      }
    // reflection symmetry of non-precessing modes (quad_mirror): every mode's mirror present,
    // conj(h_a(-f)) = sigma_a h_abar(f), read off the inputs as V_ab = sigma_a U_{abar b} for all b,
    // with U zero between opposite-sign m and U_{abar bbar} = sigma_a sigma_b conj(U_ab); checked
    // to 1e-10 of the largest |U|, |V| (FP64 inputs), so the positive form equals the general one
    int mir[RIFT_MAXM];
    bool ok = true;
    for (int a = 0; a < M && ok; ++a) {
      mir[a] = -1;
      for (int b = 0; b < M; ++b)
        if (c.mode[b].l == c.mode[a].l && c.mode[b].m == -c.mode[a].m) mir[a] = b;
      ok = mir[a] >= 0;
    }
    const double tol = 1e-10 * std::max(umax, vmax);
    // U, V of stored modes (a, b) of detector k
    auto Uab = [&](int k, int a, int b, int comp) { return d->U[2 * ((k * M + perm[a]) * M + perm[b]) + comp]; };
    auto Vab = [&](int k, int a, int b, int comp) { return d->V[2 * ((k * M + perm[a]) * M + perm[b]) + comp]; };
    int sig[RIFT_MAXM];
    for (int a = 0; a < M && ok; ++a) {
      sig[a] = 0;
      for (int sv = 1; sv >= -1 && !sig[a]; sv -= 2) {
        bool match = true;
        for (int k = 0; k < K && match; ++k)
          for (int b = 0; b < M && match; ++b)
            match = std::fabs(Vab(k, a, b, 0) - sv * Uab(k, mir[a], b, 0)) <= tol &&
                    std::fabs(Vab(k, a, b, 1) - sv * Uab(k, mir[a], b, 1)) <= tol;
        if (match) sig[a] = sv;
      }
      ok = sig[a] != 0;
    }
    for (int a = 0; a < M && ok; ++a) {
      ok = sig[mir[a]] == sig[a];
      for (int b = 0; b < M && ok; ++b)
        for (int k = 0; k < K && ok; ++k) {
          if ((long long)c.mode[a].m * c.mode[b].m < 0)
            ok = std::fabs(Uab(k, a, b, 0)) <= tol && std::fabs(Uab(k, a, b, 1)) <= tol;
          else
            ok = std::fabs(Uab(k, mir[a], mir[b], 0) - sig[a] * sig[b] * Uab(k, a, b, 0)) <= tol &&
                 std::fabs(Uab(k, mir[a], mir[b], 1) + sig[a] * sig[b] * Uab(k, a, b, 1)) <= tol;
        }
    }
    if (ok) {
      c.mirror = 1;
      c.sigma_neg = 0u;
      int stored[RIFT_MAXM];
      for (int j = 0; j < RIFT_MAXM; ++j)
        stored[j] = (c.canon_mask >> j & 1u) ? __builtin_popcount(c.canon_mask & ((1u << j) - 1u)) : -1;
      for (int j = 0; j < RIFT_MAXM; ++j)
        if (stored[j] >= 0 && sig[stored[j]] < 0) c.sigma_neg |= 1u << j;
      c.coef_off = (long long)cv.size();
      c.ncoef = (kMirrorPairs * K + 1) / 2;
      cv.resize(cv.size() + (size_t)c.ncoef, make_float4(0.f, 0.f, 0.f, 0.f));
      float2 *g = reinterpret_cast<float2 *>(cv.data() + c.coef_off);
      for (int i = 0; i < kMirrorPairs; ++i) {
        const int code = mirror_pair(i);
        const int ja = (code >> 5) & 31, jb = code & 31;
        const int a = stored[ja], b = stored[jb];
        if (a < 0 || b < 0) continue;   // absent modes (their mirrors are absent too): zero
        const double w = mirror_weight(ja, jb);
        for (int k = 0; k < K; ++k)
          g[(size_t)i * K + k] = make_float2((float)(w * Uab(k, a, b, 0)), (float)(w * Uab(k, a, b, 1)));
      }
    }
  }
  return RIFT_OK;
}

template <typename T>
rift_status grow(rift_ile *h, T *&p, size_t &cap, size_t need) {
  if (need <= cap) return RIFT_OK;
  if (p) cache_dev_free(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cache_dev_alloc((void **)&p, sizeof(T) * need);
  if (e != cudaSuccess) return fail(h, e == cudaErrorMemoryAllocation ? RIFT_ENOMEM : RIFT_ECUDA,
                                    std::string("scratch allocation: ") + cudaGetErrorString(e));
  cap = need;
  return RIFT_OK;
}

// Device scratch of the Monte Carlo runner for np points, max_items cells per round,
// ebuf per-sample slots (adaptive), nb bins and hb histogram blocks per point.
rift_status ensure_scratch(rift_ile *h, int np, size_t max_items, size_t ebuf, int nb, int hb) {
  McScratch &S = h->sc;
  rift_status s;
  if (np > h->cap_np) {
    cache_dev_free(S.acc); cache_dev_free(S.rp); cache_dev_free(S.counters);
    cache_host_free(S.rp_host); cache_host_free(S.acc_host);
    S.acc = nullptr; S.rp = nullptr; S.counters = nullptr; S.rp_host = nullptr; S.acc_host = nullptr;
    h->cap_np = 0;
    cudaError_t e;
    if ((e = cache_dev_alloc((void **)&S.acc, sizeof(AccState) * np)) != cudaSuccess ||
        (e = cache_dev_alloc((void **)&S.rp, sizeof(RoundPt) * np)) != cudaSuccess ||
        (e = cache_dev_alloc((void **)&S.counters, sizeof(uint32_t) * 2)) != cudaSuccess ||
        (e = cache_host_alloc((void **)&S.rp_host, sizeof(RoundPt) * np)) != cudaSuccess ||
        (e = cache_host_alloc((void **)&S.acc_host, sizeof(AccState) * np)) != cudaSuccess)
      return fail(h, RIFT_ENOMEM, std::string("scratch allocation: ") + cudaGetErrorString(e));
    h->cap_np = np;
  }
  if ((s = grow(h, S.partials, h->cap_items, max_items)) != RIFT_OK) return s;
  if (ebuf) {
    if ((s = grow(h, S.ell, h->cap_ebuf, ebuf)) != RIFT_OK) return s;
    if ((s = grow(h, S.bins, h->cap_bins, ebuf)) != RIFT_OK) return s;
  }
  if (nb > 0) {
    if ((s = grow(h, S.hist, h->cap_hist, (size_t)np * hb * 3 * nb)) != RIFT_OK) return s;
    if ((s = grow(h, S.tables, h->cap_tab, (size_t)2 * np * 3 * (RIFT_MAXBINS + 1))) != RIFT_OK) return s;
    if ((s = grow(h, S.lnw, h->cap_lnw, (size_t)2 * np * 3 * RIFT_MAXBINS)) != RIFT_OK) return s;
  }
  S.max_items = h->cap_items;
  S.hblocks = hb;
  return RIFT_OK;
}

// Refinement of heavy samples: candidate and scratch buffers for np points and max_items work
// items per round, and each point's state reset (no correction yet).
rift_status ensure_refine(rift_ile *h, int np, size_t max_items, cudaStream_t st) {
  rift_status s;
  if ((s = grow(h, h->cand, h->cap_cand, max_items * RIFT_CAND_PER_ITEM)) != RIFT_OK) return s;
  if ((s = grow(h, h->cmax, h->cap_cmax, max_items)) != RIFT_OK) return s;
  if ((s = grow(h, h->rscratch, h->cap_rscratch, refine_scratch_bytes(np))) != RIFT_OK) return s;
  if (np > h->cap_rstate) {
    cache_dev_free(h->rstate);
    cache_host_free(h->rstate_host);
    h->rstate = nullptr;
    h->rstate_host = nullptr;
    h->cap_rstate = 0;
    cudaError_t e;
    if ((e = cache_dev_alloc((void **)&h->rstate, sizeof(RefineState) * np)) != cudaSuccess ||
        (e = cache_host_alloc((void **)&h->rstate_host, sizeof(RefineState) * np)) != cudaSuccess)
      return fail(h, RIFT_ENOMEM, std::string("scratch allocation: ") + cudaGetErrorString(e));
    h->cap_rstate = np;
  }
  for (int p = 0; p < np; ++p) {
    std::memset(&h->rstate_host[p], 0, sizeof(RefineState));
    h->rstate_host[p].mref = -INFINITY;
  }
  RIFT_CK(h, cudaMemcpyAsync(h->rstate, h->rstate_host, sizeof(RefineState) * np, cudaMemcpyHostToDevice, st));
  return RIFT_OK;
}

// Host staging of create(): pinned memory from the buffer cache up to kPinnedStageMax bytes,
// pageable beyond.  Pinned memory goes back to the cache only once the stream that reads it has
// drained (sync_on names that stream).
constexpr size_t kPinnedStageMax = size_t(256) << 20;
struct HostStage {
  unsigned char *p = nullptr;
  bool pinned = false;
  cudaStream_t st = nullptr;
  bool reading = false;
  std::vector<unsigned char> pageable;
  cudaError_t get(size_t bytes) {
    if (bytes <= kPinnedStageMax) {
      void *q = nullptr;
      cudaError_t e = cache_host_alloc(&q, bytes);
      if (e == cudaSuccess) {
        p = static_cast<unsigned char *>(q);
        pinned = true;
        return e;
      }
      cudaGetLastError();
    }
    try {
      pageable.resize(bytes);
    } catch (...) {
      return cudaErrorMemoryAllocation;
    }
    p = pageable.data();
    return cudaSuccess;
  }
  void sync_on(cudaStream_t s) { st = s; reading = true; }
  void release() {
    if (pinned && p) {
      if (reading) cudaStreamSynchronize(st);
      cache_host_free(p);
    }
    p = nullptr;
    pinned = false;
  }
  ~HostStage() { release(); }
};

// Time origins tau0 = q_t0_gps - t_ref_gps of every point's detectors, [n][RIFT_MAX_DET] (FP64).
const double *fill_tau0(const rift_ile_desc *descs, int n, double *t0) {
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < RIFT_MAX_DET; ++k)
      t0[(size_t)i * RIFT_MAX_DET + k] = k < descs[i].n_det ? descs[i].q_t0_gps[k] - descs[i].t_ref_gps : 0.0;
  return t0;
}

rift_status create_impl(const rift_ile_desc *descs, int n, rift_ile **out) {
  if (!out) return RIFT_EINVAL;
  *out = nullptr;
  if (!descs || n < 1) return RIFT_EINVAL;
  host_par::Pool::get().wake();   // the Q conversion below runs on the worker pool
  rift_ile *h = new (std::nothrow) rift_ile();
  if (!h) return RIFT_ENOMEM;
  h->n_points = n;
  h->K = descs[0].n_det;
  h->interp = descs[0].interp;
  h->stream = (cudaStream_t)descs[0].cuda_stream;
  std::vector<float4> cv;
  std::vector<double2> uv64;
  // host copy of the arena's Q blocks followed by the points' time origins tau0: pinned (from the
  // buffer cache), so the upload is one asynchronous DMA, up to kPinnedStageMax bytes; pageable
  // beyond that (large batches)
  std::vector<long long> qoff(n);
  size_t qtot = 0;
  for (int i = 0; i < n; ++i) {
    qoff[i] = (long long)qtot;
    qtot += q_block_size(descs[i]);
  }
  HostStage stage;
  const size_t q_bytes = sizeof(float2) * std::max<size_t>(qtot, 2);
  if (stage.get(q_bytes + sizeof(double) * (size_t)n * RIFT_MAX_DET) != cudaSuccess) {
    rift_status s = fail(h, RIFT_ENOMEM, "host staging buffer");
    rift_ile_destroy(h);
    return s;
  }
  float2 *qh = reinterpret_cast<float2 *>(stage.p);
  double *t0h = reinterpret_cast<double *>(stage.p + q_bytes);
  h->pts.resize(n);
  for (int i = 0; i < n; ++i) {
    if (descs[i].n_det != h->K) { rift_status s = fail(h, RIFT_EINVAL, "points differ in n_det"); rift_ile_destroy(h); return s; }
    rift_status s = build_point(h, &descs[i], h->pts[i], qh + qoff[i], qoff[i], cv, uv64);
    if (s != RIFT_OK) {
      fprintf(stderr, "rift_ile_create: point %d: %s\n", i, h->err.c_str());
      rift_ile_destroy(h);
      return s;
    }
    h->max_M = std::max(h->max_M, h->pts[i].c.M);
    h->max_pairK = std::max(h->max_pairK, h->pts[i].c.ncoef);
    h->all_qhalf = (i == 0 || h->all_qhalf) && h->pts[i].c.qhalf;
    if (descs[i].interp != descs[0].interp) {
      rift_status s2 = fail(h, RIFT_EINVAL, "points differ in interp");
      rift_ile_destroy(h);
      return s2;
    }
  }
  if (n == 1 && h->pts[0].c.grouped && h->pts[0].c.mirror) {
    h->mirror0 = new (std::nothrow) MirrorCoefParam;
    if (!h->mirror0) { rift_status s1 = fail(h, RIFT_ENOMEM, "host allocation"); rift_ile_destroy(h); return s1; }
    std::memcpy(h->mirror0->g, cv.data() + h->pts[0].c.coef_off, sizeof(h->mirror0->g));
  } else if (n == 1 && h->pts[0].c.grouped) {
    h->canon0 = new (std::nothrow) CanonCoefParam;
    if (!h->canon0) { rift_status s1 = fail(h, RIFT_ENOMEM, "host allocation"); rift_ile_destroy(h); return s1; }
    std::memcpy(h->canon0->g, cv.data() + h->pts[0].c.coef_off, sizeof(h->canon0->g));
  }
  if (fault_is("alloc")) {
    rift_status s0 = fail(h, RIFT_ENOMEM, "injected fault: device allocation failed");
    fprintf(stderr, "rift_ile_create: %s\n", h->err.c_str());
    rift_ile_destroy(h);
    return s0;
  }
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess) {
    fprintf(stderr, "rift_ile_create: %s\n", cudaGetErrorString(e));
    rift_ile_destroy(h);
    return RIFT_ECUDA;
  }
  // merged-row blocks after all Q blocks (16-byte aligned: every block holds an even number of rows
  // of an even width); only the Q blocks travel from the host
  size_t qmerged = 0;
  for (int i = 0; i < n; ++i) {
    PointC &c = h->pts[i].c;
    if (!c.qhalf) continue;
    c.qh_rel = (long long)(qtot + qmerged) - c.q_off;
    qmerged += (size_t)c.K * c.T * c.Mhp;
  }
  // the per-point constants and coefficients in a second staging buffer (sizes known only now)
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t b_pc = sizeof(PointC) * n, b_pd = sizeof(PointD) * n, b_cv = sizeof(float4) * cv.size(),
               b_uv = sizeof(double2) * uv64.size();
  HostStage small;
  if (small.get(al(b_pc) + al(b_pd) + al(b_cv) + al(b_uv)) != cudaSuccess) {
    rift_status s1 = fail(h, RIFT_ENOMEM, "host staging buffer");
    rift_ile_destroy(h);
    return s1;
  }
  PointC *pc = reinterpret_cast<PointC *>(small.p);
  PointD *pdv = reinterpret_cast<PointD *>(small.p + al(b_pc));
  float4 *cvh = reinterpret_cast<float4 *>(small.p + al(b_pc) + al(b_pd));
  double2 *uvh = reinterpret_cast<double2 *>(small.p + al(b_pc) + al(b_pd) + al(b_cv));
  for (int i = 0; i < n; ++i) { pc[i] = h->pts[i].c; pdv[i] = h->pts[i].d; }
  if (b_cv) std::memcpy(cvh, cv.data(), b_cv);
  if (b_uv) std::memcpy(uvh, uv64.data(), b_uv);
  rift_status s = RIFT_OK;
  stage.sync_on(h->stream);   // the copies below read the staging buffers
  small.sync_on(h->stream);
  if ((e = cache_dev_alloc((void **)&h->pts_dev, sizeof(PointC) * n)) != cudaSuccess ||
      (e = cache_dev_alloc((void **)&h->q_arena, sizeof(float2) * std::max<size_t>(qtot + qmerged, 2))) != cudaSuccess ||
      (e = cache_dev_alloc((void **)&h->c_arena, sizeof(float4) * std::max<size_t>(cv.size(), 1))) != cudaSuccess ||
      (e = cache_dev_alloc((void **)&h->flags, sizeof(uint32_t))) != cudaSuccess ||
      (e = fault_is("h2d") ? cudaErrorInvalidValue : cudaSuccess) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->pts_dev, pc, b_pc, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->q_arena, qh, sizeof(float2) * qtot, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->c_arena, cvh, b_cv, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
      (e = qmerged ? launch_merge_rows(h->pts_dev, n, h->q_arena, h->stream) : cudaSuccess) != cudaSuccess ||
      (e = cache_dev_alloc((void **)&h->pd_dev, sizeof(PointD) * n)) != cudaSuccess ||
      (e = cache_dev_alloc((void **)&h->uv64, sizeof(double2) * std::max<size_t>(uv64.size(), 1))) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->pd_dev, pdv, b_pd, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->uv64, uvh, b_uv, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->flags, 0, sizeof(uint32_t), h->stream)) != cudaSuccess ||
      (e = cache_dev_alloc((void **)&h->tau0, sizeof(double) * (size_t)n * RIFT_MAX_DET)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->tau0, fill_tau0(descs, n, t0h), sizeof(double) * (size_t)n * RIFT_MAX_DET,
                           cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
    s = (e == cudaErrorMemoryAllocation) ? RIFT_ENOMEM : RIFT_ECUDA;
    fprintf(stderr, "rift_ile_create: %s\n", cudaGetErrorString(e));
    stage.release();   // after the handle's stream has drained
    small.release();
    rift_ile_destroy(h);
    return s;
  }
  *out = h;
  return RIFT_OK;
}

rift_status check_opts(rift_ile *h, const rift_mc_opts *o) {
  if (!o) return fail(h, RIFT_EINVAL, "null options");
  if (o->n_per_round == 0 || o->max_evals == 0) return fail(h, RIFT_EINVAL, "n_per_round and max_evals must be > 0");
  if (!(o->d_lo > 0) || !(o->d_hi > o->d_lo)) return fail(h, RIFT_EINVAL, "need 0 < d_lo < d_hi");
  if (o->proposal == RIFT_PROPOSAL_ADAPTIVE) {
    if (o->n_bins < 2 || o->n_bins > RIFT_MAXBINS) return fail(h, RIFT_EINVAL, "n_bins out of range [2, 256]");
    if (!(o->beta > 0) || !(o->floor_eps > 0) || !(o->floor_eps <= 1)) return fail(h, RIFT_EINVAL, "bad beta / floor_eps");
    if (o->tables) {
      const int sets = o->tables_per_point ? h->n_points : 1;
      for (int q = 0; q < 3 * sets; ++q) {
        const float *c = o->tables + (size_t)q * (o->n_bins + 1);
        if (c[0] != 0.f || c[o->n_bins] != 1.f) return fail(h, RIFT_EINVAL, "tables must start at 0 and end at 1");
        for (int b = 0; b < o->n_bins; ++b)
          if (!(c[b + 1] > c[b])) return fail(h, RIFT_EINVAL, "tables must be strictly increasing");
      }
    }
  } else if (o->proposal == RIFT_PROPOSAL_LEARNED) {
    if (!o->mdn && !h->head_given)
      return fail(h, RIFT_EINVAL, "learned proposal needs opts.mdn or rift_ile_set_proposal_head");
    if (o->fallback_neff > 0.0) {   // the adaptive sampler it falls back to
      if (o->n_bins < 2 || o->n_bins > RIFT_MAXBINS) return fail(h, RIFT_EINVAL, "n_bins out of range [2, 256]");
      if (!(o->beta > 0) || !(o->floor_eps > 0) || !(o->floor_eps <= 1)) return fail(h, RIFT_EINVAL, "bad beta / floor_eps");
      if (o->tables) return fail(h, RIFT_EINVAL, "the fallback starts from the prior's tables (opts.tables must be NULL)");
    }
  } else if (o->proposal != RIFT_PROPOSAL_PRIOR) {
    return fail(h, RIFT_EINVAL, "unknown proposal");
  }
  if (o->tables_out && o->proposal != RIFT_PROPOSAL_ADAPTIVE)
    return fail(h, RIFT_EINVAL, "tables_out needs the adaptive proposal");
  if (o->refine && (o->resume || o->save)) return fail(h, RIFT_EINVAL, "refine does not combine with resume or save");
  if (!(o->fallback_neff >= 0.0)) return fail(h, RIFT_EINVAL, "fallback_neff must be >= 0");
  if (o->fallback_neff > 0.0 && o->proposal != RIFT_PROPOSAL_LEARNED)
    return fail(h, RIFT_EINVAL, "fallback_neff applies to the learned proposal only");
  return RIFT_OK;
}

// rs (optional): the refinement of heavy samples, whose corrections replace the FP32 log weights of
// the refined samples by their FP64 values in the sums; the largest weight is then the largest
// refined one when the sample at the maximum was refined.
void fill_result(const AccState &a, rift_mc_result *r, const RefineState *rs = nullptr) {
  r->acc_max = a.m;
  r->acc_s1 = a.s1 + a.c1;
  r->acc_s2 = a.s2 + a.c2;
  r->n_evals = a.n;
  r->n_refined = 0;
  double wmax = 1.0;
  if (rs && rs->n > 0 && a.n > 0) {
    const double f = std::exp(rs->mref - a.m);
    r->acc_s1 += rs->d1 * f;
    r->acc_s2 += rs->d2 * f * f;
    const double w64 = std::exp(rs->l64max - a.m);
    wmax = (rs->l32max == a.m) ? w64 : std::max(1.0, w64);
    r->n_refined = (int)rs->n;
  }
  const double n = (double)a.n;
  if (a.n == 0 || !(r->acc_s1 > 0)) {
    r->lnL_marg = -INFINITY; r->n_eff = 0; r->n_eff_kish = 0; r->sigma = INFINITY;
    return;
  }
  r->lnL_marg = a.m + std::log(r->acc_s1) - std::log(n);
  r->n_eff = r->acc_s1 / wmax;
  r->n_eff_kish = r->acc_s1 * r->acc_s1 / r->acc_s2;
  r->sigma = (a.n > 1) ? std::sqrt(std::max(n * r->acc_s2 / (r->acc_s1 * r->acc_s1) - 1.0, 0.0) / (n - 1.0)) : INFINITY;
}

// Status of a device status word read back from the handle.
rift_status flags_status(rift_ile *h, uint32_t f) {
  if (f & RIFT_FLAG_TIMEOUT_BIT) return fail(h, RIFT_ETIMEOUT, "a bounded wait for a shared-memory copy expired");
  if (f & RIFT_FLAG_WINDOW) return fail(h, RIFT_EWINDOW, "interpolation taps left the Q window");
  if (f & RIFT_FLAG_NONFINITE) return fail(h, RIFT_ENONFINITE, "non-finite log-likelihood");
  return RIFT_OK;
}

rift_status read_flags(rift_ile *h) {
  uint32_t f = 0;
  RIFT_CK(h, cudaMemcpyAsync(&f, h->flags, sizeof(f), cudaMemcpyDeviceToHost, h->stream));
  RIFT_CK(h, cudaMemsetAsync(h->flags, 0, sizeof(uint32_t), h->stream));
  RIFT_CK(h, cudaStreamSynchronize(h->stream));
  return flags_status(h, f);
}

int taps_of(int interp) { return interp == 3 ? 4 : (interp == 1 ? 2 : 1); }

// Strata (log2) for rounds of n samples of point P: about `target` samples per cell, the split
// between sky and time chosen to minimise the expected Q window of a cell (time-of-flight
// spread over the cell's sky patch plus the cell's share of the time prior, in Q rows).
void choose_strata(const PointC &P, uint32_t n, int ls[3], int target = 640) {
  ls[0] = ls[1] = ls[2] = 0;
  int L = 0;
  while (L < 15 && ((uint64_t)target << (L + 1)) <= n) ++L;
  double best = 1e300;
  for (int a = 0; a <= L; ++a)
    for (int b = 0; a + b <= L; ++b) {
      const int c = L - a - b;
      double rows = 0.0;
      for (int k = 0; k < P.K; ++k) {
        const double R = std::sqrt((double)P.det[k].P[0] * P.det[k].P[0] + (double)P.det[k].P[1] * P.det[k].P[1] +
                                   (double)P.det[k].P[2] * P.det[k].P[2]);
        rows += R * (2.0 * kPi / (1 << a) + 2.0 / (1 << b)) * 0.5 + (double)P.A / (1 << c);
      }
      if (rows < best - 1e-9) { best = rows; ls[0] = a; ls[1] = b; ls[2] = c; }
    }
}

// Strata of a time-marginalised round: about `target` draws per cell over (ra, sin dec) only,
// two ra cells per sin dec cell (the ra range is pi times the sin dec range).
void choose_strata_sky(uint32_t n, int ls[3], int target) {
  int L = 0;
  while (L < 15 && ((uint64_t)target << (L + 1)) <= n) ++L;
  ls[1] = L / 2;
  ls[0] = L - ls[1];
  ls[2] = 0;
}

// Launch shape of the cell kernel: tm (0 sampled time, 1 time quadrature, 2 the quadrature's GEMM
// form, taken when every point has merged rows and the block holds the GEMM's arrays with the
// harmonics of the setup), the harmonics rows reserved in shared memory, the window budget and the
// dynamic shared memory of a block.
struct CellShape {
  int tm, ys_modes;
  long long budget;
  size_t smem;
};
CellShape cell_shape(const rift_ile *h, int K, int NT, int time_marg, int ys_modes, int coef_f4, int nb, int smem_sm) {
  const int block = RIFT_CELL_BLOCK;
  CellShape c{};
  if (time_marg && h->all_qhalf) {
    const size_t fixed = cells_smem_fixed(K, 0, coef_f4, nb, block);
    const long long budget = ((long long)RIFT_CELLS_MAX_DYN_SMEM - (long long)fixed) & ~15ll;
    const TgLayout T = tg_layout(K, NT, RIFT_MAXMH, (unsigned)std::max(0ll, budget));
    if (budget > 0 && T.rmax >= 64 && (long long)(T.end - T.S) >= 8ll * h->max_M * block) {
      c.tm = 2;
      c.ys_modes = 0;
      c.budget = budget;
      c.smem = fixed + (size_t)budget;
      return c;
    }
  }
  c.tm = time_marg ? 1 : 0;
  c.ys_modes = ys_modes;
  const size_t fixed = cells_smem_fixed(K, ys_modes, coef_f4, nb, block);
  long long budget = ((long long)smem_sm / h->smem_split - (long long)fixed - 2048) & ~15ll;
  c.budget = std::max(16ll * 1024, std::min(160ll * 1024, budget));
  c.smem = fixed + (size_t)c.budget;
  return c;
}

int log2_pow2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return ((1 << l) == v) ? l : -1;
}

rift_status ensure_learned(rift_ile *h) {
  const int np = h->n_points;
  if (!h->gmm) {
    RIFT_CK(h, cache_dev_alloc((void **)&h->gmm, sizeof(float) * (size_t)np * RIFT_GMM_FLOATS));
    RIFT_CK(h, cache_dev_alloc((void **)&h->gcst, sizeof(float) * (size_t)np * 4));
    RIFT_CK(h, cache_dev_alloc((void **)&h->head, sizeof(float) * (size_t)np * RIFT_MDN_HEAD));
    RIFT_CK(h, cache_dev_alloc((void **)&h->summ, sizeof(float) * (size_t)np * RIFT_MDN_SUMMARY));
  }
  return RIFT_OK;
}

// The learned proposal of every point for distance prior [d_lo, d_hi]: per-point constants
// (FP64 here), then the network on each point's summary (opts.mdn) or the given heads.
rift_status prepare_learned(rift_ile *h, const rift_mc_opts *o, cudaStream_t st) {
  rift_status s = ensure_learned(h);
  if (s != RIFT_OK) return s;
  const int np = h->n_points;
  std::vector<float> c((size_t)np * 4);
  for (int p = 0; p < np; ++p) {
    const double tspan = h->pts[p].t_hi - h->pts[p].t_lo;
    const double lnspan = std::log(o->d_hi) - std::log(o->d_lo);
    // time integrated by quadrature: the box and the prior of (ra, sin dec, cos incl, ln D) only
    const double lt = o->time_marg ? 0.0 : std::log(tspan);
    c[4 * p + 0] = (float)(std::log(2.0 * kPi) + std::log(2.0) + lt + std::log(2.0) + std::log(lnspan));
    c[4 * p + 1] = (float)(-std::log(2.0 * kPi) - std::log(2.0) - lt - std::log(2.0) + std::log(3.0) -
                           std::log(o->d_hi * o->d_hi * o->d_hi - o->d_lo * o->d_lo * o->d_lo));
    c[4 * p + 2] = (float)std::log(o->d_lo);
    c[4 * p + 3] = (float)lnspan;
  }
  RIFT_CK(h, cudaMemcpyAsync(h->gcst, c.data(), sizeof(float) * c.size(), cudaMemcpyHostToDevice, st));
  if (o->mdn) {
    RIFT_CK(h, launch_summary(h->pts_dev, h->q_arena, h->c_arena, h->tau0, np, h->summ, st));
    RIFT_CK(h, launch_mdn_gmm(static_cast<const rift_mdn *>(o->mdn), h->summ, h->gcst, np, h->head, h->gmm, h->flags, st));
  } else {
    RIFT_CK(h, launch_gmm_from_head(h->head, h->gcst, np, h->gmm, st));
  }
  RIFT_CK(h, cudaStreamSynchronize(st));
  return RIFT_OK;
}

// Sampler state between calls (rift_mc_opts.resume / save): everything the next round of a
// single-point run depends on.
struct McStateBlob {
  uint32_t magic, version;
  uint64_t seed;
  uint32_t point_id, n_per_round;
  int32_t K, M, T, proposal, n_bins, ls[3], time_marg, pad2;
  double beta, floor_eps, d_lo, d_hi;
  uint32_t rounds, pad;
  uint64_t evals;
  AccState acc;
  float tables[3 * (RIFT_MAXBINS + 1)];
  float lnw[3 * RIFT_MAXBINS];
};
static_assert(sizeof(McStateBlob) <= RIFT_MC_STATE_BYTES, "state blob larger than RIFT_MC_STATE_BYTES");
constexpr uint32_t kStateMagic = 0x53464952u;   // "RIFS"

void state_header(const rift_ile *h, const rift_mc_opts *o, const int ls[3], McStateBlob &b) {
  std::memset(&b, 0, sizeof(b));
  b.magic = kStateMagic;
  b.version = 2;
  b.seed = o->seed;
  b.point_id = o->point_id;
  b.n_per_round = o->n_per_round;
  b.K = h->pts[0].c.K; b.M = h->pts[0].c.M; b.T = h->pts[0].c.T;
  b.proposal = o->proposal;
  b.n_bins = (o->proposal == RIFT_PROPOSAL_ADAPTIVE) ? o->n_bins : 0;
  for (int d = 0; d < 3; ++d) b.ls[d] = ls[d];
  b.time_marg = o->time_marg ? 1 : 0;
  b.beta = o->beta; b.floor_eps = o->floor_eps; b.d_lo = o->d_lo; b.d_hi = o->d_hi;
}

bool state_matches(const McStateBlob &a, const McStateBlob &b) {
  return a.magic == b.magic && a.version == b.version && a.seed == b.seed && a.point_id == b.point_id &&
         a.n_per_round == b.n_per_round && a.K == b.K && a.M == b.M && a.T == b.T && a.proposal == b.proposal &&
         a.n_bins == b.n_bins && a.ls[0] == b.ls[0] && a.ls[1] == b.ls[1] && a.ls[2] == b.ls[2] &&
         a.time_marg == b.time_marg &&
         a.beta == b.beta && a.floor_eps == b.floor_eps && a.d_lo == b.d_lo && a.d_hi == b.d_hi;
}

// The Monte Carlo round loop of Eq. (lnLmarg) for np points of the handle, with the scratch S.
rift_status run_mc(rift_ile *h, const rift_mc_opts *o, int np, McScratch &S, rift_mc_result *res) {
  const int K = h->K, NT = taps_of(h->interp);
  const bool learned = (o->proposal == RIFT_PROPOSAL_LEARNED);
  const bool fallback = learned && o->fallback_neff > 0.0;
  // table machinery: the adaptive proposal, or learned points that may fall back to it
  const bool adaptive = (o->proposal == RIFT_PROPOSAL_ADAPTIVE) || fallback;
  const int nb = adaptive ? o->n_bins : 0;
  const uint32_t npr = o->n_per_round;
  std::vector<int> lsv(3 * np);
  if (learned) {
    rift_status s2 = prepare_learned(h, o, h->stream);
    if (s2 != RIFT_OK) return s2;
  }
  for (int p = 0; p < np; ++p) {
    int *ls = &lsv[3 * p];
    if (learned) {
      ls[0] = ls[1] = ls[2] = 0;
    } else if (o->strata[0] == 0 && o->strata[1] == 0 && o->strata[2] == 0) {
      if (o->time_marg) choose_strata_sky(npr, ls, std::max(16, h->cell_target / 5));   // a draw costs ~J samples
      else choose_strata(h->pts[p].c, npr, ls, h->cell_target);
    } else {
      for (int d = 0; d < 3; ++d) ls[d] = log2_pow2(o->strata[d]);
      if (ls[0] < 0 || ls[1] < 0 || ls[2] < 0) return fail(h, RIFT_EINVAL, "strata must be powers of two");
      if ((1 << (ls[0] + ls[1] + ls[2])) > RIFT_MAX_CELLS) return fail(h, RIFT_EINVAL, "more than RIFT_MAX_CELLS cells");
      if (o->time_marg && ls[2] != 0) return fail(h, RIFT_EINVAL, "time-marginalised rounds are not stratified in t");
    }
  }
  cudaStream_t st = h->stream;
  if ((o->resume || o->save) && (np != 1 || h->n_points != 1))
    return fail(h, RIFT_EINVAL, "resume/save need a single-point handle");
  if ((o->resume || o->save) && fallback) return fail(h, RIFT_EINVAL, "resume/save do not record a fallback");
  McStateBlob hdr, in{};
  if (o->resume || o->save) state_header(h, o, lsv.data(), hdr);
  if (o->resume) {
    std::memcpy(&in, o->resume, sizeof(in));
    if (!state_matches(in, hdr)) return fail(h, RIFT_EINVAL, "resume state does not match this handle and options");
  }
  // accumulators and round-0 tables
  for (int p = 0; p < np; ++p) {
    std::memset(&S.acc_host[p], 0, sizeof(AccState));
    S.acc_host[p].m = -INFINITY;
  }
  if (o->resume) S.acc_host[0] = in.acc;
  RIFT_CK(h, cudaMemcpyAsync(S.acc, S.acc_host, sizeof(AccState) * np, cudaMemcpyHostToDevice, st));
  int cur = 0;
  const size_t tstride = (size_t)3 * (nb + 1), wstride = (size_t)3 * nb;
  if (adaptive && o->resume) {
    RIFT_CK(h, cudaMemcpyAsync(S.tables, in.tables, sizeof(float) * tstride, cudaMemcpyHostToDevice, st));
    RIFT_CK(h, cudaMemcpyAsync(S.lnw, in.lnw, sizeof(float) * wstride, cudaMemcpyHostToDevice, st));
  } else if (adaptive) {
    float u[3 * (RIFT_MAXBINS + 1)];
    const float *src = o->tables;
    if (!src) {
      for (int d = 0; d < 3; ++d)
        for (int b = 0; b <= nb; ++b) u[d * (nb + 1) + b] = (float)((double)b / nb);
      src = u;
    }
    // (both buffers when learned points may fall back: a point that has not adapted yet reads
    // whichever buffer the round reads)
    for (int buf = 0; buf < (fallback ? 2 : 1); ++buf)
      for (int p = 0; p < np; ++p) {
        const float *sp = (o->tables && o->tables_per_point) ? src + p * tstride : src;
        RIFT_CK(h, cudaMemcpyAsync(S.tables + ((size_t)buf * np + p) * tstride, sp, sizeof(float) * tstride,
                                   cudaMemcpyHostToDevice, st));
      }
    RIFT_CK(h, cudaStreamSynchronize(st));
    // lnw of the round-0 tables (every point): rp is only read for its flags with part == nullptr
    for (int p = 0; p < np; ++p) {
      std::memset(&S.rp_host[p], 0, sizeof(RoundPt));
      S.rp_host[p].proposal = 1;
      S.rp_host[p].ncell = 1;
    }
    RIFT_CK(h, cudaMemcpyAsync(S.rp, S.rp_host, sizeof(RoundPt) * np, cudaMemcpyHostToDevice, st));
    for (int buf = 0; buf < (fallback ? 2 : 1); ++buf)
      RIFT_CK(h, launch_tables_points(nullptr, 0, S.rp, np, nb, 0.0, S.tables + (size_t)buf * np * tstride,
                                      S.lnw + (size_t)buf * np * wstride, st));
  }
  const int block = RIFT_CELL_BLOCK;
  int smem_sm = 0;
  RIFT_CK(h, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device));
  // a single point in the grouped layout passes its coefficients as a kernel parameter (when the
  // kernel has that variant): no shared-memory copy of them, so the Q windows get the room
  const CanonCoefParam *cc = (np == 1 && h->canon0 && NT == 4 && !learned && !o->time_marg) ? h->canon0 : nullptr;
  const MirrorCoefParam *mp = (np == 1 && h->mirror0 && NT == 4 && !learned && !o->time_marg) ? h->mirror0 : nullptr;
  const int coef_f4 = (cc || mp) ? 0 : h->max_pairK;
  // a mirror-symmetric point with all 21 modes keeps its harmonics in registers (no shared buffer)
  const CellShape shp = cell_shape(h, K, NT, o->time_marg, (mp && h->pts[0].c.M == RIFT_MAXM) ? 0 : h->max_M,
                                   coef_f4, nb, smem_sm);
  const int ys_modes = shp.ys_modes, tm = shp.tm;
  const long long budget = shp.budget;
  const size_t smem = shp.smem;
  int bps = cells_blocks_per_sm(K, NT, smem, block, tm);
  if (bps < 1) return fail(h, RIFT_EUNSUPPORTED, "cell kernel does not fit on an SM");
  CellLaunch L{};
  L.seed = o->seed;
  L.d_lo3 = (float)(o->d_lo * o->d_lo * o->d_lo);
  L.d_span3 = (float)(o->d_hi * o->d_hi * o->d_hi - o->d_lo * o->d_lo * o->d_lo);
  L.pts = h->pts_dev;
  L.rp = S.rp;
  L.n_points = np;
  L.win_budget = (int)budget;
  L.n_items = S.counters;
  L.queue = S.counters + 1;
  L.qa = h->q_arena;
  L.ca = h->c_arena;
  L.partials = S.partials;
  L.dbg_ell = (np == 1) ? o->dbg_ell : nullptr;
  L.ell_buf = adaptive ? S.ell : nullptr;
  L.bin_buf = adaptive ? S.bins : nullptr;
  L.flags = h->flags;
  L.max_M = ys_modes;
  L.merged = (mp && ys_modes == 0 && h->pts[0].c.qhalf && h->pts[0].c.Mh == RIFT_MAXMH) ? 1 : 0;
  const bool refine = o->refine && !o->time_marg;
  if (refine) {
    rift_status rs0 = ensure_refine(h, np, S.max_items, st);
    if (rs0 != RIFT_OK) return rs0;
    L.cand = h->cand;
    L.cmax = h->cmax;
  }
  const double lo3 = o->d_lo * o->d_lo * o->d_lo, span3 = o->d_hi * o->d_hi * o->d_hi - lo3;
  L.max_pairK = coef_f4;
  L.max_nb = nb;
  L.learned = learned ? 1 : 0;
  L.fault_nan = fault_is("nan_sample") ? 1 : 0;
  L.fault_stall = fault_is("stage_timeout") ? 1 : 0;
  L.tmarg = tm;
  std::vector<uint64_t> evals(np, 0);
  std::vector<int> rounds(np, 0), done(np, 0), nrun(np, 0);
  std::vector<int> prop(np, learned ? 2 : (adaptive ? 1 : 0)), fb_round(np, -1);
  int r0 = 0;
  if (o->resume) {
    evals[0] = in.evals;
    rounds[0] = (int)in.rounds;
    r0 = rounds[0];
    const double n_eff = in.acc.s1 + in.acc.c1;
    if (n_eff >= o->n_eff_target || evals[0] >= o->max_evals || (o->max_rounds > 0 && rounds[0] >= o->max_rounds))
      done[0] = 1;
  }
  int launches = 0;
  double kms = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (o->timing) {
    RIFT_CK(h, cudaEventCreate(&ev0));
    RIFT_CK(h, cudaEventCreate(&ev1));
  }
  rift_status status = RIFT_OK;
  for (int r = r0;; ++r) {
    uint32_t items = 0;
    for (int p = 0; p < np; ++p) {
      RoundPt &R = S.rp_host[p];
      std::memset(&R, 0, sizeof(R));
      R.item0 = items;
      R.ell_off = -1;
      R.dbg_off = -1;
      nrun[p] = 0;
      if (done[p]) continue;
      const uint32_t n = (uint32_t)std::min<uint64_t>(npr, o->max_evals - evals[p]);
      const int *ls = &lsv[3 * p];
      int l0 = ls[0], l1 = ls[1], l2 = ls[2];
      if ((uint64_t)n < (1ull << (l0 + l1 + l2))) l0 = l1 = l2 = 0;   // (learned points: lsv is 0)
      const uint32_t C = 1u << (l0 + l1 + l2);
      R.n = n;
      R.ncell = C;
      R.base = n / C;
      R.rem = n % C;
      R.round = (uint32_t)rounds[p];
      R.point_id = (np == 1) ? o->point_id : (uint32_t)p;
      R.ls0 = l0; R.ls1 = l1; R.ls2 = l2;
      R.proposal = prop[p];
      R.nb = nb;
      R.gmm = (prop[p] == 2) ? h->gmm + (size_t)p * RIFT_GMM_FLOATS : nullptr;
      R.tmarg = o->time_marg ? 1 : 0;
      R.lcorr0 = (float)std::log((double)n / ((double)C * (R.base + 1.0)));
      R.lcorr1 = R.base ? (float)std::log((double)n / ((double)C * R.base)) : 0.f;
      if (o->time_marg) {   // runs of consecutive draws across cells (chunks unused)
        R.chunks = 0;
        R.nitem = (n + RIFT_TMARG_CHUNK - 1) / RIFT_TMARG_CHUNK;
      } else {
        R.chunks = (R.base + (R.rem ? 1u : 0u) + RIFT_CHUNK - 1) / RIFT_CHUNK;
        R.nitem = C * R.chunks;
      }
      R.ell_off = adaptive ? (long long)p * npr : -1;
      R.dbg_off = (np == 1 && o->dbg_ell) ? (long long)rounds[p] * npr : -1;
      R.tab = adaptive ? S.tables + ((size_t)cur * np + p) * tstride : nullptr;
      R.lnw = adaptive ? S.lnw + ((size_t)cur * np + p) * wstride : nullptr;
      items += R.nitem;
      nrun[p] = (int)n;
    }
    if (items == 0) break;
    if (items > S.max_items) { status = fail(h, RIFT_EINVAL, "work items exceed the scratch"); break; }
    if (o->dbg_tables && adaptive && np == 1)
      RIFT_CK(h, cudaMemcpyAsync(o->dbg_tables + (size_t)(r - r0) * tstride, S.tables + (size_t)cur * np * tstride,
                                 sizeof(float) * tstride, cudaMemcpyDeviceToDevice, st));
    const uint32_t cnt[2] = {items, 0u};
    RIFT_CK(h, cudaMemcpyAsync(S.rp, S.rp_host, sizeof(RoundPt) * np, cudaMemcpyHostToDevice, st));
    RIFT_CK(h, cudaMemcpyAsync(S.counters, cnt, sizeof(cnt), cudaMemcpyHostToDevice, st));
    const int grid = (int)std::max<uint32_t>(1, std::min<uint32_t>(items, (uint32_t)(h->num_sms * bps)));
    if (o->timing) RIFT_CK(h, cudaEventRecord(ev0, st));
    RIFT_CK(h, launch_cells(K, NT, L, grid, block, smem, st, cc, h->pts[0].c.canon_sparse, mp));
    if (o->timing) RIFT_CK(h, cudaEventRecord(ev1, st));
    RIFT_CK(h, launch_merge_points(S.partials, S.rp, np, S.acc, st));
    launches += 2;
    if (refine) {
      RIFT_CK(h, launch_refine(h->pts_dev, h->pd_dev, h->uv64, h->q_arena, S.rp, S.acc, h->cmax, h->cand, np, o->seed, lo3,
                               span3, h->rscratch, h->rstate, h->flags, st));
      launches += 3;
    }
    const bool adapt_now = adaptive && (o->adapt_rounds < 0 || r < o->adapt_rounds);
    if (adapt_now) {
      RIFT_CK(h, launch_hist_points(S.ell, S.bins, S.rp, np, S.acc, (float)o->beta, nb, S.hist, S.hblocks, st));
      RIFT_CK(h, launch_tables_points(S.hist, S.hblocks, S.rp, np, nb, o->floor_eps,
                                      S.tables + (size_t)(1 - cur) * np * tstride,
                                      S.lnw + (size_t)(1 - cur) * np * wstride, st));
      launches += 2;
    }
    RIFT_CK(h, cudaMemcpyAsync(S.acc_host, S.acc, sizeof(AccState) * np, cudaMemcpyDeviceToHost, st));
    RIFT_CK(h, cudaStreamSynchronize(st));
    if (o->timing) {
      float ms = 0.f;
      RIFT_CK(h, cudaEventElapsedTime(&ms, ev0, ev1));
      kms += ms;
    }
    if (adapt_now) {
      // points that are not adapting keep their tables: copy them into the new buffer
      cur = 1 - cur;
    }
    bool any = false;
    for (int p = 0; p < np; ++p) {
      if (!nrun[p]) continue;
      evals[p] += (uint64_t)nrun[p];
      rounds[p] += 1;
      const AccState &a = S.acc_host[p];
      const double n_eff = a.s1 + a.c1;
      if (n_eff >= o->n_eff_target || evals[p] >= o->max_evals || (o->max_rounds > 0 && rounds[p] >= o->max_rounds))
        done[p] = 1;
      else
        any = true;
      // fallback of the learned proposal: a learned round whose own draws have n_eff below the
      // threshold (degenerate weights) hands the point to the adaptive sampler for its remaining rounds
      if (!done[p] && fallback && prop[p] == 2 && a.round_neff < o->fallback_neff) {
        prop[p] = 1;
        fb_round[p] = rounds[p];
      }
    }
    if (!any) break;
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (o->tables_out && adaptive && status == RIFT_OK) {
    // the buffer the next round would read: rebuilt from the last round if it adapted
    for (int p = 0; p < np; ++p)
      RIFT_CK(h, cudaMemcpyAsync(o->tables_out + p * tstride, S.tables + ((size_t)cur * np + p) * tstride,
                                 sizeof(float) * tstride, cudaMemcpyDeviceToHost, st));
    RIFT_CK(h, cudaStreamSynchronize(st));
  }
  if (o->save && status == RIFT_OK) {
    McStateBlob outb = hdr;
    outb.rounds = (uint32_t)rounds[0];
    outb.evals = evals[0];
    outb.acc = S.acc_host[0];
    if (adaptive) {
      RIFT_CK(h, cudaMemcpyAsync(outb.tables, S.tables + (size_t)cur * tstride, sizeof(float) * tstride,
                                 cudaMemcpyDeviceToHost, st));
      RIFT_CK(h, cudaMemcpyAsync(outb.lnw, S.lnw + (size_t)cur * wstride, sizeof(float) * wstride,
                                 cudaMemcpyDeviceToHost, st));
      RIFT_CK(h, cudaStreamSynchronize(st));
    }
    std::memset(o->save, 0, RIFT_MC_STATE_BYTES);
    std::memcpy(o->save, &outb, sizeof(outb));
  }
  // the refinement's corrections and the status word, read back behind one synchronisation
  uint32_t fword = 0;
  if (refine)
    RIFT_CK(h, cudaMemcpyAsync(h->rstate_host, h->rstate, sizeof(RefineState) * np, cudaMemcpyDeviceToHost, st));
  RIFT_CK(h, cudaMemcpyAsync(&fword, h->flags, sizeof(fword), cudaMemcpyDeviceToHost, st));
  RIFT_CK(h, cudaMemsetAsync(h->flags, 0, sizeof(uint32_t), st));
  RIFT_CK(h, cudaStreamSynchronize(st));
  rift_status fl = flags_status(h, fword);
  for (int p = 0; p < np; ++p) {
    fill_result(S.acc_host[p], &res[p], refine ? &h->rstate_host[p] : nullptr);
    res[p].rounds = rounds[p];
    res[p].fallback_round = fb_round[p];
    res[p].kernel_ms = (p == 0) ? kms : 0.0;
    res[p].kernel_launches = (p == 0) ? launches : 0;
    for (int d = 0; d < 3; ++d) res[p].strata[d] = 1 << lsv[3 * p + d];
    rift_status sp = (status != RIFT_OK) ? status : fl;
    if (sp == RIFT_OK && res[p].n_eff < o->n_eff_target) sp = RIFT_ENOTCONVERGED;
    res[p].status = sp;
  }
  if (status != RIFT_OK) return status;
  if (fl != RIFT_OK) return fl;
  for (int p = 0; p < np; ++p)
    if (res[p].status == RIFT_ENOTCONVERGED) return RIFT_ENOTCONVERGED;
  return RIFT_OK;
}

}  // namespace

extern "C" {

const char *rift_status_str(rift_status s) {
  switch (s) {
    case RIFT_OK: return "ok";
    case RIFT_EINVAL: return "invalid argument";
    case RIFT_EWINDOW: return "Q window does not cover the requested times";
    case RIFT_ENOMEM: return "out of memory";
    case RIFT_ECUDA: return "CUDA error";
    case RIFT_ETIMEOUT: return "bounded device wait expired";
    case RIFT_ENONFINITE: return "non-finite likelihood";
    case RIFT_ENOTCONVERGED: return "max_evals reached before n_eff target";
    case RIFT_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *rift_ile_last_error(const rift_ile *h) { return h ? h->err.c_str() : "null handle"; }
int rift_ile_n_points(const rift_ile *h) { return h ? h->n_points : 0; }

unsigned rift_ile_forms(const rift_ile *h, int point) {
  if (!h || point < 0 || point >= h->n_points) return 0u;
  const PointC &c = h->pts[point].c;
  return (c.grouped ? 1u : 0u) | (c.canon_sparse ? 2u : 0u) | (c.mirror ? 4u : 0u) | (c.qhalf ? 8u : 0u);
}

rift_status rift_ile_create(const rift_ile_desc *desc, rift_ile **out) { return create_impl(desc, 1, out); }

rift_status rift_ile_batch_create(const rift_ile_desc *descs, int n_points, rift_ile **out) {
  return create_impl(descs, n_points, out);
}

void rift_ile_destroy(rift_ile *h) {
  if (!h) return;
  // the buffers go back to the cache for other handles: nothing of this handle may still run
  cudaStreamSynchronize(h->stream);
  if (h->gstream) cudaStreamSynchronize(h->gstream);
  cache_dev_free(h->pts_dev);
  cache_dev_free(h->q_arena);
  cache_dev_free(h->c_arena);
  cache_dev_free(h->flags);
  McScratch &S = h->sc;
  cache_dev_free(S.acc);
  cache_dev_free(S.partials);
  cache_dev_free(S.rp);
  cache_dev_free(S.counters);
  cache_dev_free(S.ell);
  cache_dev_free(S.bins);
  cache_dev_free(S.hist);
  cache_dev_free(S.tables);
  cache_dev_free(S.lnw);
  cache_host_free(S.rp_host);
  cache_host_free(S.acc_host);
  cache_dev_free(h->stage);
  cache_dev_free(h->tau0);
  cache_dev_free(h->head);
  cache_dev_free(h->summ);
  cache_dev_free(h->gmm);
  cache_dev_free(h->gcst);
  cache_dev_free(h->last);
  cache_dev_free(h->hidx);
  cache_dev_free(h->pst);
  cache_dev_free(h->ctl);
  cache_host_free(h->ctl_host);
  cache_host_free(h->pst_host);
  cache_dev_free(h->pd_dev);
  cache_dev_free(h->uv64);
  cache_dev_free(h->cand);
  cache_dev_free(h->cmax);
  cache_dev_free(h->rscratch);
  cache_dev_free(h->rstate);
  cache_host_free(h->rstate_host);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  delete h->canon0;
  delete h->mirror0;
  delete h;
}

rift_status rift_ile_check(rift_ile *h) {
  if (!h) return RIFT_EINVAL;
  return read_flags(h);
}

rift_status rift_ile_lnL(rift_ile *h, size_t n, const float *ra, const float *dec, const float *t, const float *psi,
                         const float *phi, const float *incl, const float *dist, float *lnL_out) {
  if (!h) return RIFT_EINVAL;
  if (n == 0) return RIFT_OK;
  if (!ra || !dec || !t || !psi || !phi || !incl || !dist || !lnL_out) return fail(h, RIFT_EINVAL, "null sample array");
  const Point &p = h->pts[0];
  RIFT_CK(h, launch_lnl_array(h->K, h->pts_dev, p.c, h->q_arena, h->c_arena, n, ra, dec, t, psi, phi, incl, dist,
                              lnL_out, h->flags, h->stream));
  return RIFT_OK;
}

rift_status rift_ile_lnL_tmarg(rift_ile *h, size_t n, const float *ra, const float *dec, const float *psi,
                               const float *phi, const float *incl, const float *dist, float *out) {
  if (!h) return RIFT_EINVAL;
  if (n == 0) return RIFT_OK;
  if (!ra || !dec || !psi || !phi || !incl || !dist || !out) return fail(h, RIFT_EINVAL, "null draw array");
  const Point &p = h->pts[0];
  RIFT_CK(h, launch_lnl_tmarg(h->K, h->pts_dev, p.c, h->q_arena, h->c_arena, n, ra, dec, psi, phi, incl, dist, out,
                              h->flags, h->stream));
  return RIFT_OK;
}

rift_status rift_ile_lnL_host(rift_ile *h, size_t n, const float *ra, const float *dec, const float *t,
                              const float *psi, const float *phi, const float *incl, const float *dist,
                              float *lnL_out) {
  if (!h) return RIFT_EINVAL;
  if (n == 0) return RIFT_OK;
  if (!ra || !dec || !t || !psi || !phi || !incl || !dist || !lnL_out) return fail(h, RIFT_EINVAL, "null sample array");
  if (n > h->stage_n) {
    cache_dev_free(h->stage);
    h->stage = nullptr;
    h->stage_n = 0;
    RIFT_CK(h, cache_dev_alloc((void **)&h->stage, sizeof(float) * 8 * n));
    h->stage_n = n;
  }
  float *s = h->stage;
  const float *src[7] = {ra, dec, t, psi, phi, incl, dist};
  for (int j = 0; j < 7; ++j)
    RIFT_CK(h, cudaMemcpyAsync(s + (size_t)j * n, src[j], sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
  const Point &p = h->pts[0];
  RIFT_CK(h, launch_lnl_array(h->K, h->pts_dev, p.c, h->q_arena, h->c_arena, n, s, s + n, s + 2 * n, s + 3 * n,
                              s + 4 * n, s + 5 * n, s + 6 * n, s + 7 * n, h->flags, h->stream));
  RIFT_CK(h, cudaMemcpyAsync(lnL_out, s + 7 * n, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
  return read_flags(h);
}

rift_status rift_ile_draw(rift_ile *h, const rift_mc_opts *o, uint32_t round, const float *tables, size_t n,
                          float *theta_out, float *lpq_out, int *bins_out) {
  if (!h) return RIFT_EINVAL;
  rift_status s = check_opts(h, o);
  if (s != RIFT_OK) return s;
  if (!theta_out || !lpq_out) return fail(h, RIFT_EINVAL, "null output");
  if (n == 0) return RIFT_OK;
  if (n > 0xFFFFFFFFull) return fail(h, RIFT_EINVAL, "n too large");
  const bool tab = (o->proposal == RIFT_PROPOSAL_ADAPTIVE) && tables;
  const bool learned = (o->proposal == RIFT_PROPOSAL_LEARNED);
  const int nb = tab ? o->n_bins : 0;
  if ((s = ensure_scratch(h, 1, 1, 0, tab ? nb : 0, 1)) != RIFT_OK) return s;
  if (learned && (s = prepare_learned(h, o, h->stream)) != RIFT_OK) return s;
  McScratch &S = h->sc;
  int ls[3];
  if (learned) {
    ls[0] = ls[1] = ls[2] = 0;
  } else if (o->strata[0] == 0 && o->strata[1] == 0 && o->strata[2] == 0) {
    choose_strata(h->pts[0].c, (uint32_t)n, ls, h->cell_target);
  } else {
    for (int d = 0; d < 3; ++d) ls[d] = log2_pow2(o->strata[d]);
    if (ls[0] < 0 || ls[1] < 0 || ls[2] < 0) return fail(h, RIFT_EINVAL, "strata must be powers of two");
  }
  if ((uint64_t)n < (1ull << (ls[0] + ls[1] + ls[2]))) ls[0] = ls[1] = ls[2] = 0;
  RoundPt &R = S.rp_host[0];
  std::memset(&R, 0, sizeof(R));
  const uint32_t C = 1u << (ls[0] + ls[1] + ls[2]);
  R.n = (uint32_t)n; R.ncell = C; R.base = R.n / C; R.rem = R.n % C;
  R.round = round; R.point_id = o->point_id;
  R.ls0 = ls[0]; R.ls1 = ls[1]; R.ls2 = ls[2];
  R.proposal = learned ? 2 : (tab ? 1 : 0); R.nb = nb;
  R.gmm = learned ? h->gmm : nullptr;
  R.lcorr0 = (float)std::log((double)R.n / ((double)C * (R.base + 1.0)));
  R.lcorr1 = R.base ? (float)std::log((double)R.n / ((double)C * R.base)) : 0.f;
  R.chunks = (R.base + (R.rem ? 1u : 0u) + RIFT_CHUNK - 1) / RIFT_CHUNK;
  R.nitem = C * R.chunks;
  R.ell_off = -1; R.dbg_off = -1;
  if (tab) {
    RIFT_CK(h, cudaMemcpyAsync(S.tables, tables, sizeof(float) * 3 * (nb + 1), cudaMemcpyDeviceToDevice, h->stream));
    R.tab = S.tables;
    R.lnw = S.lnw;
  }
  RIFT_CK(h, cudaMemcpyAsync(S.rp, S.rp_host, sizeof(RoundPt), cudaMemcpyHostToDevice, h->stream));
  if (tab) RIFT_CK(h, launch_tables_points(nullptr, 0, S.rp, 1, nb, 0.0, S.tables, S.lnw, h->stream));
  CellLaunch L{};
  L.seed = o->seed;
  L.d_lo3 = (float)(o->d_lo * o->d_lo * o->d_lo);
  L.d_span3 = (float)(o->d_hi * o->d_hi * o->d_hi - o->d_lo * o->d_lo * o->d_lo);
  L.pts = h->pts_dev;
  L.rp = S.rp;
  L.n_points = 1;
  L.max_nb = nb;
  DrawOut d{theta_out, lpq_out, bins_out};
  RIFT_CK(h, launch_draw_cells(L, d, (uint32_t)n, h->stream));
  RIFT_CK(h, cudaStreamSynchronize(h->stream));
  return RIFT_OK;
}

rift_status rift_ile_marginalize(rift_ile *h, const rift_mc_opts *o, rift_mc_result *res) {
  if (!h || !res) return RIFT_EINVAL;
  rift_status s = check_opts(h, o);
  if (s != RIFT_OK) return s;
  std::memset(res, 0, sizeof(*res));
  const bool adaptive = (o->proposal == RIFT_PROPOSAL_ADAPTIVE) ||
                        (o->proposal == RIFT_PROPOSAL_LEARNED && o->fallback_neff > 0.0);
  const int nb = adaptive ? o->n_bins : 0;
  const int hb = std::max(1, std::min(64, (int)(o->n_per_round / 8192)));
  const size_t items = (size_t)RIFT_MAX_CELLS + o->n_per_round / (o->time_marg ? RIFT_TMARG_CHUNK : RIFT_CHUNK) + 1;
  if ((s = ensure_scratch(h, 1, items, adaptive ? o->n_per_round : 0, nb, hb)) != RIFT_OK) return s;
  return run_mc(h, o, 1, h->sc, res);
}

rift_status batch_run(rift_ile *h, const rift_mc_opts *o, rift_mc_result *res, bool keep_ell);

rift_status rift_ile_batch_marginalize(rift_ile *h, const rift_mc_opts *o, rift_mc_result *res) {
  return batch_run(h, o, res, false);
}

}  // extern "C"

rift_status batch_run(rift_ile *h, const rift_mc_opts *o, rift_mc_result *res, bool keep_ell) {
  if (!h || !res) return RIFT_EINVAL;
  rift_status s = check_opts(h, o);
  if (s != RIFT_OK) return s;
  if (o->resume || o->save) return fail(h, RIFT_EUNSUPPORTED, "resume/save: single-point marginalisation only");
  const int np = h->n_points;
  std::memset(res, 0, sizeof(*res) * np);
  const bool learned = (o->proposal == RIFT_PROPOSAL_LEARNED);
  const bool fallback = learned && o->fallback_neff > 0.0;
  // table machinery: the adaptive proposal, or learned points that may fall back to it
  const bool adaptive = (o->proposal == RIFT_PROPOSAL_ADAPTIVE) || fallback;
  const int nb = adaptive ? o->n_bins : 0;
  const int hb = std::max(1, std::min(64, (int)(o->n_per_round / 8192)));
  std::vector<int> lsv(3 * np);
  size_t items = 0;
  for (int p = 0; p < np; ++p) {
    int *ls = &lsv[3 * p];
    if (learned) {
      ls[0] = ls[1] = ls[2] = 0;
    } else if (o->strata[0] == 0 && o->strata[1] == 0 && o->strata[2] == 0) {
      if (o->time_marg) choose_strata_sky(o->n_per_round, ls, std::max(16, h->cell_target / 5));
      else choose_strata(h->pts[p].c, o->n_per_round, ls, h->cell_target);
    } else {
      for (int d = 0; d < 3; ++d) ls[d] = log2_pow2(o->strata[d]);
      if (ls[0] < 0 || ls[1] < 0 || ls[2] < 0) return fail(h, RIFT_EINVAL, "strata must be powers of two");
      if ((1 << (ls[0] + ls[1] + ls[2])) > RIFT_MAX_CELLS) return fail(h, RIFT_EINVAL, "more than RIFT_MAX_CELLS cells");
      if (o->time_marg && ls[2] != 0) return fail(h, RIFT_EINVAL, "time-marginalised rounds are not stratified in t");
    }
    items += ((size_t)1 << (ls[0] + ls[1] + ls[2])) + o->n_per_round / (o->time_marg ? RIFT_TMARG_CHUNK : RIFT_CHUNK) + 1;
  }
  const bool keep = adaptive || keep_ell;
  if ((s = ensure_scratch(h, np, items, keep ? (size_t)np * o->n_per_round : 0, nb, hb)) != RIFT_OK) return s;
  if (keep_ell && !h->last) RIFT_CK(h, cache_dev_alloc((void **)&h->last, sizeof(RoundPt) * np));
  McScratch &S = h->sc;
  if (np > h->cap_pst) {
    cache_dev_free(h->pst); cache_host_free(h->pst_host);
    h->pst = nullptr; h->pst_host = nullptr; h->cap_pst = 0;
    RIFT_CK(h, cache_dev_alloc((void **)&h->pst, sizeof(PtState) * np));
    RIFT_CK(h, cache_host_alloc((void **)&h->pst_host, sizeof(PtState) * np));
    h->cap_pst = np;
  }
  if (!h->ctl) {
    RIFT_CK(h, cache_dev_alloc((void **)&h->ctl, sizeof(RoundCtl)));
    RIFT_CK(h, cache_host_alloc((void **)&h->ctl_host, sizeof(RoundCtl)));
  }
  if (!h->gstream) RIFT_CK(h, cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
  cudaStream_t st = h->gstream;
  RIFT_CK(h, cudaStreamSynchronize(h->stream));   // inputs uploaded on the handle's stream
  const int K = h->K, NT = taps_of(h->interp);
  if (learned && (s = prepare_learned(h, o, st)) != RIFT_OK) return s;
  // initial state
  for (int p = 0; p < np; ++p) {
    std::memset(&S.acc_host[p], 0, sizeof(AccState));
    S.acc_host[p].m = -INFINITY;
    std::memset(&h->pst_host[p], 0, sizeof(PtState));
    for (int d = 0; d < 3; ++d) h->pst_host[p].ls[d] = lsv[3 * p + d];
    h->pst_host[p].prop = learned ? 2 : (adaptive ? 1 : 0);
    h->pst_host[p].fb_round = -1;
    std::memset(&S.rp_host[p], 0, sizeof(RoundPt));
  }
  std::memset(h->ctl_host, 0, sizeof(RoundCtl));
  h->ctl_host->round = -1;
  RIFT_CK(h, cudaMemcpyAsync(S.acc, S.acc_host, sizeof(AccState) * np, cudaMemcpyHostToDevice, st));
  RIFT_CK(h, cudaMemcpyAsync(h->pst, h->pst_host, sizeof(PtState) * np, cudaMemcpyHostToDevice, st));
  RIFT_CK(h, cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(RoundCtl), cudaMemcpyHostToDevice, st));
  const size_t tstride = (size_t)3 * (nb + 1);
  BatchCtl B{};
  B.npr = o->n_per_round;
  B.np = np;
  B.max_evals = o->max_evals;
  B.n_eff_target = o->n_eff_target;
  B.max_rounds = o->max_rounds;
  B.adaptive = adaptive ? 1 : 0;
  B.adapt_rounds = o->adapt_rounds;
  B.nb = nb;
  B.tables = S.tables;
  B.lnw = S.lnw;
  B.learned = learned ? 1 : 0;
  B.keep_ell = keep_ell ? 1 : 0;
  B.gmm = h->gmm;
  B.last = keep_ell ? h->last : nullptr;
  B.tmarg = o->time_marg ? 1 : 0;
  B.point_id1 = o->point_id;
  B.fallback_neff = fallback ? o->fallback_neff : 0.0;
  if (adaptive) {
    float u[3 * (RIFT_MAXBINS + 1)];
    const float *src = o->tables;
    if (!src) {
      for (int d = 0; d < 3; ++d)
        for (int b = 0; b <= nb; ++b) u[d * (nb + 1) + b] = (float)((double)b / nb);
      src = u;
    }
    // both table buffers hold the round-0 tables when learned points may fall back: a point that
    // has not adapted yet reads whichever buffer the round reads
    for (int buf = 0; buf < (fallback ? 2 : 1); ++buf)
      for (int p = 0; p < np; ++p) {
        const float *sp = (o->tables && o->tables_per_point) ? src + p * tstride : src;
        RIFT_CK(h, cudaMemcpyAsync(S.tables + ((size_t)buf * np + p) * tstride, sp, sizeof(float) * tstride,
                                   cudaMemcpyHostToDevice, st));
      }
    RIFT_CK(h, cudaStreamSynchronize(st));
    for (int p = 0; p < np; ++p) { S.rp_host[p].proposal = 1; S.rp_host[p].ncell = 1; }
    RIFT_CK(h, cudaMemcpyAsync(S.rp, S.rp_host, sizeof(RoundPt) * np, cudaMemcpyHostToDevice, st));
    for (int buf = 0; buf < (fallback ? 2 : 1); ++buf)
      RIFT_CK(h, launch_tables_points(nullptr, 0, S.rp, np, nb, 0.0, S.tables + (size_t)buf * np * tstride,
                                      S.lnw + (size_t)buf * np * 3 * nb, st));
    for (int p = 0; p < np; ++p) { S.rp_host[p].proposal = 0; S.rp_host[p].ncell = 0; }
  }
  RIFT_CK(h, cudaMemcpyAsync(S.rp, S.rp_host, sizeof(RoundPt) * np, cudaMemcpyHostToDevice, st));
  // launch shape of the persistent cell kernel
  const int block = RIFT_CELL_BLOCK;
  int smem_sm = 0;
  RIFT_CK(h, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device));
  const CellShape shp = cell_shape(h, K, NT, o->time_marg, h->max_M, h->max_pairK, nb, smem_sm);
  const int tm = shp.tm;
  const long long budget = shp.budget;
  const size_t smem = shp.smem;
  const int bps = cells_blocks_per_sm(K, NT, smem, block, tm);
  if (bps < 1) return fail(h, RIFT_EUNSUPPORTED, "cell kernel does not fit on an SM");
  CellLaunch L{};
  L.seed = o->seed;
  L.d_lo3 = (float)(o->d_lo * o->d_lo * o->d_lo);
  L.d_span3 = (float)(o->d_hi * o->d_hi * o->d_hi - o->d_lo * o->d_lo * o->d_lo);
  L.pts = h->pts_dev;
  L.rp = S.rp;
  L.n_points = np;
  L.win_budget = (int)budget;
  L.n_items = &h->ctl->n_items;
  L.queue = &h->ctl->queue;
  L.qa = h->q_arena;
  L.ca = h->c_arena;
  L.partials = S.partials;
  L.ell_buf = keep ? S.ell : nullptr;
  L.bin_buf = keep ? S.bins : nullptr;
  L.flags = h->flags;
  L.max_M = shp.ys_modes;
  L.max_pairK = h->max_pairK;
  L.max_nb = nb;
  L.learned = learned ? 1 : 0;
  L.fault_nan = fault_is("nan_sample") ? 1 : 0;
  L.fault_stall = fault_is("stage_timeout") ? 1 : 0;
  L.tmarg = tm;
  const bool refine = o->refine && !o->time_marg;
  if (refine) {
    rift_status rs0 = ensure_refine(h, np, S.max_items, st);
    if (rs0 != RIFT_OK) return rs0;
    L.cand = h->cand;
    L.cmax = h->cmax;
  }
  const double lo3 = o->d_lo * o->d_lo * o->d_lo, span3 = o->d_hi * o->d_hi * o->d_hi - lo3;
  const int grid = h->num_sms * bps;
  // capture G rounds: update -> cells -> merge -> (refine) -> (adaptive) hist -> tables
  const int G = std::max(1, h->graph_rounds);
  // every argument the captured launches take by value (pointers included): an equal key means the
  // cached graph launches exactly these kernels with these arguments
  std::vector<unsigned char> key;
  auto put = [&key](const void *x, size_t nbytes) {
    const unsigned char *c = static_cast<const unsigned char *>(x);
    key.insert(key.end(), c, c + nbytes);
  };
  const float beta_f = (float)o->beta;
  const double eps_d = o->floor_eps;
  const int ints[9] = {K, NT, grid, block, (int)smem, G, adaptive ? 1 : 0, nb, S.hblocks};
  put(&B, sizeof(B));
  put(&L, sizeof(L));
  put(ints, sizeof(ints));
  put(&beta_f, sizeof(beta_f));
  put(&eps_d, sizeof(eps_d));
  const void *ptrs[12] = {h->pst, S.acc, S.rp, h->ctl, S.partials, S.ell, S.hist,
                          refine ? h->rscratch : nullptr, refine ? h->rstate : nullptr, h->pd_dev, h->uv64, h->flags};
  put(ptrs, sizeof(ptrs));
  const double refd[2] = {refine ? lo3 : 0.0, refine ? span3 : 0.0};
  put(refd, sizeof(refd));
  if (!h->gexec || key != h->gkey) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->gkey.clear();
    cudaGraph_t graph = nullptr;
    RIFT_CK(h, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    for (int g = 0; g < G && ce == cudaSuccess; ++g) {
      if ((ce = launch_round_update(B, h->pst, S.acc, S.rp, h->ctl, st)) != cudaSuccess) break;
      if ((ce = launch_cells(K, NT, L, grid, block, smem, st)) != cudaSuccess) break;
      if ((ce = launch_merge_points(S.partials, S.rp, np, S.acc, st)) != cudaSuccess) break;
      if (refine && (ce = launch_refine(h->pts_dev, h->pd_dev, h->uv64, h->q_arena, S.rp, S.acc, h->cmax, h->cand, np, o->seed,
                                        lo3, span3, h->rscratch, h->rstate, h->flags, st)) != cudaSuccess)
        break;
      if (adaptive) {
        if ((ce = launch_hist_ctl(S.ell, S.bins, S.rp, np, S.acc, beta_f, nb, S.hist, S.hblocks, h->ctl, st)) !=
            cudaSuccess)
          break;
        if ((ce = launch_tables_ctl(S.hist, S.hblocks, S.rp, np, nb, eps_d, B, h->ctl, st)) != cudaSuccess) break;
      }
    }
    cudaError_t ee = cudaStreamEndCapture(st, &graph);
    if (ce != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(h, ce, "graph capture"); }
    if (ee != cudaSuccess) return cuda_fail(h, ee, "cudaStreamEndCapture");
    ee = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ee != cudaSuccess) { h->gexec = nullptr; return cuda_fail(h, ee, "cudaGraphInstantiate"); }
    h->gkey = key;
  }
  cudaGraphExec_t exec = h->gexec;
  // replay until a round update finds no active point (all results accounted)
  uint64_t max_np_evals = o->max_evals;
  const uint64_t rounds_cap = (max_np_evals + o->n_per_round - 1) / o->n_per_round + 2;
  const uint64_t replay_cap = (o->max_rounds > 0 ? std::min<uint64_t>(rounds_cap, o->max_rounds + 2) : rounds_cap) / G + 2;
  int replays = 0;
  rift_status status = RIFT_OK;
  for (;;) {
    cudaError_t e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(RoundCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { status = cuda_fail(h, e, "graph replay"); break; }
    ++replays;
    if (h->ctl_host->active == 0) break;
    if ((uint64_t)replays > replay_cap) { status = fail(h, RIFT_ETIMEOUT, "batched run did not terminate"); break; }
  }
  if (status != RIFT_OK) return status;
  RIFT_CK(h, cudaMemcpyAsync(S.acc_host, S.acc, sizeof(AccState) * np, cudaMemcpyDeviceToHost, st));
  RIFT_CK(h, cudaMemcpyAsync(h->pst_host, h->pst, sizeof(PtState) * np, cudaMemcpyDeviceToHost, st));
  if (refine)
    RIFT_CK(h, cudaMemcpyAsync(h->rstate_host, h->rstate, sizeof(RefineState) * np, cudaMemcpyDeviceToHost, st));
  RIFT_CK(h, cudaStreamSynchronize(st));
  if (o->tables_out && adaptive) {
    // Round r reads table buffer (number of adapting rounds before r) mod 2 and an adapting round
    // writes the other one, so after a point's last round its next proposal is in buffer
    // min(rounds, adapt_rounds) mod 2; later rounds of other points do not touch its slot.
    const size_t tstride = (size_t)3 * (nb + 1);
    for (int p = 0; p < np; ++p) {
      const long long rp_ = h->pst_host[p].rounds;
      const long long na = (o->adapt_rounds < 0) ? rp_ : std::min<long long>(rp_, o->adapt_rounds);
      const size_t buf = (size_t)(na & 1);
      RIFT_CK(h, cudaMemcpyAsync(o->tables_out + p * tstride, S.tables + (buf * np + p) * tstride,
                                 sizeof(float) * tstride, cudaMemcpyDeviceToHost, st));
    }
    RIFT_CK(h, cudaStreamSynchronize(st));
  }
  rift_status fl = read_flags(h);
  rift_status overall = fl;
  for (int p = 0; p < np; ++p) {
    fill_result(S.acc_host[p], &res[p], refine ? &h->rstate_host[p] : nullptr);
    res[p].rounds = h->pst_host[p].rounds;
    res[p].kernel_launches = (p == 0) ? replays * G * ((adaptive ? 5 : 3) + (refine ? 3 : 0)) : 0;
    res[p].fallback_round = h->pst_host[p].fb_round;
    for (int d = 0; d < 3; ++d) res[p].strata[d] = 1 << lsv[3 * p + d];
    rift_status sp = fl;
    if (sp == RIFT_OK && res[p].n_eff < o->n_eff_target) sp = RIFT_ENOTCONVERGED;
    res[p].status = sp;
    if (overall == RIFT_OK && sp != RIFT_OK) overall = sp;
  }
  return overall;
}

extern "C" {

rift_status rift_ile_batch_summary(rift_ile *h, float *out_dev) {
  if (!h || !out_dev) return RIFT_EINVAL;
  RIFT_CK(h, launch_summary(h->pts_dev, h->q_arena, h->c_arena, h->tau0, h->n_points, out_dev, h->stream));
  RIFT_CK(h, cudaStreamSynchronize(h->stream));
  return RIFT_OK;
}

rift_status rift_ile_set_proposal_head(rift_ile *h, const float *head_host) {
  if (!h || !head_host) return RIFT_EINVAL;
  rift_status s = ensure_learned(h);
  if (s != RIFT_OK) return s;
  RIFT_CK(h, cudaMemcpy(h->head, head_host, sizeof(float) * (size_t)h->n_points * RIFT_MDN_HEAD,
                        cudaMemcpyHostToDevice));
  h->head_given = true;
  return RIFT_OK;
}

rift_status rift_ile_boxes(rift_ile *h, double d_lo, double d_hi, float *out) {
  if (!h || !out || !(d_lo > 0) || !(d_hi > d_lo)) return RIFT_EINVAL;
  for (int p = 0; p < h->n_points; ++p) {
    float *o = out + (size_t)p * 10;
    const double a[5] = {0.0, -1.0, h->pts[p].t_lo, -1.0, std::log(d_lo)};
    const double b[5] = {2.0 * kPi, 1.0, h->pts[p].t_hi, 1.0, std::log(d_hi)};
    for (int d = 0; d < 5; ++d) { o[d] = (float)a[d]; o[5 + d] = (float)b[d]; }
  }
  return RIFT_OK;
}

// Arguments the row and harvest kernels need to re-draw the samples of a run made with `o`.
static CellLaunch rows_launch(const rift_ile *h, const rift_mc_opts *o) {
  CellLaunch L{};
  L.seed = o->seed;
  L.d_lo3 = (float)(o->d_lo * o->d_lo * o->d_lo);
  L.d_span3 = (float)(o->d_hi * o->d_hi * o->d_hi - o->d_lo * o->d_lo * o->d_lo);
  L.pts = h->pts_dev;
  L.n_points = h->n_points;
  return L;
}

rift_status rift_ile_batch_harvest(rift_ile *h, const rift_mc_opts *o, int H, double beta, float *theta_dev,
                                   rift_mc_result *res) {
  if (!h || !o || !theta_dev || !res || H < 1 || !(beta > 0)) return RIFT_EINVAL;
  rift_status s = batch_run(h, o, res, true);
  if (s != RIFT_OK && s != RIFT_ENOTCONVERGED) return s;
  const int np = h->n_points;
  McScratch &S = h->sc;
  const size_t need = (size_t)np * H;
  if (need > h->cap_hidx) {
    cache_dev_free(h->hidx);
    h->hidx = nullptr;
    h->cap_hidx = 0;
    RIFT_CK(h, cache_dev_alloc((void **)&h->hidx, sizeof(int) * need));
    h->cap_hidx = need;
  }
  cudaStream_t st = h->gstream;
  RIFT_CK(h, launch_resample(S.ell, h->last, S.acc, np, (float)beta, H, h->hidx, st));
  const CellLaunch L = rows_launch(h, o);
  RIFT_CK(h, launch_harvest_theta(L, h->last, h->hidx, H, theta_dev, st));
  RIFT_CK(h, cudaStreamSynchronize(st));
  return s;
}

rift_status rift_ile_samples(rift_ile *h, const rift_mc_opts *o, size_t cap, float *out_dev, uint64_t *n_out,
                             rift_mc_result *res) {
  if (!h || !o || !res || !n_out || (cap > 0 && !out_dev)) return RIFT_EINVAL;
  rift_status s = batch_run(h, o, res, true);
  if (s != RIFT_OK && s != RIFT_ENOTCONVERGED) return s;
  const int np = h->n_points;
  cudaStream_t st = h->gstream;
  const CellLaunch L = rows_launch(h, o);
  RIFT_CK(h, launch_rows(L, h->last, h->sc.ell, nullptr, cap, RIFT_SAMPLE_COLS, np, out_dev, st));
  std::vector<RoundPt> last(np);
  RIFT_CK(h, cudaMemcpyAsync(last.data(), h->last, sizeof(RoundPt) * np, cudaMemcpyDeviceToHost, st));
  RIFT_CK(h, cudaStreamSynchronize(st));
  for (int p = 0; p < np; ++p) n_out[p] = last[p].n;
  return s;
}

rift_status rift_ile_posterior(rift_ile *h, const rift_mc_opts *o, int H, float *out_dev, int *idx_dev,
                               rift_mc_result *res) {
  if (!h || !o || !res || !out_dev || H < 1) return RIFT_EINVAL;
  rift_status s = batch_run(h, o, res, true);
  if (s != RIFT_OK && s != RIFT_ENOTCONVERGED) return s;
  const int np = h->n_points;
  int *idx = idx_dev;
  if (!idx) {
    const size_t need = (size_t)np * H;
    if (need > h->cap_hidx) {
      cache_dev_free(h->hidx);
      h->hidx = nullptr;
      h->cap_hidx = 0;
      RIFT_CK(h, cache_dev_alloc((void **)&h->hidx, sizeof(int) * need));
      h->cap_hidx = need;
    }
    idx = h->hidx;
  }
  cudaStream_t st = h->gstream;
  RIFT_CK(h, launch_resample(h->sc.ell, h->last, h->sc.acc, np, 1.0f, H, idx, st));
  const CellLaunch L = rows_launch(h, o);
  RIFT_CK(h, launch_rows(L, h->last, h->sc.ell, idx, (size_t)H, RIFT_POSTERIOR_COLS, np, out_dev, st));
  if (o->time_marg) {
    RIFT_CK(h, cudaMemsetAsync(h->flags, 0, sizeof(uint32_t), st));
    RIFT_CK(h, launch_tdraw(h->K, h->interp, h->pts_dev, np, h->max_pairK / h->K, h->max_M, h->q_arena, h->c_arena,
                            h->last, o->seed, H, out_dev, h->flags, st));
  }
  RIFT_CK(h, cudaStreamSynchronize(st));
  if (o->time_marg) {
    const rift_status f = read_flags(h);
    if (f != RIFT_OK) return f;
  }
  return s;
}


rift_status rift_source_frame(int n_det, const double *det_tensor, const double *det_pos, int n_modes, const int *lm,
                              double t_ref_gps, double d_ref_mpc, size_t n, const double *src, double *coef,
                              double *tk) {
  const int K = n_det, M = n_modes;
  if (K < 1 || K > RIFT_MAX_DET || M < 1 || M > RIFT_MAX_MODES) return RIFT_EINVAL;
  if (!det_tensor || !det_pos || !lm || !(d_ref_mpc > 0) || !std::isfinite(t_ref_gps)) return RIFT_EINVAL;
  if (n == 0) return RIFT_OK;
  if (!src || !coef || !tk) return RIFT_EINVAL;
  // the detectors and modes as the likelihood kernels hold them, with times in seconds
  PointC c;
  std::memset(&c, 0, sizeof(c));
  c.K = K; c.M = M; c.fs = 1.f; c.dref = (float)d_ref_mpc;
  split(gmst_rad(t_ref_gps) / (2.0 * kPi), c.g_hi, c.g_lo);
  int perm[RIFT_MAX_MODES];
  for (int a = 0; a < M; ++a) {
    const int l = lm[2 * a], m = lm[2 * a + 1];
    if (l < 2 || l > 4 || m < -l || m > l) return RIFT_EINVAL;
    for (int b = 0; b < a; ++b)
      if (lm[2 * b] == l && lm[2 * b + 1] == m) return RIFT_EINVAL;
    perm[a] = a;
  }
  std::sort(perm, perm + M, [&](int x, int y) {
    return lm[2 * x] != lm[2 * y] ? lm[2 * x] < lm[2 * y] : lm[2 * x + 1] < lm[2 * y + 1];
  });
  for (int a = 0; a < M; ++a) {
    swsh_terms(lm[2 * perm[a]], lm[2 * perm[a] + 1], c.mode[a]);
    c.canon_mask |= 1u << canon_index(c.mode[a].l, c.mode[a].m);
  }
  for (int j = 0; j < RIFT_MAXM; ++j) {
    ModeC t;
    swsh_terms(canon_l(j), canon_m(j), t);
    for (int r = 0; r < t.nterm; ++r) c.ccoef[j][r] = t.coef[r];
  }
  for (int k = 0; k < K; ++k) {
    const double *t = det_tensor + 9 * k;
    DetC &D = c.det[k];
    D.d[0] = (float)t[0]; D.d[1] = (float)t[1]; D.d[2] = (float)t[2];
    D.d[3] = (float)t[4]; D.d[4] = (float)t[5]; D.d[5] = (float)t[8];
    for (int i = 0; i < 3; ++i) split(det_pos[3 * k + i] / kC, D.P[i], D.Plo[i]);
  }
  std::vector<float> in(8 * n);
  for (size_t i = 0; i < n; ++i) {
    const double *q = src + 7 * i;
    for (int j = 0; j < 7; ++j)
      if (!std::isfinite(q[j])) return RIFT_EINVAL;
    if (!(q[6] > 0)) return RIFT_EINVAL;
    in[i] = (float)q[0];
    in[n + i] = (float)q[1];
    split(q[2], in[2 * n + i], in[3 * n + i]);
    in[4 * n + i] = (float)q[3];
    in[5 * n + i] = (float)q[4];
    in[6 * n + i] = (float)q[5];
    in[7 * n + i] = (float)q[6];
  }
  PointC *pd = nullptr;
  float *sd = nullptr;
  float2 *cd = nullptr, *td = nullptr;
  std::vector<float2> cf(n * K * M), tf(n * K);
  cudaError_t e;
  if ((e = cudaMalloc(&pd, sizeof(PointC))) == cudaSuccess && (e = cudaMalloc(&sd, sizeof(float) * in.size())) == cudaSuccess &&
      (e = cudaMalloc(&cd, sizeof(float2) * cf.size())) == cudaSuccess &&
      (e = cudaMalloc(&td, sizeof(float2) * tf.size())) == cudaSuccess &&
      (e = cudaMemcpy(pd, &c, sizeof(PointC), cudaMemcpyHostToDevice)) == cudaSuccess &&
      (e = cudaMemcpy(sd, in.data(), sizeof(float) * in.size(), cudaMemcpyHostToDevice)) == cudaSuccess &&
      (e = launch_source_frame(K, pd, n, sd, cd, td, nullptr)) == cudaSuccess &&
      (e = cudaMemcpy(cf.data(), cd, sizeof(float2) * cf.size(), cudaMemcpyDeviceToHost)) == cudaSuccess)
    e = cudaMemcpy(tf.data(), td, sizeof(float2) * tf.size(), cudaMemcpyDeviceToHost);
  cudaFree(pd);
  cudaFree(sd);
  cudaFree(cd);
  cudaFree(td);
  if (e != cudaSuccess) return (e == cudaErrorMemoryAllocation) ? RIFT_ENOMEM : RIFT_ECUDA;
  for (size_t i = 0; i < n; ++i)
    for (int k = 0; k < K; ++k) {
      tk[i * K + k] = (double)tf[i * K + k].x + (double)tf[i * K + k].y;
      for (int a = 0; a < M; ++a) {   // stored (canonical) order -> the caller's order
        const float2 v = cf[(i * K + k) * M + a];
        double *o = coef + 2 * ((i * K + k) * M + perm[a]);
        o[0] = v.x;
        o[1] = v.y;
      }
    }
  return RIFT_OK;
}

rift_status rift_ile_get_tune(const rift_ile *h, rift_tune *out) {
  if (!h || !out) return RIFT_EINVAL;
  out->cell_samples = h->cell_target;
  out->smem_split = h->smem_split;
  out->ms = 0.0;
  return RIFT_OK;
}

rift_status rift_ile_set_tune(rift_ile *h, const rift_tune *t) {
  if (!h || !t) return RIFT_EINVAL;
  if (t->cell_samples < 64 || t->cell_samples > 65536 || t->smem_split < 1 || t->smem_split > 8)
    return fail(h, RIFT_EINVAL, "tune out of range");
  h->cell_target = t->cell_samples;
  h->smem_split = t->smem_split;
  return RIFT_OK;
}

rift_status rift_ile_autotune(rift_ile *h, const rift_mc_opts *o, int reps, rift_tune *best) {
  if (!h || !o || !best || reps < 1) return RIFT_EINVAL;
  rift_status s = check_opts(h, o);
  if (s != RIFT_OK) return s;
  rift_mc_opts t = *o;
  t.max_evals = (uint64_t)o->n_per_round * reps;
  t.n_eff_target = 1e300;
  t.dbg_ell = nullptr;
  t.dbg_tables = nullptr;
  t.timing = 0;
  t.max_rounds = reps;
  t.resume = nullptr;
  t.save = nullptr;
  t.tables_out = nullptr;
  const int old_target = h->cell_target, old_ctas = h->smem_split;
  const int targets[5] = {320, 640, 960, 1280, 2048}, splits[4] = {2, 3, 4, 6};
  std::vector<rift_mc_result> res((size_t)h->n_points);
  double best_ms = 1e300;
  rift_tune b{old_target, old_ctas, 0.0};
  cudaEvent_t e0, e1;
  RIFT_CK(h, cudaEventCreate(&e0));
  RIFT_CK(h, cudaEventCreate(&e1));
  for (int ti = 0; ti < 5; ++ti)
    for (int si = 0; si < 4; ++si) {
      const int c = splits[si];
      h->cell_target = targets[ti];
      h->smem_split = c;
      // one untimed call (first-use costs), then the timed one
      for (int pass = 0; pass < 2; ++pass) {
        RIFT_CK(h, cudaDeviceSynchronize());
        RIFT_CK(h, cudaEventRecord(e0, 0));
        s = (h->n_points > 1) ? rift_ile_batch_marginalize(h, &t, res.data()) : rift_ile_marginalize(h, &t, res.data());
        RIFT_CK(h, cudaEventRecord(e1, 0));
        RIFT_CK(h, cudaEventSynchronize(e1));
        if (s != RIFT_OK && s != RIFT_ENOTCONVERGED) {
          h->cell_target = old_target;
          h->smem_split = old_ctas;
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return s;
        }
      }
      float ms = 0.f;
      RIFT_CK(h, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        b.cell_samples = targets[ti];
        b.smem_split = c;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->cell_target = b.cell_samples;
  h->smem_split = b.smem_split;
  b.ms = best_ms / reps;
  *best = b;
  return RIFT_OK;
}

}  // extern "C"

// Internal entry used by the allocation-free entry point (noalloc.cu): the runner with
// caller-provided scratch.
rift_status rift_internal_run_static(rift_ile *h, const rift_mc_opts *o, McScratch &S, rift_mc_result *res) {
  if (!h || !res) return RIFT_EINVAL;
  rift_status s = check_opts(h, o);
  if (s != RIFT_OK) return s;
  std::memset(res, 0, sizeof(*res));
  return run_mc(h, o, 1, S, res);
}

rift_status rift_internal_fail(rift_ile *h, rift_status s, const char *msg) { return fail(h, s, msg); }
