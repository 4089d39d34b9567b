// C ABI of the extrinsic-likelihood library: validation, per-point constants (FP64
// on the host, once per point), device arenas, and the Monte Carlo round loop.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rift_ile.h"
#include "rift_device.cuh"
#include "rift_internal.h"

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

struct Point {
  PointC c;
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
  // scratch (owned)
  uint32_t *flags = nullptr;
  Part *partials = nullptr;
  int max_parts = 0;
  AccState *acc = nullptr;
  size_t acc_n = 0;
  float *ell_buf = nullptr;
  uint32_t *bin_buf = nullptr;
  size_t ebuf_n = 0;
  unsigned long long *hist_part = nullptr;
  size_t hist_n = 0;
  float *tables = nullptr;  // [2][3][nb+1] ping-pong
  float *lnw = nullptr;     // [2][3][nb]
  int tab_nb = 0;
  float *stage = nullptr;   // lnL_host staging [8][n]
  size_t stage_n = 0;
  int max_M = 0;
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
rift_status build_point(rift_ile *h, const rift_ile_desc *d, Point &P, std::vector<float2> &qv,
                        std::vector<float4> &cv) {
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
  c.fs = (float)d->fs;
  if ((double)c.fs != d->fs) return fail(h, RIFT_EINVAL, "fs must be exactly representable in float32");
  c.dref = (float)d->d_ref_mpc;
  const double g = gmst_rad(d->t_ref_gps) / (2.0 * kPi);
  split(g, c.g_hi, c.g_lo);
  split((d->t_hi - d->t_lo) * d->fs, c.A, c.Alo);
  c.t_lo = (float)d->t_lo;
  c.t_span = (float)(d->t_hi - d->t_lo);
  P.t_lo = d->t_lo; P.t_hi = d->t_hi;
  // modes
  for (int a = 0; a < M; ++a) {
    const int l = d->lm[2 * a], m = d->lm[2 * a + 1];
    if (l < 2 || l > 4 || m < -l || m > l) return fail(h, RIFT_EINVAL, "mode (l,m) outside 2<=l<=4, |m|<=l");
    for (int b = 0; b < a; ++b)
      if (d->lm[2 * b] == l && d->lm[2 * b + 1] == m) return fail(h, RIFT_EINVAL, "duplicate mode");
    swsh_terms(l, m, c.mode[a]);
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
  for (int i = 0; i < K * M * T * 2; ++i)
    if (!std::isfinite(d->Q[i])) return fail(h, RIFT_EINVAL, "non-finite Q");
  // Q arena block: [K][T][Mp] complex64, zero padded
  c.q_off = (long long)qv.size();
  qv.resize(qv.size() + (size_t)K * T * c.Mp, make_float2(0.f, 0.f));
  float2 *qb = qv.data() + c.q_off;
  for (int k = 0; k < K; ++k)
    for (int a = 0; a < M; ++a)
      for (int j = 0; j < T; ++j) {
        const double *q = d->Q + 2 * (((size_t)k * M + a) * T + j);
        qb[((size_t)k * T + j) * c.Mp + a] = make_float2((float)q[0], (float)q[1]);
      }
  // pair coefficients [pair][K] = (U, V) upper triangle, off-diagonal doubled
  c.uv_off = (long long)cv.size();
  for (int a = 0; a < M; ++a)
    for (int b = a; b < M; ++b)
      for (int k = 0; k < K; ++k) {
        const double f = (a == b) ? 1.0 : 2.0;
        const double *u = d->U + 2 * ((k * M + a) * M + b), *v = d->V + 2 * ((k * M + a) * M + b);
        cv.push_back(make_float4((float)(f * u[0]), (float)(f * u[1]), (float)(f * v[0]), (float)(f * v[1])));
      }
  return RIFT_OK;
}

rift_status ensure_scratch(rift_ile *h, int parts, size_t ebuf, int nb, int hist_parts) {
  if (parts > h->max_parts) {
    if (h->partials) cudaFree(h->partials);
    h->partials = nullptr;
    RIFT_CK(h, cudaMalloc(&h->partials, sizeof(Part) * parts));
    h->max_parts = parts;
  }
  if (ebuf > h->ebuf_n) {
    if (h->ell_buf) cudaFree(h->ell_buf);
    if (h->bin_buf) cudaFree(h->bin_buf);
    h->ell_buf = nullptr; h->bin_buf = nullptr;
    RIFT_CK(h, cudaMalloc(&h->ell_buf, sizeof(float) * ebuf));
    RIFT_CK(h, cudaMalloc(&h->bin_buf, sizeof(uint32_t) * ebuf));
    h->ebuf_n = ebuf;
  }
  if (nb > 0) {
    const size_t need = (size_t)hist_parts * 3 * nb;
    if (need > h->hist_n) {
      if (h->hist_part) cudaFree(h->hist_part);
      h->hist_part = nullptr;
      RIFT_CK(h, cudaMalloc(&h->hist_part, sizeof(unsigned long long) * need));
      h->hist_n = need;
    }
    if (nb != h->tab_nb) {
      if (h->tables) cudaFree(h->tables);
      if (h->lnw) cudaFree(h->lnw);
      h->tables = nullptr; h->lnw = nullptr;
      RIFT_CK(h, cudaMalloc(&h->tables, sizeof(float) * 2 * 3 * (nb + 1)));
      RIFT_CK(h, cudaMalloc(&h->lnw, sizeof(float) * 2 * 3 * nb));
      h->tab_nb = nb;
    }
  }
  return RIFT_OK;
}

rift_status create_impl(const rift_ile_desc *descs, int n, rift_ile **out) {
  if (!out) return RIFT_EINVAL;
  *out = nullptr;
  if (!descs || n < 1) return RIFT_EINVAL;
  rift_ile *h = new (std::nothrow) rift_ile();
  if (!h) return RIFT_ENOMEM;
  h->n_points = n;
  h->K = descs[0].n_det;
  h->stream = (cudaStream_t)descs[0].cuda_stream;
  std::vector<float2> qv;
  std::vector<float4> cv;
  h->pts.resize(n);
  for (int i = 0; i < n; ++i) {
    if (descs[i].n_det != h->K) { rift_status s = fail(h, RIFT_EINVAL, "points differ in n_det"); rift_ile_destroy(h); return s; }
    rift_status s = build_point(h, &descs[i], h->pts[i], qv, cv);
    if (s != RIFT_OK) {
      fprintf(stderr, "rift_ile_create: point %d: %s\n", i, h->err.c_str());
      rift_ile_destroy(h);
      return s;
    }
    h->max_M = std::max(h->max_M, h->pts[i].c.M);
  }
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess) {
    fprintf(stderr, "rift_ile_create: %s\n", cudaGetErrorString(e));
    rift_ile_destroy(h);
    return RIFT_ECUDA;
  }
  std::vector<PointC> pc(n);
  for (int i = 0; i < n; ++i) pc[i] = h->pts[i].c;
  rift_status s = RIFT_OK;
  if ((e = cudaMalloc(&h->pts_dev, sizeof(PointC) * n)) != cudaSuccess ||
      (e = cudaMalloc(&h->q_arena, sizeof(float2) * std::max<size_t>(qv.size(), 2))) != cudaSuccess ||
      (e = cudaMalloc(&h->c_arena, sizeof(float4) * std::max<size_t>(cv.size(), 1))) != cudaSuccess ||
      (e = cudaMalloc(&h->flags, sizeof(uint32_t))) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->pts_dev, pc.data(), sizeof(PointC) * n, cudaMemcpyHostToDevice, h->stream)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(h->q_arena, qv.data(), sizeof(float2) * qv.size(), cudaMemcpyHostToDevice, h->stream)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(h->c_arena, cv.data(), sizeof(float4) * cv.size(), cudaMemcpyHostToDevice, h->stream)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(h->flags, 0, sizeof(uint32_t), h->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
    s = (e == cudaErrorMemoryAllocation) ? RIFT_ENOMEM : RIFT_ECUDA;
    fprintf(stderr, "rift_ile_create: %s\n", cudaGetErrorString(e));
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
      for (int d = 0; d < 3; ++d) {
        const float *c = o->tables + d * (o->n_bins + 1);
        if (c[0] != 0.f || c[o->n_bins] != 1.f) return fail(h, RIFT_EINVAL, "tables must start at 0 and end at 1");
        for (int b = 0; b < o->n_bins; ++b)
          if (!(c[b + 1] > c[b])) return fail(h, RIFT_EINVAL, "tables must be strictly increasing");
      }
    }
  } else if (o->proposal == RIFT_PROPOSAL_LEARNED) {
    return fail(h, RIFT_EUNSUPPORTED, "learned proposal: use rift_mdn_* entry points");
  } else if (o->proposal != RIFT_PROPOSAL_PRIOR) {
    return fail(h, RIFT_EINVAL, "unknown proposal");
  }
  return RIFT_OK;
}

void fill_result(const AccState &a, rift_mc_result *r) {
  r->acc_max = a.m;
  r->acc_s1 = a.s1 + a.c1;
  r->acc_s2 = a.s2 + a.c2;
  r->n_evals = a.n;
  const double n = (double)a.n;
  if (a.n == 0 || !(r->acc_s1 > 0)) {
    r->lnL_marg = -INFINITY; r->n_eff = 0; r->n_eff_kish = 0; r->sigma = INFINITY;
    return;
  }
  r->lnL_marg = a.m + std::log(r->acc_s1) - std::log(n);
  r->n_eff = r->acc_s1;
  r->n_eff_kish = r->acc_s1 * r->acc_s1 / r->acc_s2;
  r->sigma = (a.n > 1) ? std::sqrt(std::max(n * r->acc_s2 / (r->acc_s1 * r->acc_s1) - 1.0, 0.0) / (n - 1.0)) : INFINITY;
}

rift_status read_flags(rift_ile *h) {
  uint32_t f = 0;
  RIFT_CK(h, cudaMemcpyAsync(&f, h->flags, sizeof(f), cudaMemcpyDeviceToHost, h->stream));
  RIFT_CK(h, cudaMemsetAsync(h->flags, 0, sizeof(uint32_t), h->stream));
  RIFT_CK(h, cudaStreamSynchronize(h->stream));
  if (f & RIFT_FLAG_WINDOW) return fail(h, RIFT_EWINDOW, "interpolation taps left the Q window");
  if (f & RIFT_FLAG_NONFINITE) return fail(h, RIFT_ENONFINITE, "non-finite log-likelihood");
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

rift_status rift_ile_create(const rift_ile_desc *desc, rift_ile **out) { return create_impl(desc, 1, out); }

rift_status rift_ile_batch_create(const rift_ile_desc *descs, int n_points, rift_ile **out) {
  return create_impl(descs, n_points, out);
}

void rift_ile_destroy(rift_ile *h) {
  if (!h) return;
  if (h->stream || true) cudaStreamSynchronize(h->stream);
  cudaFree(h->pts_dev);
  cudaFree(h->q_arena);
  cudaFree(h->c_arena);
  cudaFree(h->flags);
  cudaFree(h->partials);
  cudaFree(h->acc);
  cudaFree(h->ell_buf);
  cudaFree(h->bin_buf);
  cudaFree(h->hist_part);
  cudaFree(h->tables);
  cudaFree(h->lnw);
  cudaFree(h->stage);
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

rift_status rift_ile_lnL_host(rift_ile *h, size_t n, const float *ra, const float *dec, const float *t,
                              const float *psi, const float *phi, const float *incl, const float *dist,
                              float *lnL_out) {
  if (!h) return RIFT_EINVAL;
  if (n == 0) return RIFT_OK;
  if (!ra || !dec || !t || !psi || !phi || !incl || !dist || !lnL_out) return fail(h, RIFT_EINVAL, "null sample array");
  if (n > h->stage_n) {
    cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_n = 0;
    RIFT_CK(h, cudaMalloc(&h->stage, sizeof(float) * 8 * n));
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
  if (n > 0xFFFFFFFFull) return fail(h, RIFT_EINVAL, "n too large");
  const int nb = (o->proposal == RIFT_PROPOSAL_ADAPTIVE) ? o->n_bins : 0;
  if ((s = ensure_scratch(h, 1, 0, nb, 1)) != RIFT_OK) return s;
  McParams prm{};
  prm.seed = o->seed; prm.round = round; prm.n = (uint32_t)n; prm.point_id = o->point_id;
  prm.proposal = (nb > 0 && tables) ? 1 : 0;
  prm.nb = nb;
  prm.d_lo3 = (float)(o->d_lo * o->d_lo * o->d_lo);
  prm.d_span3 = (float)(o->d_hi * o->d_hi * o->d_hi - o->d_lo * o->d_lo * o->d_lo);
  if (prm.proposal) {
    RIFT_CK(h, cudaMemcpyAsync(h->tables, tables, sizeof(float) * 3 * (nb + 1), cudaMemcpyDeviceToDevice, h->stream));
    RIFT_CK(h, launch_tables(nullptr, 0, nb, 0.0, h->tables, h->lnw, h->stream));
    prm.tables = h->tables; prm.lnw = h->lnw;
  }
  DrawOut d{theta_out, lpq_out, bins_out};
  RIFT_CK(h, launch_draw(h->K, h->pts_dev, h->pts[0].c, prm, d, h->stream));
  return RIFT_OK;
}

rift_status rift_ile_marginalize(rift_ile *h, const rift_mc_opts *o, rift_mc_result *res) {
  if (!h || !res) return RIFT_EINVAL;
  rift_status s = check_opts(h, o);
  if (s != RIFT_OK) return s;
  std::memset(res, 0, sizeof(*res));
  const Point &p = h->pts[0];
  const int block = RIFT_MC_BLOCK;
  const bool adaptive = (o->proposal == RIFT_PROPOSAL_ADAPTIVE);
  const int nb = adaptive ? o->n_bins : 0;
  const size_t smem = rift_point_smem_bytes(h->K, p.c.npair, nb, block, p.c.M);
  if (smem > 200 * 1024) return fail(h, RIFT_EUNSUPPORTED, "shared memory footprint too large");
  int bps = mc_round_blocks_per_sm(h->K, smem, block);
  if (bps < 1) bps = 1;
  const uint32_t npr = o->n_per_round;
  int grid = std::max(1, std::min<int>(h->num_sms * bps, (int)((npr + block - 1) / block)));
  const int hist_grid = std::max(1, std::min(h->num_sms, (int)((npr + 255) / 256)));
  if ((s = ensure_scratch(h, grid, adaptive ? npr : 0, nb, hist_grid)) != RIFT_OK) return s;
  if (!h->acc) RIFT_CK(h, cudaMalloc(&h->acc, sizeof(AccState)));
  AccState a0{};
  a0.m = -INFINITY;
  RIFT_CK(h, cudaMemcpyAsync(h->acc, &a0, sizeof(a0), cudaMemcpyHostToDevice, h->stream));
  int cur = 0;
  if (adaptive) {
    if (o->tables) {
      RIFT_CK(h, cudaMemcpyAsync(h->tables, o->tables, sizeof(float) * 3 * (nb + 1), cudaMemcpyHostToDevice, h->stream));
    } else {
      std::vector<float> u(3 * (nb + 1));
      for (int d = 0; d < 3; ++d)
        for (int b = 0; b <= nb; ++b) u[d * (nb + 1) + b] = (float)((double)b / nb);
      RIFT_CK(h, cudaMemcpyAsync(h->tables, u.data(), sizeof(float) * u.size(), cudaMemcpyHostToDevice, h->stream));
      RIFT_CK(h, cudaStreamSynchronize(h->stream));
    }
    RIFT_CK(h, launch_tables(nullptr, 0, nb, 0.0, h->tables, h->lnw, h->stream));
  }
  McParams prm{};
  prm.seed = o->seed; prm.point_id = o->point_id; prm.nb = nb;
  prm.d_lo3 = (float)(o->d_lo * o->d_lo * o->d_lo);
  prm.d_span3 = (float)(o->d_hi * o->d_hi * o->d_hi - o->d_lo * o->d_lo * o->d_lo);
  prm.partials = h->partials; prm.flags = h->flags;
  uint64_t evals = 0;
  AccState a{};
  int r = 0;
  int launches = 0;
  double kms = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (o->timing) {
    RIFT_CK(h, cudaEventCreate(&ev0));
    RIFT_CK(h, cudaEventCreate(&ev1));
  }
  for (;; ++r) {
    const uint64_t left = o->max_evals - evals;
    prm.round = (uint32_t)r;
    prm.n = (uint32_t)std::min<uint64_t>(npr, left);
    prm.proposal = adaptive ? 1 : 0;
    prm.tables = adaptive ? h->tables + cur * 3 * (nb + 1) : nullptr;
    prm.lnw = adaptive ? h->lnw + cur * 3 * nb : nullptr;
    prm.dbg_ell = o->dbg_ell;
    prm.dbg_off = (long long)r * npr;
    prm.ell_buf = adaptive ? h->ell_buf : nullptr;
    prm.bin_buf = adaptive ? h->bin_buf : nullptr;
    if (o->dbg_tables && adaptive)
      RIFT_CK(h, cudaMemcpyAsync(o->dbg_tables + (size_t)r * 3 * (nb + 1), prm.tables, sizeof(float) * 3 * (nb + 1),
                                 cudaMemcpyDeviceToDevice, h->stream));
    const int g = std::max(1, std::min<int>(grid, (int)((prm.n + block - 1) / block)));
    if (o->timing) RIFT_CK(h, cudaEventRecord(ev0, h->stream));
    RIFT_CK(h, launch_mc_round(h->K, h->pts_dev, p.c, h->q_arena, h->c_arena, prm, g, block, h->stream));
    if (o->timing) RIFT_CK(h, cudaEventRecord(ev1, h->stream));
    RIFT_CK(h, launch_merge(h->partials, g, h->acc, h->stream));
    launches += 2;
    const bool adapt_now = adaptive && (o->adapt_rounds < 0 || r < o->adapt_rounds);
    if (adapt_now) {
      const int hg = std::max(1, std::min(hist_grid, (int)((prm.n + 255) / 256)));
      RIFT_CK(h, launch_hist(h->ell_buf, h->bin_buf, prm.n, h->acc, (float)o->beta, nb, h->hist_part, hg, h->stream));
      RIFT_CK(h, launch_tables(h->hist_part, hg, nb, o->floor_eps, h->tables + (1 - cur) * 3 * (nb + 1),
                               h->lnw + (1 - cur) * 3 * nb, h->stream));
      launches += 2;
    }
    RIFT_CK(h, cudaMemcpyAsync(&a, h->acc, sizeof(a), cudaMemcpyDeviceToHost, h->stream));
    RIFT_CK(h, cudaStreamSynchronize(h->stream));
    if (o->timing) {
      float ms = 0.f;
      RIFT_CK(h, cudaEventElapsedTime(&ms, ev0, ev1));
      kms += ms;
    }
    if (adapt_now) cur = 1 - cur;
    evals += prm.n;
    const double n_eff = a.s1 + a.c1;
    if (n_eff >= o->n_eff_target || evals >= o->max_evals || (o->max_rounds > 0 && r + 1 >= o->max_rounds)) break;
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  fill_result(a, res);
  res->rounds = r + 1;
  res->kernel_ms = kms;
  res->kernel_launches = launches;
  s = read_flags(h);
  if (s == RIFT_OK && res->n_eff < o->n_eff_target) s = RIFT_ENOTCONVERGED;
  res->status = s;
  return s;
}

rift_status rift_ile_batch_marginalize(rift_ile *h, const rift_mc_opts *o, rift_mc_result *res) {
  (void)o; (void)res;
  return fail(h, RIFT_EUNSUPPORTED, "batched marginalisation not built yet");
}

}  // extern "C"

// Internal accessors used by the allocation-free entry point (noalloc.cu).
rift_status rift_internal_point0(rift_ile *h, const PointC **host, const PointC **dev, const float2 **qa,
                                 const float4 **ca, int *K, int *num_sms, uint32_t **flags, cudaStream_t *st) {
  if (!h || h->pts.empty()) return RIFT_EINVAL;
  *host = &h->pts[0].c;
  *dev = h->pts_dev;
  *qa = h->q_arena;
  *ca = h->c_arena;
  *K = h->K;
  *num_sms = h->num_sms;
  *flags = h->flags;
  *st = h->stream;
  return RIFT_OK;
}

rift_status rift_internal_fail(rift_ile *h, rift_status s, const char *msg) { return fail(h, s, msg); }

rift_status rift_internal_validate_opts(rift_ile *h, const rift_mc_opts *o) { return check_opts(h, o); }
