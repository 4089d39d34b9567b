// Mode inner products of Eq. (QUV) on the device, from frequency-domain mode waveforms, data
// and noise weights:
//   Q_{k,lm}(tau_j) = 2 df sum_f exp(2 pi i f tau_j) conj(h_lm(f)) d_k(f) w_k(f),
//   U_{k,lm,l'm'}   = 2 df sum_f conj(h_lm(f)) h_l'm'(f) w_k(f),
//   V_{k,lm,l'm'}   = 2 df sum_f h_lm(-f) h_l'm'(f) w_k(f),
// w_k = band / S_k (Eq. overlap).  The grid is f = nu df (integer nu) and tau_j = tau0_k + j / fs
// with n = fs / df an integer, so exp(2 pi i f tau_j) = exp(2 pi i nu df tau0_k)
// exp(2 pi i (nu j mod n) / n): the first factor is folded into the per-bin data term on the host
// in FP64, the second comes from an exact integer index.  Sums are FP32 over blocks of 32 bins
// added into double-float totals.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rift_ile.h"
#include "rift_device.cuh"
#include "rift_internal.h"
#include "host_par.h"

namespace {

constexpr int kQThreads = 128;   // grid times per CTA
constexpr int kQModes = 7;       // modes per CTA
constexpr int kChunk = 256;      // band bins staged per pass

__device__ __forceinline__ void df_acc(df &acc, float v) { acc = df_add_f(acc, v); }

// Partial Q of detector blockIdx.z / slices over bin slice blockIdx.z % slices, modes
// [blockIdx.y * kQModes, +kQModes), grid times [blockIdx.x * kQTimes, +kQTimes): thread t takes the
// times j = base + t and base + t + kQThreads, so every staged product is used twice.  The band is
// cut into slices of whole chunks so that enough CTAs run; quv_q_reduce_kernel adds the slices.
// X[a][b] = conj(h_a(f_b)) B_k(f_b) is formed per staged chunk; each time's twiddle index nu_b j
// mod n advances by j between consecutive bins of the same run and is recomputed at run starts.
// Qp: [slices][K][M][nt] complex double.
constexpr int kQPerThread = 2;
constexpr int kQTimes = kQThreads * kQPerThread;   // grid times per CTA

__global__ void __launch_bounds__(kQThreads) quv_q_kernel(const float2 *__restrict__ H, const float2 *__restrict__ Bk,
                                                          const int *__restrict__ nu, const int *__restrict__ run_start,
                                                          int nb, int M, int nt, int n, int slices,
                                                          double2 *__restrict__ Qp) {
  __shared__ float2 sX[kQModes][kChunk];
  __shared__ int sNu[kChunk], sRun[kChunk], sBlk[kChunk / 16];
  const int k = blockIdx.z / slices, slice = blockIdx.z % slices, a0 = blockIdx.y * kQModes;
  const int nchunk = (nb + kChunk - 1) / kChunk, per = (nchunk + slices - 1) / slices;
  const int b_begin = min(nb, slice * per * kChunk), b_end = min(nb, (slice + 1) * per * kChunk);
  const int ma = min(kQModes, M - a0);
  int jt[kQPerThread];
#pragma unroll
  for (int q = 0; q < kQPerThread; ++q) jt[q] = blockIdx.x * kQTimes + threadIdx.x + q * kQThreads;
  df accr[kQPerThread][kQModes], acci[kQPerThread][kQModes];
#pragma unroll
  for (int q = 0; q < kQPerThread; ++q)
#pragma unroll
    for (int a = 0; a < kQModes; ++a) { accr[q][a] = df{0.f, 0.f}; acci[q][a] = df{0.f, 0.f}; }
  const float inv_n2 = 2.0f / (float)n;
  // per time: exp(2 pi i j / n), the twiddle's step between consecutive bins of a run; the
  // twiddle itself and its integer index
  float sts[kQPerThread], stc[kQPerThread], sn[kQPerThread], cs[kQPerThread];
  int idx[kQPerThread];
#pragma unroll
  for (int q = 0; q < kQPerThread; ++q) {
    sincospif((float)(jt[q] % n) * inv_n2, &sts[q], &stc[q]);
    sn[q] = 0.f;
    cs[q] = 1.f;
    idx[q] = 0;
  }
  for (int b0 = b_begin; b0 < b_end; b0 += kChunk) {
    const int cb = min(kChunk, b_end - b0);
    __syncthreads();
    for (int t = threadIdx.x; t < cb * kQModes; t += blockDim.x) {
      const int a = t / cb, b = t - a * cb;
      float2 x = make_float2(0.f, 0.f);
      if (a < ma) {
        const float2 h = H[(size_t)(a0 + a) * nb + b0 + b];
        const float2 c = Bk[(size_t)k * nb + b0 + b];
        x = make_float2(h.x * c.x + h.y * c.y, h.x * c.y - h.y * c.x);   // conj(h) c
      }
      sX[a][b] = x;
    }
    for (int t = threadIdx.x; t < cb; t += blockDim.x) { sNu[t] = nu[b0 + t]; sRun[t] = run_start[b0 + t]; }
    // blocks of 16 bins inside the chunk with no run starting after their first bin
    for (int g = threadIdx.x; g < kChunk / 16; g += blockDim.x) {
      bool whole = 16 * g + 16 <= cb;
      for (int u = 1; u < 16 && whole; ++u) whole = run_start[b0 + 16 * g + u] == 0;
      sBlk[g] = whole ? 1 : 0;
    }
    __syncthreads();
    float pr[kQPerThread][kQModes], pi[kQPerThread][kQModes];
#pragma unroll
    for (int q = 0; q < kQPerThread; ++q)
#pragma unroll
      for (int a = 0; a < kQModes; ++a) { pr[q][a] = 0.f; pi[q][a] = 0.f; }
    // one bin's products with the current twiddles into the FP32 partial sums; the partial sums
    // go into the double-float totals every 32 bins and at the end of the chunk
    auto products = [&](int b) {
#pragma unroll
      for (int a = 0; a < kQModes; ++a) {
        const float2 x = sX[a][b];
#pragma unroll
        for (int q = 0; q < kQPerThread; ++q) {
          pr[q][a] = fmaf(x.x, cs[q], fmaf(-x.y, sn[q], pr[q][a]));
          pi[q][a] = fmaf(x.x, sn[q], fmaf(x.y, cs[q], pi[q][a]));
        }
      }
    };
    auto fold = [&](int b) {
      if ((b & 31) == 31 || b == cb - 1) {
#pragma unroll
        for (int q = 0; q < kQPerThread; ++q)
#pragma unroll
          for (int a = 0; a < kQModes; ++a) {
            df_acc(accr[q][a], pr[q][a]);
            df_acc(acci[q][a], pi[q][a]);
            pr[q][a] = 0.f;
            pi[q][a] = 0.f;
          }
      }
    };
    // the twiddle exp(2 pi i (nu_b j mod n) / n): exact (integer index into sincospi) at the start
    // of a run of consecutive bins and every 16 bins; in between rotated by the time's step
    // exp(2 pi i j / n), so its error stays within about 16 roundings
    auto twiddle = [&](int b) {
      const bool restart = b == 0 || sRun[b];
      const bool exact = restart || (b & 15) == 0;
#pragma unroll
      for (int q = 0; q < kQPerThread; ++q) {
        if (restart) idx[q] = (int)(((long long)sNu[b] * jt[q]) % n);
        else { idx[q] += jt[q]; if (idx[q] >= n) idx[q] -= n; }
        if (exact) {
          sincospif((float)idx[q] * inv_n2, &sn[q], &cs[q]);
        } else {
          const float c2 = fmaf(cs[q], stc[q], -sn[q] * sts[q]);
          sn[q] = fmaf(sn[q], stc[q], cs[q] * sts[q]);
          cs[q] = c2;
        }
      }
    };
    for (int b = 0; b < cb;) {
      if ((b & 15) == 0 && sBlk[b >> 4]) {
        // 16 bins of one run (a run may start at the first): the same twiddles as bin by bin,
        // without the per-bin index and run bookkeeping
        twiddle(b);
        products(b);
#pragma unroll
        for (int u = 1; u < 16; ++u) {
#pragma unroll
          for (int q = 0; q < kQPerThread; ++q) {
            const float c2 = fmaf(cs[q], stc[q], -sn[q] * sts[q]);
            sn[q] = fmaf(sn[q], stc[q], cs[q] * sts[q]);
            cs[q] = c2;
          }
          products(b + u);
        }
        fold(b + 15);
#pragma unroll
        for (int q = 0; q < kQPerThread; ++q)   // the index of bin b + 15
          idx[q] = (int)(((long long)idx[q] + 15ll * jt[q]) % n);
        b += 16;
      } else {
        twiddle(b);
        products(b);
        fold(b);
        ++b;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kQPerThread; ++q)
    if (jt[q] < nt) {
#pragma unroll
      for (int a = 0; a < kQModes; ++a)
        if (a < ma)
          Qp[(((size_t)slice * (gridDim.z / slices) + k) * M + a0 + a) * nt + jt[q]] =
              make_double2((double)accr[q][a].hi + (double)accr[q][a].lo, (double)acci[q][a].hi + (double)acci[q][a].lo);
    }
}

// Q[k][m][j] = qscale[k] times the sum over the slices of Qp, in slice order (FP64); qscale undoes
// the power-of-two scalings of the data term and the waveforms.
__global__ void quv_q_reduce_kernel(const double2 *__restrict__ Qp, int slices, size_t count, size_t per_det,
                                    const double *__restrict__ qscale, double2 *__restrict__ Q) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double re = 0.0, im = 0.0;
  for (int s = 0; s < slices; ++s) {
    const double2 v = Qp[(size_t)s * count + i];
    re += v.x;
    im += v.y;
  }
  const double sc = qscale[i / per_det];
  Q[i] = make_double2(re * sc, im * sc);
}

// U and V of detector blockIdx.y, pair (a, b) = blockIdx.x: the block's threads stride over the band
// bins (coalesced loads), each keeping FP32 sums of its bins, then a block reduction in
// double-float.  Hw[k][b] = h_b w_k (formed on the host in FP64, so the size of 1/S stays out of
// FP32), Hm[a] = h_a(-f); scale[k] undoes the power-of-two scalings and carries 2 df.
constexpr int kUVThreads = 256;

__device__ __forceinline__ df df_shfl_down(df v, int o) {
  return df{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}

__global__ void __launch_bounds__(kUVThreads) quv_uv_kernel(const float2 *__restrict__ H, const float2 *__restrict__ Hm,
                                                            const float2 *__restrict__ Hw, int nb, int M,
                                                            double2 *__restrict__ U, double2 *__restrict__ V,
                                                            const double *__restrict__ scale) {
  __shared__ df sred[4][kUVThreads / 32];
  const int pidx = blockIdx.x, k = blockIdx.y;
  const int a = pidx / M, b = pidx - a * M;
  const float2 *ha = H + (size_t)a * nb, *hma = Hm + (size_t)a * nb, *yb = Hw + ((size_t)k * M + b) * nb;
  float pur = 0.f, pui = 0.f, pvr = 0.f, pvi = 0.f;
  for (int i = threadIdx.x; i < nb; i += kUVThreads) {
    const float2 x = ha[i], y = yb[i], z = hma[i];
    pur = fmaf(x.x, y.x, fmaf(x.y, y.y, pur));     // conj(x) y
    pui = fmaf(x.x, y.y, fmaf(-x.y, y.x, pui));
    pvr = fmaf(z.x, y.x, fmaf(-z.y, y.y, pvr));    // z y
    pvi = fmaf(z.x, y.y, fmaf(z.y, y.x, pvi));
  }
  df v[4] = {df{pur, 0.f}, df{pui, 0.f}, df{pvr, 0.f}, df{pvi, 0.f}};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = df_add(v[c], df_shfl_down(v[c], o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) sred[c][wid] = v[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    df t[4] = {df{0.f, 0.f}, df{0.f, 0.f}, df{0.f, 0.f}, df{0.f, 0.f}};
    for (int w = 0; w < kUVThreads / 32; ++w)
#pragma unroll
      for (int c = 0; c < 4; ++c) t[c] = df_add(t[c], sred[c][w]);
    const size_t o = ((size_t)k * M + a) * M + b;
    const double sc = scale[k];
    U[o] = make_double2(sc * ((double)t[0].hi + t[0].lo), sc * ((double)t[1].hi + t[1].lo));
    V[o] = make_double2(sc * ((double)t[2].hi + t[2].lo), sc * ((double)t[3].hi + t[3].lo));
  }
}

// Power of two that brings the largest magnitude of a set near 1 (1 for an all-zero set).
double unit_scale(double vmax) { return vmax > 0.0 && std::isfinite(vmax) ? std::ldexp(1.0, -std::ilogb(vmax)) : 1.0; }

thread_local std::string g_quv_err;
thread_local double g_quv_ms[2] = {0.0, 0.0};   // quv_q_kernel, quv_uv_kernel of the last call

rift_status quv_fail(rift_status s, const std::string &m) {
  g_quv_err = m;
  return s;
}

// Device buffer from the process-wide buffer cache, given back when the call returns (the call
// drains its stream before that, see StreamDrain).
struct DevBuf {
  void *p = nullptr;
  ~DevBuf() { if (p) cache_dev_free(p); }
};

// Drains the stream at every exit once device work has been queued on it, so buffers go back to
// the cache only when no work in flight reads them.
struct StreamDrain {
  cudaStream_t st = nullptr;
  bool armed = false;
  ~StreamDrain() { if (armed) cudaStreamSynchronize(st); }
};

// Pinned host staging from the buffer cache.
struct HostBuf {
  void *p = nullptr;
  ~HostBuf() { if (p) cache_host_free(p); }
};

}  // namespace

extern "C" {

const char *rift_quv_last_error(void) { return g_quv_err.c_str(); }

void rift_quv_kernel_ms(double out[2]) {
  if (!out) return;
  out[0] = g_quv_ms[0];
  out[1] = g_quv_ms[1];
}

rift_status rift_quv(const rift_ile_fd_desc *d, double *Q, double *U, double *V) {
  if (!d || !Q || !U || !V) return quv_fail(RIFT_EINVAL, "null argument");
  const int K = d->n_det, M = d->n_modes, nf = d->n_f, nt = d->n_t;
  if (K < 1 || K > RIFT_MAX_DET || M < 1 || M > RIFT_MAX_MODES || nf < 1 || nt < 1)
    return quv_fail(RIFT_EINVAL, "sizes out of range");
  if (!d->nu || !d->hlm || !d->data || !d->weight || !d->mirror || !d->q_t0_gps)
    return quv_fail(RIFT_EINVAL, "null array in descriptor");
  if (!(d->df > 0) || !(d->fs > 0)) return quv_fail(RIFT_EINVAL, "df and fs must be positive");
  const double nd = d->fs / d->df;
  const long long n = llround(nd);
  if (n < 2 || std::fabs(nd - (double)n) > 1e-9 * nd || n > (1ll << 30))
    return quv_fail(RIFT_EINVAL, "fs / df must be an integer (the Q grid and the frequency grid share it)");
  if ((long long)nt > n) return quv_fail(RIFT_EINVAL, "n_t exceeds fs / df samples");
  host_par::Pool::get().wake();   // the passes over the bins below run on the worker pool
  // band bins: weight nonzero in some detector (in bin order; parts of the bin range on the
  // worker pool, joined in part order); every mirror index in range
  constexpr int kParts = 8;
  std::vector<int> bpart[kParts];
  int bad_mirror[kParts] = {};
  parallel_parts(nf, 16384, kParts, [&](int part, int i0, int i1) {
    std::vector<int> &v = bpart[part];
    for (int i = i0; i < i1; ++i) {
      bad_mirror[part] |= (d->mirror[i] < 0) | (d->mirror[i] >= nf);
      bool in = false;
      for (int k = 0; k < K; ++k) in = in || d->weight[(size_t)k * nf + i] != 0.0;
      if (in) v.push_back(i);
    }
  });
  std::vector<int> band;
  for (int t = 0; t < kParts; ++t) {
    if (bad_mirror[t]) return quv_fail(RIFT_EINVAL, "mirror index out of range");
    band.insert(band.end(), bpart[t].begin(), bpart[t].end());
  }
  const int nb = (int)band.size();
  if (nb == 0) return quv_fail(RIFT_EINVAL, "no bin has a nonzero weight");
  // per band bin, in parallel over bin ranges: validity, the twiddle index nu mod n, the data term
  // B_k = 2 df w_k d_k exp(2 pi i nu df tau0_k) (FP64), and the largest component magnitudes of
  // the waveforms, the data terms and the weighted waveforms (for the power-of-two scalings below)
  std::vector<double> Bd(2 * (size_t)K * nb);
  std::vector<int> nuv(nb), run(nb);
  struct PartMax {
    double h = 0.0, b[RIFT_MAX_DET] = {}, w[RIFT_MAX_DET] = {};
    int bad = 0;   // 1 non-finite waveform, 2 bad weight, 3 non-finite data
  };
  PartMax pm[kParts];
  auto cabs = [](const double *z) { return std::max(std::fabs(z[0]), std::fabs(z[1])); };
  // exp(2 pi i nu df tau0_k) of a bin: exact (fmod, cos, sin) at the start of a part, of a run of
  // consecutive nu and every 32 bins, otherwise the previous bin's value times exp(2 pi i df tau0_k)
  constexpr double kTwoPi = 2.0 * 3.14159265358979323846;
  double wre[RIFT_MAX_DET], wim[RIFT_MAX_DET];
  for (int k = 0; k < K; ++k) {
    const double ph = kTwoPi * std::fmod(d->df * (d->q_t0_gps[k] - d->t_ref_gps), 1.0);
    wre[k] = std::cos(ph);
    wim[k] = std::sin(ph);
  }
  parallel_parts(nb, 2048, kParts, [&](int part, int b0, int b1) {
    PartMax &r = pm[part];
    double cre[RIFT_MAX_DET] = {}, cim[RIFT_MAX_DET] = {};
    int since = 0;
    for (int b = b0; b < b1 && !r.bad; ++b) {
      const bool exact = b == b0 || d->nu[band[b]] != d->nu[band[b - 1]] + 1 || ++since == 32;
      if (exact) since = 0;
      const int i = band[b], im = d->mirror[i];
      long long v = d->nu[i] % n;
      if (v < 0) v += n;
      nuv[b] = (int)v;
      double hb = 0.0;   // largest component of the bin's waveforms
      for (int a = 0; a < M; ++a) {
        const double *h = d->hlm + 2 * ((size_t)a * nf + i), *hm = d->hlm + 2 * ((size_t)a * nf + im);
        if (!std::isfinite(h[0]) || !std::isfinite(h[1]) || !std::isfinite(hm[0]) || !std::isfinite(hm[1])) {
          r.bad = 1;
          break;
        }
        hb = std::max(hb, cabs(h));
        r.h = std::max(r.h, std::max(cabs(h), cabs(hm)));
      }
      for (int k = 0; k < K && !r.bad; ++k) {
        const double w = d->weight[(size_t)k * nf + i];
        const double *x = d->data + 2 * ((size_t)k * nf + i);
        if (!std::isfinite(w) || w < 0.0) { r.bad = 2; break; }
        if (!std::isfinite(x[0]) || !std::isfinite(x[1])) { r.bad = 3; break; }
        if (exact) {
          const double tau0 = d->q_t0_gps[k] - d->t_ref_gps;
          const double ph = kTwoPi * std::fmod((double)d->nu[i] * d->df * tau0, 1.0);
          cre[k] = std::cos(ph);
          cim[k] = std::sin(ph);
        } else {
          const double c2 = cre[k] * wre[k] - cim[k] * wim[k];
          cim[k] = cre[k] * wim[k] + cim[k] * wre[k];
          cre[k] = c2;
        }
        const double c = cre[k], sn = cim[k], f = 2.0 * d->df * w;
        double *bd = &Bd[2 * ((size_t)k * nb + b)];
        bd[0] = f * (x[0] * c - x[1] * sn);
        bd[1] = f * (x[0] * sn + x[1] * c);
        r.b[k] = std::max(r.b[k], cabs(bd));
        r.w[k] = std::max(r.w[k], w * hb);
      }
    }
  });
  double hmax = 0.0;
  std::vector<double> bmax(K, 0.0), wmax(K, 0.0);
  for (int t = 0; t < kParts; ++t) {
    if (pm[t].bad == 1) return quv_fail(RIFT_EINVAL, "non-finite mode waveform in the band");
    if (pm[t].bad == 2) return quv_fail(RIFT_EINVAL, "weights must be finite and non-negative");
    if (pm[t].bad == 3) return quv_fail(RIFT_EINVAL, "non-finite data in the band");
    hmax = std::max(hmax, pm[t].h);
    for (int k = 0; k < K; ++k) {
      bmax[k] = std::max(bmax[k], pm[t].b[k]);
      wmax[k] = std::max(wmax[k], pm[t].w[k]);
    }
  }
  for (int b = 0; b < nb; ++b) run[b] = (b == 0 || nuv[b] != (nuv[b - 1] + 1) % n) ? 1 : 0;
  // operands rescaled by powers of two so that FP32 holds them whatever the strain units
  const double sH = unit_scale(hmax);
  std::vector<double> sB(K), sW(K), qscale(K), uvscale(K);
  for (int k = 0; k < K; ++k) {
    sB[k] = unit_scale(bmax[k]);
    sW[k] = unit_scale(wmax[k]);
    qscale[k] = 1.0 / (sH * sB[k]);
    uvscale[k] = 2.0 * d->df / (sH * sW[k]);
  }
  // FP32 operands in one pinned staging buffer: H [M][nb], Hm [M][nb], B [K][nb], Hw [K][M][nb],
  // then the twiddle indices, the run starts and the U/V scales
  const size_t nH = (size_t)M * nb, nB = (size_t)K * nb, nHw = (size_t)K * M * nb;
  const size_t o_Hm = nH, o_B = 2 * nH, o_Hw = 2 * nH + nB, n_f2 = 2 * nH + nB + nHw;
  const size_t stage_bytes = sizeof(float2) * n_f2 + sizeof(int) * 2 * (size_t)nb + sizeof(double) * (2 * K + 1);
  HostBuf hs;
  cudaError_t e;
  if ((e = cache_host_alloc(&hs.p, stage_bytes)) != cudaSuccess)
    return quv_fail(e == cudaErrorMemoryAllocation ? RIFT_ENOMEM : RIFT_ECUDA, cudaGetErrorString(e));
  float2 *F2 = static_cast<float2 *>(hs.p);
  float2 *H = F2, *Hm = F2 + o_Hm, *B = F2 + o_B, *Hw = F2 + o_Hw;
  int *nu_h = reinterpret_cast<int *>(F2 + n_f2), *run_h = nu_h + nb;
  double *sc_h = reinterpret_cast<double *>(run_h + nb);   // 8-byte aligned: 2 nb ints follow the float2s
  std::memcpy(nu_h, nuv.data(), sizeof(int) * nb);
  std::memcpy(run_h, run.data(), sizeof(int) * nb);
  for (int k = 0; k < K; ++k) {
    sc_h[k] = uvscale[k];
    sc_h[K + k] = qscale[k];
  }
  parallel_parts(nb, 2048, kParts, [&](int, int b0, int b1) {
    for (int b = b0; b < b1; ++b) {
      const int i = band[b];
      for (int a = 0; a < M; ++a) {
        const double *h = d->hlm + 2 * ((size_t)a * nf + i), *hm = d->hlm + 2 * ((size_t)a * nf + d->mirror[i]);
        H[(size_t)a * nb + b] = make_float2((float)(h[0] * sH), (float)(h[1] * sH));
        Hm[(size_t)a * nb + b] = make_float2((float)(hm[0] * sH), (float)(hm[1] * sH));
        for (int k = 0; k < K; ++k) {
          const double w = d->weight[(size_t)k * nf + i] * sW[k];
          Hw[((size_t)k * M + a) * nb + b] = make_float2((float)(h[0] * w), (float)(h[1] * w));
        }
      }
      for (int k = 0; k < K; ++k) {
        const double *bd = &Bd[2 * ((size_t)k * nb + b)];
        B[(size_t)k * nb + b] = make_float2((float)(bd[0] * sB[k]), (float)(bd[1] * sB[k]));
      }
    }
  });
  cudaStream_t st = (cudaStream_t)d->cuda_stream;
  DevBuf dF2, dnu, dsc, dQ, dU, dV, dQp;
  StreamDrain drain;
  drain.st = st;
  // bin slices: about four CTAs per SM in all
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int ctas = ((nt + kQTimes - 1) / kQTimes) * ((M + kQModes - 1) / kQModes) * K;
  const int nchunk = (nb + kChunk - 1) / kChunk;
  const int slices = std::max(1, std::min(nchunk, (4 * nsm + ctas - 1) / ctas));
  if ((e = cache_dev_alloc(&dF2.p, sizeof(float2) * n_f2)) != cudaSuccess ||
      (e = cache_dev_alloc(&dnu.p, sizeof(int) * 2 * (size_t)nb)) != cudaSuccess ||
      (e = cache_dev_alloc(&dsc.p, sizeof(double) * 2 * K)) != cudaSuccess ||
      (e = cache_dev_alloc(&dQ.p, sizeof(double2) * (size_t)K * M * nt)) != cudaSuccess ||
      (e = cache_dev_alloc(&dQp.p, sizeof(double2) * (size_t)slices * K * M * nt)) != cudaSuccess ||
      (e = cache_dev_alloc(&dU.p, sizeof(double2) * (size_t)K * M * M)) != cudaSuccess ||
      (e = cache_dev_alloc(&dV.p, sizeof(double2) * (size_t)K * M * M)) != cudaSuccess)
    return quv_fail(e == cudaErrorMemoryAllocation ? RIFT_ENOMEM : RIFT_ECUDA, cudaGetErrorString(e));
  drain.armed = true;
  if ((e = cudaMemcpyAsync(dF2.p, F2, sizeof(float2) * n_f2, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dnu.p, nu_h, sizeof(int) * 2 * (size_t)nb, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dsc.p, sc_h, sizeof(double) * 2 * K, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return quv_fail(RIFT_ECUDA, cudaGetErrorString(e));
  const float2 *dH = static_cast<const float2 *>(dF2.p), *dHm = dH + o_Hm, *dB = dH + o_B, *dHw = dH + o_Hw;
  const int *dnu_p = static_cast<const int *>(dnu.p), *drun_p = dnu_p + nb;
  // CUDA events around each kernel on the call's stream (rift_quv_kernel_ms)
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  for (int i = 0; i < 3; ++i)
    if ((e = cudaEventCreate(&ev[i])) != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
      return quv_fail(RIFT_ECUDA, cudaGetErrorString(e));
    }
  dim3 gq((nt + kQTimes - 1) / kQTimes, (M + kQModes - 1) / kQModes, K * slices);
  cudaEventRecord(ev[0], st);
  quv_q_kernel<<<gq, kQThreads, 0, st>>>(dH, dB, dnu_p, drun_p, nb, M, nt, (int)n, slices, (double2 *)dQp.p);
  const size_t qcount = (size_t)K * M * nt;
  quv_q_reduce_kernel<<<(unsigned)((qcount + 255) / 256), 256, 0, st>>>(
      (const double2 *)dQp.p, slices, qcount, (size_t)M * nt, (const double *)dsc.p + K, (double2 *)dQ.p);
  cudaEventRecord(ev[1], st);
  dim3 guv(M * M, K);
  quv_uv_kernel<<<guv, kUVThreads, 0, st>>>(dH, dHm, dHw, nb, M, (double2 *)dU.p, (double2 *)dV.p,
                                            (const double *)dsc.p);
  cudaEventRecord(ev[2], st);
  if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaEventSynchronize(ev[2])) == cudaSuccess) {
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    g_quv_ms[0] = a;
    g_quv_ms[1] = b;
  }
  for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess ||
      (e = cudaMemcpyAsync(Q, dQ.p, sizeof(double2) * (size_t)K * M * nt, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(U, dU.p, sizeof(double2) * (size_t)K * M * M, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(V, dV.p, sizeof(double2) * (size_t)K * M * M, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return quv_fail(RIFT_ECUDA, cudaGetErrorString(e));
  return RIFT_OK;
}

rift_status rift_ile_create_fd(const rift_ile_fd_desc *d, rift_ile **out) {
  if (!d || !out) return quv_fail(RIFT_EINVAL, "null argument");
  const size_t K = (size_t)std::max(d->n_det, 0), M = (size_t)std::max(d->n_modes, 0), T = (size_t)std::max(d->n_t, 0);
  std::vector<double> Q(2 * K * M * T), U(2 * K * M * M), V(2 * K * M * M);
  rift_status s = rift_quv(d, Q.data(), U.data(), V.data());
  if (s != RIFT_OK) return s;
  // U_ab and U_ba (V_ab and V_ba) are separate sums: make U Hermitian and V symmetric exactly
  for (size_t k = 0; k < K; ++k)
    for (size_t a = 0; a < M; ++a)
      for (size_t b = a; b < M; ++b) {
        double *u1 = &U[2 * ((k * M + a) * M + b)], *u2 = &U[2 * ((k * M + b) * M + a)];
        double *v1 = &V[2 * ((k * M + a) * M + b)], *v2 = &V[2 * ((k * M + b) * M + a)];
        const double ur = 0.5 * (u1[0] + u2[0]), ui = 0.5 * (u1[1] - u2[1]);
        const double vr = 0.5 * (v1[0] + v2[0]), vi = 0.5 * (v1[1] + v2[1]);
        u1[0] = ur; u1[1] = ui; u2[0] = ur; u2[1] = -ui;
        v1[0] = vr; v1[1] = vi; v2[0] = vr; v2[1] = vi;
      }
  rift_ile_desc c;
  std::memset(&c, 0, sizeof(c));
  c.n_det = d->n_det; c.det_tensor = d->det_tensor; c.det_pos = d->det_pos;
  c.n_modes = d->n_modes; c.lm = d->lm; c.n_t = d->n_t; c.Q = Q.data(); c.q_t0_gps = d->q_t0_gps;
  c.fs = d->fs; c.U = U.data(); c.V = V.data(); c.t_ref_gps = d->t_ref_gps; c.d_ref_mpc = d->d_ref_mpc;
  c.t_lo = d->t_lo; c.t_hi = d->t_hi; c.interp = d->interp; c.cuda_stream = d->cuda_stream;
  return rift_ile_create(&c, out);
}

}  // extern "C"
