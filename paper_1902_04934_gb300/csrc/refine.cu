// Refinement of heavy samples (rift_mc_opts.refine): the samples that carry an estimate resting
// on a few draws are evaluated again in FP64, and the estimate uses those values.
//
// After a round's merge, per point: the candidates (the two largest log weights of every warp of
// every work item, written by the cell kernel) within B nats of the running maximum are chosen,
// B the largest of 1..24 that keeps them at RIFT_REFINE_CAP at most (refine_select_kernel); each
// chosen sample is drawn again from its Philox counters and evaluated in FP64 by one warp
// (refine_eval_kernel): the same draw as the sampler (prior transforms, stratification, inverse
// CDF of the round's tables), the detector response and delay, the -2Y_lm, the interpolated Q
// (from its FP32 copy), and the quadratic form of Eq. (def:lnL:Decomposed) with U and V in FP64;
// then refine_fold_kernel adds e^{l64 - m} - e^{l32 - m} (and the squares) to the point's
// corrections in a fixed order.  The host applies them to the accumulator at return.
#include <cmath>
#include <cstdint>

#include "../../include/rift_ile.h"
#include "rift_device.cuh"
#include "rift_internal.h"

namespace {

constexpr double kPiD = 3.14159265358979323846;

__device__ __forceinline__ double u_of(uint32_t x) { return ((double)(x >> 9) + 0.5) * 1.1920928955078125e-07; }

__device__ __forceinline__ uint32_t cell_of_r(const RoundPt &R, uint32_t i) {
  const uint32_t big = R.rem * (R.base + 1u);
  return (i < big) ? i / (R.base + 1u) : R.rem + (i - big) / R.base;
}

// Sample i of round R in FP64: (ra, sin dec, t, psi, phi, (1 + cos incl)/2, D) and ln p - ln q.
struct DrawD {
  double ra, sd, t, psi, phi, cf, D, lpq;
};

__device__ DrawD draw_fp64(const PointD &P, const RoundPt &R, uint32_t i, unsigned long long seed, double lo3,
                           double span3) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint4 a = philox4x32_10(make_uint4(i, R.round, 0u, R.point_id), key);
  const uint4 b = philox4x32_10(make_uint4(i, R.round, 1u, R.point_id), key);
  const uint32_t cell = cell_of_r(R, i);
  const uint32_t C = 1u << (R.ls0 + R.ls1 + R.ls2);
  const uint32_t c0 = cell & ((1u << R.ls0) - 1u);
  const uint32_t c1 = (cell >> R.ls0) & ((1u << R.ls1) - 1u);
  const uint32_t c2 = cell >> (R.ls0 + R.ls1);
  double U[3];
  U[0] = ((double)c0 + u_of(a.x)) / (double)(1u << R.ls0);
  U[1] = ((double)c1 + u_of(a.y)) / (double)(1u << R.ls1);
  U[2] = ((double)c2 + u_of(a.z)) / (double)(1u << R.ls2);
  DrawD d;
  const double n_c = (cell < R.rem) ? (double)R.base + 1.0 : (double)R.base;
  d.lpq = (C > 1u) ? log((double)R.n / ((double)C * n_c)) : 0.0;
  double x[3] = {U[0], U[1], U[2]};
  if (R.proposal == 1) {
    const int nb = R.nb;
    for (int q = 0; q < 3; ++q) {
      const float *cdf = R.tab + q * (nb + 1);
      int lo = 0, hi = nb;   // largest bin with cdf[bin] <= U
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if ((double)cdf[mid] <= U[q]) lo = mid; else hi = mid;
      }
      const double pb = (double)cdf[lo + 1] - (double)cdf[lo];
      x[q] = ((double)lo + (U[q] - (double)cdf[lo]) / pb) / (double)nb;
      d.lpq -= log((double)nb * pb);
    }
  }
  d.ra = 2.0 * kPiD * x[0];
  d.sd = 2.0 * x[1] - 1.0;
  d.t = P.t_lo + P.t_span * x[2];
  d.psi = kPiD * u_of(a.w);
  d.phi = 2.0 * kPiD * u_of(b.x);
  d.cf = u_of(b.y);
  d.D = cbrt(lo3 + u_of(b.z) * span3);
  return d;
}

// The part of ln L of a drawn sample that detector k contributes, in FP64, computed by one warp:
// lane a < M owns mode a (its harmonic, its row of the quadratic form and its part of the linear
// term); returns (Re F_k conj(Y) qbar_k, |F_k|^2 conj(Y)^T U_k Y + Re(conj(F_k)^2 Y^T V_k Y)) summed
// over the warp.  FP64 runs at a small fraction of the FP32 rate here, so the detectors go to
// separate warps (separate schedulers) and the draw and geometry are repeated by each.
__device__ double2 detector_fp64_warp(const PointD &P, const double2 *__restrict__ uv, const float2 *__restrict__ qa,
                                      const DrawD &d, int k, uint32_t &flags) {
  const int lane = threadIdx.x & 31;
  const int K = P.K, M = P.M;
  // sky: n = (cos dec cos(ra - GMST), cos dec sin(ra - GMST), sin dec) in the Earth-fixed frame
  const double ang = d.ra - 2.0 * kPiD * P.g;
  double sa, ca;
  sincos(ang, &sa, &ca);
  const double cd = sqrt(fmax(0.0, 1.0 - d.sd * d.sd));
  const double nx = cd * ca, ny = cd * sa, nz = d.sd;
  double s2p, c2p;
  sincos(2.0 * d.psi, &s2p, &c2p);
  const double ex = -sa, ey = ca;
  const double fx = -d.sd * ca, fy = -d.sd * sa, fz = cd;
  // harmonic of this lane's mode: powers of cos, sin(incl/2) and e^{i m phi} by products
  double yr = 0.0, yi = 0.0;
  if (lane < M) {
    const double ch = sqrt(d.cf), sh = sqrt(1.0 - d.cf);
    double cp[9], sp[9];
    cp[0] = 1.0; sp[0] = 1.0;
    for (int j = 1; j < 9; ++j) { cp[j] = cp[j - 1] * ch; sp[j] = sp[j - 1] * sh; }
    double v = 0.0;
    const int l = P.ml[lane];
    for (int r = 0; r < P.nterm[lane]; ++r) {
      const int kc = P.kc[lane][r];
      v += P.coef[lane][r] * cp[kc] * sp[2 * l - kc];
    }
    double s1, c1;
    sincos(d.phi, &s1, &c1);
    const int am = abs(P.mm[lane]);
    double er = 1.0, ei = 0.0;
    for (int j = 0; j < am; ++j) {
      const double t = er * c1 - ei * s1;
      ei = er * s1 + ei * c1;
      er = t;
    }
    yr = v * er;
    yi = (P.mm[lane] < 0) ? -v * ei : v * ei;
  }
  const int NT = (P.interp == 3) ? 4 : (P.interp == 1 ? 2 : 1);
  const int first = (NT == 4) ? -1 : 0;
  const double *dd = P.d[k];
  const double dex = dd[0] * ex + dd[1] * ey;
  const double dey = dd[1] * ex + dd[3] * ey;
  const double dez = dd[2] * ex + dd[4] * ey;
  const double dfx = dd[0] * fx + dd[1] * fy + dd[2] * fz;
  const double dfy = dd[1] * fx + dd[3] * fy + dd[4] * fz;
  const double dfz = dd[2] * fx + dd[4] * fy + dd[5] * fz;
  const double fr0 = (ex * dex + ey * dey) - (fx * dfx + fy * dfy + fz * dfz);
  const double fi0 = 2.0 * (fx * dex + fy * dey + fz * dez);
  const double Fr = c2p * fr0 - s2p * fi0, Fi = s2p * fr0 + c2p * fi0;
  // Q index of t + delay_k
  double s = P.c0[k] + (d.t - P.t_lo) * P.fs - (P.P[k][0] * nx + P.P[k][1] * ny + P.P[k][2] * nz);
  if (NT == 1) s += 0.5;
  const double fl = floor(s);
  const double mu = s - fl;
  int i0 = (int)fl + first;
  if (i0 < 0 || i0 + NT > P.T) {
    flags |= RIFT_FLAG_WINDOW;
    i0 = min(max(i0, 0), P.T - NT);
  }
  double w[4];
  if (NT == 4) {
    const double a1 = mu + 1.0, b1 = mu - 1.0, c1 = mu - 2.0;
    w[0] = -mu * b1 * c1 / 6.0;
    w[1] = a1 * b1 * c1 * 0.5;
    w[2] = -a1 * mu * c1 * 0.5;
    w[3] = a1 * mu * b1 / 6.0;
  } else if (NT == 2) {
    w[0] = 1.0 - mu; w[1] = mu; w[2] = 0.0; w[3] = 0.0;
  } else {
    w[0] = 1.0; w[1] = 0.0; w[2] = 0.0; w[3] = 0.0;
  }
  double lin = 0.0;
  if (lane < M) {
    // linear term of this mode: Re(F conj(Y_a) qbar_a)
    double qr = 0.0, qi = 0.0;
    for (int r = 0; r < NT; ++r) {
      const float2 q = qa[P.q_off + ((long long)k * P.T + i0 + r) * P.Mp + lane];
      qr += w[r] * (double)q.x;
      qi += w[r] * (double)q.y;
    }
    const double zr = yr * qr + yi * qi, zi = yr * qi - yi * qr;   // conj(Y) qbar
    lin = Fr * zr - Fi * zi;
  }
  // row a of conj(Y)^T U Y and Y^T V Y
  double ar = 0.0, br = 0.0, bi = 0.0;
  const double2 *Uk = uv + P.uv_off + (size_t)k * M * M;
  const double2 *Vk = uv + P.uv_off + (size_t)(K + k) * M * M;
  for (int bm = 0; bm < M; ++bm) {
    const double ybr = __shfl_sync(0xffffffffu, yr, bm), ybi = __shfl_sync(0xffffffffu, yi, bm);
    if (lane < M) {
      const double2 u = Uk[(size_t)lane * M + bm], v = Vk[(size_t)lane * M + bm];
      const double pr = yr * ybr + yi * ybi, pi = yr * ybi - yi * ybr;   // conj(Y_a) Y_b
      const double qr2 = yr * ybr - yi * ybi, qi2 = yr * ybi + yi * ybr; // Y_a Y_b
      ar += pr * u.x - pi * u.y;
      br += qr2 * v.x - qi2 * v.y;
      bi += qr2 * v.y + qi2 * v.x;
    }
  }
  const double gr = Fr * Fr - Fi * Fi, gi = -2.0 * Fr * Fi;   // conj(F)^2
  double quad = (Fr * Fr + Fi * Fi) * ar + (gr * br - gi * bi);
  for (int o = 16; o > 0; o >>= 1) {
    lin += __shfl_xor_sync(0xffffffffu, lin, o);
    quad += __shfl_xor_sync(0xffffffffu, quad, o);
  }
  return make_double2(lin, quad);
}

constexpr int kBuckets = 24;
constexpr int kSelThreads = 1024;   // threads of the one block per point

// Per point (one block): the round's candidates within B nats of the running maximum, in the order
// (thread t of the block, its items t, t + kSelThreads, ..., warp, rank); B as in the header.  Items
// whose largest log weight lies 24 nats or more below are skipped whole.  Learned and
// time-marginalised rounds choose none.
__global__ void __launch_bounds__(kSelThreads) refine_select_kernel(const RoundPt *__restrict__ rp,
                                                            const AccState *__restrict__ acc,
                                                            const float *__restrict__ cmax,
                                                            const float2 *__restrict__ cand, uint2 *__restrict__ list,
                                                            int *__restrict__ count) {
  __shared__ int hist[kBuckets];
  __shared__ int scan[kSelThreads];
  __shared__ int s_B;
  const int p = blockIdx.x, t = threadIdx.x;
  const RoundPt R = rp[p];
  if (R.n == 0 || R.proposal == 2 || R.tmarg) {
    if (t == 0) count[p] = 0;
    return;
  }
  // the maximum is a float log weight (converted exactly): the distances below it in float
  const float Mx = (float)acc[p].m;
  const long long ni = (long long)R.nitem;   // thread t takes items t, t + kSelThreads, ... (coalesced)
  if (t < kBuckets) hist[t] = 0;
  __syncthreads();
  for (long long it = t; it < ni; it += kSelThreads) {
    const float pm = cmax[R.item0 + it];
    if (!(Mx - pm < (float)kBuckets)) continue;
    const float2 *c = cand + (R.item0 + it) * RIFT_CAND_PER_ITEM;
    for (int q = 0; q < RIFT_CAND_PER_ITEM; ++q) {
      const float l = c[q].x;
      if (!isfinite(l)) continue;
      const float dl = fmaxf(0.f, Mx - l);
      if (dl < (float)kBuckets) atomicAdd(&hist[(int)dl], 1);
    }
  }
  __syncthreads();
  if (t == 0) {
    int B = 0, cum = 0;
    for (int b = 0; b < kBuckets; ++b) {
      cum += hist[b];
      if (cum > RIFT_REFINE_CAP) break;
      B = b + 1;
    }
    s_B = B;
  }
  __syncthreads();
  const float B = (float)s_B;
  int mine = 0;
  for (long long it = t; it < ni; it += kSelThreads) {
    const float pm = cmax[R.item0 + it];
    if (!(Mx - pm < B)) continue;
    const float2 *c = cand + (R.item0 + it) * RIFT_CAND_PER_ITEM;
    for (int q = 0; q < RIFT_CAND_PER_ITEM; ++q) {
      const float l = c[q].x;
      if (isfinite(l) && fmaxf(0.f, Mx - l) < B) ++mine;
    }
  }
  scan[t] = mine;
  __syncthreads();
  for (int o = 1; o < kSelThreads; o <<= 1) {
    const int v = (t >= o) ? scan[t - o] : 0;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  int off = scan[t] - mine;
  for (long long it = t; it < ni; it += kSelThreads) {
    const float pm = cmax[R.item0 + it];
    if (!(Mx - pm < B)) continue;
    const float2 *c = cand + (R.item0 + it) * RIFT_CAND_PER_ITEM;
    for (int q = 0; q < RIFT_CAND_PER_ITEM; ++q) {
      const float l = c[q].x;
      if (isfinite(l) && fmaxf(0.f, Mx - l) < B && off < RIFT_REFINE_CAP)
        list[(size_t)p * RIFT_REFINE_CAP + off++] = make_uint2(__float_as_uint(c[q].y), __float_as_uint(l));
    }
  }
  if (t == kSelThreads - 1) count[p] = min(scan[kSelThreads - 1], RIFT_REFINE_CAP);
}

// One block per chosen sample, one warp per detector: (l32, l64) with l64 = FP64 lnL + FP64
// ln p - ln q.
__global__ void __launch_bounds__(32 * RIFT_MAXK) refine_eval_kernel(
    const PointD *__restrict__ pd, const double2 *__restrict__ uv, const float2 *__restrict__ qa,
    const RoundPt *__restrict__ rp, const uint2 *__restrict__ list, const int *__restrict__ count,
    unsigned long long seed, double lo3, double span3, double2 *__restrict__ out, uint32_t *flags_out) {
  __shared__ double2 part[RIFT_MAXK];
  const int p = blockIdx.y, j = blockIdx.x, k = threadIdx.x >> 5;
  if (j >= count[p]) return;
  const RoundPt R = rp[p];
  const PointD &P = pd[p];
  const uint2 e = list[(size_t)p * RIFT_REFINE_CAP + j];
  uint32_t flags = 0u;
  const DrawD d = draw_fp64(P, R, e.x, seed, lo3, span3);
  if (k < P.K) {
    const double2 v = detector_fp64_warp(P, uv, qa, d, k, flags);
    if ((threadIdx.x & 31) == 0) part[k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double lin = 0.0, quad = 0.0;
    for (int q = 0; q < P.K; ++q) { lin += part[q].x; quad += part[q].y; }
    const double x = P.dref / d.D;
    out[(size_t)p * RIFT_REFINE_CAP + j] = make_double2((double)__uint_as_float(e.y), x * lin - 0.25 * x * x * quad + d.lpq);
  }
  if (flags) atomicOr(flags_out, flags);
}

// Per point, one warp: the chosen samples' corrections, the exponentials lane-parallel and the
// sums in a fixed shuffle order (deterministic); the largest refined l64 kept with its l32.
__global__ void __launch_bounds__(32) refine_fold_kernel(const AccState *__restrict__ acc, const int *__restrict__ count,
                                                         const double2 *__restrict__ out, RefineState *__restrict__ rs) {
  const int p = blockIdx.x, lane = threadIdx.x;
  const int n = count[p];
  if (n == 0) return;
  RefineState s = rs[p];
  const double Mx = acc[p].m;
  if (!(s.mref >= Mx)) {
    const double f = (s.n == 0) ? 0.0 : exp(s.mref - Mx);
    s.d1 *= f;
    s.d2 *= f * f;
    s.mref = Mx;
  }
  double d1 = 0.0, d2 = 0.0, l64 = -INFINITY, l32 = -INFINITY;
  int cnt = 0;
  for (int j = lane; j < n; j += 32) {
    const double2 v = out[(size_t)p * RIFT_REFINE_CAP + j];
    if (!isfinite(v.y)) continue;
    const double e32 = exp(v.x - s.mref), e64 = exp(v.y - s.mref);
    d1 += e64 - e32;
    d2 += e64 * e64 - e32 * e32;
    if (v.y > l64) { l64 = v.y; l32 = v.x; }
    ++cnt;
  }
  for (int o = 16; o > 0; o >>= 1) {
    d1 += __shfl_xor_sync(0xffffffffu, d1, o);
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    const double ol64 = __shfl_xor_sync(0xffffffffu, l64, o), ol32 = __shfl_xor_sync(0xffffffffu, l32, o);
    if (ol64 > l64 || (ol64 == l64 && ol32 > l32)) { l64 = ol64; l32 = ol32; }
  }
  if (lane == 0) {
    s.d1 += d1;
    s.d2 += d2;
    if (cnt > 0 && (s.n == 0 || l64 > s.l64max)) { s.l64max = l64; s.l32max = l32; }
    s.n += (unsigned long long)cnt;
    rs[p] = s;
  }
}

}  // namespace

size_t refine_scratch_bytes(int np) {
  return ((size_t)np * RIFT_REFINE_CAP * sizeof(uint2) + 255) / 256 * 256 + ((size_t)np * sizeof(int) + 255) / 256 * 256 +
         (size_t)np * RIFT_REFINE_CAP * sizeof(double2);
}

cudaError_t launch_refine(const PointC *pts, const PointD *pd, const double2 *uv64, const float2 *qa,
                          const RoundPt *rp, const AccState *acc, const float *cmax, const float2 *cand, int np,
                          unsigned long long seed, double d_lo3, double d_span3, void *scratch,
                          RefineState *rs, uint32_t *flags, cudaStream_t st) {
  (void)pts;
  if (np <= 0) return cudaSuccess;
  unsigned char *b = static_cast<unsigned char *>(scratch);
  uint2 *list = reinterpret_cast<uint2 *>(b);
  b += ((size_t)np * RIFT_REFINE_CAP * sizeof(uint2) + 255) / 256 * 256;
  int *count = reinterpret_cast<int *>(b);
  b += ((size_t)np * sizeof(int) + 255) / 256 * 256;
  double2 *out = reinterpret_cast<double2 *>(b);
  refine_select_kernel<<<np, kSelThreads, 0, st>>>(rp, acc, cmax, cand, list, count);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  refine_eval_kernel<<<dim3(RIFT_REFINE_CAP, (unsigned)np), 32 * RIFT_MAXK, 0, st>>>(pd, uv64, qa, rp, list, count, seed,
                                                                             d_lo3, d_span3, out, flags);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  refine_fold_kernel<<<np, 32, 0, st>>>(acc, count, out, rs);
  return cudaGetLastError();
}
