// Kernels of the extrinsic-likelihood hot path (sm_103a).
//
//  mc_round     : Philox draw -> prior/proposal transform -> response, delay, -2Y_lm
//                 -> Q gather + interpolation -> linear and quadratic terms -> lnL
//                 -> log weight -> per-thread log-sum-exp -> warp-shuffle block merge
//                 (Eq. def:lnL:Decomposed inside Eq. lnLmarg; Sec. II.B-C)
//  merge        : FP64 fixed-order merge of block partials into the point's running
//                 compensated accumulator
//  hist, tables : adaptive proposal update (Sec. III.B: the sampling prior is rebuilt
//                 from the most recent chunk of samples)
//  lnl_array    : per-sample lnL at caller-supplied samples
//  draw         : the samples of one round, for inspection
#include <cfloat>
#include <cmath>

#include "rift_device.cuh"
#include "rift_internal.h"

namespace {

constexpr float kTwoPi = 6.283185307179586f;
constexpr float kNegInf = -INFINITY;

__device__ __forceinline__ void load_point(const PointC *src, PointC *dst) {
  const int n = sizeof(PointC) / sizeof(int);
  const int *s = reinterpret_cast<const int *>(src);
  int *d = reinterpret_cast<int *>(dst);
  for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ void draw_uniforms(unsigned long long seed, uint32_t i, uint32_t round, uint32_t point,
                                              float u[8]) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint4 a = philox4x32_10(make_uint4(i, round, 0u, point), key);
  const uint4 b = philox4x32_10(make_uint4(i, round, 1u, point), key);
  u[0] = bits_to_u(a.x); u[1] = bits_to_u(a.y); u[2] = bits_to_u(a.z); u[3] = bits_to_u(a.w);
  u[4] = bits_to_u(b.x); u[5] = bits_to_u(b.y); u[6] = bits_to_u(b.z); u[7] = bits_to_u(b.w);
}

// Piecewise-constant inverse CDF of one adapted coordinate: fraction x of the range
// (double-float) and the bin.  The bin is the largest b with cdf[b] <= u.
__device__ __forceinline__ df inv_cdf(const float *cdf, int nb, float u, int &b) {
  int lo = 0, hi = nb;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (cdf[mid] <= u) lo = mid; else hi = mid;
  }
  b = lo;
  const float c0 = cdf[lo], c1 = cdf[lo + 1];
  const df num = two_sum(u, -c0);
  const df den = two_sum(c1, -c0);
  const float f = __fdiv_rn(num.hi + num.lo, den.hi + den.lo);
  const df bf = two_sum((float)b, f);
  const float fnb = (float)nb;
  const float qh = __fdiv_rn(bf.hi, fnb);
  const float r = __fmaf_rn(-qh, fnb, bf.hi);
  const float ql = __fdiv_rn(r + bf.lo, fnb);
  return fast_two_sum(qh, ql);
}

struct Drawn {
  df x0, x1, x2;   // fractions of the ra, sin dec, t ranges
  float u3, u4, u5, u6;
  float lpq;       // ln p - ln q
  uint32_t bins;   // packed adapted bins (8 bits each)
};

__device__ __forceinline__ Drawn draw_sample(const McParams &prm, uint32_t point, uint32_t i, const float *tab,
                                             const float *lnw) {
  float u[8];
  draw_uniforms(prm.seed, i, prm.round, point, u);
  Drawn d;
  d.u3 = u[3]; d.u4 = u[4]; d.u5 = u[5]; d.u6 = u[6];
  if (prm.proposal == 0) {
    d.x0 = df{u[0], 0.f}; d.x1 = df{u[1], 0.f}; d.x2 = df{u[2], 0.f};
    d.lpq = 0.f; d.bins = 0u;
  } else {
    const int nb = prm.nb;
    int b0, b1, b2;
    d.x0 = inv_cdf(tab, nb, u[0], b0);
    d.x1 = inv_cdf(tab + (nb + 1), nb, u[1], b1);
    d.x2 = inv_cdf(tab + 2 * (nb + 1), nb, u[2], b2);
    d.lpq = lnw[b0] + lnw[nb + b1] + lnw[2 * nb + b2];
    d.bins = (uint32_t)b0 | ((uint32_t)b1 << 8) | ((uint32_t)b2 << 16);
  }
  return d;
}

// Geometry of a drawn sample: response, time index per detector, distance factor, -2Y_lm.
template <int K>
__device__ __forceinline__ void geometry_drawn(const PointC &P, const McParams &prm, const Drawn &d, SampleGeo &g,
                                               float2 *Ys, int ystride) {
  // sidereal hour-angle offset in turns: v = ra/2pi - GMST/2pi (double-float)
  const df v = df_add(d.x0, df{-P.g_hi, -P.g_lo});
  float s0, c0;
  sincospif(2.f * v.hi, &s0, &c0);
  const float ares = kTwoPi * v.lo;
  const float ca = c0 - s0 * ares, sa = s0 + c0 * ares;   // cos, sin of (ra - GMST)
  const df sd = df_add_f(df{2.f * d.x1.hi, 2.f * d.x1.lo}, -1.f);
  const float cd = 2.f * sqrtf(d.x1.hi * (1.f - d.x1.hi));
  float s2p, c2p;
  sincospif(2.f * d.u3, &s2p, &c2p);                      // 2 psi = 2 pi u3
  df base[K];
  const df tf = df_mul(df{P.A, P.Alo}, d.x2);             // (t - t_lo) fs
#pragma unroll
  for (int k = 0; k < K; ++k) base[k] = df_add(df{P.det[k].c0, P.det[k].c0lo}, tf);
  response_delay<K>(P, ca, sa, sd, cd, c2p, s2p, g, base);
  const float D3 = fmaf(d.u6, prm.d_span3, prm.d_lo3);
  g.x = P.dref * rcbrtf(D3);
  float sphi, cphi;
  sincospif(2.f * d.u4, &sphi, &cphi);
  swsh_modes(P, sqrtf(d.u5), sqrtf(1.f - d.u5), cphi, sphi, Ys, ystride);
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

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <int K, int NT>
__global__ void __launch_bounds__(RIFT_MC_BLOCK, 4) mc_round_kernel(const PointC *__restrict__ pts, const float2 *__restrict__ qa,
                                                        const float4 *__restrict__ ca, McParams prm) {
  extern __shared__ __align__(16) unsigned char smem[];
  PointC &P = *reinterpret_cast<PointC *>(smem);
  load_point(pts, &P);
  __syncthreads();
  size_t off = align16(sizeof(PointC));
  float4 *C = reinterpret_cast<float4 *>(smem + off);
  off = align16(off + sizeof(float4) * (size_t)P.npair * K);
  float *tab = reinterpret_cast<float *>(smem + off);
  float *lnw = tab + 3 * (prm.nb + 1);
  if (prm.proposal != 0) off = align16(off + sizeof(float) * (size_t)(3 * (prm.nb + 1) + 3 * prm.nb));
  float2 *Ys = reinterpret_cast<float2 *>(smem + off) + threadIdx.x;
  const int ystride = blockDim.x;
  const float4 *cg = ca + P.uv_off;
  for (int j = threadIdx.x; j < P.npair * K; j += blockDim.x) C[j] = cg[j];
  if (prm.proposal != 0) {
    for (int j = threadIdx.x; j < 3 * (prm.nb + 1); j += blockDim.x) tab[j] = prm.tables[j];
    for (int j = threadIdx.x; j < 3 * prm.nb; j += blockDim.x) lnw[j] = prm.lnw[j];
  }
  __syncthreads();
  const float2 *Q = qa + P.q_off;

  float m = kNegInf, s1 = 0.f, s2 = 0.f, cnt = 0.f;
  uint32_t flags = 0u;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < prm.n; i += gridDim.x * blockDim.x) {
    const Drawn d = draw_sample(prm, prm.point_id, i, tab, lnw);
    SampleGeo g;
    geometry_drawn<K>(P, prm, d, g, Ys, ystride);
    const float lin = linear_term<K, NT>(P, Q, g, Ys, ystride, flags);
    const float quad = quad_term<K>(P, C, g, Ys, ystride);
    const float lnL = g.x * fmaf(-0.25f * g.x, quad, lin);
    const float ell = lnL + d.lpq;
    if (prm.dbg_ell) prm.dbg_ell[prm.dbg_off + i] = ell;
    if (prm.ell_buf) { prm.ell_buf[i] = ell; prm.bin_buf[i] = d.bins; }
    if (isfinite(ell)) { lse_push(ell, m, s1, s2); cnt += 1.f; }
    else flags |= RIFT_FLAG_NONFINITE;
  }
  // warp merge
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float m2 = __shfl_xor_sync(0xffffffffu, m, o);
    const float a2 = __shfl_xor_sync(0xffffffffu, s1, o);
    const float b2 = __shfl_xor_sync(0xffffffffu, s2, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    lse_merge(m, s1, s2, m2, a2, b2);
  }
  flags = __reduce_or_sync(0xffffffffu, flags);
  __shared__ float4 wpart[32];
  __shared__ uint32_t wflag[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { wpart[wid] = make_float4(m, s1, s2, cnt); wflag[wid] = flags; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float M = kNegInf, S1 = 0.f, S2 = 0.f, N = 0.f;
    uint32_t F = 0u;
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) {
      lse_merge(M, S1, S2, wpart[w].x, wpart[w].y, wpart[w].z);
      N += wpart[w].w;
      F |= wflag[w];
    }
    prm.partials[blockIdx.x] = Part{(double)M, (double)S1, (double)S2, (double)N};
    if (F) atomicOr(prm.flags, F);
  }
}

__device__ __forceinline__ void d_merge(double &m, double &s1, double &s2, double &n, double m2, double t1, double t2,
                                        double n2) {
  n += n2;
  if (m2 > m) {
    double tm = m, a = s1, b = s2;
    m = m2; s1 = t1; s2 = t2; m2 = tm; t1 = a; t2 = b;
  }
  if (m2 == -INFINITY) return;
  const double e = exp(m2 - m);
  s1 += t1 * e;
  s2 += t2 * e * e;
}

__device__ __forceinline__ void neumaier(double &s, double &c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
  s = t;
}

__global__ void merge_kernel(const Part *__restrict__ part, int nparts, AccState *acc) {
  __shared__ double sm[256][4];
  double m = -INFINITY, s1 = 0.0, s2 = 0.0, n = 0.0;
  for (int j = threadIdx.x; j < nparts; j += blockDim.x) {
    const Part p = part[j];
    d_merge(m, s1, s2, n, p.m, p.s1, p.s2, p.n);
  }
  sm[threadIdx.x][0] = m; sm[threadIdx.x][1] = s1; sm[threadIdx.x][2] = s2; sm[threadIdx.x][3] = n;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double a = sm[threadIdx.x][0], b = sm[threadIdx.x][1], c = sm[threadIdx.x][2], d = sm[threadIdx.x][3];
      d_merge(a, b, c, d, sm[threadIdx.x + w][0], sm[threadIdx.x + w][1], sm[threadIdx.x + w][2],
              sm[threadIdx.x + w][3]);
      sm[threadIdx.x][0] = a; sm[threadIdx.x][1] = b; sm[threadIdx.x][2] = c; sm[threadIdx.x][3] = d;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double M = sm[0][0], S1 = sm[0][1], S2 = sm[0][2], N = sm[0][3];
    acc->round_max = M;
    if (N > 0.0 && M != -INFINITY) {
      if (M > acc->m) {
        const double f = (acc->m == -INFINITY) ? 0.0 : exp(acc->m - M);
        acc->s1 *= f; acc->c1 *= f; acc->s2 *= f * f; acc->c2 *= f * f;
        acc->m = M;
      }
      const double e = exp(M - acc->m);
      neumaier(acc->s1, acc->c1, S1 * e);
      neumaier(acc->s2, acc->c2, S2 * e * e);
    }
    acc->n += (unsigned long long)N;
  }
}

// Adaptive histogram: w^beta = exp(beta (l - max_round)) accumulated per bin of each
// adapted coordinate in 32.32 fixed point (integer adds: order independent, deterministic).
__global__ void hist_kernel(const float *__restrict__ ell, const uint32_t *__restrict__ bins, uint32_t n,
                            const AccState *acc, float beta, int nb, unsigned long long *part) {
  extern __shared__ unsigned long long h[];
  for (int j = threadIdx.x; j < 3 * nb; j += blockDim.x) h[j] = 0ull;
  __syncthreads();
  const float mx = (float)acc->round_max;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float l = ell[i];
    if (!isfinite(l)) continue;
    const float w = expf(beta * (l - mx));
    const unsigned long long q = __float2ull_rn(w * 4294967296.0f);
    const uint32_t b = bins[i];
    atomicAdd(&h[b & 255u], q);
    atomicAdd(&h[nb + ((b >> 8) & 255u)], q);
    atomicAdd(&h[2 * nb + ((b >> 16) & 255u)], q);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < 3 * nb; j += blockDim.x) part[(size_t)blockIdx.x * 3 * nb + j] = h[j];
}

// New proposal tables: p_b = (1 - eps) h_b / sum h + eps / nb; cdf = cumsum (FP64) rounded
// to float32 with cdf[0] = 0, cdf[nb] = 1; lnw_b = -ln(nb (cdf[b+1] - cdf[b])).
__global__ void tables_kernel(const unsigned long long *__restrict__ part, int nparts, int nb, double eps,
                              float *tables, float *lnw) {
  __shared__ double hs[3 * RIFT_MAXBINS];
  for (int j = threadIdx.x; j < 3 * nb; j += blockDim.x) {
    unsigned long long t = 0ull;
    if (part) for (int p = 0; p < nparts; ++p) t += part[(size_t)p * 3 * nb + j];
    hs[j] = (double)t;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int d = threadIdx.x;
    double S = 0.0;
    for (int b = 0; b < nb; ++b) S += hs[d * nb + b];
    float *cdf = tables + d * (nb + 1);
    if (part) {
      double c = 0.0;
      cdf[0] = 0.f;
      double tot = 0.0;
      for (int b = 0; b < nb; ++b) tot += (S > 0.0 ? (1.0 - eps) * hs[d * nb + b] / S : 0.0) + eps / nb;
      if (S <= 0.0) tot = 1.0;
      for (int b = 0; b < nb; ++b) {
        const double pb = (S > 0.0 ? (1.0 - eps) * hs[d * nb + b] / S + eps / nb : 1.0 / nb);
        c += pb;
        cdf[b + 1] = (float)(c / tot);
      }
      cdf[nb] = 1.f;
    }
    for (int b = 0; b < nb; ++b)
      lnw[d * nb + b] = (float)(-log((double)nb * ((double)cdf[b + 1] - (double)cdf[b])));
  }
}

template <int K, int NT>
__global__ void __launch_bounds__(128) lnl_array_kernel(const PointC *__restrict__ pts, const float2 *__restrict__ qa,
                                                         const float4 *__restrict__ ca, size_t n,
                                                         const float *__restrict__ ra, const float *__restrict__ dec,
                                                         const float *__restrict__ t, const float *__restrict__ psi,
                                                         const float *__restrict__ phi,
                                                         const float *__restrict__ incl,
                                                         const float *__restrict__ dist, float *__restrict__ out,
                                                         uint32_t *flags_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  PointC &P = *reinterpret_cast<PointC *>(smem);
  load_point(pts, &P);
  __syncthreads();
  size_t off = align16(sizeof(PointC));
  float4 *C = reinterpret_cast<float4 *>(smem + off);
  off = align16(off + sizeof(float4) * (size_t)P.npair * K);
  float2 *Ys = reinterpret_cast<float2 *>(smem + off) + threadIdx.x;
  const int ystride = blockDim.x;
  const float4 *cg = ca + P.uv_off;
  for (int j = threadIdx.x; j < P.npair * K; j += blockDim.x) C[j] = cg[j];
  __syncthreads();
  const float2 *Q = qa + P.q_off;
  uint32_t flags = 0u;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    // ra/2pi - GMST/2pi in double-float turns
    const float r = ra[i];
    const float ph = __fmul_rn(r, 0.15915494309189535f);
    const float pl = __fmaf_rn(r, 0.15915494309189535f, -ph) + r * 6.4206382e-09f;
    const df v = df_add(fast_two_sum(ph, pl), df{-P.g_hi, -P.g_lo});
    float s0, c0;
    sincospif(2.f * v.hi, &s0, &c0);
    const float ares = kTwoPi * v.lo;
    const float cA = c0 - s0 * ares, sA = s0 + c0 * ares;
    float sdh, cd;
    sincosf(dec[i], &sdh, &cd);
    float s2p, c2p;
    sincosf(2.f * psi[i], &s2p, &c2p);
    const float tf = __fmul_rn(t[i], P.fs);
    const df tfs = fast_two_sum(tf, __fmaf_rn(t[i], P.fs, -tf));
    df base[K];
#pragma unroll
    for (int k = 0; k < K; ++k) base[k] = df_add(df{P.det[k].ct, P.det[k].ctlo}, tfs);
    SampleGeo g;
    response_delay<K>(P, cA, sA, df{sdh, 0.f}, cd, c2p, s2p, g, base);
    g.x = __fdiv_rn(P.dref, dist[i]);
    float sphi, cphi, ch, sh;
    sincosf(phi[i], &sphi, &cphi);
    sincosf(0.5f * incl[i], &sh, &ch);
    swsh_modes(P, ch, sh, cphi, sphi, Ys, ystride);
    const float lin = linear_term<K, NT>(P, Q, g, Ys, ystride, flags);
    const float quad = quad_term<K>(P, C, g, Ys, ystride);
    const float lnL = g.x * fmaf(-0.25f * g.x, quad, lin);
    if (!isfinite(lnL)) flags |= RIFT_FLAG_NONFINITE;
    out[i] = lnL;
  }
  if (flags) atomicOr(flags_out, flags);
}

__global__ void draw_kernel(const PointC *__restrict__ pts, McParams prm, DrawOut o) {
  __shared__ __align__(16) PointC P;
  extern __shared__ float dtab[];
  load_point(pts, &P);
  float *tab = dtab;
  float *lnw = dtab + 3 * (prm.nb + 1);
  if (prm.proposal != 0) {
    for (int j = threadIdx.x; j < 3 * (prm.nb + 1); j += blockDim.x) tab[j] = prm.tables[j];
    for (int j = threadIdx.x; j < 3 * prm.nb; j += blockDim.x) lnw[j] = prm.lnw[j];
  }
  __syncthreads();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= prm.n) return;
  const Drawn d = draw_sample(prm, prm.point_id, i, tab, lnw);
  const size_t n = prm.n;
  o.theta[0 * n + i] = kTwoPi * (d.x0.hi + d.x0.lo);
  o.theta[1 * n + i] = (2.f * d.x1.hi - 1.f) + 2.f * d.x1.lo;
  o.theta[2 * n + i] = P.t_lo + P.t_span * (d.x2.hi + d.x2.lo);
  o.theta[3 * n + i] = 3.14159265358979f * d.u3;
  o.theta[4 * n + i] = kTwoPi * d.u4;
  o.theta[5 * n + i] = 2.f * d.u5 - 1.f;
  o.theta[6 * n + i] = cbrtf(fmaf(d.u6, prm.d_span3, prm.d_lo3));
  o.lpq[i] = d.lpq;
  if (o.bins) {
    o.bins[0 * n + i] = (int)(d.bins & 255u);
    o.bins[1 * n + i] = (int)((d.bins >> 8) & 255u);
    o.bins[2 * n + i] = (int)((d.bins >> 16) & 255u);
  }
}

template <int K, int NT>
cudaError_t mc_round_k(const PointC *pt_dev, const float2 *qa, const float4 *ca, const McParams &prm, int grid,
                       int block, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(mc_round_kernel<K, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  mc_round_kernel<K, NT><<<grid, block, smem, st>>>(pt_dev, qa, ca, prm);
  return cudaGetLastError();
}

template <int K, int NT>
cudaError_t lnl_array_k(const PointC *pt_dev, const float2 *qa, const float4 *ca, size_t n, const float *ra,
                        const float *dec, const float *t, const float *psi, const float *phi, const float *incl,
                        const float *dist, float *out, uint32_t *flags, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(lnl_array_kernel<K, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int block = 128;
  const unsigned grid = (unsigned)((n + block - 1) / block);
  lnl_array_kernel<K, NT><<<grid, block, smem, st>>>(pt_dev, qa, ca, n, ra, dec, t, psi, phi, incl, dist, out, flags);
  return cudaGetLastError();
}

template <int K, int NT>
int occ_k(size_t smem, int block) {
  int nb = 0;
  cudaFuncSetAttribute(mc_round_kernel<K, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mc_round_kernel<K, NT>, block, smem);
  return nb;
}

int taps_of(int interp) { return interp == 3 ? 4 : (interp == 1 ? 2 : 1); }

}  // namespace

size_t rift_point_smem_bytes(int K, int npair, int nb, int block, int M) {
  size_t off = (sizeof(PointC) + 15) & ~size_t(15);
  off = (off + sizeof(float4) * (size_t)npair * K + 15) & ~size_t(15);
  if (nb > 0) off = (off + sizeof(float) * (size_t)(3 * (nb + 1) + 3 * nb) + 15) & ~size_t(15);
  return off + sizeof(float2) * (size_t)M * block;
}

int mc_round_blocks_per_sm(int K, size_t smem, int block) {
  switch (K) {
    case 1: return occ_k<1, 4>(smem, block);
    case 2: return occ_k<2, 4>(smem, block);
    case 3: return occ_k<3, 4>(smem, block);
    case 4: return occ_k<4, 4>(smem, block);
    default: return 0;
  }
}

#define RIFT_DISPATCH_KT(K, NT, CALL)                                           \
  switch ((K) * 8 + (NT)) {                                                     \
    case 1 * 8 + 1: return CALL(1, 1); case 1 * 8 + 2: return CALL(1, 2); case 1 * 8 + 4: return CALL(1, 4); \
    case 2 * 8 + 1: return CALL(2, 1); case 2 * 8 + 2: return CALL(2, 2); case 2 * 8 + 4: return CALL(2, 4); \
    case 3 * 8 + 1: return CALL(3, 1); case 3 * 8 + 2: return CALL(3, 2); case 3 * 8 + 4: return CALL(3, 4); \
    case 4 * 8 + 1: return CALL(4, 1); case 4 * 8 + 2: return CALL(4, 2); case 4 * 8 + 4: return CALL(4, 4); \
    default: return cudaErrorInvalidValue;                                      \
  }

cudaError_t launch_mc_round(int K, const PointC *pt_dev, const PointC &ph, const float2 *qa, const float4 *ca,
                            const McParams &prm, int grid, int block, cudaStream_t st) {
  const size_t smem = rift_point_smem_bytes(K, ph.npair, prm.proposal ? prm.nb : 0, block, ph.M);
#define RIFT_MC(KK, TT) mc_round_k<KK, TT>(pt_dev, qa, ca, prm, grid, block, smem, st)
  RIFT_DISPATCH_KT(K, taps_of(ph.interp), RIFT_MC)
#undef RIFT_MC
}

cudaError_t launch_merge(const Part *partials, int nparts, AccState *acc, cudaStream_t st) {
  merge_kernel<<<1, 256, 0, st>>>(partials, nparts, acc);
  return cudaGetLastError();
}

cudaError_t launch_hist(const float *ell, const uint32_t *bins, uint32_t n, const AccState *acc, float beta, int nb,
                        unsigned long long *part, int grid, cudaStream_t st) {
  hist_kernel<<<grid, 256, sizeof(unsigned long long) * 3 * nb, st>>>(ell, bins, n, acc, beta, nb, part);
  return cudaGetLastError();
}

cudaError_t launch_tables(const unsigned long long *part, int nparts, int nb, double floor_eps, float *tables,
                          float *lnw, cudaStream_t st) {
  tables_kernel<<<1, 256, 0, st>>>(part, nparts, nb, floor_eps, tables, lnw);
  return cudaGetLastError();
}

cudaError_t launch_lnl_array(int K, const PointC *pt_dev, const PointC &ph, const float2 *qa, const float4 *ca,
                             size_t n, const float *ra, const float *dec, const float *t, const float *psi,
                             const float *phi, const float *incl, const float *dist, float *out, uint32_t *flags,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t smem = rift_point_smem_bytes(K, ph.npair, 0, 128, ph.M);
#define RIFT_LA(KK, TT) lnl_array_k<KK, TT>(pt_dev, qa, ca, n, ra, dec, t, psi, phi, incl, dist, out, flags, smem, st)
  RIFT_DISPATCH_KT(K, taps_of(ph.interp), RIFT_LA)
#undef RIFT_LA
}

cudaError_t launch_draw(int K, const PointC *pt_dev, const PointC &ph, const McParams &prm, DrawOut o,
                        cudaStream_t st) {
  (void)K; (void)ph;
  if (prm.n == 0) return cudaSuccess;
  const int block = 128;
  const unsigned grid = (prm.n + block - 1) / block;
  const size_t smem = prm.proposal ? sizeof(float) * (3 * (prm.nb + 1) + 3 * prm.nb) : 0;
  draw_kernel<<<grid, block, smem, st>>>(pt_dev, prm, o);
  return cudaGetLastError();
}
