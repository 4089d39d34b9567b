// Per-sample likelihood at caller-supplied samples (sm_103a): Eq. (def:lnL:Decomposed)
// with the Q taps gathered from global memory.  The Monte Carlo rounds live in mc.cu.
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

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Stage the coefficients of the point's quadratic form into shared memory: the positive form's
// table for a mirror-symmetric point (kernels compiled for three detectors and cubic taps), the
// pair layout otherwise.  The region holds npair * K float4, at least the mirror table's ncoef.
template <int K, int NT>
__device__ __forceinline__ void stage_quad_coef(const PointC &P, const float4 *__restrict__ ca, float4 *C) {
  const bool mir = kCanonPath<K, NT> && P.mirror;
  const float4 *cg = ca + (mir ? P.coef_off : P.uv_off);
  const int n = mir ? P.ncoef : P.npair * K;
  for (int j = threadIdx.x; j < n; j += blockDim.x) C[j] = cg[j];
}

// Quadratic form of a caller draw with harmonics Ys and real factors d (phi in radians).
template <int K, int NT>
__device__ __forceinline__ float quad_caller(const PointC &P, const float4 *C, const SampleGeo &g, const float2 *Ys,
                                             int ystride, float phi, const float (&d)[RIFT_MAXM]) {
  if constexpr (kCanonPath<K, NT>) {
    if (P.mirror) return quad_mirror_at<K>(reinterpret_cast<const float2 *>(C), g, d, P.sigma_neg, phi);
  }
  (void)phi;
  (void)d;
  return quad_term<K>(P, C, g, Ys, ystride);
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
  stage_quad_coef<K, NT>(P, ca, C);
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
    float dj[RIFT_MAXM];
    swsh_canonical_t<kCanonPath<K, NT>>(P, ch, sh, cphi, sphi, Ys, ystride, dj);
    const float lin = linear_term<K, NT>(P, Q, g, Ys, ystride, flags);
    const float quad = quad_caller<K, NT>(P, C, g, Ys, ystride, phi[i], dj);
    const float lnL = g.x * fmaf(-0.25f * g.x, quad, lin);
    if (!isfinite(lnL)) flags |= RIFT_FLAG_NONFINITE;
    out[i] = lnL;
  }
  if (flags) atomicOr(flags_out, flags);
}

// Geometry, harmonics and quadratic form of a caller draw (ra, dec, psi, phi, incl, D) whose time
// is integrated: g.s[k] is the Q index of the first quadrature time t_lo + 1/(2 fs) plus the time
// of flight to detector k.  Returns the quadratic form.
template <int K, int NT>
__device__ __forceinline__ float tmarg_setup(const PointC &P, const float4 *C, float r, float dec, float psi,
                                             float phi, float incl, float dist, SampleGeo &g, float2 *Ys,
                                             int ystride) {
  const float ph = __fmul_rn(r, 0.15915494309189535f);
  const float pl = __fmaf_rn(r, 0.15915494309189535f, -ph) + r * 6.4206382e-09f;
  const df v = df_add(fast_two_sum(ph, pl), df{-P.g_hi, -P.g_lo});
  float s0, c0;
  sincospif(2.f * v.hi, &s0, &c0);
  const float ares = kTwoPi * v.lo;
  const float cA = c0 - s0 * ares, sA = s0 + c0 * ares;
  float sdh, cd;
  sincosf(dec, &sdh, &cd);
  float s2p, c2p;
  sincosf(2.f * psi, &s2p, &c2p);
  df base[K];
#pragma unroll
  for (int k = 0; k < K; ++k) base[k] = df_add_f(df{P.det[k].c0, P.det[k].c0lo}, 0.5f);   // t_0 = t_lo + 1/(2 fs)
  response_delay<K>(P, cA, sA, df{sdh, 0.f}, cd, c2p, s2p, g, base);
  g.x = __fdiv_rn(P.dref, dist);
  float sphi, cphi, ch, sh;
  sincosf(phi, &sphi, &cphi);
  sincosf(0.5f * incl, &sh, &ch);
  float dj[RIFT_MAXM];
  swsh_canonical_t<kCanonPath<K, NT>>(P, ch, sh, cphi, sphi, Ys, ystride, dj);
  return quad_caller<K, NT>(P, C, g, Ys, ystride, phi, dj);
}

// Time-marginalised likelihood of caller draws (ra, dec, psi, phi, incl, D): Eq. (lnL:tmarg)
// by the midpoint rule on the Q sampling interval (tmarg_term).
template <int K, int NT>
__global__ void __launch_bounds__(128) lnl_tmarg_array_kernel(
    const PointC *__restrict__ pts, const float2 *__restrict__ qa, const float4 *__restrict__ ca, size_t n,
    const float *__restrict__ ra, const float *__restrict__ dec, const float *__restrict__ psi,
    const float *__restrict__ phi, const float *__restrict__ incl, const float *__restrict__ dist,
    float *__restrict__ out, uint32_t *flags_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  PointC &P = *reinterpret_cast<PointC *>(smem);
  load_point(pts, &P);
  __syncthreads();
  size_t off = align16(sizeof(PointC));
  float4 *C = reinterpret_cast<float4 *>(smem + off);
  off = align16(off + sizeof(float4) * (size_t)P.npair * K);
  float2 *Ys = reinterpret_cast<float2 *>(smem + off) + threadIdx.x;
  const int ystride = blockDim.x;
  stage_quad_coef<K, NT>(P, ca, C);
  __syncthreads();
  const float2 *Q = qa + P.q_off;
  uint32_t flags = 0u;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    SampleGeo g;
    const float quad = tmarg_setup<K, NT>(P, C, ra[i], dec[i], psi[i], phi[i], incl[i], dist[i], g, Ys, ystride);
    const float lm = tmarg_term<K, NT>(P, Q, g.s, g.F, Ys, ystride, g.x, quad, flags);
    if (!isfinite(lm)) flags |= RIFT_FLAG_NONFINITE;
    out[i] = lm;
  }
  if (flags) atomicOr(flags_out, flags);
}

// Event times of resampled time-marginalised draws (grid: slots x points): row h of point p,
// out[p][h] = (ra, dec, t, psi, phi, incl, D, lnL), gets t = t_j drawn from the conditional on the
// quadrature grid (tmarg_pick) with the uniform of Philox block 3 of counter (h, 0, point) (the
// sampler's streams use blocks 0-2), and lnL = lnL(t_j).  Rows that are NaN stay NaN.
template <int K, int NT>
__global__ void __launch_bounds__(128) tdraw_kernel(const PointC *__restrict__ pts, const float2 *__restrict__ qa,
                                                     const float4 *__restrict__ ca, const RoundPt *__restrict__ last,
                                                     unsigned long long seed, int H, float *__restrict__ out,
                                                     uint32_t *flags_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int p = blockIdx.y;
  PointC &P = *reinterpret_cast<PointC *>(smem);
  load_point(pts + p, &P);
  __syncthreads();
  size_t off = align16(sizeof(PointC));
  float4 *C = reinterpret_cast<float4 *>(smem + off);
  off = align16(off + sizeof(float4) * (size_t)P.npair * K);
  float2 *Ys = reinterpret_cast<float2 *>(smem + off) + threadIdx.x;
  const int ystride = blockDim.x;
  stage_quad_coef<K, NT>(P, ca, C);
  __syncthreads();
  const float2 *Q = qa + P.q_off;
  uint32_t flags = 0u;
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h < H) {
    float *o = out + ((size_t)p * H + h) * 8;
    if (!isnan(o[0])) {
      const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
      const uint4 b = philox4x32_10(make_uint4((uint32_t)h, 0u, 3u, last[p].point_id), key);
      SampleGeo g;
      const float quad = tmarg_setup<K, NT>(P, C, o[0], o[1], o[3], o[4], o[5], o[6], g, Ys, ystride);
      float l;
      const int j = tmarg_pick<K, NT>(P, Q, g.s, g.F, Ys, ystride, g.x, quad, bits_to_u(b.x), l, flags);
      if (j < 0) {
        o[2] = NAN; o[7] = NAN;
        flags |= RIFT_FLAG_NONFINITE;
      } else {
        o[2] = P.t_lo + ((float)j + 0.5f) / P.fs;
        o[7] = l;
      }
    }
  }
  if (flags) atomicOr(flags_out, flags);
}

template <int K, int NT>
cudaError_t lnl_tmarg_k(const PointC *pt_dev, const float2 *qa, const float4 *ca, size_t n, const float *ra,
                        const float *dec, const float *psi, const float *phi, const float *incl, const float *dist,
                        float *out, uint32_t *flags, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(lnl_tmarg_array_kernel<K, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int block = 128;
  const unsigned grid = (unsigned)((n + block - 1) / block);
  lnl_tmarg_array_kernel<K, NT><<<grid, block, smem, st>>>(pt_dev, qa, ca, n, ra, dec, psi, phi, incl, dist, out,
                                                          flags);
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
cudaError_t tdraw_k(const PointC *pts, const float2 *qa, const float4 *ca, const RoundPt *last,
                    unsigned long long seed, int np, int H, float *out, uint32_t *flags, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(tdraw_kernel<K, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int block = 128;
  const dim3 grid((unsigned)((H + block - 1) / block), (unsigned)np);
  tdraw_kernel<K, NT><<<grid, block, smem, st>>>(pts, qa, ca, last, seed, H, out, flags);
  return cudaGetLastError();
}

int taps_of(int interp) { return interp == 3 ? 4 : (interp == 1 ? 2 : 1); }

// Detector-frame coefficients and arrival times of sources (physical injections): for source i,
// coef[i][k][a] = x conj(F_k) Y_a (stored modes a, canonical order) and tk[i][k] = t + delay_k as
// (hi, lo) of a double-float, with the response, time of flight and harmonics of the likelihood
// kernels.  P holds the detectors with P.det[k].P = x_k / c in seconds (a sampling rate of 1), so
// the double-float "index" of response_delay is a time.  src: [8][n] = ra, dec, t (hi, lo), psi,
// phi, incl, D.
template <int K>
__global__ void __launch_bounds__(128) source_frame_kernel(const PointC *__restrict__ pts, size_t n,
                                                            const float *__restrict__ src, float2 *__restrict__ coef,
                                                            float2 *__restrict__ tk) {
  __shared__ __align__(16) PointC P;
  load_point(pts, &P);
  __syncthreads();
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float r = src[i], dec = src[n + i], psi = src[4 * n + i], phi = src[5 * n + i], incl = src[6 * n + i];
  const float ph = __fmul_rn(r, 0.15915494309189535f);
  const float pl = __fmaf_rn(r, 0.15915494309189535f, -ph) + r * 6.4206382e-09f;
  const df v = df_add(fast_two_sum(ph, pl), df{-P.g_hi, -P.g_lo});
  float s0, c0;
  sincospif(2.f * v.hi, &s0, &c0);
  const float ares = kTwoPi * v.lo;
  const float cA = c0 - s0 * ares, sA = s0 + c0 * ares;
  float sdh, cd, s2p, c2p;
  sincosf(dec, &sdh, &cd);
  sincosf(2.f * psi, &s2p, &c2p);
  df base[K];
#pragma unroll
  for (int k = 0; k < K; ++k) base[k] = df{src[2 * n + i], src[3 * n + i]};
  SampleGeo g;
  response_delay<K>(P, cA, sA, df{sdh, 0.f}, cd, c2p, s2p, g, base);
  const float x = __fdiv_rn(P.dref, src[7 * n + i]);
  float sphi, cphi, ch, sh;
  sincosf(phi, &sphi, &cphi);
  sincosf(0.5f * incl, &sh, &ch);
  float2 Y[RIFT_MAXM];
  swsh_canonical(P, ch, sh, cphi, sphi, Y, 1);
  for (int k = 0; k < K; ++k) {
    const float2 F = g.F[k];
    for (int a = 0; a < P.M; ++a) {
      // x conj(F) Y
      const float2 y = Y[a];
      coef[(i * K + k) * P.M + a] = make_float2(x * (F.x * y.x + F.y * y.y), x * (F.x * y.y - F.y * y.x));
    }
    tk[i * K + k] = make_float2(g.s[k].hi, g.s[k].lo);
  }
}

}  // namespace

cudaError_t launch_source_frame(int K, const PointC *pt_dev, size_t n, const float *src, float2 *coef, float2 *tk,
                                cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 127) / 128);
  switch (K) {
    case 1: source_frame_kernel<1><<<grid, 128, 0, st>>>(pt_dev, n, src, coef, tk); break;
    case 2: source_frame_kernel<2><<<grid, 128, 0, st>>>(pt_dev, n, src, coef, tk); break;
    case 3: source_frame_kernel<3><<<grid, 128, 0, st>>>(pt_dev, n, src, coef, tk); break;
    case 4: source_frame_kernel<4><<<grid, 128, 0, st>>>(pt_dev, n, src, coef, tk); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

size_t rift_point_smem_bytes(int K, int npair, int nb, int block, int M) {
  size_t off = (sizeof(PointC) + 15) & ~size_t(15);
  off = (off + sizeof(float4) * (size_t)npair * K + 15) & ~size_t(15);
  if (nb > 0) off = (off + sizeof(float) * (size_t)(3 * (nb + 1) + 3 * nb) + 15) & ~size_t(15);
  return off + sizeof(float2) * (size_t)M * block;
}

#define RIFT_DISPATCH_KT(K, NT, CALL)                                           \
  switch ((K) * 8 + (NT)) {                                                     \
    case 1 * 8 + 1: return CALL(1, 1); case 1 * 8 + 2: return CALL(1, 2); case 1 * 8 + 4: return CALL(1, 4); \
    case 2 * 8 + 1: return CALL(2, 1); case 2 * 8 + 2: return CALL(2, 2); case 2 * 8 + 4: return CALL(2, 4); \
    case 3 * 8 + 1: return CALL(3, 1); case 3 * 8 + 2: return CALL(3, 2); case 3 * 8 + 4: return CALL(3, 4); \
    case 4 * 8 + 1: return CALL(4, 1); case 4 * 8 + 2: return CALL(4, 2); case 4 * 8 + 4: return CALL(4, 4); \
    default: return cudaErrorInvalidValue;                                      \
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

// Merged rows (grid: blocks x points): row (k, t) of point p, slot h < Mh, is its Q row's entry for
// stored mode h_a[h]; slots up to Mhp are zero.
__global__ void __launch_bounds__(256) merge_rows_kernel(const PointC *__restrict__ pts, float2 *__restrict__ qa) {
  const PointC &P = pts[blockIdx.y];
  if (!P.qhalf) return;
  const long long n = (long long)P.K * P.T * P.Mhp;
  float2 *out = qa + P.q_off + P.qh_rel;
  const float2 *in = qa + P.q_off;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int hh = (int)(i % P.Mhp);
    const long long row = i / P.Mhp;
    out[i] = (hh < P.Mh) ? in[row * P.Mp + P.h_a[hh]] : make_float2(0.f, 0.f);
  }
}

cudaError_t launch_merge_rows(const PointC *pts, int np, float2 *qa, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  merge_rows_kernel<<<dim3(32, (unsigned)np), 256, 0, st>>>(pts, qa);
  return cudaGetLastError();
}

cudaError_t launch_lnl_tmarg(int K, const PointC *pt_dev, const PointC &ph, const float2 *qa, const float4 *ca,
                             size_t n, const float *ra, const float *dec, const float *psi, const float *phi,
                             const float *incl, const float *dist, float *out, uint32_t *flags, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t smem = rift_point_smem_bytes(K, ph.npair, 0, 128, ph.M);
#define RIFT_LT(KK, TT) lnl_tmarg_k<KK, TT>(pt_dev, qa, ca, n, ra, dec, psi, phi, incl, dist, out, flags, smem, st)
  RIFT_DISPATCH_KT(K, taps_of(ph.interp), RIFT_LT)
#undef RIFT_LT
}


cudaError_t launch_tdraw(int K, int interp, const PointC *pts, int np, int max_npair, int max_M, const float2 *qa,
                         const float4 *ca, const RoundPt *last, unsigned long long seed, int H, float *out,
                         uint32_t *flags, cudaStream_t st) {
  if (np == 0 || H == 0) return cudaSuccess;
  const size_t smem = rift_point_smem_bytes(K, max_npair, 0, 128, max_M);
#define RIFT_TD(KK, TT) tdraw_k<KK, TT>(pts, qa, ca, last, seed, np, H, out, flags, smem, st)
  RIFT_DISPATCH_KT(K, taps_of(interp), RIFT_TD)
#undef RIFT_TD
}
