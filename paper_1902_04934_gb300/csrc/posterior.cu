// Extrinsic posterior samples from a marginalisation (Eq. (lnLmarg) read as a posterior: the draws
// of a round weighted by w_i = L_i p_i / q_i are samples of p(theta | d) at the intrinsic point;
// Sec. VI: the same integration yields the extrinsic distributions).
//
//   rows_kernel      re-draws sample i of a point's last round from its index (same Philox
//                    stream and proposal as the cell kernel) and writes its parameters, lnL and
//                    ln p - ln q;
//   resample_kernel  systematic resampling of a point's last round with probabilities
//                    proportional to exp(beta (l_i - max l)), cumulative sums in FP64.
// The event time of time-marginalised draws is drawn in kernels.cu (tdraw_kernel).
#include <cmath>

#include "draw.cuh"
#include "rift_device.cuh"
#include "rift_internal.h"

namespace {

constexpr float kPi = 3.14159265358979f;
constexpr float kTwoPi = 6.283185307179586f;

// Parameters of draw d: ra, dec, t (NaN when the time is integrated out), psi, phi, incl, D.
// dec and incl come from the sampled sin dec and (1 + cos incl)/2 by atan2, which keeps them
// accurate near the poles.
__device__ __forceinline__ void theta_of(const PointC &P, const Drawn &d, bool tmarg, float *o) {
  o[0] = kTwoPi * (d.x0.hi + d.x0.lo);
  const float sd = (2.f * d.x1.hi - 1.f) + 2.f * d.x1.lo;
  const float cd = cos_dec_of(d.x1);
  o[1] = atan2f(sd, cd);
  o[2] = tmarg ? NAN : P.t_lo + P.t_span * (d.x2.hi + d.x2.lo);
  o[3] = kPi * d.u_psi;
  o[4] = kTwoPi * d.u_phi;
  o[5] = 2.f * atan2f(sqrtf(1.f - d.c_frac), sqrtf(d.c_frac));
  o[6] = d.dist;
}

// Row s of point p (grid: slots x points): sample i = idx[p][s] (idx NULL: i = s) of the point's
// last round -> out[p][s][0..ncol): the 7 parameters, lnL = l_i - (ln p - ln q), and (ncol 9)
// ln p - ln q.  Slots without a sample (past the round, or idx < 0) are NaN.
__global__ void rows_kernel(CellLaunch L, const RoundPt *__restrict__ last, const float *__restrict__ ell,
                            const int *__restrict__ idx, size_t n_slots, int ncol, float *__restrict__ out) {
  const int p = blockIdx.y;
  const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  const RoundPt R = last[p];
  float *o = out + ((size_t)p * n_slots + s) * ncol;
  const long long i = idx ? (long long)idx[(size_t)p * n_slots + s] : (long long)s;
  if (i < 0 || (uint64_t)i >= R.n || R.ell_off < 0) {
    for (int q = 0; q < ncol; ++q) o[q] = NAN;
    return;
  }
  const uint32_t ii = (uint32_t)i;
  const uint32_t big = R.rem * (R.base + 1u);
  const uint32_t cell = (ii < big) ? ii / (R.base + 1u) : R.rem + (ii - big) / R.base;
  const PointC *P = L.pts + p;
  Drawn d;
  if (R.proposal == 2)
    d = R.tmarg ? draw_learned<1>(L.seed, R, ii, R.gmm, P->dref, L.d_lo3, L.d_span3)
                : draw_learned<0>(L.seed, R, ii, R.gmm, P->dref, L.d_lo3, L.d_span3);
  else
    d = draw_cell_sample(L.seed, R, ii, cell, R.tab, R.lnw, P->dref, L.d_lo3, L.d_span3);
  theta_of(*P, d, R.tmarg != 0, o);
  o[7] = ell[R.ell_off + ii] - d.lpq;
  if (ncol > 8) o[8] = d.lpq;
}

// Block-wide inclusive scan of one double per thread (256 threads), added to `carry`; returns
// this thread's inclusive sum and (prev) the inclusive sum of the thread before it, which is
// `carry` for thread 0: bitwise the value that thread computed, so that consecutive rows share
// their boundary exactly.
__device__ __forceinline__ double block_scan(double v, double carry, double *wsum, double *wlast, double &prev) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) wsum[wid] = v;
  __syncthreads();
  double off = 0.0;
  for (int q = 0; q < wid; ++q) off += wsum[q];
  const double inc = (v + off) + carry;
  if (lane == 31) wlast[wid] = inc;
  __syncthreads();
  const double up = __shfl_up_sync(0xffffffffu, inc, 1);
  prev = lane > 0 ? up : (wid > 0 ? wlast[wid - 1] : carry);
  return inc;
}

// First slot h (0..H) whose target (h + 1/2) tot / H is >= c.
__device__ __forceinline__ int first_slot_at(double c, double tot, int H) {
  double g = ceil(c * (double)H / tot - 0.5);
  int h = (int)fmin(fmax(g, 0.0), (double)H);
  while (h > 0 && ((double)(h - 1) + 0.5) * tot / (double)H >= c) --h;
  while (h < H && ((double)h + 0.5) * tot / (double)H < c) ++h;
  return h;
}

// One CTA (256 threads) per point: slot h takes the first sample i of the last round with
// C_i > (h + 1/2) C_{n-1} / H, C the cumulative sums of w_i = exp(beta (l_i - max l)) (w = 0 for
// non-finite l).  Two passes of the same scan: the first gives the total C_{n-1}, the second
// assigns every slot whose target falls in [C_{i-1}, C_i) to sample i.
__global__ void __launch_bounds__(256) resample_kernel(const float *__restrict__ ell, const RoundPt *__restrict__ last,
                                                       const AccState *__restrict__ acc, float beta, int H,
                                                       int *__restrict__ idx) {
  __shared__ double wsum[8], wlast[8];
  __shared__ double carry_s;
  const int p = blockIdx.x;
  const RoundPt R = last[p];
  int *out = idx + (size_t)p * H;
  for (int h = threadIdx.x; h < H; h += blockDim.x) out[h] = -1;
  if (R.n == 0 || R.ell_off < 0) return;
  __syncthreads();
  const float mx = (float)acc[p].round_max;
  const float *e = ell + R.ell_off;
  double tot = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    double carry = 0.0;
    for (uint32_t b = 0; b < R.n; b += blockDim.x) {
      const uint32_t i = b + threadIdx.x;
      const float l = (i < R.n) ? e[i] : -INFINITY;
      const double w = isfinite(l) ? (double)expf(beta * (l - mx)) : 0.0;
      double prev;
      const double inc = block_scan(w, carry, wsum, wlast, prev);
      if (pass == 1 && i < R.n && inc > prev) {
        const int h0 = first_slot_at(prev, tot, H), h1 = first_slot_at(inc, tot, H);
        for (int h = h0; h < h1; ++h) out[h] = (int)i;
      }
      if (threadIdx.x == blockDim.x - 1) carry_s = inc;
      __syncthreads();
      carry = carry_s;
      __syncthreads();
    }
    tot = carry;
    if (!(tot > 0.0)) return;
  }
}

}  // namespace

cudaError_t launch_rows(const CellLaunch &L, const RoundPt *last, const float *ell, const int *idx, size_t n_slots,
                        int ncol, int np, float *out, cudaStream_t st) {
  if (n_slots == 0 || np == 0) return cudaSuccess;
  const int block = 128;
  const dim3 g((unsigned)((n_slots + block - 1) / block), (unsigned)np);
  rows_kernel<<<g, block, 0, st>>>(L, last, ell, idx, n_slots, ncol, out);
  return cudaGetLastError();
}

cudaError_t launch_resample(const float *ell, const RoundPt *last, const AccState *acc, int np, float beta, int H,
                            int *idx, cudaStream_t st) {
  if (np == 0 || H == 0) return cudaSuccess;
  resample_kernel<<<np, 256, 0, st>>>(ell, last, acc, beta, H, idx);
  return cudaGetLastError();
}
