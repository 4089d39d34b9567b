// Learned proposal: mixture-density network over (ra, sin dec, t, cos incl, ln D), its
// training (weighted negative log likelihood of harvested posterior samples, Adam), the
// per-point summary it is conditioned on.
//
// Network: s (64) -> 256 -> 256 (GELU, erf form) -> 88 = 8 logits + 8x5 means + 8x5 log
// sigmas; weights bfloat16 (rounded from a float32 master copy), accumulation float32.  The
// forward pass runs on the tensor cores (tcgen05, 128 points per CTA, activations split into two
// bfloat16 terms); loss and backward take one CTA per point; weight gradients are sums over
// points in point order (the same bits on every run).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rift_ile.h"
#include "rift_device.cuh"
#include "rift_internal.h"
#include "tc.cuh"

namespace {

constexpr int NI = 64, NH = 256, NC = 8, ND = 5, NO = NC * (1 + 2 * ND);
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NPARAM = OFF_B3 + NO;
static_assert(NPARAM == RIFT_MDN_PARAMS, "parameter count in the header is out of date");
constexpr float LS_MIN = -8.f, LS_MAX = 4.f;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}
__device__ __forceinline__ float bf(const __nv_bfloat16 *w, int i) { return __bfloat162float(w[i]); }

// dot of a bfloat16 row (16-byte aligned, n multiple of 8) with a float vector in shared memory
__device__ __forceinline__ float row_dot(const __nv_bfloat16 *row, const float *x, int n, float acc) {
  const uint4 *r = reinterpret_cast<const uint4 *>(row);
  for (int q = 0; q < n / 8; ++q) {
    const uint4 v = __ldg(r + q);
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(h[e]);
      acc = fmaf(f.x, x[8 * q + 2 * e], acc);
      acc = fmaf(f.y, x[8 * q + 2 * e + 1], acc);
    }
  }
  return acc;
}

// ---------------------------------------------------------------------------------------------
// Forward pass on the tensor cores (tcgen05), 128 points per CTA.  Each layer is D = A W^T: A
// holds the layer's inputs (rows = points), W the weight rows (neurons), both BF16 in shared
// memory in the K-major layout of tc.cuh, D is FP32 in tensor memory.  The FP32 inputs are split
// into two BF16 terms, a = hi + lo with hi = bf16(a) and lo = bf16(a - hi), and both are multiplied
// by the (exactly BF16) weights, so the inputs keep about 16 significant bits.  Sixteen warps:
// warp w reads the tensor-memory lanes of rows 32 (w % 4) .. + 31 (the quarter its position in a
// warpgroup allows) and the columns of group w / 4, applying bias, GELU and the split on the way
// to the next layer's operand.  The next weights are staged by asynchronous copies while the
// warps work through the previous layer's results.  Tensor-memory columns: layer 1 [0, 256),
// layer 2 [0, 128) and [128, 256) (the two halves of W2 staged in turn), the head [0, 96).
// ---------------------------------------------------------------------------------------------
constexpr int TC_P = 128;                        // points per CTA (tensor-memory lanes)
constexpr int TC_THREADS = 512;                  // 4 lane quarters x 4 column groups
constexpr int NO_PAD = 96;                       // head rows padded to a multiple of 16
constexpr int TC_OP = TC_P * NH * 2;             // bytes of one activation operand (K up to 256)
constexpr int TC_WB = 128 * NH * 2;              // weight buffer: W1 (256 x 64), half of W2, W3 padded
// dynamic shared memory: weight buffer, activation operands (hi, lo), biases; 224 KB are requested,
// so the block has the SM to itself and the operand reads of any descriptor stay in the allocation
constexpr int TC_SMEM_USED = TC_WB + 2 * TC_OP + (2 * NH + NO_PAD) * 4;
constexpr int TC_SMEM = 224 * 1024;
static_assert(TC_SMEM_USED <= TC_SMEM, "forward operands exceed the shared memory");
constexpr uint32_t TC_COLS = 256;                // tensor-memory columns held by a CTA

// Rows [n0, n0 + R) of a row-major BF16 weight matrix with Kd columns into the K-major layout with
// R rows (rows at or past n_end zero-filled), as 16-byte asynchronous copies: consecutive threads
// take 8 rows of one 16-byte column group, so a warp reads 64 contiguous bytes of each of 8 rows
// and writes 512 contiguous bytes.  Completed by tc_copies_done.
__device__ __forceinline__ void tc_load_w(unsigned char *dst, const __nv_bfloat16 *Wm, int n0, int R, int Kd,
                                          int n_end) {
  const int KG = Kd / 8;
  for (int i = threadIdx.x; i < R * KG; i += blockDim.x) {
    const int n = ((i >> 3) / KG) * 8 + (i & 7), kg = (i >> 3) % KG;
    const bool in = n0 + n < n_end;
    const __nv_bfloat16 *src = Wm + (in ? (size_t)(n0 + n) * Kd + 8 * kg : 0);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                     tc::smem_u32(dst + tc::kmajor_off((uint32_t)n, 8u * kg, (uint32_t)R))),
                 "l"(src), "r"(in ? 16 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void tc_copies_done() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Row r, columns [c, c + 16) of both activation operands from 16 FP32 values.
__device__ __forceinline__ void tc_store16(unsigned char *Ahi, unsigned char *Alo, int r, int c, const float (&a)[16]) {
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    __nv_bfloat162 hi[4], lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float x0 = a[8 * g + 2 * e], x1 = a[8 * g + 2 * e + 1];
      const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
      hi[e] = __halves2bfloat162(h0, h1);
      lo[e] = __halves2bfloat162(__float2bfloat16_rn(x0 - __bfloat162float(h0)),
                                 __float2bfloat16_rn(x1 - __bfloat162float(h1)));
    }
    const uint32_t off = tc::kmajor_off((uint32_t)r, (uint32_t)(c + 8 * g), TC_P);
    *reinterpret_cast<uint4 *>(Ahi + off) = *reinterpret_cast<const uint4 *>(hi);
    *reinterpret_cast<uint4 *>(Alo + off) = *reinterpret_cast<const uint4 *>(lo);
  }
}

// D (+)= A W^T for the 128 x Kd operands (hi, lo) and the N weight rows staged with R = N rows;
// issued by one thread, K steps of 16, the first product overwriting D.
__device__ __forceinline__ void tc_layer(uint32_t d, uint32_t ahi, uint32_t alo, uint32_t wb, int Kd, int N) {
  const uint32_t idesc = tc::idesc_bf16_f32(TC_P, N);
  const uint32_t lbo_a = TC_P * 16, lbo_w = (uint32_t)N * 16;
  for (int s = 0; s < Kd / 16; ++s) {
    const uint64_t bd = tc::desc_kmajor(wb + 2u * s * lbo_w, lbo_w, 128);
    tc::mma_bf16(d, tc::desc_kmajor(ahi + 2u * s * lbo_a, lbo_a, 128), bd, idesc, s > 0 ? 1u : 0u);
    tc::mma_bf16(d, tc::desc_kmajor(alo + 2u * s * lbo_a, lbo_a, 128), bd, idesc, 1u);
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1) mdn_forward_tc_kernel(const __nv_bfloat16 *__restrict__ W,
                                                                      const float *__restrict__ S, int P,
                                                                      float *__restrict__ head,
                                                                      float *__restrict__ cache,
                                                                      uint32_t *__restrict__ status) {
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char *Wb = sm, *Ahi = sm + TC_WB, *Alo = sm + TC_WB + TC_OP;
  float *bias = reinterpret_cast<float *>(sm + TC_WB + 2 * TC_OP);   // b1 [NH], b2 [NH], b3 [NO_PAD]
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, wq = t >> 5;
  const int row = 32 * (wq & 3) + (t & 31), cg = wq >> 2;   // the thread's row and column group
  const int p = blockIdx.x * TC_P + row;
  const bool valid = p < P;
  if (wq == 0) {
    tc::tmem_alloc(&tslot, TC_COLS);
    tc::tmem_relinquish();
  }
  if (t == 0) tc::mbar_init(&bar, 1);
  tc_load_w(Wb, W + OFF_W1, 0, NH, NI, NH);
  for (int i = t; i < NH; i += TC_THREADS) {
    bias[i] = bf(W, OFF_B1 + i);
    bias[NH + i] = bf(W, OFF_B2 + i);
  }
  if (t < NO_PAD) bias[2 * NH + t] = t < NO ? bf(W, OFF_B3 + t) : 0.f;
  {
    float a[16];   // the row's summary features [16 cg, 16 cg + 16)
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = valid ? S[(size_t)p * NI + 16 * cg + j] : 0.f;
    tc_store16(Ahi, Alo, row, 16 * cg, a);
  }
  tc_copies_done();
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = tslot, trow = tm + ((uint32_t)(32 * (wq & 3)) << 16);
  const uint32_t ahi = tc::smem_u32(Ahi), alo = tc::smem_u32(Alo), wb = tc::smem_u32(Wb);
  uint32_t phase = 0;
  // every thread waits for the products in flight; all agree on the outcome
  auto wait_products = [&]() {
    const bool ok = __syncthreads_and(tc::mbar_wait(&bar, phase) ? 1 : 0) != 0;
    if (ok) phase ^= 1u;
    tc::fence_after_sync();
    return ok;
  };
  // staged weights and operands written by the threads visible to the tensor core, earlier
  // tensor-memory loads done
  auto operands_ready = [&]() {
    tc_copies_done();
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  // the row's hidden-layer columns [64 cg, 64 cg + 64): a = D + b (cached), next operand GELU(a)
  auto hidden = [&](const float *b, int cache_off) {
#pragma unroll 1
    for (int c = 64 * cg; c < 64 * cg + 64; c += 16) {
      float a[16];
      tc::ld_row16(trow + (uint32_t)c, a);
#pragma unroll
      for (int j = 0; j < 16; ++j) a[j] += b[c + j];
      if (cache && valid) {
        float4 *o = reinterpret_cast<float4 *>(cache + (size_t)p * 2 * NH + cache_off + c);
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = make_float4(a[4 * j], a[4 * j + 1], a[4 * j + 2], a[4 * j + 3]);
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) a[j] = gelu(a[j]);
      tc_store16(Ahi, Alo, row, c, a);
    }
  };
  bool ok = true;
  do {
    // layer 1: a1 = W1 s + b1, h1 = GELU(a1); the first half of W2 is staged meanwhile
    if (t == 0) { tc_layer(tm, ahi, alo, wb, NI, NH); tc::commit(&bar); }
    if (!(ok = wait_products())) break;
    tc_load_w(Wb, W + OFF_W2, 0, NH / 2, NH, NH);
    hidden(bias, 0);
    operands_ready();
    // layer 2, one half of the neurons at a time: a2 = W2 h1 + b2, h2 = GELU(a2)
    if (t == 0) { tc_layer(tm, ahi, alo, wb, NH, NH / 2); tc::commit(&bar); }
    if (!(ok = wait_products())) break;
    tc_load_w(Wb, W + OFF_W2, NH / 2, NH / 2, NH, NH);
    operands_ready();
    if (t == 0) { tc_layer(tm + NH / 2, ahi, alo, wb, NH, NH / 2); tc::commit(&bar); }
    if (!(ok = wait_products())) break;
    tc_load_w(Wb, W + OFF_W3, 0, NO_PAD, NH, NO);
    hidden(bias + NH, NH);
    operands_ready();
    // head = W3 h2 + b3 (columns 16 j for j = cg, cg + 4)
    if (t == 0) { tc_layer(tm, ahi, alo, wb, NH, NO_PAD); tc::commit(&bar); }
    if (!(ok = wait_products())) break;
    for (int c = 16 * cg; c < NO_PAD; c += 64) {
      float a[16];
      tc::ld_row16(trow + (uint32_t)c, a);
      if (valid)
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c + j < NO) head[(size_t)p * NO + c + j] = a[j] + bias[2 * NH + c + j];
    }
  } while (false);
  if (!ok) {
    // an expired wait: flag it, wait (bounded) once more for the products in flight, then free
    // the tensor memory
    if (t == 0) atomicOr(status, RIFT_FLAG_TIMEOUT_BIT);
    tc::mbar_wait(&bar, phase);
  }
  tc_copies_done();
  tc::fence_before_sync();
  __syncthreads();
  if (wq == 0) tc::tmem_dealloc(tm, TC_COLS);
}

// head[p] = MLP(S[p]) for P points on the tensor cores, cache[p] = (a1, a2) when given; an expired
// wait sets RIFT_FLAG_TIMEOUT_BIT in *status.
cudaError_t launch_forward(const __nv_bfloat16 *W, const float *S, int P, float *head, float *cache,
                           uint32_t *status, cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(mdn_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (e != cudaSuccess) return e;
  mdn_forward_tc_kernel<<<(P + TC_P - 1) / TC_P, TC_THREADS, TC_SMEM, st>>>(W, S, P, head, cache, status);
  return cudaGetLastError();
}

// Weighted NLL of each point's H samples: loss[p] and dL/dhead[p] (scaled by `scale`).
// theta: [P][H][5] (ra, sin dec, t, cos incl, ln D); w: [P][H]; box: [P][2][5] (a, b).
__global__ void __launch_bounds__(128) mdn_loss_kernel(const float *__restrict__ head, const float *__restrict__ th,
                                                       const float *__restrict__ w, const float *__restrict__ box,
                                                       int H, float scale, float *__restrict__ gout,
                                                       float *__restrict__ loss) {
  const int p = blockIdx.x;
  __shared__ float hd[NO], lpi[NC], isg[NC * ND], lsc[NC * ND];
  __shared__ float red[NO + 1][4];
  const int t = threadIdx.x;
  if (t < NO) hd[t] = head[(size_t)p * NO + t];
  __syncthreads();
  if (t == 0) {
    float mx = -INFINITY;
    for (int j = 0; j < NC; ++j) mx = fmaxf(mx, hd[j]);
    float se = 0.f;
    for (int j = 0; j < NC; ++j) se += expf(hd[j] - mx);
    for (int j = 0; j < NC; ++j) lpi[j] = hd[j] - mx - logf(se);
  }
  if (t < NC * ND) {
    const float l = fminf(fmaxf(hd[NC + NC * ND + t], LS_MIN), LS_MAX);
    lsc[t] = l;
    isg[t] = expf(-l);
  }
  __syncthreads();
  float acc[NO + 1];
#pragma unroll
  for (int q = 0; q <= NO; ++q) acc[q] = 0.f;
  const float *a = box + (size_t)p * 10, *b = a + 5;
  for (int j = t; j < H; j += blockDim.x) {
    float wj = w[(size_t)p * H + j];
    float z[ND], jac = 0.f;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const float v = th[((size_t)p * H + j) * ND + d];
      if (!isfinite(v)) wj = 0.f;   // an empty harvest slot carries no weight
      // samples on the edge of the box (float rounding) are kept just inside it
      const float x = fminf(fmaxf((isfinite(v) ? v - a[d] : 0.f) / (b[d] - a[d]), 1e-6f), 1.f - 1e-6f);
      z[d] = logf(x) - log1pf(-x);
      jac += logf(b[d] - a[d]) + logf(x) + log1pf(-x);
    }
    float comp[NC], mx = -INFINITY;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float s = lpi[c];
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        const float u = (z[d] - hd[NC + c * ND + d]) * isg[c * ND + d];
        s -= 0.5f * u * u + lsc[c * ND + d] + 0.91893853320467274f;
      }
      comp[c] = s;
      mx = fmaxf(mx, s);
    }
    float se = 0.f;
#pragma unroll
    for (int c = 0; c < NC; ++c) se += expf(comp[c] - mx);
    const float lq = mx + logf(se);
    acc[NO] -= wj * (lq - jac);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float r = expf(comp[c] - lq) * wj;
      acc[c] -= r;
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        const float u = (z[d] - hd[NC + c * ND + d]) * isg[c * ND + d];
        acc[NC + c * ND + d] -= r * u * isg[c * ND + d];
        acc[NC + NC * ND + c * ND + d] -= r * (u * u - 1.f);
      }
    }
    // + w pi_c (the softmax normalisation)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] += wj * expf(lpi[c]);
  }
  // block reduction (warp shuffles, then the four warps in a fixed order)
  const int lane = t & 31, wid = t >> 5;
#pragma unroll
  for (int q = 0; q <= NO; ++q) {
    float v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[q][wid] = v;
  }
  __syncthreads();
  for (int q = t; q <= NO; q += blockDim.x) {
    const float v = red[q][0] + red[q][1] + red[q][2] + red[q][3];
    if (q < NO) {
      float g = v * scale;
      if (q >= NC + NC * ND) {
        const float raw = hd[q];
        if (!(raw > LS_MIN && raw < LS_MAX)) g = 0.f;
      }
      gout[(size_t)p * NO + q] = g;
    } else {
      loss[p] = v;
    }
  }
}

// Backpropagation of dL/dhead through the MLP to the pre-activation gradients of both hidden layers
// of point p: ga[p][0..NH) = dL/da1, ga[p][NH..2NH) = dL/da2 (the weight gradients are the sums over
// points of their outer products, formed by mdn_wgrad_kernel in a fixed order).
__global__ void __launch_bounds__(256) mdn_backward_kernel(const __nv_bfloat16 *__restrict__ W,
                                                           const float *__restrict__ cache,
                                                           const float *__restrict__ gout, int P,
                                                           float *__restrict__ ga) {
  const int p = blockIdx.x;
  if (p >= P) return;
  __shared__ float ga2[NH], go[NO];
  const int t = threadIdx.x;
  if (t < NO) go[t] = gout[(size_t)p * NO + t];
  const float a1 = cache[(size_t)p * 2 * NH + t], a2 = cache[(size_t)p * 2 * NH + NH + t];
  __syncthreads();
  float gh2 = 0.f;
  for (int o = 0; o < NO; ++o) gh2 = fmaf(go[o], bf(W, OFF_W3 + o * NH + t), gh2);
  ga2[t] = gh2 * gelu_grad(a2);
  __syncthreads();
  float gh1 = 0.f;
  for (int j = 0; j < NH; ++j) gh1 = fmaf(ga2[j], bf(W, OFF_W2 + j * NH + t), gh1);
  ga[(size_t)p * 2 * NH + t] = gh1 * gelu_grad(a1);
  ga[(size_t)p * 2 * NH + NH + t] = ga2[t];
}

// Weight gradients as sums over the P points, each parameter by one thread in point order (the
// same bits on every run): W3[o][t] += go[p][o] h2[p][t], b3[o] += go[p][o], W2[j][t] += ga2[p][j]
// h1[p][t], b2[j] += ga2[p][j], W1[j][i] += ga1[p][j] s[p][i], b1[j] += ga1[p][j], with h = GELU(a)
// recomputed from the cached pre-activations.
__global__ void __launch_bounds__(256) mdn_wgrad_kernel(const float *__restrict__ S, const float *__restrict__ cache,
                                                        const float *__restrict__ gout,
                                                        const float *__restrict__ ga, int P,
                                                        float *__restrict__ grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NPARAM) return;
  float acc = 0.f;
  if (e >= OFF_B3) {
    const int o = e - OFF_B3;
    for (int p = 0; p < P; ++p) acc += gout[(size_t)p * NO + o];
  } else if (e >= OFF_W3) {
    const int o = (e - OFF_W3) / NH, t = (e - OFF_W3) % NH;
    for (int p = 0; p < P; ++p) acc = fmaf(gout[(size_t)p * NO + o], gelu(cache[(size_t)p * 2 * NH + NH + t]), acc);
  } else if (e >= OFF_B2) {
    const int j = e - OFF_B2;
    for (int p = 0; p < P; ++p) acc += ga[(size_t)p * 2 * NH + NH + j];
  } else if (e >= OFF_W2) {
    const int j = (e - OFF_W2) / NH, t = (e - OFF_W2) % NH;
    for (int p = 0; p < P; ++p) acc = fmaf(ga[(size_t)p * 2 * NH + NH + j], gelu(cache[(size_t)p * 2 * NH + t]), acc);
  } else if (e >= OFF_B1) {
    const int j = e - OFF_B1;
    for (int p = 0; p < P; ++p) acc += ga[(size_t)p * 2 * NH + j];
  } else {
    const int j = (e - OFF_W1) / NI, i = (e - OFF_W1) % NI;
    for (int p = 0; p < P; ++p) acc = fmaf(ga[(size_t)p * 2 * NH + j], S[(size_t)p * NI + i], acc);
  }
  grad[e] += acc;
}

// Adam (Kingma & Ba 2015) on the float32 master copy, bfloat16 weights refreshed, gradient cleared.
__global__ void mdn_adam_kernel(float *master, __nv_bfloat16 *w, float *grad, float *m, float *v, int n, float lr,
                                float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = grad[i];
  const float mm = 0.9f * m[i] + 0.1f * g;
  const float vv = 0.999f * v[i] + 0.001f * g * g;
  m[i] = mm;
  v[i] = vv;
  const float x = master[i] - lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
  master[i] = x;
  w[i] = __float2bfloat16_rn(x);
  grad[i] = 0.f;
}

__global__ void mdn_round_kernel(const float *master, __nv_bfloat16 *w, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = __float2bfloat16_rn(master[i]);
}

// Per-point learned proposal for the sampler (layout RIFT_GMM_FLOATS) from the head; the
// mixture weights are normalised in FP64 and rounded to float32 before their float32
// cumulative sum, so the component choice can be reproduced exactly.  cst: [P][4] =
// (sum ln(b - a), constant of ln p5, ln D_lo, ln D_hi - ln D_lo).
__global__ void mdn_gmm_kernel(const float *__restrict__ head, const float *__restrict__ cst, int P,
                               float *__restrict__ gmm) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float *h = head + (size_t)p * NO;
  float *G = gmm + (size_t)p * RIFT_GMM_FLOATS;
  double mx = -INFINITY;
  for (int j = 0; j < NC; ++j) mx = fmax(mx, (double)h[j]);
  double e[NC], se = 0.0;
  for (int j = 0; j < NC; ++j) { e[j] = exp((double)h[j] - mx); se += e[j]; }
  float cw = 0.f;
  for (int j = 0; j < NC; ++j) {
    const double pi = e[j] / se;
    G[j] = (float)log(pi);
    cw = __fadd_rn(cw, (float)pi);
    G[8 + j] = cw;
  }
  for (int q = 0; q < NC * ND; ++q) {
    const float l = fminf(fmaxf(h[NC + NC * ND + q], LS_MIN), LS_MAX);
    G[16 + q] = h[NC + q];
    G[56 + q] = l;
    G[96 + q] = expf(-l);
  }
  for (int q = 0; q < 4; ++q) G[136 + q] = cst[(size_t)p * 4 + q];
  for (int q = 140; q < RIFT_GMM_FLOATS; ++q) G[q] = 0.f;
}

// Summary of each point (64 features, layout as in the header).  One CTA per point.
__global__ void __launch_bounds__(256) summary_kernel(const PointC *__restrict__ pts, const float2 *__restrict__ qa,
                                                      const float4 *__restrict__ ca, const double *__restrict__ tau0,
                                                      float *__restrict__ out) {
  __shared__ __align__(16) PointC P;
  __shared__ float red[8][8];
  __shared__ float feats[NI];
  __shared__ float tm22[RIFT_MAXK];
  const int p = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
  {
    const int *src = reinterpret_cast<const int *>(pts + p);
    int *dst = reinterpret_cast<int *>(&P);
    for (int i = t; i < (int)(sizeof(PointC) / 4); i += blockDim.x) dst[i] = src[i];
  }
  if (t < NI) feats[t] = 0.f;
  __syncthreads();
  const int K = P.K, T = P.T;
  const float2 *Q = qa + P.q_off;
  int nf = 0;
  for (int k = 0; k < K; ++k) {
    const float t0 = (float)tau0[(size_t)p * RIFT_MAXK + k];
    for (int mi = 0; mi < 2; ++mi) {
      const int want_m = mi == 0 ? 2 : -2;
      int a = -1;
      for (int q = 0; q < P.M; ++q)
        if (P.mode[q].l == 2 && P.mode[q].m == want_m) a = q;
      if (a < 0) {
        if (mi == 0 && t == 0) tm22[k] = 0.f;
        nf += 5;
        continue;
      }
      // pass 1: max |Q|^2
      float mx = 0.f;
      for (int j = t; j < T; j += blockDim.x) {
        const float2 q = Q[((size_t)k * T + j) * P.Mp + a];
        mx = fmaxf(mx, __fadd_rn(__fmul_rn(q.x, q.x), __fmul_rn(q.y, q.y)));
      }
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) red[0][wid] = mx;
      __syncthreads();
      mx = red[0][0];
      for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[0][w]);
      __syncthreads();
      // pass 2: weights (|Q|^2 / max)^4: normalisation, mean time, weighted Q
      float sw = 0.f, st = 0.f, sr = 0.f, si = 0.f;
      for (int j = t; j < T; j += blockDim.x) {
        const float2 q = Q[((size_t)k * T + j) * P.Mp + a];
        const float r = __fadd_rn(__fmul_rn(q.x, q.x), __fmul_rn(q.y, q.y)) / mx;
        const float r2 = r * r, w = r2 * r2;
        sw += w; st += w * ((float)j / P.fs); sr += w * q.x; si += w * q.y;
      }
      float v[4] = {sw, st, sr, si};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0) red[1 + q][wid] = v[q];
      }
      __syncthreads();
      float S[4];
      for (int q = 0; q < 4; ++q) {
        S[q] = 0.f;
        for (int w = 0; w < 8; ++w) S[q] += red[1 + q][w];
      }
      const float tmr = S[1] / S[0];   // mean time relative to the first sample
      __syncthreads();
      // pass 3: spread about the mean
      float sv = 0.f;
      for (int j = t; j < T; j += blockDim.x) {
        const float2 q = Q[((size_t)k * T + j) * P.Mp + a];
        const float r = __fadd_rn(__fmul_rn(q.x, q.x), __fmul_rn(q.y, q.y)) / mx;
        const float r2 = r * r, w = r2 * r2;
        const float d = (float)j / P.fs - tmr;
        sv += w * d * d;
      }
      for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
      if (lane == 0) red[5][wid] = sv;
      __syncthreads();
      if (t == 0) {
        float V = 0.f;
        for (int w = 0; w < 8; ++w) V += red[5][w];
        const float tm = t0 + tmr;
        const float ph = atan2f(S[3], S[2]);
        feats[nf + 0] = tm;
        feats[nf + 1] = sqrtf(V / S[0]);
        feats[nf + 2] = (logf(mx) * 4.f + logf(S[0] / (float)T)) / 8.f;
        feats[nf + 3] = cosf(ph);
        feats[nf + 4] = sinf(ph);
        if (mi == 0) tm22[k] = tm;
      }
      __syncthreads();
      nf += 5;
    }
  }
  if (t == 0) {
    // log sqrt(U_aa) of (2,2), (2,-2) per detector, from the diagonal pair coefficients
    const int M = P.M;
    for (int k = 0; k < K; ++k)
      for (int mi = 0; mi < 2; ++mi) {
        const int want_m = mi == 0 ? 2 : -2;
        int a = -1;
        for (int q = 0; q < M; ++q)
          if (P.mode[q].l == 2 && P.mode[q].m == want_m) a = q;
        float f = 0.f;
        if (a >= 0) {
          const int pair = pair_slot(a, a, M);
          f = 0.5f * logf(ca[P.uv_off + (size_t)pair * K + k].x);
        }
        if (nf < NI) feats[nf] = f;
        ++nf;
      }
    for (int i = 0; i < K; ++i)
      for (int j = i + 1; j < K; ++j) {
        if (nf < NI) feats[nf] = tm22[i] - tm22[j];
        ++nf;
      }
  }
  __syncthreads();
  if (t < NI) out[(size_t)p * NI + t] = feats[t];
}

}  // namespace

struct rift_mdn {
  float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  __nv_bfloat16 *w = nullptr;
  int step = 0;
  std::string err;
  // training scratch
  float *head = nullptr, *cache = nullptr, *gout = nullptr, *loss = nullptr, *ga = nullptr;
  int cap = 0;
  uint32_t *status = nullptr;   // device word: RIFT_FLAG_TIMEOUT_BIT after an expired wait of the forward pass
};

namespace {

rift_status mfail(rift_mdn *m, rift_status s, const std::string &msg) {
  if (m) m->err = msg;
  return s;
}

#define MCK(m, call)                                                                        \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return mfail(m, RIFT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

thread_local double g_forward_ms = 0.0;   // device time of the last rift_mdn_forward kernel (this thread)

// Reads and clears the forward pass's status word (after the call's work has finished).
rift_status check_status(rift_mdn *m) {
  uint32_t f = 0;
  MCK(m, cudaMemcpy(&f, m->status, sizeof f, cudaMemcpyDeviceToHost));
  if (!f) return RIFT_OK;
  MCK(m, cudaMemset(m->status, 0, sizeof f));
  return mfail(m, RIFT_ETIMEOUT, "a bounded wait of the tensor-core forward pass expired");
}

rift_status mdn_scratch(rift_mdn *m, int P) {
  if (P <= m->cap) return RIFT_OK;
  cudaFree(m->head); cudaFree(m->cache); cudaFree(m->gout); cudaFree(m->loss); cudaFree(m->ga);
  m->head = m->cache = m->gout = m->loss = m->ga = nullptr;
  m->cap = 0;
  MCK(m, cudaMalloc(&m->head, sizeof(float) * (size_t)P * NO));
  MCK(m, cudaMalloc(&m->cache, sizeof(float) * (size_t)P * 2 * NH));
  MCK(m, cudaMalloc(&m->ga, sizeof(float) * (size_t)P * 2 * NH));
  MCK(m, cudaMalloc(&m->gout, sizeof(float) * (size_t)P * NO));
  MCK(m, cudaMalloc(&m->loss, sizeof(float) * (size_t)P));
  m->cap = P;
  return RIFT_OK;
}

// Philox-based initialisation: uniform(-1, 1) * sqrt(3 / fan_in) (variance 1 / fan_in), biases 0.
void init_params(uint64_t seed, std::vector<float> &out) {
  out.assign(NPARAM, 0.f);
  auto fill = [&](int off, int rows, int cols, uint32_t tag) {
    const double sc = std::sqrt(3.0 / cols);
    for (int i = 0; i < rows * cols; ++i) {
      // Philox4x32-10 of (i, tag, 0, 0) with the seed as key; first word
      uint32_t c0 = (uint32_t)i, c1 = tag, c2 = 0, c3 = 0;
      uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
      for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n1 = (uint32_t)p1, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1,
                       n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
      }
      const double u = ((c0 >> 9) + 0.5) / 8388608.0;
      out[off + i] = (float)((2.0 * u - 1.0) * sc);
    }
  };
  fill(OFF_W1, NH, NI, 1);
  fill(OFF_W2, NH, NH, 2);
  fill(OFF_W3, NO, NH, 3);
}

}  // namespace

extern "C" {

rift_status rift_mdn_create(uint64_t seed, rift_mdn **out) {
  if (!out) return RIFT_EINVAL;
  *out = nullptr;
  rift_mdn *m = new (std::nothrow) rift_mdn();
  if (!m) return RIFT_ENOMEM;
  std::vector<float> init;
  init_params(seed, init);
  cudaError_t e;
  if ((e = cudaMalloc(&m->master, sizeof(float) * NPARAM)) != cudaSuccess ||
      (e = cudaMalloc(&m->m, sizeof(float) * NPARAM)) != cudaSuccess ||
      (e = cudaMalloc(&m->v, sizeof(float) * NPARAM)) != cudaSuccess ||
      (e = cudaMalloc(&m->grad, sizeof(float) * NPARAM)) != cudaSuccess ||
      (e = cudaMalloc(&m->w, sizeof(__nv_bfloat16) * NPARAM)) != cudaSuccess ||
      (e = cudaMalloc(&m->status, sizeof(uint32_t))) != cudaSuccess ||
      (e = cudaMemset(m->status, 0, sizeof(uint32_t))) != cudaSuccess ||
      (e = cudaMemcpy(m->master, init.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(m->m, 0, sizeof(float) * NPARAM)) != cudaSuccess ||
      (e = cudaMemset(m->v, 0, sizeof(float) * NPARAM)) != cudaSuccess ||
      (e = cudaMemset(m->grad, 0, sizeof(float) * NPARAM)) != cudaSuccess) {
    rift_mdn_destroy(m);
    return e == cudaErrorMemoryAllocation ? RIFT_ENOMEM : RIFT_ECUDA;
  }
  mdn_round_kernel<<<(NPARAM + 255) / 256, 256>>>(m->master, m->w, NPARAM);
  if (cudaDeviceSynchronize() != cudaSuccess) { rift_mdn_destroy(m); return RIFT_ECUDA; }
  *out = m;
  return RIFT_OK;
}

void rift_mdn_destroy(rift_mdn *m) {
  if (!m) return;
  cudaFree(m->master); cudaFree(m->m); cudaFree(m->v); cudaFree(m->grad); cudaFree(m->w);
  cudaFree(m->head); cudaFree(m->cache); cudaFree(m->gout); cudaFree(m->loss); cudaFree(m->ga);
  cudaFree(m->status);
  delete m;
}

const char *rift_mdn_last_error(const rift_mdn *m) { return m ? m->err.c_str() : "null handle"; }

rift_status rift_mdn_set_params(rift_mdn *m, const float *host) {
  if (!m || !host) return RIFT_EINVAL;
  MCK(m, cudaMemcpy(m->master, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
  MCK(m, cudaMemset(m->m, 0, sizeof(float) * NPARAM));
  MCK(m, cudaMemset(m->v, 0, sizeof(float) * NPARAM));
  MCK(m, cudaMemset(m->grad, 0, sizeof(float) * NPARAM));
  m->step = 0;
  mdn_round_kernel<<<(NPARAM + 255) / 256, 256>>>(m->master, m->w, NPARAM);
  MCK(m, cudaDeviceSynchronize());
  return RIFT_OK;
}

rift_status rift_mdn_get_params(rift_mdn *m, float *host, int which) {
  if (!m || !host) return RIFT_EINVAL;
  if (which == 0) {
    MCK(m, cudaMemcpy(host, m->master, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
  } else {
    std::vector<__nv_bfloat16> b(NPARAM);
    MCK(m, cudaMemcpy(b.data(), m->w, sizeof(__nv_bfloat16) * NPARAM, cudaMemcpyDeviceToHost));
    for (int i = 0; i < NPARAM; ++i) host[i] = __bfloat162float(b[i]);
  }
  return RIFT_OK;
}

rift_status rift_mdn_forward(rift_mdn *m, int n, const float *summ_dev, float *head_dev) {
  if (!m || n < 0 || (n && (!summ_dev || !head_dev))) return RIFT_EINVAL;
  if (n == 0) return RIFT_OK;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  MCK(m, cudaEventCreate(&ev[0]));
  if (cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return mfail(m, RIFT_ECUDA, "cudaEventCreate");
  }
  cudaError_t e = cudaEventRecord(ev[0], 0);
  if (e == cudaSuccess) e = launch_forward(m->w, summ_dev, n, head_dev, nullptr, m->status, 0);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess && cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) g_forward_ms = ms;
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  MCK(m, e);
  return check_status(m);
}

double rift_mdn_forward_ms(void) { return g_forward_ms; }

rift_status rift_mdn_loss_grad(rift_mdn *m, int n, const float *summ_dev, const float *theta_dev, const float *w_dev,
                               int H, const float *box_dev, double *loss_out, float *grad_host) {
  if (!m || n < 1 || H < 1 || !summ_dev || !theta_dev || !w_dev || !box_dev) return RIFT_EINVAL;
  rift_status s = mdn_scratch(m, n);
  if (s != RIFT_OK) return s;
  MCK(m, cudaMemset(m->grad, 0, sizeof(float) * NPARAM));
  MCK(m, launch_forward(m->w, summ_dev, n, m->head, m->cache, m->status, 0));
  mdn_loss_kernel<<<n, 128>>>(m->head, theta_dev, w_dev, box_dev, H, 1.f / n, m->gout, m->loss);
  mdn_backward_kernel<<<n, 256>>>(m->w, m->cache, m->gout, n, m->ga);
  mdn_wgrad_kernel<<<(NPARAM + 255) / 256, 256>>>(summ_dev, m->cache, m->gout, m->ga, n, m->grad);
  MCK(m, cudaGetLastError());
  std::vector<float> l(n);
  MCK(m, cudaMemcpy(l.data(), m->loss, sizeof(float) * n, cudaMemcpyDeviceToHost));
  double tot = 0.0;
  for (float x : l) tot += x;
  if (loss_out) *loss_out = tot / n;
  if (grad_host) MCK(m, cudaMemcpy(grad_host, m->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
  MCK(m, cudaMemset(m->grad, 0, sizeof(float) * NPARAM));
  return check_status(m);
}

rift_status rift_mdn_train(rift_mdn *m, int n, const float *summ_dev, const float *theta_dev, const float *w_dev,
                           int H, const float *box_dev, int steps, int batch, double lr, double *loss_per_step) {
  if (!m || n < 1 || H < 1 || steps < 0 || !summ_dev || !theta_dev || !w_dev || !box_dev || !(lr > 0))
    return RIFT_EINVAL;
  if (batch < 1 || batch > n) batch = n;
  rift_status s = mdn_scratch(m, batch);
  if (s != RIFT_OK) return s;
  for (int it = 0; it < steps; ++it) {
    const int p0 = (int)(((long long)it * batch) % n);
    const int nb = std::min(batch, n - p0);
    const float *S = summ_dev + (size_t)p0 * NI;
    const float *th = theta_dev + (size_t)p0 * H * ND;
    const float *w = w_dev + (size_t)p0 * H;
    const float *bx = box_dev + (size_t)p0 * 10;
    MCK(m, launch_forward(m->w, S, nb, m->head, m->cache, m->status, 0));
    mdn_loss_kernel<<<nb, 128>>>(m->head, th, w, bx, H, 1.f / nb, m->gout, m->loss);
    mdn_backward_kernel<<<nb, 256>>>(m->w, m->cache, m->gout, nb, m->ga);
    mdn_wgrad_kernel<<<(NPARAM + 255) / 256, 256>>>(S, m->cache, m->gout, m->ga, nb, m->grad);
    m->step += 1;
    const float bc1 = 1.f - std::pow(0.9f, (float)m->step), bc2 = 1.f - std::pow(0.999f, (float)m->step);
    mdn_adam_kernel<<<(NPARAM + 255) / 256, 256>>>(m->master, m->w, m->grad, m->m, m->v, NPARAM, (float)lr, bc1, bc2);
    MCK(m, cudaGetLastError());
    if (loss_per_step) {
      std::vector<float> l(nb);
      MCK(m, cudaMemcpy(l.data(), m->loss, sizeof(float) * nb, cudaMemcpyDeviceToHost));
      double tot = 0.0;
      for (float x : l) tot += x;
      loss_per_step[it] = tot / nb;
    }
  }
  MCK(m, cudaDeviceSynchronize());
  return check_status(m);
}

}  // extern "C"

// ---------------------------------------------------------------- used by capi.cu
cudaError_t launch_summary(const PointC *pts, const float2 *qa, const float4 *ca, const double *tau0, int np,
                           float *out, cudaStream_t st) {
  summary_kernel<<<np, 256, 0, st>>>(pts, qa, ca, tau0, out);
  return cudaGetLastError();
}

cudaError_t launch_mdn_gmm(const rift_mdn *m, const float *summ, const float *cst, int np, float *head_scratch,
                           float *gmm, uint32_t *flags, cudaStream_t st) {
  const cudaError_t e = launch_forward(m->w, summ, np, head_scratch, nullptr, flags, st);
  if (e != cudaSuccess) return e;
  mdn_gmm_kernel<<<(np + 127) / 128, 128, 0, st>>>(head_scratch, cst, np, gmm);
  return cudaGetLastError();
}

cudaError_t launch_gmm_from_head(const float *head, const float *cst, int np, float *gmm, cudaStream_t st) {
  mdn_gmm_kernel<<<(np + 127) / 128, 128, 0, st>>>(head, cst, np, gmm);
  return cudaGetLastError();
}

