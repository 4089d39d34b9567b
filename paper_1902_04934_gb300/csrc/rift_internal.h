// Host-side view of the kernels (launch wrappers) shared by the C-ABI translation unit.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

struct PointC;

// Threads per block of the fused likelihood kernel.
#define RIFT_MC_BLOCK 256

// Block partial of the log-sum-exp: max, sum e^{l-max}, sum e^{2(l-max)}, count.
struct __align__(32) Part {
  double m, s1, s2, n;
};

// Running log-sum-exp state of one point (FP64, Neumaier-compensated sums).
struct AccState {
  double m;       // max log weight so far
  double s1, c1;  // sum e^{l-m} and its compensation
  double s2, c2;  // sum e^{2(l-m)} and its compensation
  double round_max; // max log weight of the last round (adaptive histograms)
  unsigned long long n;
  unsigned long long pad;
};

// Per-launch Monte Carlo parameters.
struct McParams {
  unsigned long long seed;
  uint32_t round;
  uint32_t n;          // samples this round (per point)
  uint32_t point_id;   // counter word 3 (single point)
  int proposal;        // 0 prior, 1 tables
  int nb;              // bins per adapted coordinate
  int pad;
  float d_lo3, d_span3;
  const float *tables; // device [3][nb+1]
  const float *lnw;    // device [3][nb]: -ln(nb p_b)
  float *dbg_ell;      // optional [.. + n]
  long long dbg_off;
  float *ell_buf;      // adaptive scratch [n]
  uint32_t *bin_buf;   // adaptive scratch [n], bins packed 3 x 8 bits
  Part *partials;   // [grid] (m, s1, s2, n)
  uint32_t *flags;
};

struct DrawOut {
  float *theta;  // [7][n]
  float *lpq;    // [n]
  int *bins;     // [3][n] or null
};

size_t rift_point_smem_bytes(int K, int npair, int nb, int block, int M);

cudaError_t launch_mc_round(int K, const PointC *pt_dev, const PointC &pt_host, const float2 *q_arena,
                            const float4 *c_arena, const McParams &prm, int grid, int block, cudaStream_t st);
cudaError_t launch_merge(const Part *partials, int nparts, AccState *acc, cudaStream_t st);
cudaError_t launch_hist(const float *ell, const uint32_t *bins, uint32_t n, const AccState *acc, float beta,
                        int nb, unsigned long long *part, int grid, cudaStream_t st);
cudaError_t launch_tables(const unsigned long long *part, int nparts, int nb, double floor_eps, float *tables,
                          float *lnw, cudaStream_t st);
cudaError_t launch_lnl_array(int K, const PointC *pt_dev, const PointC &pt_host, const float2 *q_arena,
                             const float4 *c_arena, size_t n, const float *ra, const float *dec, const float *t,
                             const float *psi, const float *phi, const float *incl, const float *dist, float *out,
                             uint32_t *flags, cudaStream_t st);
cudaError_t launch_draw(int K, const PointC *pt_dev, const PointC &pt_host, const McParams &prm, DrawOut o,
                        cudaStream_t st);
int mc_round_blocks_per_sm(int K, size_t smem, int block);
