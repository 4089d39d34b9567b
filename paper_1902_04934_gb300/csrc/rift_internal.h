// Host-side view of the kernels (launch wrappers) shared by the C-ABI translation unit.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

struct PointC;

// Threads per block of the fused likelihood kernel.
#define RIFT_MC_BLOCK 256
// Threads per block of the cell kernel, and samples per work item at most.
#define RIFT_CELL_BLOCK 256
#define RIFT_CHUNK 2048
// Draws per work item in time-marginalised rounds: an item is a run of consecutive draws of a
// point (across cells), one per thread, so every item but a point's last is one full pass of a CTA
// (a draw costs about J samples; items of part-filled passes leave threads idle).
#define RIFT_TMARG_CHUNK RIFT_CELL_BLOCK
// Dynamic shared memory the cell kernels may take (their attribute).
#define RIFT_CELLS_MAX_DYN_SMEM (220 * 1024)

// Shared-memory layout of the time-quadrature GEMM of the cell kernel (time-marginalised rounds
// whose points all have merged rows) inside its window buffer of `budget` bytes: byte offsets,
// 16-byte aligned, of the per-draw arrays of an item (RIFT_CELL_BLOCK draws) and the rows `rmax`
// (a multiple of 8) of the row-sum block S ([rmax][33] floats) and of each of the two staged Q
// buffers ([rmax][maxmh] complex64).  The draws' harmonics share the S and Q space during setup.
#define RIFT_TG_SROW 33
struct TgLayout {
  unsigned G, W, R0, CX, XX, KEY, POS, LT, LN, GM, S, QS, end;
  int rmax;
};
inline __host__ __device__ unsigned tg_al16(unsigned x) { return (x + 15u) & ~15u; }
inline __host__ __device__ TgLayout tg_layout(int K, int NT, int maxmh, unsigned budget) {
  const unsigned B = RIFT_CELL_BLOCK;
  TgLayout t;
  unsigned o = 0;
  t.G = o;   o = tg_al16(o + 16u * (unsigned)K * (unsigned)(maxmh / 2) * B);   // float4 [K][maxmh/2][B]
  t.W = o;   o = tg_al16(o + 4u * (unsigned)(K * NT) * B);                    // float [K][NT][B]
  t.R0 = o;  o = tg_al16(o + 4u * (unsigned)K * B);                           // int [K][B]
  t.CX = o;  o = tg_al16(o + 4u * B);                                          // -x quad / 4
  t.XX = o;  o = tg_al16(o + 4u * B);                                          // x = D_ref / D
  t.KEY = o; o = tg_al16(o + 8u * B);                                          // (sort key, thread)
  t.POS = o; o = tg_al16(o + 4u * B);                                          // slot of each thread
  t.LT = o;  o = tg_al16(o + 8u * B);                                          // (max, sum) per thread
  t.LN = o;  o = tg_al16(o + 4u * B);                                          // lnL per slot
  t.GM = o;  o = tg_al16(o + 8u * (unsigned)K * (B / 32u));                     // group min, max of r0
  const unsigned row = 4u * RIFT_TG_SROW + 2u * 8u * (unsigned)maxmh;
  t.rmax = (budget > o) ? (int)(((budget - o) / row) & ~7u) : 0;
  t.S = o;   o = tg_al16(o + 4u * RIFT_TG_SROW * (unsigned)(t.rmax > 0 ? t.rmax : 0));
  t.QS = o;  o = tg_al16(o + 2u * 8u * (unsigned)maxmh * (unsigned)(t.rmax > 0 ? t.rmax : 0));
  t.end = o;
  return t;
}

// Block partial of the log-sum-exp: max, sum e^{l-max}, sum e^{2(l-max)}, count.
struct __align__(32) Part {
  double m, s1, s2, n;
};

// Refinement of heavy samples (rift_mc_opts.refine), per point: the corrections of the sums,
// sum over refined samples of e^{l64 - mref} - e^{l32 - mref} (and of the squares), relative to
// mref, the running maximum when they were last folded; the largest refined FP64 log weight and the
// FP32 value it replaced; the number of refined samples.
struct RefineState {
  double mref, d1, d2, l64max, l32max;
  unsigned long long n;
};
// Candidates kept per work item: the two largest log weights of each warp.
#define RIFT_CAND_PER_ITEM (2 * (RIFT_CELL_BLOCK / 32))

// Running log-sum-exp state of one point (FP64, Neumaier-compensated sums).
struct AccState {
  double m;       // max log weight so far
  double s1, c1;  // sum e^{l-m} and its compensation
  double s2, c2;  // sum e^{2(l-m)} and its compensation
  double round_max; // max log weight of the last round (adaptive histograms)
  unsigned long long n;
  unsigned long long pad;
  double round_neff;  // n_eff of the last round's draws alone: sum w / max w over the round
};

// One point's part of a Monte Carlo round (device array over points).
struct RoundPt {
  uint32_t n;              // samples this round (0: point inactive)
  uint32_t ncell;          // cells: S_ra S_sd S_t, 0 if inactive
  uint32_t base, rem;      // n = base * ncell + rem; cells [0, rem) hold base + 1 samples
  uint32_t item0;          // first work item of this point in the round
  uint32_t chunks;         // work items per cell (each at most RIFT_CHUNK samples); 0 if tmarg
  uint32_t nitem;          // work items of this point: ncell * chunks (tmarg: ceil(n / RIFT_TMARG_CHUNK))
  uint32_t round;          // Philox counter word 1
  uint32_t point_id;       // Philox counter word 3
  uint32_t ls0, ls1, ls2;  // log2 of the strata in effect
  int proposal;            // 0 prior, 1 tables
  int nb;                  // bins per adapted coordinate
  float lcorr0, lcorr1;    // ln(n / (C (base+1))), ln(n / (C base)): stratified-estimator weights
  long long ell_off;       // offset of the point's samples in the per-sample buffers (-1: none)
  long long dbg_off;       // offset in the caller's dbg_ell (-1: none)
  const float *tab;        // [3][nb+1] float32 CDF tables
  const float *lnw;        // [3][nb]   -ln(nb p_b)
  const float *gmm;        // [RIFT_GMM_FLOATS] learned proposal of the point (proposal 2)
  int tmarg;               // time marginalised by quadrature: the t table stays uniform
  int pad_;
};

// Learned proposal of one point as the sampler reads it (floats): ln pi[8], float32 cumulative
// pi[8], mu[8][5], ln sigma[8][5], 1/sigma[8][5], sum_d ln(b_d - a_d), the constant part of
// ln p5, ln D_lo, ln D_hi - ln D_lo, pad.
#define RIFT_GMM_FLOATS 144

// Arguments of the cell kernel.
struct CellLaunch {
  unsigned long long seed;
  float d_lo3, d_span3;
  const PointC *pts;
  const RoundPt *rp;
  int n_points;
  int win_budget;              // bytes of shared memory for staged Q windows
  const uint32_t *n_items;     // device: work items of this round
  uint32_t *queue;             // device: work-item counter (reset to 0 before the launch)
  const float2 *qa;
  const float4 *ca;
  Part *partials;              // [n_items]
  float *dbg_ell;
  float *ell_buf;
  uint32_t *bin_buf;
  uint32_t *flags;
  int max_M;                   // largest mode count over the points (shared-memory layout)
  int max_pairK;               // largest npair * K over the points
  int max_nb;                  // largest bin count (0 if no point uses tables)
  int learned;                 // points sample from their learned proposal (R.proposal 2; a point that
                               // fell back to the adaptive proposal draws from its tables)
  int fault_nan;               // injected fault: sample 0 of round 0 of every point has a NaN log weight
  int fault_stall;             // injected fault: window copies announced on the mbarrier but never issued
  int tmarg;                   // the event time is marginalised by quadrature (Eq. lnL:tmarg)
  int merged;                  // single mirror-symmetric point with all 21 modes whose 9 mirror
                               // pairs of Q merge (P.qhalf, P.Mh = 12): merged rows (cells_kernel_mp)
  float2 *cand;                // optional [items][RIFT_CAND_PER_ITEM]: (log weight, sample index bits)
                               // of the two largest log weights of each warp of each item
  float *cmax;                 // with cand: [items] the item's largest log weight
};

// Device-side round control of a batched run replayed as a CUDA graph.
struct RoundCtl {
  uint32_t n_items;       // work items of the prepared round
  uint32_t queue;         // work-queue counter of the cell kernel
  uint32_t active;        // points in the prepared round
  int round;              // number of the prepared round
  int adapt_now;          // the prepared round rebuilds tables afterwards
  int tabbuf;             // table buffer read by the prepared round
  int pad0, pad1;
};

// Per-point progress of a batched run (device).
struct PtState {
  unsigned long long evals;
  int rounds;
  int done;
  int ls[3];
  int prop;       // proposal of the point's next round (learned points may fall back to adaptive)
  int fb_round;   // first round on the adaptive proposal after a fallback, -1 if none
  int pad;
};

// Options of a batched run, as the device round-update kernel sees them.
struct BatchCtl {
  uint32_t npr;             // samples per round
  int np;                   // points
  unsigned long long max_evals;
  double n_eff_target;
  int max_rounds;           // 0: none
  int adaptive;
  int adapt_rounds;         // < 0: always
  int nb;
  float *tables;            // [2][np][3][nb+1]
  float *lnw;               // [2][np][3][nb]
  int learned;              // points sample from their learned proposals (gmm)
  int keep_ell;             // keep per-sample log weights of every round (harvest)
  const float *gmm;         // [np][RIFT_GMM_FLOATS]
  RoundPt *last;            // [np] the last round each point ran (harvest)
  int tmarg;                // the event time is marginalised by quadrature
  uint32_t point_id1;       // Philox point word of a single-point handle (batches use the point index)
  double fallback_neff;     // learned points switch to the adaptive proposal after a round whose own
                            // n_eff is below this (0: never)
};

// Scratch of the Monte Carlo runner (device pointers unless noted).
struct McScratch {
  AccState *acc;               // [np]
  Part *partials;              // [max_items]
  RoundPt *rp;                 // [np]
  uint32_t *counters;          // [2]: work items of the round, work-queue counter
  float *ell;                  // [np * n_per_round] adaptive per-sample log weights
  uint32_t *bins;              // [np * n_per_round] adaptive bins
  unsigned long long *hist;    // [np][hblocks][3][nb]
  float *tables;               // [2][np][3][RIFT_MAXBINS + 1]
  float *lnw;                  // [2][np][3][RIFT_MAXBINS]
  size_t max_items;
  int hblocks;
  RoundPt *rp_host;            // host mirror [np]
  AccState *acc_host;          // host mirror [np]
};

struct DrawOut {
  float *theta;  // [7][n]
  float *lpq;    // [n]
  int *bins;     // [3][n] or null
};

size_t rift_point_smem_bytes(int K, int npair, int nb, int block, int M);

cudaError_t launch_lnl_array(int K, const PointC *pt_dev, const PointC &pt_host, const float2 *q_arena,
                             const float4 *c_arena, size_t n, const float *ra, const float *dec, const float *t,
                             const float *psi, const float *phi, const float *incl, const float *dist, float *out,
                             uint32_t *flags, cudaStream_t st);
cudaError_t launch_lnl_tmarg(int K, const PointC *pt_dev, const PointC &ph, const float2 *qa, const float4 *ca,
                             size_t n, const float *ra, const float *dec, const float *psi, const float *phi,
                             const float *incl, const float *dist, float *out, uint32_t *flags, cudaStream_t st);

// Detector-frame coefficients and arrival times of sources (kernels.cu)
cudaError_t launch_source_frame(int K, const PointC *pt_dev, size_t n, const float *src, float2 *coef, float2 *tk,
                                cudaStream_t st);

// Cell kernel (mc.cu)
size_t cells_smem_fixed(int K, int max_M, int max_pairK, int max_nb, int block);
cudaError_t launch_cells(int K, int ntap, const CellLaunch &L, int grid, int block, size_t smem, cudaStream_t st,
                         const CanonCoefParam *cc = nullptr, int cc_sparse = 0, const MirrorCoefParam *mp = nullptr);
int cells_blocks_per_sm(int K, int ntap, size_t smem, int block, int tmarg = 0);
// Merged Q rows of every point that has them, gathered from the point's uploaded Q block.
cudaError_t launch_merge_rows(const PointC *pts, int np, float2 *qa, cudaStream_t st);
// Refinement of heavy samples after a round's merge: choose each point's samples from the items'
// candidates, evaluate them in FP64, fold the corrections into RefineState.  `scratch` holds
// np * RIFT_REFINE_CAP uint2 + np int + np * RIFT_REFINE_CAP double2 (refine_scratch_bytes).
struct PointD;
size_t refine_scratch_bytes(int np);
cudaError_t launch_refine(const PointC *pts, const PointD *pd, const double2 *uv64, const float2 *qa,
                          const RoundPt *rp, const AccState *acc, const float *cmax, const float2 *cand, int np,
                          unsigned long long seed, double d_lo3, double d_span3, void *scratch,
                          RefineState *rs, uint32_t *flags, cudaStream_t st);
cudaError_t launch_merge_points(const Part *partials, const RoundPt *rp, int n_points, AccState *acc,
                                cudaStream_t st);
cudaError_t launch_hist_points(const float *ell, const uint32_t *bins, const RoundPt *rp, int n_points,
                               const AccState *acc, float beta, int nb, unsigned long long *part, int hblocks,
                               cudaStream_t st);
cudaError_t launch_tables_points(const unsigned long long *part, int hblocks, const RoundPt *rp, int n_points,
                                 int nb, double floor_eps, float *tables, float *lnw, cudaStream_t st);
cudaError_t launch_draw_cells(const CellLaunch &L, DrawOut o, uint32_t n, cudaStream_t st);
cudaError_t launch_round_update(const BatchCtl &B, PtState *st_dev, const AccState *acc, RoundPt *rp, RoundCtl *ctl,
                                cudaStream_t st);
cudaError_t launch_hist_ctl(const float *ell, const uint32_t *bins, const RoundPt *rp, int n_points,
                            const AccState *acc, float beta, int nb, unsigned long long *part, int hblocks,
                            const RoundCtl *ctl, cudaStream_t st);
cudaError_t launch_harvest_theta(const CellLaunch &L, const RoundPt *last, const int *idx, int H, float *theta,
                                 cudaStream_t st);
cudaError_t launch_summary(const PointC *pts, const float2 *qa, const float4 *ca, const double *tau0, int np,
                           float *out, cudaStream_t st);
struct rift_mdn;
cudaError_t launch_mdn_gmm(const rift_mdn *m, const float *summ, const float *cst, int np, float *head_scratch,
                           float *gmm, uint32_t *flags, cudaStream_t st);
cudaError_t launch_gmm_from_head(const float *head, const float *cst, int np, float *gmm, cudaStream_t st);
// device and pinned host buffers of handles, recycled through a process-wide cache (cache.cu);
// a buffer is given back only when no work in flight uses it
cudaError_t cache_dev_alloc(void **p, size_t n);
cudaError_t cache_host_alloc(void **p, size_t n);
void cache_dev_free(void *p);
void cache_host_free(void *p);

// posterior samples (posterior.cu, kernels.cu)
cudaError_t launch_rows(const CellLaunch &L, const RoundPt *last, const float *ell, const int *idx, size_t n_slots,
                        int ncol, int np, float *out, cudaStream_t st);
cudaError_t launch_resample(const float *ell, const RoundPt *last, const AccState *acc, int np, float beta, int H,
                            int *idx, cudaStream_t st);
cudaError_t launch_tdraw(int K, int interp, const PointC *pts, int np, int max_npair, int max_M, const float2 *qa,
                         const float4 *ca, const RoundPt *last, unsigned long long seed, int H, float *out,
                         uint32_t *flags, cudaStream_t st);
cudaError_t launch_tables_ctl(const unsigned long long *part, int hblocks, const RoundPt *rp, int n_points, int nb,
                              double floor_eps, const BatchCtl &B, const RoundCtl *ctl, cudaStream_t st);

#define RIFT_FLAG_TIMEOUT_BIT 4u
