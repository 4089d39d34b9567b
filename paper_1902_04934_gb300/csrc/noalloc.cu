// rift_ile_marginalize_static: the marginalisation of rift_ile_marginalize with its
// scratch memory (block partials, running accumulator, adaptive histograms, tables and
// per-sample buffers) taken from one file-scope device array instead of cudaMalloc.
//
// Callers this is for: programs that hand (nearly) all device memory to another
// allocator at start-up, or that must not allocate or free device memory after
// initialisation (allocation can fail under such a pool, and cudaMalloc/cudaFree can
// synchronise the device).  Such a caller creates its handles during start-up and then
// only calls this entry point, which allocates nothing.
//
// The array below exists once per device that loads the library and stays allocated
// until the process exits.  Host code cannot use the name `g_static_scratch` as a device
// address (on the host it names a stand-in object); the device address is obtained with
// cudaGetSymbolAddress, once per device, with that device current, by the first call made
// on that device.  That first call should therefore come before any stream capture.
// All calls on one device share the array: calls whose work overlaps on the GPU race.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/rift_ile.h"
#include "rift_device.cuh"
#include "rift_internal.h"

namespace {

constexpr int kBlock = RIFT_MC_BLOCK;
constexpr int kMaxBlocks = RIFT_STATIC_MAX_BLOCKS;
constexpr int kMaxHistBlocks = 64;
constexpr size_t kAlign = 256;

constexpr size_t al(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// layout of the scratch array
constexpr size_t kOffAcc = 0;
constexpr size_t kOffPart = al(kOffAcc + sizeof(AccState));
constexpr size_t kOffHist = al(kOffPart + sizeof(Part) * kMaxBlocks);
constexpr size_t kOffTab = al(kOffHist + sizeof(unsigned long long) * kMaxHistBlocks * 3 * RIFT_MAXBINS);
constexpr size_t kOffLnw = al(kOffTab + sizeof(float) * 2 * 3 * (RIFT_MAXBINS + 1));
constexpr size_t kOffEll = al(kOffLnw + sizeof(float) * 2 * 3 * RIFT_MAXBINS);
constexpr size_t kOffBin = al(kOffEll + sizeof(float) * RIFT_STATIC_MAX_ROUND);
constexpr size_t kBytes = al(kOffBin + sizeof(uint32_t) * RIFT_STATIC_MAX_ROUND);
static_assert(kBytes == RIFT_STATIC_SCRATCH_BYTES, "scratch size in the header is out of date");

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up on first use).
cudaError_t scratch_address(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

// Internal accessors of the handle, defined in capi.cu.
rift_status rift_internal_point0(rift_ile *h, const PointC **host, const PointC **dev, const float2 **qa,
                                 const float4 **ca, int *K, int *num_sms, uint32_t **flags, cudaStream_t *st);
rift_status rift_internal_fail(rift_ile *h, rift_status s, const char *msg);
rift_status rift_internal_validate_opts(rift_ile *h, const rift_mc_opts *o);

extern "C" rift_status rift_ile_marginalize_static(rift_ile *h, const rift_mc_opts *o, rift_mc_result *res) {
  if (!h || !res) return RIFT_EINVAL;
  rift_status s = rift_internal_validate_opts(h, o);
  if (s != RIFT_OK) return s;
  const PointC *ph = nullptr, *pd = nullptr;
  const float2 *qa = nullptr;
  const float4 *ca = nullptr;
  int K = 0, sms = 0;
  uint32_t *flags = nullptr;
  cudaStream_t st = nullptr;
  if ((s = rift_internal_point0(h, &ph, &pd, &qa, &ca, &K, &sms, &flags, &st)) != RIFT_OK) return s;
  const bool adaptive = (o->proposal == RIFT_PROPOSAL_ADAPTIVE);
  const int nb = adaptive ? o->n_bins : 0;
  if (adaptive && o->n_per_round > (uint32_t)RIFT_STATIC_MAX_ROUND)
    return rift_internal_fail(h, RIFT_EINVAL,
                              "rift_ile_marginalize_static: n_per_round exceeds RIFT_STATIC_MAX_ROUND "
                              "(the static scratch holds one adaptive round of at most that many samples)");
  if (o->dbg_tables || o->timing)
    return rift_internal_fail(h, RIFT_EINVAL, "rift_ile_marginalize_static: dbg_tables and timing are not supported");
  unsigned char *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return rift_internal_fail(h, RIFT_ECUDA, cudaGetErrorString(e));
  AccState *acc = reinterpret_cast<AccState *>(base + kOffAcc);
  Part *parts = reinterpret_cast<Part *>(base + kOffPart);
  unsigned long long *hist = reinterpret_cast<unsigned long long *>(base + kOffHist);
  float *tables = reinterpret_cast<float *>(base + kOffTab);
  float *lnw = reinterpret_cast<float *>(base + kOffLnw);
  float *ell = reinterpret_cast<float *>(base + kOffEll);
  uint32_t *bins = reinterpret_cast<uint32_t *>(base + kOffBin);

  const size_t smem = rift_point_smem_bytes(K, ph->npair, nb, kBlock, ph->M);
  if (smem > 200 * 1024) return rift_internal_fail(h, RIFT_EUNSUPPORTED, "shared memory footprint too large");
  int bps = mc_round_blocks_per_sm(K, smem, kBlock);
  if (bps < 1) bps = 1;
  const uint32_t npr = o->n_per_round;
  const int grid = std::max(1, std::min(std::min(sms * bps, kMaxBlocks), (int)((npr + kBlock - 1) / kBlock)));
  const int hist_grid = std::max(1, std::min(kMaxHistBlocks, (int)((npr + 255) / 256)));

  // the array keeps the previous call's contents: reset the accumulator, set round-0 tables
  AccState a0;
  std::memset(&a0, 0, sizeof(a0));
  a0.m = -INFINITY;
#define RIFT_SCK(call)                                                               \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) return rift_internal_fail(h, RIFT_ECUDA, cudaGetErrorString(e_)); \
  } while (0)
  RIFT_SCK(cudaMemcpyAsync(acc, &a0, sizeof(a0), cudaMemcpyHostToDevice, st));
  int cur = 0;
  if (adaptive) {
    float u[3 * (RIFT_MAXBINS + 1)];
    const float *src = o->tables;
    if (!src) {
      for (int d = 0; d < 3; ++d)
        for (int b = 0; b <= nb; ++b) u[d * (nb + 1) + b] = (float)((double)b / nb);
      src = u;
    }
    RIFT_SCK(cudaMemcpyAsync(tables, src, sizeof(float) * 3 * (nb + 1), cudaMemcpyHostToDevice, st));
    RIFT_SCK(cudaStreamSynchronize(st));   // the source may be on this stack frame
    RIFT_SCK(launch_tables(nullptr, 0, nb, 0.0, tables, lnw, st));
  }
  McParams prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.seed = o->seed; prm.point_id = o->point_id; prm.nb = nb;
  prm.d_lo3 = (float)(o->d_lo * o->d_lo * o->d_lo);
  prm.d_span3 = (float)(o->d_hi * o->d_hi * o->d_hi - o->d_lo * o->d_lo * o->d_lo);
  prm.partials = parts; prm.flags = flags;
  uint64_t evals = 0;
  AccState a;
  std::memset(&a, 0, sizeof(a));
  int r = 0, launches = 0;
  for (;; ++r) {
    prm.round = (uint32_t)r;
    prm.n = (uint32_t)std::min<uint64_t>(npr, o->max_evals - evals);
    prm.proposal = adaptive ? 1 : 0;
    prm.tables = adaptive ? tables + cur * 3 * (nb + 1) : nullptr;
    prm.lnw = adaptive ? lnw + cur * 3 * nb : nullptr;
    prm.dbg_ell = o->dbg_ell;
    prm.dbg_off = (long long)r * npr;
    prm.ell_buf = adaptive ? ell : nullptr;
    prm.bin_buf = adaptive ? bins : nullptr;
    const int g = std::max(1, std::min<int>(grid, (int)((prm.n + kBlock - 1) / kBlock)));
    RIFT_SCK(launch_mc_round(K, pd, *ph, qa, ca, prm, g, kBlock, st));
    RIFT_SCK(launch_merge(parts, g, acc, st));
    launches += 2;
    const bool adapt_now = adaptive && (o->adapt_rounds < 0 || r < o->adapt_rounds);
    if (adapt_now) {
      const int hg = std::max(1, std::min(hist_grid, (int)((prm.n + 255) / 256)));
      RIFT_SCK(launch_hist(ell, bins, prm.n, acc, (float)o->beta, nb, hist, hg, st));
      RIFT_SCK(launch_tables(hist, hg, nb, o->floor_eps, tables + (1 - cur) * 3 * (nb + 1), lnw + (1 - cur) * 3 * nb,
                             st));
      launches += 2;
    }
    RIFT_SCK(cudaMemcpyAsync(&a, acc, sizeof(a), cudaMemcpyDeviceToHost, st));
    RIFT_SCK(cudaStreamSynchronize(st));
    if (adapt_now) cur = 1 - cur;
    evals += prm.n;
    const double n_eff = a.s1 + a.c1;
    if (n_eff >= o->n_eff_target || evals >= o->max_evals || (o->max_rounds > 0 && r + 1 >= o->max_rounds)) break;
  }
#undef RIFT_SCK
  std::memset(res, 0, sizeof(*res));
  res->acc_max = a.m;
  res->acc_s1 = a.s1 + a.c1;
  res->acc_s2 = a.s2 + a.c2;
  res->n_evals = a.n;
  const double n = (double)a.n;
  if (a.n == 0 || !(res->acc_s1 > 0)) {
    res->lnL_marg = -INFINITY; res->sigma = INFINITY;
  } else {
    res->lnL_marg = a.m + std::log(res->acc_s1) - std::log(n);
    res->n_eff = res->acc_s1;
    res->n_eff_kish = res->acc_s1 * res->acc_s1 / res->acc_s2;
    res->sigma = (a.n > 1) ? std::sqrt(std::max(n * res->acc_s2 / (res->acc_s1 * res->acc_s1) - 1.0, 0.0) / (n - 1.0))
                           : INFINITY;
  }
  res->rounds = r + 1;
  res->kernel_launches = launches;
  s = rift_ile_check(h);
  if (s == RIFT_OK && res->n_eff < o->n_eff_target) s = RIFT_ENOTCONVERGED;
  res->status = s;
  return s;
}
