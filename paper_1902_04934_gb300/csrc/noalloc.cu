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
// address (on the host it names a stand-in object); every call looks the device address up
// with cudaGetSymbolAddress, with the caller's device current, and checks the result.  The
// first call on a device is the set-up: the lookup may load the library's device code there
// (which is when the array is allocated), so that first call should come before any stream
// capture.  Later lookups only read the runtime's symbol table; looking the address up on
// every call, rather than keeping it, keeps it valid after cudaDeviceReset, which unloads the
// module and may place the array elsewhere when it is loaded again.
// The learned proposal is refused: its per-handle network buffers would be allocated.
// All calls on one device share the array: calls whose work overlaps on the GPU race.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <string>

#include "../../include/rift_ile.h"
#include "rift_device.cuh"
#include "rift_internal.h"

namespace {

constexpr int kHist = 64;          // histogram blocks per round
// work items of one round: cells plus extra chunks of large cells (adaptive rounds are
// capped at RIFT_STATIC_MAX_ROUND samples; prior rounds of any size use at most this many
// items because the runner rejects more; time-marginalised rounds, in items of at most
// RIFT_TMARG_CHUNK = RIFT_CHUNK / 8 draws, are capped at an eighth of the prior-round limit)
constexpr size_t kItems = (size_t)RIFT_MAX_CELLS + RIFT_STATIC_MAX_PRIOR_ROUND / RIFT_CHUNK + 1;
constexpr size_t kAlign = 256;

constexpr size_t al(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// layout of the scratch array (one point)
constexpr size_t kOffAcc = 0;
constexpr size_t kOffPart = al(kOffAcc + sizeof(AccState));
constexpr size_t kOffRp = al(kOffPart + sizeof(Part) * kItems);
constexpr size_t kOffCnt = al(kOffRp + sizeof(RoundPt));
constexpr size_t kOffHist = al(kOffCnt + sizeof(uint32_t) * 2);
constexpr size_t kOffTab = al(kOffHist + sizeof(unsigned long long) * kHist * 3 * RIFT_MAXBINS);
constexpr size_t kOffLnw = al(kOffTab + sizeof(float) * 2 * 3 * (RIFT_MAXBINS + 1));
constexpr size_t kOffEll = al(kOffLnw + sizeof(float) * 2 * 3 * RIFT_MAXBINS);
constexpr size_t kOffBin = al(kOffEll + sizeof(float) * RIFT_STATIC_MAX_ROUND);
constexpr size_t kBytes = al(kOffBin + sizeof(uint32_t) * RIFT_STATIC_MAX_ROUND);
static_assert(kBytes == RIFT_STATIC_SCRATCH_BYTES, "scratch size in the header is out of date");
static_assert(RIFT_CHUNK == 8 * RIFT_TMARG_CHUNK, "the time-marginalised round limit assumes items of RIFT_CHUNK / 8");

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kBytes];

namespace {

// Device address of the scratch array on the current device.
cudaError_t scratch_address(unsigned char **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char *>(p);
  return cudaSuccess;
}

}  // namespace

// Defined in capi.cu: the Monte Carlo runner with caller-provided scratch.
rift_status rift_internal_run_static(rift_ile *h, const rift_mc_opts *o, McScratch &S, rift_mc_result *res);
rift_status rift_internal_fail(rift_ile *h, rift_status s, const char *msg);

extern "C" rift_status rift_ile_marginalize_static(rift_ile *h, const rift_mc_opts *o, rift_mc_result *res) {
  if (!h || !res || !o) return RIFT_EINVAL;
  if (o->proposal == RIFT_PROPOSAL_ADAPTIVE && o->n_per_round > (uint32_t)RIFT_STATIC_MAX_ROUND)
    return rift_internal_fail(h, RIFT_EINVAL,
                              "rift_ile_marginalize_static: n_per_round exceeds RIFT_STATIC_MAX_ROUND "
                              "(the static scratch holds one adaptive round of at most that many samples)");
  if (o->n_per_round > (uint32_t)RIFT_STATIC_MAX_PRIOR_ROUND)
    return rift_internal_fail(h, RIFT_EINVAL,
                              "rift_ile_marginalize_static: n_per_round exceeds RIFT_STATIC_MAX_PRIOR_ROUND "
                              "(the static scratch holds the partials of at most that many samples per round)");
  if (o->time_marg && o->n_per_round > (uint32_t)(RIFT_STATIC_MAX_PRIOR_ROUND / 8))
    return rift_internal_fail(h, RIFT_EINVAL,
                              "rift_ile_marginalize_static: time-marginalised rounds hold at most "
                              "RIFT_STATIC_MAX_PRIOR_ROUND / 8 draws (work items of at most 256 draws)");
  if (o->proposal == RIFT_PROPOSAL_LEARNED)
    return rift_internal_fail(h, RIFT_EINVAL,
                              "rift_ile_marginalize_static: the learned proposal is not supported (its network "
                              "buffers are allocated per handle)");
  if (o->dbg_tables || o->timing)
    return rift_internal_fail(h, RIFT_EINVAL, "rift_ile_marginalize_static: dbg_tables and timing are not supported");
  if (o->refine)
    return rift_internal_fail(h, RIFT_EINVAL,
                              "rift_ile_marginalize_static: refine is not supported (its candidate buffers are "
                              "allocated per handle)");
  if (o->proposal == RIFT_PROPOSAL_ADAPTIVE && (o->n_bins < 2 || o->n_bins > RIFT_MAXBINS))
    return rift_internal_fail(h, RIFT_EINVAL, "n_bins out of range [2, 256]");
  unsigned char *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return rift_internal_fail(h, RIFT_ECUDA, cudaGetErrorString(e));
  // host mirrors of the one point's round descriptor and accumulator live on this stack frame
  RoundPt rp_host;
  AccState acc_host;
  McScratch S;
  std::memset(&S, 0, sizeof(S));
  S.acc = reinterpret_cast<AccState *>(base + kOffAcc);
  S.partials = reinterpret_cast<Part *>(base + kOffPart);
  S.rp = reinterpret_cast<RoundPt *>(base + kOffRp);
  S.counters = reinterpret_cast<uint32_t *>(base + kOffCnt);
  S.hist = reinterpret_cast<unsigned long long *>(base + kOffHist);
  S.tables = reinterpret_cast<float *>(base + kOffTab);
  S.lnw = reinterpret_cast<float *>(base + kOffLnw);
  S.ell = reinterpret_cast<float *>(base + kOffEll);
  S.bins = reinterpret_cast<uint32_t *>(base + kOffBin);
  S.max_items = kItems;
  S.hblocks = std::max(1, std::min(kHist, (int)(o->n_per_round / 8192)));
  S.rp_host = &rp_host;
  S.acc_host = &acc_host;
  // everything the runner reads from the array is (re)initialised by it: the accumulator,
  // the round-0 tables, the round descriptor and the work counters
  return rift_internal_run_static(h, o, S, res);
}
