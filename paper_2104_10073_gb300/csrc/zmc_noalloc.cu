// zmc_noalloc.cu -- batched integration that allocates no memory.
//
// zmc_integrate_noalloc runs the same sampling and merge kernels as
// zmc_integrate, but everything it needs beyond the caller's descriptor table
// (host) and result array (device) -- the launch header, the work list, the
// per-integrand device descriptors and the per-chunk partial sums -- lives in
// one fixed array that is part of the library's device image.  It creates no
// context, calls no cudaMalloc / cudaFree / cudaHostAlloc, and uses a static
// host buffer for staging.
//
// Who needs this: code that may not allocate device memory at the point where
// it wants an integral -- a framework that owns all device memory through its
// own pool and forbids side allocations, a latency-bound loop where an
// allocation's implicit device synchronisation or its failure on a nearly full
// device is not acceptable, or a caller that cannot afford zmc_create's arena.
//
// Costs and rules:
//   * the array below (ZMC_NOALLOC_SCRATCH_BYTES) is reserved on a device once
//     the library's device code is loaded there (with CUDA's lazy module
//     loading, at the latest on the first call on that device) and stays
//     reserved until the process exits;
//   * the tables are uploaded from a static (pageable) host buffer; before a
//     call overwrites that buffer it waits until the previous call's upload has
//     completed on the GPU (an event recorded after the upload), so a call may
//     block until the previous call's stream has reached its upload;
//   * every call uses the same array and it keeps the last call's contents;
//     the call re-uploads the tables and zeroes the work counters itself, and
//     every partial-sum record is written before it is read;
//   * calls whose GPU work overlaps (different streams, or different host
//     threads on one stream without ordering) race on the array: order them;
//   * the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) and creates the upload event, with that device
//     current; make that first call before any stream capture.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "zmc_runtime.h"

namespace {

constexpr size_t kScratchBytes = ZMC_NOALLOC_SCRATCH_BYTES;
constexpr size_t kMaxFns = ZMC_NOALLOC_MAX_FNS;
constexpr uint32_t kQuints = 104;  // the default chunk, so results equal zmc_integrate's
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr size_t r256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }
constexpr size_t kOffHdr = 0;
constexpr size_t kOffEnt = r256(sizeof(zmc::LaunchHdr));

// Host staging of the tables (header | entries | merge list | descriptors),
// laid out exactly as in the device array, sized for kMaxFns integrands.
constexpr size_t kHostBytes = kOffEnt + r256(kMaxFns * sizeof(zmc::Entry)) +
                              r256(kMaxFns * sizeof(const zmc::FnDev *)) +
                              r256(kMaxFns * sizeof(zmc::FnDev));
alignas(256) unsigned char g_host_stage[kHostBytes];
uint32_t g_order[kMaxFns];
std::mutex g_mu;
unsigned char *g_scratch_dev[kMaxDevices];  // device address of the array, per device
cudaEvent_t g_upload_ev[kMaxDevices];       // recorded after each call's table upload
cudaEvent_t g_last_upload = nullptr;        // the event of the last call, any device

}  // namespace

using namespace zmc;

extern "C" zmc_status zmc_integrate_noalloc(const zmc_desc *desc, size_t n, zmc_result *out,
                                            void *stream) {
  if (!desc || !out || n == 0) return set_error(ZMC_EINVAL, "need n >= 1 descriptors and an output");
  if (n > kMaxFns)
    return set_error(ZMC_EINVAL, "zmc_integrate_noalloc takes at most %zu integrands (got %zu)",
                     kMaxFns, n);
  std::lock_guard<std::mutex> g(g_mu);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(ZMC_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(ZMC_EINVAL, "device %d out of range", dev);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(ZMC_ECUDA, "scratch address lookup: %s", cudaGetErrorString(e));
    g_scratch_dev[dev] = static_cast<unsigned char *>(p);
  }
  if (!g_upload_ev[dev]) {
    e = cudaEventCreateWithFlags(&g_upload_ev[dev], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      g_upload_ev[dev] = nullptr;
      return set_error(ZMC_ECUDA, "upload event: %s", cudaGetErrorString(e));
    }
  }
  unsigned char *dbase = g_scratch_dev[dev];

  // layout for this call
  const size_t off_mrg = kOffEnt + r256(n * sizeof(Entry));
  const size_t off_fns = off_mrg + r256(n * sizeof(const FnDev *));
  const size_t off_rec = off_fns + r256(n * sizeof(FnDev));
  const uint64_t chunk = chunk_samples_of(kQuints);
  uint64_t chunks = 0;
  for (size_t i = 0; i < n; ++i) {
    if (desc[i].n_samples == 0 || desc[i].n_samples > (1ull << 62))
      return set_error(ZMC_EINVAL, "descriptor %zu: bad n_samples", i);
    chunks += (desc[i].n_samples + chunk - 1) / chunk;
  }
  const uint64_t need = off_rec + chunks * sizeof(float2);
  if (need > kScratchBytes)
    return set_error(ZMC_ENOMEM,
                     "zmc_integrate_noalloc needs %llu bytes of scratch; its fixed array holds "
                     "%zu (at most ~%llu samples in total)",
                     static_cast<unsigned long long>(need), kScratchBytes,
                     static_cast<unsigned long long>((kScratchBytes - off_rec) / sizeof(float2) *
                                                     chunk));

  // the previous call's upload must have read the staging buffer before it is
  // rewritten (a pageable asynchronous copy need not have consumed its source
  // when cudaMemcpyAsync returns)
  if (g_last_upload) {
    e = cudaEventSynchronize(g_last_upload);
    if (e != cudaSuccess)
      return set_error(ZMC_ECUDA, "previous upload: %s", cudaGetErrorString(e));
    g_last_upload = nullptr;
  }

  // host tables
  LaunchHdr *hdr = reinterpret_cast<LaunchHdr *>(g_host_stage + kOffHdr);
  Entry *ents = reinterpret_cast<Entry *>(g_host_stage + kOffEnt);
  const FnDev **mrg = reinterpret_cast<const FnDev **>(g_host_stage + off_mrg);
  FnDev *fns = reinterpret_cast<FnDev *>(g_host_stage + off_fns);
  const FnDev *dfns = reinterpret_cast<const FnDev *>(dbase + off_fns);
  float2 *drec = reinterpret_cast<float2 *>(dbase + off_rec);
  uint64_t rec = 0;
  for (size_t i = 0; i < n; ++i) {
    zmc_status st = precompute(desc[i], &fns[i], nullptr, nullptr);
    if (st != ZMC_OK) return set_error(st, "descriptor %zu: %s", i, zmc_last_error(nullptr));
    fns[i].rec = drec + rec;
    fns[i].out = out + i;
    rec += (desc[i].n_samples + chunk - 1) / chunk;
    mrg[i] = dfns + i;
    g_order[i] = static_cast<uint32_t>(i);
  }
  std::sort(g_order, g_order + n, [&](uint32_t a, uint32_t b) {
    if (desc[a].family != desc[b].family) return desc[a].family < desc[b].family;
    if (fns[a].variant != fns[b].variant) return fns[a].variant < fns[b].variant;
    return a < b;
  });
  std::memset(hdr, 0, sizeof(LaunchHdr));  // work counters start at zero
  uint64_t item = 0;
  int cur = -1;
  for (size_t k = 0; k < n; ++k) {
    const uint32_t i = g_order[k];
    const int f = static_cast<int>(desc[i].family);
    while (cur < f) {
      ++cur;
      hdr->item_begin[cur] = hdr->item_end[cur] = item;
    }
    ents[k].item_begin = item;
    ents[k].fn = dfns + i;
    ents[k].chunk_begin = 0;
    item += (desc[i].n_samples + chunk - 1) / chunk;
    hdr->item_end[f] = item;
  }
  while (cur < 3) {
    ++cur;
    hdr->item_begin[cur] = hdr->item_end[cur] = item;
  }
  hdr->n_entries = static_cast<uint32_t>(n);
  hdr->n_merge = static_cast<uint32_t>(n);
  hdr->quints_per_lane = kQuints;

  // launch shape: the persistent grid of each family kernel on this device
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(ZMC_ECUDA, "device query: %s", cudaGetErrorString(e));
  cudaStream_t str = static_cast<cudaStream_t>(stream);
  e = cudaMemcpyAsync(dbase, g_host_stage, off_rec, cudaMemcpyHostToDevice, str);
  if (e != cudaSuccess) return set_error(ZMC_ECUDA, "table upload: %s", cudaGetErrorString(e));
  e = cudaEventRecord(g_upload_ev[dev], str);
  if (e != cudaSuccess) {
    // the copy may still read the staging buffer: wait for it here instead
    cudaStreamSynchronize(str);
    return set_error(ZMC_ECUDA, "upload event: %s", cudaGetErrorString(e));
  }
  g_last_upload = g_upload_ev[dev];
  for (int f = 0; f < 4; ++f) {
    const uint64_t items = hdr->item_end[f] - hdr->item_begin[f];
    if (items == 0) continue;
    const uint64_t per_sm = static_cast<uint64_t>(std::max(batched_max_blocks_per_sm(f, 256), 1));
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(sms * per_sm, (items + 7) / 8));
    e = launch_batched(f, reinterpret_cast<const Entry *>(dbase + kOffEnt),
                       reinterpret_cast<LaunchHdr *>(dbase + kOffHdr),
                       static_cast<unsigned>(grid), 256, str);
    if (e != cudaSuccess) return set_error(ZMC_ECUDA, "sampling launch: %s", cudaGetErrorString(e));
  }
  const unsigned mgrid = static_cast<unsigned>(std::min<size_t>((n + 7) / 8, static_cast<size_t>(sms) * 16));
  e = launch_merge(reinterpret_cast<const FnDev *const *>(dbase + off_mrg),
                   reinterpret_cast<const LaunchHdr *>(dbase + kOffHdr), mgrid, str);
  if (e != cudaSuccess) return set_error(ZMC_ECUDA, "merge launch: %s", cudaGetErrorString(e));
  return ZMC_OK;
}
