// Host runtime internals shared by zmc_runtime.cpp (context, arena, plans) and
// zmc_serving.cpp (continuous-batching scheduler).  Not part of the C ABI.
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "zmc_internal.h"

namespace zmc {

// Thread-local error text + status helper.
zmc_status set_error(zmc_status st, const char *fmt, ...);

// First-fit sub-allocator over one device buffer (256-byte granules, coalescing
// free list).  All device memory a context uses comes from here.
class Arena {
 public:
  void init(char *base, size_t bytes);
  // nullptr when no free range is large enough.
  void *alloc(size_t bytes);
  void release(void *p);
  size_t used() const { return used_; }
  size_t size() const { return size_; }
  size_t largest_free() const;

 private:
  char *base_ = nullptr;
  size_t size_ = 0;
  size_t used_ = 0;
  std::map<size_t, size_t> free_;       // offset -> length
  std::map<size_t, size_t> allocated_;  // offset -> length
  mutable std::mutex mu_;
};

// Derived device form of one descriptor (validation + FP64 precompute).
zmc_status precompute(const zmc_desc &d, FnDev *fn, PlainFn *plain, double *volume);

// Launch-shape choice for the per-family persistent kernels.
struct LaunchShape {
  unsigned block = 256;
  unsigned blocks_per_sm[4] = {0, 0, 0, 0};  // 0 -> occupancy maximum
};

// One autotuner result (zmc_tune.cpp): a family kernel's launch geometry, or
// (quints > 0) a table shape class's chunk length and per-family unroll.
struct TuneChoice {
  unsigned block = 256;
  unsigned blocks_per_sm = 0;
  unsigned quints = 0;
  unsigned unroll[4] = {1, 1, 1, 1};
  float ms = 0.0f;
};
constexpr uint32_t kTuneQuints[] = {26, 52, 104, 208};  // chunk lengths the tuner tries

struct Job;

}  // namespace zmc

struct zmc_plan;

namespace zmc {
// Side streams and events that run the family kernels of one launch
// concurrently: forked from a main stream and joined back into it (also inside
// a stream capture, where the fork and join become graph edges).  A family
// kernel's blocks then fill the SMs that the previous family's last chunks
// leave idle, instead of waiting for its tail.
struct FamilyFork {
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[3] = {nullptr, nullptr, nullptr};
  cudaError_t init();
  void destroy();
};
// Launch the batched kernels of the families with present[f] on `main`,
// concurrently when more than one is present.
cudaError_t launch_families(FamilyFork &ff, const Entry *entries, LaunchHdr *hdr,
                            const unsigned *grid, const unsigned *block, const bool *present,
                            cudaStream_t main, const unsigned *unroll = nullptr);
// The generator-only kernel (zmc_kernels.cu): grid x 256 threads, per_thread
// Philox blocks each (a multiple of 4), one folded word per thread into out.
cudaError_t launch_philox_rate(uint32_t per_thread, unsigned grid, uint32_t *out,
                               cudaStream_t stream);
}  // namespace zmc

struct zmc_ctx {
  int device = 0;
  int sms = 0;
  std::string gpu_name;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  zmc::FamilyFork fork;  // concurrent family kernels of one launch
  char *arena_base = nullptr;
  bool own_arena = false;
  zmc::Arena arena;
  uint32_t quints_per_lane = 16;
  uint32_t max_chunks_per_iter = 0;
  uint32_t serving_share = 0;  // serving: 0 oldest job first, > 0 equal shares of >= this
  uint64_t serving_cut_backlog = 0;  // serving: backlog below which launches end at a job
  uint32_t autotune = 0;  // ZMC_TUNE_* flags
  std::string tune_cache_path;
  zmc::LaunchShape shape;
  int max_blocks_per_sm[4] = {0, 0, 0, 0};
  int kernel_regs[zmc::kMaxUnroll][4] = {};  // registers per thread of each family kernel
  std::map<std::string, zmc::TuneChoice> tune_cache;  // autotuner results by key
  std::atomic<bool> poisoned{false};
  std::recursive_mutex api_mu;  // serialises API calls that use the stream

  // pinned staging for host <-> device copies of the blocking calls
  void *stage = nullptr;
  size_t stage_bytes = 0;

  // serving
  bool serving = false;
  struct ServingState *srv = nullptr;  // owned; created by serving_start
};

namespace zmc {
zmc_status ctx_cuda_fail(zmc_ctx *ctx, cudaError_t err, const char *what);
zmc_status ensure_stage(zmc_ctx *ctx, size_t bytes);
unsigned family_grid(const zmc_ctx *ctx, int family, uint64_t items, int unroll = 1);
unsigned grid_for(const zmc_ctx *ctx, int family, unsigned block, unsigned bps, uint64_t items,
                  int unroll = 1);
std::string tune_key(const zmc_ctx *ctx, int family, int dim, uint32_t quints, int unroll);
void tune_cache_load(zmc_ctx *ctx);
void tune_cache_store(zmc_ctx *ctx, const std::string &key, const TuneChoice &c);
}  // namespace zmc

// Root form of a real polynomial sum_k e[k] u^k of degree <= 4 (zmc_polyroots.cpp):
//   q(u) = lead * prod_s f_s(u); slot s of type 1 is a real root, f_s = u - v[s];
//   type 2 opens a complex pair, f_s = (u - v[s])^2 + v[s+1] (v[s+1] > 0), and
//   the pair's second slot has type 3.  False when no reliable form was found
//   (the caller then keeps the coefficients).
namespace zmc {
struct RootForm {
  double lead;
  int n;            // slots used
  uint8_t type[4];
  double v[4];
};
bool poly_root_form(const double *e, int g, RootForm *out);
}  // namespace zmc

// Host thread pool (zmc_pool.cpp): fn(begin, end) over [0, n) in ranges of
// `grain`, on the calling thread and the pool's workers; returns when all ranges
// are done.  Small n runs inline.
#include <functional>
namespace zmc {
void host_parallel_for(size_t n, size_t grain, const std::function<void(size_t, size_t)> &fn);
}  // namespace zmc

// User-defined integrands (zmc_udf.cpp): one row of a udf integration; lo/hi
// hold dim values, p ZMC_NPARAM.
namespace zmc {
struct UdfRow {
  uint32_t dim = 0, func = 0, stream_id = 0;
  uint64_t n_samples = 0, seed = 0;
  const double *lo = nullptr, *hi = nullptr, *p = nullptr;
};
zmc_status udf_run(zmc_ctx *ctx, const zmc_udf *udf, const UdfRow *rows, size_t n,
                   zmc_result *out);
uint32_t udf_dim(const zmc_udf *udf);
}  // namespace zmc

// Serving state (zmc_serving.cpp).
struct ServingState;
zmc_status serving_start(zmc_ctx *ctx);
void serving_stop(zmc_ctx *ctx);
