// zmc_serving.cpp -- continuous batching of integration jobs.
//
// zmc_submit copies a job's descriptors, validates and precomputes them, and
// queues the job.  A scheduler thread owns a stream and loops:
//   1. admit queued jobs, in order, while their device block (descriptor table,
//      one 8-byte record per chunk, result rows) fits in the arena;
//   2. build one iteration of at most max_chunks_per_iter chunks over the
//      admitted jobs: oldest job first by default (each job's next chunks up to
//      the remaining budget), or equal shares for every job with work left
//      (zmc_options.serving_share);
//   3. upload the iteration's entry table and header on the copy-in stream (so
//      the copies overlap the launch before), replay the iteration graph (the
//      per-family persistent sampling kernels) on the sampling stream, and on a
//      side stream, after the graph, merge (FP64) every job whose last chunks
//      ran and copy those jobs' results to pinned staging, record an event; the
//      sampling stream goes straight on to the next graph, so the merge and the
//      copies overlap the next launch; two iteration slots are in flight at once;
//   4. when a slot's event completes, hand the finished jobs' results to
//      zmc_poll and free their device blocks.
// Checkpoints: zmc_checkpoint takes a running job off the live list; the next
// iteration (stream-ordered after every iteration that ran the job's chunks)
// uploads copies of its descriptors cut to the chunks issued so far and merges
// them into moments (out_mode 1) together with the moments the job was resumed
// from.  zmc_submit_resume starts each integrand at sample from.n of its stream
// (FnDev.s_off) and carries from as the descriptor's prior moments.
// Failures: a failed CUDA call in the loop poisons the context, every pending job
// completes with ZMC_ECUDA and later calls on the context return ZMC_ECUDA.  The
// environment variable ZMC_SERVING_FAULT_AT=<k> injects such a failure on the
// host at iteration k (for tests; no GPU fault is involved).
// A chunk's record depends only on (integrand, chunk) and the merge sums records
// in a fixed order, so a job's results are bit-identical whether it runs alone or
// mixed with others.  No kernel waits on another: every launch drains a finite
// work list and exits.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "zmc_runtime.h"

using namespace zmc;

namespace {

using Clock = std::chrono::steady_clock;

enum class JobState {
  kQueued,
  kRunning,
  kFinishing,
  kDone,
  kCancelled,
  kFailed,
  kCheckpointing,  // taken off the live list; its moments merge in the next iteration
  kCheckpointed
};

struct ServJob {
  uint64_t id = 0;
  size_t n = 0;
  std::vector<FnDev> fns;      // host copy, device pointers filled at admission
  std::vector<int> family;
  std::vector<uint64_t> nchunk;
  std::vector<uint64_t> next_chunk;
  size_t cursor = 0;           // first integrand with chunks left to issue
  uint64_t chunks_total = 0, chunks_issued = 0, samples = 0;
  size_t block_bytes = 0;
  char *dblock = nullptr;
  FnDev *d_fns = nullptr;
  zmc_result *d_out = nullptr;
  JobState state = JobState::kQueued;
  zmc_status fail_status = ZMC_OK;
  std::vector<zmc_result> results;
  std::vector<zmc_moments> ckpt;  // filled when a checkpoint completes
  uint64_t last_seq = 0;       // last iteration that touched the job
  Clock::time_point t_submit, t_done;
};

struct Slot {
  Entry *d_entries = nullptr;
  LaunchHdr *d_hdr = nullptr;
  const FnDev **d_merge = nullptr;
  zmc_result *d_results = nullptr;  // contiguous copy target of merged results
  char *h_stage = nullptr;          // pinned: entries | merge list | hdr | results
  cudaEvent_t ev = nullptr;      // the slot's last work (side stream): results staged
  cudaEvent_t ev_up = nullptr;   // its tables uploaded (copy-in stream)
  cudaEvent_t ev_run = nullptr;  // its sampling graph done (sampling stream)
  cudaGraphExec_t graph = nullptr;
  bool busy = false;
  uint64_t seq = 0;
  std::vector<std::shared_ptr<ServJob>> finishing;
  std::vector<size_t> result_off;
};

}  // namespace

struct ServingState {
  zmc_ctx *ctx = nullptr;
  std::thread thread;
  std::mutex mu;
  std::condition_variable cv_work;
  std::condition_variable cv_done;
  bool stop = false;
  std::atomic<uint64_t> wakeups{0};  // new work announced (submits, checkpoints)
  std::deque<std::shared_ptr<ServJob>> queue;
  std::vector<std::shared_ptr<ServJob>> live;
  std::deque<std::shared_ptr<ServJob>> to_merge;
  std::deque<std::shared_ptr<ServJob>> to_ckpt;  // checkpoint merges not yet issued
  std::unordered_map<uint64_t, std::shared_ptr<ServJob>> jobs;
  std::vector<std::shared_ptr<ServJob>> cancelled_pending;
  uint64_t next_id = 1;
  cudaStream_t stream = nullptr;  // sampling graphs, back to back
  cudaStream_t up = nullptr;      // host -> device tables
  cudaStream_t side = nullptr;    // merges and device -> host results
  FamilyFork fork;  // the four family kernels of an iteration run concurrently
  Slot slots[2];
  uint32_t max_chunks = 0;
  uint32_t max_entries = 0;
  uint32_t max_merge = 0;
  unsigned grid[4] = {0, 0, 0, 0};
  uint64_t seq = 0;
  zmc_serving_stats stats{};
  zmc_status thread_status = ZMC_OK;
  uint64_t fault_at = 0;  // host-side fault injection (tests): iteration that fails
  std::deque<uint64_t> finished;  // finished, not yet reported by zmc_poll_any
};

namespace {

size_t round256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

void free_job_device(ServingState *S, ServJob &j) {
  if (j.dblock) {
    S->ctx->arena.release(j.dblock);
    j.dblock = nullptr;
  }
}

// Admission: one arena block per job; its descriptor table is copied into the
// slot's pinned admission area and uploaded asynchronously from there.
bool try_admit(ServingState *S, const std::shared_ptr<ServJob> &jp, char *stage,
               size_t &stage_used, size_t stage_cap) {
  zmc_ctx *ctx = S->ctx;
  ServJob &j = *jp;
  const size_t tbytes = j.n * sizeof(FnDev);
  if (stage_used + tbytes > stage_cap) return false;
  char *blk = static_cast<char *>(ctx->arena.alloc(j.block_bytes));
  if (!blk) return false;
  j.dblock = blk;
  j.d_fns = reinterpret_cast<FnDev *>(blk);
  size_t off = round256(j.n * sizeof(FnDev));
  float2 *rec = reinterpret_cast<float2 *>(blk + off);
  off += round256(j.chunks_total * sizeof(float2));
  j.d_out = reinterpret_cast<zmc_result *>(blk + off);
  uint64_t r = 0;
  for (size_t i = 0; i < j.n; ++i) {
    j.fns[i].rec = rec + r;
    j.fns[i].out = j.d_out + i;
    r += j.nchunk[i];
  }
  char *src = stage + stage_used;
  std::memcpy(src, j.fns.data(), tbytes);
  stage_used += round256(tbytes);
  cudaError_t e = cudaMemcpyAsync(j.d_fns, src, tbytes, cudaMemcpyHostToDevice, S->up);
  if (e != cudaSuccess) {
    ctx_cuda_fail(ctx, e, "serving admission upload");
    S->thread_status = ZMC_ECUDA;
  }
  j.state = JobState::kRunning;
  if (j.chunks_total == 0) S->to_merge.push_back(jp);  // nothing left to sample
  return true;
}

zmc_status build_slot_graph(ServingState *S, Slot &sl) {
  zmc_ctx *ctx = S->ctx;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "serving capture");
  cudaError_t le = cudaMemsetAsync(sl.d_hdr, 0, sizeof(sl.d_hdr->counter), S->stream);
  const bool all[4] = {true, true, true, true};
  const unsigned block[4] = {ctx->shape.block, ctx->shape.block, ctx->shape.block,
                             ctx->shape.block};
  if (le == cudaSuccess)
    le = launch_families(S->fork, sl.d_entries, sl.d_hdr, S->grid, block, all, S->stream);
  e = cudaStreamEndCapture(S->stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return ctx_cuda_fail(ctx, le, "serving capture launch");
  }
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "serving end capture");
  e = cudaGraphInstantiate(&sl.graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "serving graph instantiate");
  return ZMC_OK;
}

constexpr size_t kAdmitBytes = 16u << 20;  // pinned admission area per slot

size_t stage_bytes(const ServingState *S) {
  return round256(S->max_entries * sizeof(Entry)) + round256(S->max_merge * sizeof(FnDev *)) +
         round256(sizeof(LaunchHdr)) + round256(S->max_merge * sizeof(zmc_result)) +
         kAdmitBytes;
}

char *admit_area(const ServingState *S, const Slot &sl) {
  return sl.h_stage + stage_bytes(S) - kAdmitBytes;
}

// Retire a completed slot: results to jobs, device blocks back to the arena.
void retire_slot(ServingState *S, Slot &sl) {
  std::lock_guard<std::mutex> g(S->mu);
  const char *res_base = sl.h_stage + round256(S->max_entries * sizeof(Entry)) +
                         round256(S->max_merge * sizeof(FnDev *)) +
                         round256(sizeof(LaunchHdr));
  const auto now = Clock::now();
  for (size_t k = 0; k < sl.finishing.size(); ++k) {
    auto &j = sl.finishing[k];
    if (j->state == JobState::kFinishing) {
      j->results.resize(j->n);
      std::memcpy(j->results.data(), res_base + sl.result_off[k] * sizeof(zmc_result),
                  j->n * sizeof(zmc_result));
      j->state = JobState::kDone;
      j->t_done = now;
      S->stats.completed++;
      S->stats.samples_done += j->samples;
      S->finished.push_back(j->id);
    } else if (j->state == JobState::kCheckpointing) {
      // the merge wrote moments (out_mode 1): estimate = mean, stderr_ = M2
      const zmc_result *r =
          reinterpret_cast<const zmc_result *>(res_base + sl.result_off[k] * sizeof(zmc_result));
      j->ckpt.resize(j->n);
      for (size_t i = 0; i < j->n; ++i) {
        j->ckpt[i].mean = r[i].estimate;
        j->ckpt[i].m2 = r[i].stderr_;
        j->ckpt[i].n = r[i].n;
        j->ckpt[i].status = ZMC_OK;
        j->ckpt[i].reserved = 0;
      }
      j->state = JobState::kCheckpointed;
    }
    free_job_device(S, *j);
  }
  sl.finishing.clear();
  sl.result_off.clear();
  sl.busy = false;
  // cancelled jobs whose last iteration has now finished
  auto &cp = S->cancelled_pending;
  for (auto it = cp.begin(); it != cp.end();) {
    if ((*it)->last_seq <= sl.seq) {
      free_job_device(S, **it);
      it = cp.erase(it);
    } else {
      ++it;
    }
  }
  S->cv_done.notify_all();
}

// The launch fill rule (zmc_serving_fill): take[i] chunks of job i, jobs in
// arrival order.  Oldest first by default: each job takes its next chunks up to
// the whole remaining budget, so a launch finishes the oldest jobs and starts
// the next ones with what is left (measured on the Poisson job stream: p99
// latency 17 ms instead of 22 ms at 300 jobs/s, 33 instead of 53 ms at 400, p50
// unchanged, against equal shares).  With a short backlog (fewer than
// cut_backlog samples left to issue over the jobs) the launch ends with the
// last chunks of the first job it completes, so that job's results do not wait
// for the newer jobs' chunks behind it; those start the next launch, which runs
// right after it.  With a long backlog every launch is filled (each launch
// costs a fixed ~50 us).  Measured (2^31-sample budget): p99 15.4 against 16.7
// ms at 300 jobs/s, 29.9 against 30.6 at 400, 364 against 360 G samples/s under
// overload.  With share > 0 every job with work left gets budget / jobs per
// pass, but at least share chunks (runs of a few chunks would turn every work
// item into an entry-table search).
void fill_launch(const uint64_t *left, size_t n, uint64_t budget, uint64_t share,
                 uint64_t cut_backlog, uint64_t chunk_samples, uint64_t *take) {
  for (size_t i = 0; i < n; ++i) take[i] = 0;
  if (share == 0) {
    uint64_t backlog = 0;  // saturating: a job may hold up to 2^62 samples per row
    for (size_t i = 0; i < n && backlog != UINT64_MAX; ++i) {
      const uint64_t s = left[i] > UINT64_MAX / chunk_samples ? UINT64_MAX
                                                               : left[i] * chunk_samples;
      backlog = backlog > UINT64_MAX - s ? UINT64_MAX : backlog + s;
    }
    const bool cut = backlog < cut_backlog;
    for (size_t i = 0; i < n && budget > 0; ++i) {
      take[i] = std::min(left[i], budget);
      budget -= take[i];
      if (cut && take[i] > 0 && take[i] == left[i]) break;
    }
    return;
  }
  std::vector<size_t> active;
  for (size_t i = 0; i < n; ++i)
    if (left[i] > 0) active.push_back(i);
  while (budget > 0 && !active.empty()) {
    const uint64_t per = std::max<uint64_t>(share, budget / active.size());
    std::vector<size_t> still;
    for (size_t i : active) {
      const uint64_t t = std::min({per, budget, left[i] - take[i]});
      take[i] += t;
      budget -= t;
      if (take[i] < left[i]) still.push_back(i);
      if (budget == 0) break;
    }
    active.swap(still);
  }
}

void scheduler_loop(ServingState *S) {
  zmc_ctx *ctx = S->ctx;
  cudaSetDevice(ctx->device);
  for (;;) {
    // retire completed slots
    for (auto &sl : S->slots) {
      if (!sl.busy) continue;
      cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaSuccess) {
        retire_slot(S, sl);
      } else if (q != cudaErrorNotReady) {
        ctx_cuda_fail(ctx, q, "serving event");
        S->thread_status = ZMC_ECUDA;
      }
    }
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->thread_status != ZMC_OK) {
      // fail everything that is still pending
      for (auto &kv : S->jobs)
        if (kv.second->state != JobState::kDone && kv.second->state != JobState::kCancelled &&
            kv.second->state != JobState::kFailed &&
            kv.second->state != JobState::kCheckpointed) {
          kv.second->state = JobState::kFailed;
          kv.second->fail_status = S->thread_status;
          S->finished.push_back(kv.first);
        }
      S->cv_done.notify_all();
      if (S->stop) return;
      S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
      continue;
    }
    // pick a free slot
    Slot *slot = nullptr;
    for (auto &sl : S->slots)
      if (!sl.busy) {
        slot = &sl;
        break;
      }
    // admission in arrival order, staged through the free slot's pinned area
    size_t used = 0;  // bytes of the slot's admission area taken this iteration
    if (slot) {
      char *area = admit_area(S, *slot);
      while (!S->queue.empty()) {
        auto j = S->queue.front();
        if (j->state == JobState::kCancelled || j->state == JobState::kCheckpointed) {
          S->queue.pop_front();
          continue;
        }
        if (j->n * sizeof(FnDev) > kAdmitBytes) {  // never fits the area: refused
          j->state = JobState::kFailed;
          j->fail_status = ZMC_ENOMEM;
          S->finished.push_back(j->id);
          S->queue.pop_front();
          S->cv_done.notify_all();
          continue;
        }
        if (!try_admit(S, j, area, used, kAdmitBytes)) break;
        S->queue.pop_front();
        S->live.push_back(j);
      }
    }
    const bool have_work = !S->live.empty() || !S->to_merge.empty() || !S->to_ckpt.empty();
    if (!slot || !have_work) {
      bool any_busy = S->slots[0].busy || S->slots[1].busy;
      if (S->stop && !any_busy) return;
      if (any_busy) {
        const uint64_t seen = S->wakeups.load(std::memory_order_acquire);
        lk.unlock();
        // wait outside the lock for the oldest busy slot, or, when a slot is
        // free, for the first of that slot's completion and new work (a job, a
        // checkpoint): a job that arrives while one launch runs is then built
        // and queued behind it at once instead of after the launch's results
        // have been copied back
        Slot *oldest = nullptr;
        for (auto &sl : S->slots)
          if (sl.busy && (!oldest || sl.seq < oldest->seq)) oldest = &sl;
        if (oldest && !slot) {
          cudaEventSynchronize(oldest->ev);
        } else if (oldest) {
          while (cudaEventQuery(oldest->ev) == cudaErrorNotReady &&
                 S->wakeups.load(std::memory_order_acquire) == seen)
            std::this_thread::yield();
        }
        continue;
      }
      if (!S->queue.empty()) {
        // admission is blocked on memory that nothing in flight will free soon
        S->cv_work.wait_for(lk, std::chrono::milliseconds(1));
        continue;
      }
      S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      if (S->stop && S->queue.empty() && S->live.empty()) return;
      continue;
    }
    // ---- build one iteration
    const uint64_t seq = ++S->seq;
    char *st = slot->h_stage;
    Entry *ents = reinterpret_cast<Entry *>(st);
    const FnDev **mrg =
        reinterpret_cast<const FnDev **>(st + round256(S->max_entries * sizeof(Entry)));
    LaunchHdr *hdr = reinterpret_cast<LaunchHdr *>(
        st + round256(S->max_entries * sizeof(Entry)) + round256(S->max_merge * sizeof(FnDev *)));
    std::vector<Entry> fam_ents[4];
    std::unordered_map<const FnDev *, uint32_t> variant_of;
    // the launch's chunks per live job (fill_launch); a run of chunks of one
    // integrand is one entry, so the entry table never holds more entries than
    // the launch has chunks
    std::vector<std::shared_ptr<ServJob>> active;
    for (auto &j : S->live)
      if (j->state == JobState::kRunning && j->chunks_issued < j->chunks_total) active.push_back(j);
    std::vector<uint64_t> left(active.size()), take(active.size());
    for (size_t q = 0; q < active.size(); ++q)
      left[q] = active[q]->chunks_total - active[q]->chunks_issued;
    fill_launch(left.data(), active.size(), std::min<uint64_t>(S->max_chunks, S->max_entries),
                ctx->serving_share, ctx->serving_share ? 0 : ctx->serving_cut_backlog,
                chunk_samples_of(ctx->quints_per_lane), take.data());
    uint32_t n_entries = 0;
    uint64_t jobs_in_iter = 0;  // jobs with work items in this launch
    for (size_t q = 0; q < active.size(); ++q) {
      if (take[q] == 0) continue;
      auto &j = active[q];
      ++jobs_in_iter;
      uint64_t want = take[q];
      while (want > 0 && j->cursor < j->n) {
        const size_t i = j->cursor;
        const uint64_t left_i = j->nchunk[i] - j->next_chunk[i];
        if (left_i == 0) {  // resumed integrand with no samples left
          ++j->cursor;
          continue;
        }
        const uint64_t t = std::min(left_i, want);
        Entry en;
        en.item_begin = t;  // the run length for now; item offsets come below
        en.fn = j->d_fns + i;
        en.chunk_begin = j->next_chunk[i];
        fam_ents[j->family[i]].push_back(en);
        variant_of[en.fn] = j->fns[i].variant;
        ++n_entries;
        j->next_chunk[i] += t;
        j->chunks_issued += t;
        want -= t;
        if (j->next_chunk[i] == j->nchunk[i]) ++j->cursor;
      }
      j->last_seq = seq;
      if (j->chunks_issued == j->chunks_total) S->to_merge.push_back(j);
    }
    // concatenate by family, each family's runs ordered by variant (stable) so
    // co-resident warps mostly run the same code path, as in a plan;
    // convert run lengths into item offsets
    std::memset(hdr, 0, sizeof *hdr);
    uint64_t item = 0;
    uint32_t k = 0;
    for (int f = 0; f < 4; ++f) {
      auto &fe = fam_ents[f];
      std::vector<uint32_t> var(fe.size());
      for (size_t q = 0; q < fe.size(); ++q) {
        const FnDev *dev = fe[q].fn;
        // the host copy of the descriptor holds the variant; find it by job
        var[q] = variant_of.at(dev);
      }
      std::vector<uint32_t> order(fe.size());
      for (size_t q = 0; q < order.size(); ++q) order[q] = static_cast<uint32_t>(q);
      std::stable_sort(order.begin(), order.end(),
                       [&](uint32_t a, uint32_t b) { return var[a] < var[b]; });
      std::vector<Entry> sorted(fe.size());
      for (size_t q = 0; q < order.size(); ++q) sorted[q] = fe[order[q]];
      fe.swap(sorted);
      hdr->item_begin[f] = item;
      for (auto &en : fam_ents[f]) {
        const uint64_t len = en.item_begin;
        en.item_begin = item;
        ents[k++] = en;
        item += len;
      }
      hdr->item_end[f] = item;
    }
    hdr->n_entries = k;
    hdr->quints_per_lane = ctx->quints_per_lane;
    // merge list: whole jobs whose chunks have all been issued
    uint32_t nm = 0;
    slot->finishing.clear();
    slot->result_off.clear();
    while (!S->to_merge.empty()) {
      auto j = S->to_merge.front();
      if (j->state != JobState::kRunning) {
        S->to_merge.pop_front();
        continue;
      }
      if (nm + j->n > S->max_merge) break;
      for (size_t i = 0; i < j->n; ++i) mrg[nm + i] = j->d_fns + i;
      slot->finishing.push_back(j);
      slot->result_off.push_back(nm);
      nm += static_cast<uint32_t>(j->n);
      j->state = JobState::kFinishing;
      j->last_seq = seq;
      S->to_merge.pop_front();
    }
    // checkpoints: descriptors cut to the chunks issued so far, merged into moments
    while (!S->to_ckpt.empty()) {
      auto j = S->to_ckpt.front();
      if (j->state != JobState::kCheckpointing) {
        S->to_ckpt.pop_front();
        continue;
      }
      const size_t tbytes = j->n * sizeof(FnDev);
      if (nm + j->n > S->max_merge || used + tbytes > kAdmitBytes) break;
      const uint64_t chunk = chunk_samples_of(ctx->quints_per_lane);
      FnDev *cut = reinterpret_cast<FnDev *>(admit_area(S, *slot) + used);
      for (size_t i = 0; i < j->n; ++i) {
        cut[i] = j->fns[i];
        cut[i].n_samples = std::min(j->next_chunk[i] * chunk, j->fns[i].n_samples);
        cut[i].out_mode = 1;
        mrg[nm + i] = j->d_fns + i;
      }
      used += round256(tbytes);
      // on the sampling stream: the launches that ran the job's chunks read the
      // table being rewritten, and they run before this copy
      cudaError_t e = cudaMemcpyAsync(j->d_fns, cut, tbytes, cudaMemcpyHostToDevice, S->stream);
      if (e != cudaSuccess) {
        ctx_cuda_fail(ctx, e, "serving checkpoint upload");
        S->thread_status = ZMC_ECUDA;
      }
      slot->finishing.push_back(j);
      slot->result_off.push_back(nm);
      nm += static_cast<uint32_t>(j->n);
      j->last_seq = seq;
      S->to_ckpt.pop_front();
    }
    hdr->n_merge = nm;
    // drop finished jobs from the live list
    S->live.erase(std::remove_if(S->live.begin(), S->live.end(),
                                 [](const std::shared_ptr<ServJob> &j) {
                                   return j->state != JobState::kRunning ||
                                          j->chunks_issued == j->chunks_total;
                                 }),
                  S->live.end());
    S->stats.iterations++;
    if (jobs_in_iter >= 2) S->stats.shared_iterations++;
    S->stats.max_jobs_per_iter = std::max(S->stats.max_jobs_per_iter, jobs_in_iter);
    lk.unlock();

    // ---- enqueue: upload tables, replay the graph, copy merged results back
    const size_t ent_bytes = round256(S->max_entries * sizeof(Entry));
    const size_t mrg_bytes = round256(S->max_merge * sizeof(FnDev *));
    const size_t hdr_bytes = round256(sizeof(LaunchHdr));
    cudaError_t e = cudaSuccess;
    if (S->fault_at != 0 && seq == S->fault_at) {
      // injected on the host: nothing of this iteration is enqueued, and it is
      // reported exactly like a failed CUDA call
      ctx_cuda_fail(ctx, cudaErrorLaunchFailure, "serving iteration (injected fault)");
      S->thread_status = ZMC_ECUDA;
      continue;
    }
    // the slot's buffers were last read by its previous iteration, which has
    // retired (its merge and copies included)
    if (k > 0)
      e = cudaMemcpyAsync(slot->d_entries, ents, k * sizeof(Entry), cudaMemcpyHostToDevice,
                          S->up);
    if (e == cudaSuccess && nm > 0)
      e = cudaMemcpyAsync(slot->d_merge, mrg, nm * sizeof(FnDev *), cudaMemcpyHostToDevice,
                          S->up);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(slot->d_hdr, hdr, sizeof(LaunchHdr), cudaMemcpyHostToDevice, S->up);
    if (e == cudaSuccess) e = cudaEventRecord(slot->ev_up, S->up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->stream, slot->ev_up, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(slot->graph, S->stream);
    if (e == cudaSuccess) e = cudaEventRecord(slot->ev_run, S->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->side, slot->ev_run, 0);
    if (e == cudaSuccess && nm > 0) {
      // the jobs merged here have no chunks in later launches, so the merge
      // overlaps the next sampling graph
      const unsigned mg = static_cast<unsigned>(
          std::min<uint64_t>((nm + 7) / 8, static_cast<uint64_t>(ctx->sms) * 16));
      e = launch_merge(slot->d_merge, slot->d_hdr, mg, S->side);
    }
    char *res_stage = st + ent_bytes + mrg_bytes + hdr_bytes;
    for (size_t q = 0; e == cudaSuccess && q < slot->finishing.size(); ++q) {
      auto &j = slot->finishing[q];
      e = cudaMemcpyAsync(res_stage + slot->result_off[q] * sizeof(zmc_result), j->d_out,
                          j->n * sizeof(zmc_result), cudaMemcpyDeviceToHost, S->side);
    }
    if (e == cudaSuccess) e = cudaEventRecord(slot->ev, S->side);
    if (e != cudaSuccess) {
      ctx_cuda_fail(ctx, e, "serving iteration");
      S->thread_status = ZMC_ECUDA;
      continue;
    }
    slot->busy = true;
    slot->seq = seq;
  }
}

}  // namespace

zmc_status serving_start(zmc_ctx *ctx) {
  auto S = std::make_unique<ServingState>();
  S->ctx = ctx;
  // default: ~2.1e9 samples per iteration (about 6 ms of sampling) whatever the
  // chunk length.  With launches cut at job ends under a short backlog, a
  // longer budget only matters under load, where fewer, longer launches pay
  // less fixed cost: against 2^30 samples, p99 15.4 against 15.7 ms at 300
  // jobs/s, 29.9 against 30.9 at 400, 364 against 360 G samples/s under
  // overload.
  S->max_chunks = ctx->max_chunks_per_iter
                      ? ctx->max_chunks_per_iter
                      : static_cast<uint32_t>(std::max<uint64_t>(
                            1024, (1ull << 31) / chunk_samples_of(ctx->quints_per_lane)));
  S->max_entries = std::max<uint32_t>(S->max_chunks, 1024);
  S->max_entries = std::min<uint32_t>(S->max_entries, 1u << 20);
  S->max_merge = 1u << 16;
  if (const char *f = std::getenv("ZMC_SERVING_FAULT_AT")) S->fault_at = std::strtoull(f, nullptr, 10);
  cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->side, cudaStreamNonBlocking);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "serving stream");
  e = S->fork.init();
  if (e != cudaSuccess) {
    S->fork.destroy();
    return ctx_cuda_fail(ctx, e, "serving side streams");
  }
  for (int f = 0; f < 4; ++f) S->grid[f] = family_grid(ctx, f, ~0ull >> 8);
  const size_t sb = stage_bytes(S.get());
  for (auto &sl : S->slots) {
    sl.d_entries = static_cast<Entry *>(ctx->arena.alloc(S->max_entries * sizeof(Entry)));
    sl.d_merge = static_cast<const FnDev **>(ctx->arena.alloc(S->max_merge * sizeof(FnDev *)));
    sl.d_hdr = static_cast<LaunchHdr *>(ctx->arena.alloc(sizeof(LaunchHdr)));
    if (!sl.d_entries || !sl.d_merge || !sl.d_hdr)
      return set_error(ZMC_ENOMEM, "serving tables do not fit the arena");
    e = cudaHostAlloc(reinterpret_cast<void **>(&sl.h_stage), sb, cudaHostAllocDefault);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "serving staging");
    e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_up, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_run, cudaEventDisableTiming);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "serving event");
    zmc_status st = build_slot_graph(S.get(), sl);
    if (st != ZMC_OK) return st;
  }
  S->stats.arena_bytes = ctx->arena.size();
  ServingState *raw = S.release();
  ctx->srv = raw;
  raw->thread = std::thread(scheduler_loop, raw);
  return ZMC_OK;
}

void serving_stop(zmc_ctx *ctx) {
  ServingState *S = ctx->srv;
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
    for (auto &j : S->queue) j->state = JobState::kCancelled;
    S->queue.clear();
    for (auto &j : S->live) j->state = JobState::kCancelled;
    S->live.clear();
    S->to_merge.clear();
    for (auto &j : S->to_ckpt)
      if (j->state == JobState::kCheckpointing) j->state = JobState::kCancelled;
    S->to_ckpt.clear();
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  if (S->thread.joinable()) S->thread.join();
  cudaStreamSynchronize(S->up);
  cudaStreamSynchronize(S->stream);
  cudaStreamSynchronize(S->side);
  for (auto &kv : S->jobs) free_job_device(S, *kv.second);
  for (auto &sl : S->slots) {
    if (sl.graph) cudaGraphExecDestroy(sl.graph);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.ev_up) cudaEventDestroy(sl.ev_up);
    if (sl.ev_run) cudaEventDestroy(sl.ev_run);
    if (sl.h_stage) cudaFreeHost(sl.h_stage);
    ctx->arena.release(sl.d_entries);
    ctx->arena.release(sl.d_merge);
    ctx->arena.release(sl.d_hdr);
  }
  cudaStreamDestroy(S->stream);
  cudaStreamDestroy(S->up);
  cudaStreamDestroy(S->side);
  S->fork.destroy();
  delete S;
  ctx->srv = nullptr;
}

namespace {

// Validate, precompute and queue a job; from (optional) holds per-integrand
// moments of samples [0, from[i].n) of its stream, taken earlier.
zmc_status submit_job(zmc_ctx *ctx, const zmc_desc *desc, const zmc_moments *from, size_t n,
                      uint64_t *job_id) {
  if (!ctx || !desc || !job_id || n == 0) return set_error(ZMC_EINVAL, "bad submit arguments");
  if (!ctx->serving || !ctx->srv) return set_error(ZMC_EINVAL, "context created without serving");
  if (ctx->poisoned) return set_error(ZMC_ECUDA, "context poisoned by an earlier CUDA error");
  ServingState *S = ctx->srv;
  auto j = std::make_shared<ServJob>();
  j->n = n;
  j->fns.resize(n);
  j->family.resize(n);
  j->nchunk.resize(n);
  j->next_chunk.assign(n, 0);
  const uint64_t chunk = chunk_samples_of(ctx->quints_per_lane);
  std::vector<uint8_t> ok(n, 1);
  host_parallel_for(n, 64, [&](size_t b, size_t e) {
    for (size_t i = b; i < e; ++i) ok[i] = precompute(desc[i], &j->fns[i], nullptr, nullptr) == ZMC_OK;
  });
  for (size_t i = 0; i < n; ++i) {
    if (!ok[i]) {
      const zmc_status st = precompute(desc[i], &j->fns[i], nullptr, nullptr);
      return set_error(st, "descriptor %zu: %s", i, zmc_last_error(nullptr));
    }
    uint64_t start = 0;
    if (from && from[i].n > 0) {
      const zmc_moments &m = from[i];
      start = m.n;
      if (m.status != ZMC_OK || start > desc[i].n_samples ||
          (start % kQuint != 0 && start != desc[i].n_samples) || !std::isfinite(m.mean) ||
          !std::isfinite(m.m2) || m.m2 < 0.0)
        return set_error(ZMC_EINVAL,
                         "descriptor %zu: resume moments need status OK, finite mean and "
                         "M2 >= 0, n <= n_samples and n a multiple of 5 (or n_samples)", i);
      FnDev &f = j->fns[i];
      f.s_off = start;
      f.n_samples = desc[i].n_samples - start;
      f.prior_n = start;
      f.prior_mean = m.mean;
      f.prior_m2 = m.m2;
    }
    j->family[i] = static_cast<int>(desc[i].family);
    j->nchunk[i] = (desc[i].n_samples - start + chunk - 1) / chunk;
    j->chunks_total += j->nchunk[i];
    j->samples += desc[i].n_samples - start;
  }
  j->block_bytes = round256(n * sizeof(FnDev)) + round256(j->chunks_total * sizeof(float2)) +
                   round256(n * sizeof(zmc_result));
  const size_t max_fns = std::min<size_t>(S->max_merge, kAdmitBytes / sizeof(FnDev));
  if (n > max_fns) return set_error(ZMC_EINVAL, "a job may hold at most %zu integrands", max_fns);
  if (j->block_bytes > ctx->arena.size())
    return set_error(ZMC_ENOMEM, "job needs %zu bytes; the arena has %zu", j->block_bytes,
                     ctx->arena.size());
  j->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) return set_error(ZMC_ECLOSED, "context is shutting down");
    j->id = S->next_id++;
    S->jobs[j->id] = j;
    S->queue.push_back(j);
    S->wakeups.fetch_add(1, std::memory_order_release);
    S->stats.submitted++;
    *job_id = j->id;
  }
  S->cv_work.notify_one();
  return ZMC_OK;
}

}  // namespace

extern "C" {

zmc_status zmc_submit(zmc_ctx *ctx, const zmc_desc *desc, size_t n, uint64_t *job_id) {
  return submit_job(ctx, desc, nullptr, n, job_id);
}

zmc_status zmc_submit_resume(zmc_ctx *ctx, const zmc_desc *desc, const zmc_moments *from,
                             size_t n, uint64_t *job_id) {
  if (!from) return set_error(ZMC_EINVAL, "null moments");
  return submit_job(ctx, desc, from, n, job_id);
}

zmc_status zmc_poll(zmc_ctx *ctx, uint64_t job_id, zmc_result *out, int32_t wait_ms) {
  if (!ctx || !ctx->srv) return set_error(ZMC_EINVAL, "context created without serving");
  ServingState *S = ctx->srv;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return set_error(ZMC_ENOTFOUND, "unknown job %llu",
                                            static_cast<unsigned long long>(job_id));
  std::shared_ptr<ServJob> j = it->second;
  auto finished = [&] {
    return j->state == JobState::kDone || j->state == JobState::kCancelled ||
           j->state == JobState::kFailed || j->state == JobState::kCheckpointed;
  };
  if (!finished()) {
    if (wait_ms == 0) return set_error(ZMC_EAGAIN, "job not finished");
    if (wait_ms < 0) {
      S->cv_done.wait(lk, finished);
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), finished)) {
      return set_error(ZMC_ETIMEOUT, "job not finished after %d ms", wait_ms);
    }
  }
  S->jobs.erase(job_id);
  if (j->state == JobState::kCancelled) return set_error(ZMC_ECLOSED, "job was cancelled");
  if (j->state == JobState::kCheckpointed)
    return set_error(ZMC_ECLOSED, "job was checkpointed");
  if (j->state == JobState::kFailed) return set_error(j->fail_status, "job failed");
  if (out) std::memcpy(out, j->results.data(), j->n * sizeof(zmc_result));
  return ZMC_OK;
}

zmc_status zmc_cancel(zmc_ctx *ctx, uint64_t job_id) {
  if (!ctx || !ctx->srv) return set_error(ZMC_EINVAL, "context created without serving");
  ServingState *S = ctx->srv;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return set_error(ZMC_ENOTFOUND, "unknown job");
  auto &j = it->second;
  if (j->state == JobState::kDone || j->state == JobState::kFailed ||
      j->state == JobState::kCancelled || j->state == JobState::kCheckpointed)
    return ZMC_OK;
  if (j->state == JobState::kQueued) {
    j->state = JobState::kCancelled;
  } else if (j->state == JobState::kRunning || j->state == JobState::kFinishing ||
             j->state == JobState::kCheckpointing) {
    j->state = JobState::kCancelled;
    // device memory is freed once the last iteration that used it has finished
    S->cancelled_pending.push_back(j);
    S->live.erase(std::remove(S->live.begin(), S->live.end(), j), S->live.end());
  }
  S->stats.cancelled++;
  S->finished.push_back(job_id);
  S->cv_done.notify_all();
  return ZMC_OK;
}

zmc_status zmc_checkpoint(zmc_ctx *ctx, uint64_t job_id, zmc_moments *out, int32_t wait_ms) {
  if (!ctx || !ctx->srv) return set_error(ZMC_EINVAL, "context created without serving");
  if (!out) return set_error(ZMC_EINVAL, "null output");
  ServingState *S = ctx->srv;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return set_error(ZMC_ENOTFOUND, "unknown job %llu",
                                            static_cast<unsigned long long>(job_id));
  std::shared_ptr<ServJob> j = it->second;
  switch (j->state) {
    case JobState::kQueued:
      // nothing ran: the moments it started from
      for (size_t i = 0; i < j->n; ++i) {
        const FnDev &f = j->fns[i];
        out[i].mean = f.prior_n ? f.prior_mean : 0.0;
        out[i].m2 = f.prior_n ? f.prior_m2 : 0.0;
        out[i].n = f.prior_n;
        out[i].status = ZMC_OK;
        out[i].reserved = 0;
      }
      j->state = JobState::kCheckpointed;
      S->jobs.erase(job_id);
      S->cv_done.notify_all();
      return ZMC_OK;
    case JobState::kRunning:
      if (j->chunks_issued == j->chunks_total)
        return set_error(ZMC_EAGAIN, "job has issued all of its samples; collect it with zmc_poll");
      j->state = JobState::kCheckpointing;
      S->live.erase(std::remove(S->live.begin(), S->live.end(), j), S->live.end());
      S->to_ckpt.push_back(j);
      S->wakeups.fetch_add(1, std::memory_order_release);
      S->cv_work.notify_one();
      break;
    case JobState::kCheckpointing:
    case JobState::kCheckpointed:
      break;
    case JobState::kFinishing:
    case JobState::kDone:
      return set_error(ZMC_EAGAIN, "job has issued all of its samples; collect it with zmc_poll");
    case JobState::kCancelled:
      return set_error(ZMC_ECLOSED, "job was cancelled");
    case JobState::kFailed:
      return set_error(j->fail_status, "job failed");
  }
  auto settled = [&] { return j->state != JobState::kCheckpointing; };
  if (!settled()) {
    if (wait_ms == 0) return set_error(ZMC_EAGAIN, "checkpoint under way");
    if (wait_ms < 0) {
      S->cv_done.wait(lk, settled);
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), settled)) {
      return set_error(ZMC_ETIMEOUT, "checkpoint not finished after %d ms", wait_ms);
    }
  }
  if (j->state == JobState::kCancelled) return set_error(ZMC_ECLOSED, "job was cancelled");
  if (j->state == JobState::kFailed) return set_error(j->fail_status, "job failed");
  std::memcpy(out, j->ckpt.data(), j->n * sizeof(zmc_moments));
  S->jobs.erase(job_id);
  return ZMC_OK;
}

zmc_status zmc_poll_any(zmc_ctx *ctx, uint64_t *job_ids, size_t cap, int32_t wait_ms,
                        size_t *n_out) {
  if (!ctx || !ctx->srv || !job_ids || !n_out || cap == 0)
    return set_error(ZMC_EINVAL, "bad zmc_poll_any arguments");
  ServingState *S = ctx->srv;
  std::unique_lock<std::mutex> lk(S->mu);
  *n_out = 0;
  auto ready = [&] { return !S->finished.empty() || S->stop; };
  if (!ready()) {
    if (wait_ms == 0) return set_error(ZMC_EAGAIN, "no finished job");
    if (wait_ms < 0) {
      S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready)) {
      return set_error(ZMC_ETIMEOUT, "no job finished within %d ms", wait_ms);
    }
  }
  size_t n = 0;
  while (n < cap && !S->finished.empty()) {
    const uint64_t id = S->finished.front();
    S->finished.pop_front();
    if (S->jobs.count(id)) job_ids[n++] = id;  // skip jobs already collected by zmc_poll
  }
  *n_out = n;
  if (n) return ZMC_OK;
  if (S->stop) return set_error(ZMC_ECLOSED, "context is shutting down");
  return set_error(ZMC_EAGAIN, "no finished job");
}

zmc_status zmc_serving_fill(const uint64_t *chunks_left, size_t n_jobs, uint64_t budget,
                            uint32_t share, uint64_t cut_backlog, uint64_t chunk_samples,
                            uint64_t *take) {
  if ((n_jobs > 0 && (!chunks_left || !take)) || chunk_samples == 0)
    return set_error(ZMC_EINVAL, "zmc_serving_fill: null array or zero chunk_samples");
  fill_launch(chunks_left, n_jobs, budget, share, cut_backlog, chunk_samples, take);
  return ZMC_OK;
}

zmc_status zmc_serving_stats_get(zmc_ctx *ctx, zmc_serving_stats *out) {
  if (!ctx || !ctx->srv || !out) return set_error(ZMC_EINVAL, "no serving state");
  ServingState *S = ctx->srv;
  std::lock_guard<std::mutex> g(S->mu);
  *out = S->stats;
  out->queued = S->queue.size();
  out->running = S->live.size();
  out->arena_used_bytes = ctx->arena.used();
  out->arena_bytes = ctx->arena.size();
  return ZMC_OK;
}

}  // extern "C"
