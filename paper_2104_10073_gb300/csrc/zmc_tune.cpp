// zmc_tune.cpp -- the autotuner's cache: launch geometry (threads per block,
// resident blocks per SM) chosen per family kernel, stored as JSON.
//
// The geometry decides only which warp runs which work item, never what an
// item computes, so tuning never changes results.  Keys name what the best
// geometry can depend on: the GPU model and SM count, the family, the chunk
// length (quints per lane), the dominant dimension of the family's samples and
// the family kernel's registers per thread (its build).
//
// File format (written by this file only):
//   {"version": 1, "entries": {
//     "<gpu>|<sms>|<family>|<quints>|<dim>|r<regs>": {"block": 256, "blocks_per_sm": 2, "ms": 0.512},
//     ...}}
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>

#include "zmc_runtime.h"

namespace zmc {

std::string tune_key(const zmc_ctx *ctx, int family, int dim) {
  std::ostringstream k;
  // the kernel's register count stands for its build: a rebuild with other
  // launch-bound knobs is timed afresh instead of reusing another build's choice
  k << ctx->gpu_name << '|' << ctx->sms << '|' << family << '|' << ctx->quints_per_lane << '|'
    << dim << "|r" << ctx->kernel_regs[family];
  return k.str();
}

void tune_cache_load(zmc_ctx *ctx) {
  ctx->tune_cache.clear();
  if (ctx->tune_cache_path.empty()) return;
  std::ifstream in(ctx->tune_cache_path);
  if (!in) return;
  std::stringstream ss;
  ss << in.rdbuf();
  const std::string s = ss.str();
  // entries look like "key": {"block": B, "blocks_per_sm": N, "ms": T}
  size_t pos = s.find("\"entries\"");
  if (pos == std::string::npos) return;
  pos = s.find('{', pos);
  if (pos == std::string::npos) return;
  ++pos;
  while (true) {
    const size_t k0 = s.find('"', pos);
    if (k0 == std::string::npos) break;
    const size_t k1 = s.find('"', k0 + 1);
    if (k1 == std::string::npos) break;
    const size_t b0 = s.find('{', k1);
    if (b0 == std::string::npos) break;
    const size_t b1 = s.find('}', b0);
    if (b1 == std::string::npos) break;
    const std::string key = s.substr(k0 + 1, k1 - k0 - 1);
    const std::string body = s.substr(b0, b1 - b0);
    unsigned block = 0, bps = 0;
    float ms = 0.0f;
    const size_t pb = body.find("\"block\""), pn = body.find("\"blocks_per_sm\""),
                 pm = body.find("\"ms\"");
    if (pb != std::string::npos && pn != std::string::npos &&
        std::sscanf(body.c_str() + body.find(':', pb) + 1, "%u", &block) == 1 &&
        std::sscanf(body.c_str() + body.find(':', pn) + 1, "%u", &bps) == 1) {
      if (pm != std::string::npos) std::sscanf(body.c_str() + body.find(':', pm) + 1, "%f", &ms);
      if ((block == 128 || block == 256) && bps >= 1 && bps <= 16) {
        TuneChoice c;
        c.block = block;
        c.blocks_per_sm = bps;
        c.ms = ms;
        ctx->tune_cache[key] = c;
      }
    }
    pos = b1 + 1;
  }
}

void tune_cache_store(zmc_ctx *ctx, const std::string &key, const TuneChoice &c) {
  ctx->tune_cache[key] = c;
  if (ctx->tune_cache_path.empty()) return;
  const std::string tmp = ctx->tune_cache_path + ".tmp";
  {
    std::ofstream out(tmp);
    if (!out) return;
    out << "{\"version\": 1, \"entries\": {\n";
    size_t i = 0;
    for (const auto &kv : ctx->tune_cache) {
      out << "  \"" << kv.first << "\": {\"block\": " << kv.second.block
          << ", \"blocks_per_sm\": " << kv.second.blocks_per_sm << ", \"ms\": " << kv.second.ms
          << "}" << (++i < ctx->tune_cache.size() ? "," : "") << "\n";
    }
    out << "}}\n";
  }
  std::rename(tmp.c_str(), ctx->tune_cache_path.c_str());
}

}  // namespace zmc
