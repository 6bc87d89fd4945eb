// zmc_tune.cpp -- the autotuner's cache, stored as JSON: launch geometry
// (threads per block, resident blocks per SM) chosen per family kernel, and the
// chunk length and per-family quint-loop unroll chosen per table shape class.
//
// The geometry decides only which warp runs which work item, never what an
// item computes.  The chunk length changes how samples are grouped before the
// FP64 merge, and the unroll how the compiler lays out a lane's loop; both
// change results within rounding only, and results are bit-identical for one
// choice.  Geometry keys name what the
// best geometry can depend on: the GPU model and SM count, the family, the chunk
// length (quints per lane), the unroll, the dominant dimension of the family's
// samples and the family kernel's registers per thread (its build).  Chunk keys
// (zmc_runtime.cpp, chunk_tune_key) name the GPU, the families present with
// their dominant dimensions and kernels' registers, and the table's size class.
//
// File format (written by this file only):
//   {"version": 2, "entries": {
//     "<gpu>|<sms>|<family>|q<quints>|u<unroll>|<dim>|r<regs>":
//         {"block": 256, "blocks_per_sm": 2, "ms": 0.512},
//     "chunk|<gpu>|<sms>|...": {"quints": 104, "unroll": [1, 2, 1, 1], "ms": 3.1},
//     ...}}
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>

#include "zmc_runtime.h"

namespace zmc {

std::string tune_key(const zmc_ctx *ctx, int family, int dim, uint32_t quints, int unroll) {
  std::ostringstream k;
  // the kernel's register count stands for its build: a rebuild with other
  // launch-bound knobs is timed afresh instead of reusing another build's choice
  k << ctx->gpu_name << '|' << ctx->sms << '|' << family << "|q" << quints << "|u" << unroll
    << '|' << dim << "|r" << ctx->kernel_regs[unroll - 1][family];
  return k.str();
}

namespace {

// The unsigned number after "name": in body, if present.
bool field_u(const std::string &body, const char *name, unsigned *out) {
  const size_t p = body.find(std::string("\"") + name + "\"");
  if (p == std::string::npos) return false;
  const size_t c = body.find(':', p);
  return c != std::string::npos && std::sscanf(body.c_str() + c + 1, " %u", out) == 1;
}

}  // namespace

void tune_cache_load(zmc_ctx *ctx) {
  ctx->tune_cache.clear();
  if (ctx->tune_cache_path.empty()) return;
  std::ifstream in(ctx->tune_cache_path);
  if (!in) return;
  std::stringstream ss;
  ss << in.rdbuf();
  const std::string s = ss.str();
  // entries look like "key": {"block": B, "blocks_per_sm": N, "ms": T} or
  // "key": {"quints": Q, "unroll": [u0, u1, u2, u3], "ms": T}
  if (s.find("\"version\": 2") == std::string::npos) return;  // older format: retune
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
    TuneChoice c;
    const size_t pm = body.find("\"ms\"");
    if (pm != std::string::npos) std::sscanf(body.c_str() + body.find(':', pm) + 1, "%f", &c.ms);
    unsigned block = 0, bps = 0, quints = 0;
    if (field_u(body, "quints", &quints)) {
      const size_t pu = body.find("\"unroll\"");
      const size_t lb = pu == std::string::npos ? pu : body.find('[', pu);
      unsigned u[4] = {0, 0, 0, 0};
      bool ok = lb != std::string::npos &&
                std::sscanf(body.c_str() + lb + 1, " %u , %u , %u , %u", &u[0], &u[1], &u[2],
                            &u[3]) == 4;
      for (unsigned x : u) ok = ok && x >= 1 && x <= static_cast<unsigned>(kMaxUnroll);
      bool known = false;
      for (uint32_t q : kTuneQuints) known = known || q == quints;
      if (ok && known) {
        c.quints = quints;
        for (int f = 0; f < 4; ++f) c.unroll[f] = u[f];
        ctx->tune_cache[key] = c;
      }
    } else if (field_u(body, "block", &block) && field_u(body, "blocks_per_sm", &bps)) {
      if ((block == 128 || block == 256) && bps >= 1 && bps <= 16) {
        c.block = block;
        c.blocks_per_sm = bps;
        ctx->tune_cache[key] = c;
      }
    }
    // a chunk entry's body holds a [...] list: continue after the entry's '}'
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
    out << "{\"version\": 2, \"entries\": {\n";
    size_t i = 0;
    for (const auto &kv : ctx->tune_cache) {
      const TuneChoice &t = kv.second;
      out << "  \"" << kv.first << "\": {";
      if (t.quints)
        out << "\"quints\": " << t.quints << ", \"unroll\": [" << t.unroll[0] << ", "
            << t.unroll[1] << ", " << t.unroll[2] << ", " << t.unroll[3] << "]";
      else
        out << "\"block\": " << t.block << ", \"blocks_per_sm\": " << t.blocks_per_sm;
      out << ", \"ms\": " << t.ms << "}" << (++i < ctx->tune_cache.size() ? "," : "") << "\n";
    }
    out << "}}\n";
  }
  std::rename(tmp.c_str(), ctx->tune_cache_path.c_str());
}

}  // namespace zmc
