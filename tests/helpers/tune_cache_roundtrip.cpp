// Host-only check of the autotune cache: load a file, add an entry, store,
// reload; prints "key block blocks_per_sm" lines of the final state, then the
// key tune_key forms for a context with known fields ("key: <key>").
#include <cstdio>

#include "zmc_runtime.h"

int main(int argc, char **argv) {
  if (argc < 3) return 2;
  zmc_ctx c;
  c.tune_cache_path = argv[1];
  zmc::tune_cache_load(&c);
  zmc::TuneChoice t;
  t.block = 128;
  t.blocks_per_sm = 3;
  t.ms = 1.5f;
  c.tune_cache_path = argv[2];
  zmc::tune_cache_store(&c, "GPU X|10|2|16|5", t);
  zmc_ctx d;
  d.tune_cache_path = argv[2];
  zmc::tune_cache_load(&d);
  for (const auto &kv : d.tune_cache)
    std::printf("%s %u %u\n", kv.first.c_str(), kv.second.block, kv.second.blocks_per_sm);
  zmc_ctx k;
  k.gpu_name = "GPU X";
  k.sms = 10;
  k.quints_per_lane = 16;
  k.kernel_regs[2] = 115;
  std::printf("key: %s\n", zmc::tune_key(&k, 2, 5).c_str());
  return 0;
}
