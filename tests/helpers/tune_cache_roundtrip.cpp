// Host-only check of the autotune cache: load a file, add a geometry entry and
// a chunk entry, store, reload; prints "key block blocks_per_sm" for geometry
// entries and "key q<quints> u<u0><u1><u2><u3>" for chunk entries of the final
// state, then the key tune_key forms for a context with known fields
// ("key: <key>").
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
  zmc::tune_cache_store(&c, "GPU X|10|2|q16|u1|5|r115", t);
  zmc::TuneChoice q;
  q.quints = 52;
  q.unroll[1] = 2;
  q.ms = 3.25f;
  zmc::tune_cache_store(&c, "chunk|GPU X|10|m5", q);
  zmc_ctx d;
  d.tune_cache_path = argv[2];
  zmc::tune_cache_load(&d);
  for (const auto &kv : d.tune_cache) {
    const zmc::TuneChoice &e = kv.second;
    if (e.quints)
      std::printf("%s q%u u%u%u%u%u\n", kv.first.c_str(), e.quints, e.unroll[0], e.unroll[1],
                  e.unroll[2], e.unroll[3]);
    else
      std::printf("%s %u %u\n", kv.first.c_str(), e.block, e.blocks_per_sm);
  }
  zmc_ctx k;
  k.gpu_name = "GPU X";
  k.sms = 10;
  k.kernel_regs[1][2] = 115;
  std::printf("key: %s\n", zmc::tune_key(&k, 2, 5, 16, 2).c_str());
  return 0;
}
