// Internal device-side layouts of the GB300 multi-function Monte Carlo path.
//
// The host runtime (zmc_runtime.cpp) turns each public zmc_desc into one FnDev
// (FP32 evaluation constants derived in FP64) and the kernels (zmc_kernels.cu,
// zmc_fam_<family>.cu, zmc_plain.cu) read only FnDev, Entry, LaunchHdr and the
// plain form's PlainFn / PlainJob.  Nothing here is part of the C ABI.
#pragma once

// This header is also compiled at run time by NVRTC for user-defined integrands
// (zmc_udf.cpp supplies minimal <cstdint>, <cstddef> and <cuda_runtime.h>);
// host-only declarations are hidden from it.
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "zmc.h"

namespace zmc {

constexpr int kMaxDim = 7;
constexpr int kWarp = 32;

// A lane's unit of work is a quint: 5 consecutive samples (starting at a multiple
// of 5) whose 5 D coordinates are the 5 D 23-bit fields of D Philox blocks (five
// fields per 128-bit block).  A chunk is 32 lanes x quints_per_lane quints.
constexpr uint32_t kQuint = 5;
__host__ __device__ constexpr uint64_t chunk_samples_of(uint32_t quints_per_lane) {
  return 32ull * kQuint * quints_per_lane;
}

// Variant code: dimension in bits 0..3 (1..12), family in bits 4..6, and in
// bits 8 and up the polynomial's variant degree (0..7) or the index of a user
// function in its module (0..63).  The sampling kernel dispatches one
// specialised body per variant.
__host__ __device__ constexpr uint32_t variant_code(uint32_t family, uint32_t dim,
                                                    uint32_t deg) {
  return (deg << 8) | (family << 4) | dim;
}

// One integrand as the sampling kernel sees it (384 bytes, 16-byte aligned).
//
// Every family's amplitude carries a power-of-two scale S (chosen on the host so
// that S times an upper bound of |f| over the box is ~2^48): the kernel sums the
// scaled values f' = S f, whose squares stay inside FP32 range for values down
// to 2^-111 of that bound, and the FP64 merge multiplies by inv_scale = 1/S
// (exact).
//
// Payload words w[] by family (FP32 unless noted; "hi/lo" pairs are an FP64
// constant split as hi = fl32(c), lo = fl32(c - hi), so that FMA chains over
// both halves carry the constant to ~2^-48 relative).  m_i = word & 0x7FFFFF is
// the 23-bit sample integer of coordinate i, u_i = m_i 2^-23, v_i = 1 + u_i.
//   HARMONIC  f = S R cos(2 pi P), P = k.x/(2 pi) - atan2(b, a)/(2 pi) in turns,
//             R = sqrt(a^2 + b^2); T_i = k_i (hi_i-lo_i)/(2 pi) 2^41 (turns per
//             unit of m_i, in units of 2^-64 turn): high word at w[i] (u32),
//             fl32(low word / 2^32) at w[7+i], fl32(2^23 - w[7+i] 2^23) at w[14+i];
//             P0 (u32, units of 2^-32 turn, minus the folded 2^23 offsets) w[21];
//             S R at w[22].  Variant degree 1 (D >= 2, every T_i equal to T): T's
//             high word at w[0], its low word (u32) at w[1], P0 + 2^-33 turn to
//             2^-64 turn (no offsets): high word w[21], low word w[2].
//   ABSLIN    s = c.x in units of 2^-F (F per integrand, host-chosen):
//             s 2^F = G0 + sum_i G_i vb_i + L, vb_i = 0x4B000000 + m_i, exact in
//             64-bit integers (modulo 2^64) plus L = l0 + sum_i g_i fl(2^23 + m_i)
//             in FP32: G_i (s32) at w[i], g_i (FP32, |g_i| <= 1/2) at w[7+i],
//             G0 (u64) at w[14] (lo), w[15] (hi), l0 at w[16], S a 2^-F at w[17].
//             Variant degree 1 (rows of >= 256 samples): the same with F such that
//             |c.x| 2^F <= 2^29 on the box, the integer sum taken modulo 2^32.
//   GAUSS     t_i = (x_i - mu_i) beta, beta = sqrt(log2(e) / 2) / sigma, so that
//             f = A 2^(-sum t_i^2);  h_i = (hi_i - lo_i) beta: hi w[i], lo w[7+i];
//             S A w[28].  Variant degree 0 ("near": mu_i / box position within
//             [-1, 2] box widths in every dimension): t_i = h_i (v_i - 1 - u0_i) + c0_i
//             with u0_i the position rounded to a multiple of 2^-22 and 1 + u0_i
//             stored (w[14+i], exact), so v_i - (1 + u0_i) is exact, and
//             c0_i = -h_i (position - u0_i) (w[21+i]).
//             Variant degree 1 ("far"): t_i = e_i + h_i u_i, e_i = (lo_i - mu_i) beta:
//             hi w[14+i], lo w[21+i].
//   POLY      factor i re-expanded in u_i in [0, 1): q_i(u) = sum_j e_ij u^j;
//             e_ij hi at w[5i+j], lo at w[35+5i+j] (factor 0 carries S).
struct alignas(16) FnDev {
  uint32_t variant;
  uint32_t stream_id;
  uint32_t key0, key1;
  uint64_t n_samples;
  float2 *rec;        // chunk records (mean', M2') of this integrand, one per chunk
  zmc_result *out;    // result row written by the merge kernel
  double volume;      // prod (hi_i - lo_i), FP64
  double inv_scale;   // 1 / S (a power of two)
  uint64_t s_off;     // absolute index of sample 0 (a multiple of 5): sample s of
                      // this descriptor is sample s_off + s of the Philox stream
  uint32_t w[72];
  // Moments (unscaled) of samples taken before this descriptor's, e.g. a
  // checkpoint of the same stream; the merge combines them with this
  // descriptor's samples (Chan).  prior_n = 0: none.
  uint64_t prior_n;
  double prior_mean;
  double prior_m2;
  uint32_t out_mode;  // merge output: 0 zmc_result (estimate, stderr), 1 zmc_moments
  uint32_t reserved;
};
static_assert(sizeof(FnDev) == 384, "FnDev layout");

// A contiguous run of chunks of one integrand inside one persistent launch.
struct Entry {
  uint64_t item_begin;   // first work-item index of this run in the launch
  const FnDev *fn;
  uint64_t chunk_begin;  // first chunk of the integrand covered by this run
};
static_assert(sizeof(Entry) == 24, "Entry layout");

// Per-launch header, device resident so that a captured graph can be replayed
// with new contents.  The work items of a launch are ordered by family; family f
// owns items [item_begin[f], item_end[f]) and is drained by its own persistent
// kernel through counter[f].
struct LaunchHdr {
  unsigned long long counter[4];     // per-family item dispensers (zeroed before a launch)
  unsigned long long item_begin[4];
  unsigned long long item_end[4];
  uint32_t n_entries;
  uint32_t n_merge;                  // integrands to merge after this launch
  uint32_t quints_per_lane;          // chunk = 160 * quints_per_lane samples
  uint32_t pad;
};

// FP64 descriptor of the plain per-integrand kernel (passed by value).
struct PlainFn {
  uint32_t family, dim, stream_id, deg;
  uint32_t key0, key1;
  uint64_t n_samples;
  double lo[kMaxDim];
  double w[kMaxDim];
  double p[ZMC_NPARAM];
};

// Plain-form merge job (one per integrand): its per-block (n, mean, M2) records.
struct PlainJob {
  const double *rec;
  uint32_t nblk;
  uint32_t pad;
  double volume;
  zmc_result *out;
};

#ifndef __CUDACC_RTC__
// The sampling path of one integrand family, defined in zmc_fam_<family>.cu.
struct FamilyOps {
  cudaError_t (*launch_batched)(const Entry *entries, LaunchHdr *hdr, unsigned grid,
                                unsigned block, cudaStream_t stream);
  int (*max_blocks_per_sm)(int block);  // resident blocks of `block` threads per SM
  cudaError_t (*launch_eval)(const FnDev *fn, uint64_t s_begin, uint32_t count, float *out,
                             cudaStream_t stream);
  int (*regs_per_thread)();  // registers of the family kernel as built (0 if unknown)
};
// Each family file is built once per quint-loop unroll (1 or 2): U1 and U2.
extern const FamilyOps kFamilyHarmonicU1, kFamilyAbslinU1, kFamilyGaussU1, kFamilyPolyU1;
extern const FamilyOps kFamilyHarmonicU2, kFamilyAbslinU2, kFamilyGaussU2, kFamilyPolyU2;
constexpr int kMaxUnroll = 2;

// Launch wrappers (zmc_kernels.cu, zmc_plain.cu).  All return the launch's
// cudaError_t; an unknown family or unroll gives cudaErrorInvalidValue.
cudaError_t launch_batched(int family, const Entry *entries, LaunchHdr *hdr, unsigned grid,
                           unsigned block, cudaStream_t stream, int unroll = 1);
cudaError_t launch_merge(const FnDev *const *fns, const LaunchHdr *hdr, unsigned grid,
                         cudaStream_t stream);
cudaError_t launch_plain(const PlainFn &fn, double *block_rec, unsigned grid,
                         cudaStream_t stream);
cudaError_t launch_plain_merge(const PlainJob *jobs, uint32_t n, cudaStream_t stream);
cudaError_t launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, size_t n,
                          cudaStream_t stream);
cudaError_t launch_eval(int family, const FnDev *fn, uint64_t s_begin, uint32_t count,
                        float *out, cudaStream_t stream);
int batched_max_blocks_per_sm(int family, int block, int unroll = 1);
int batched_regs_per_thread(int family, int unroll = 1);
unsigned plain_grid(const PlainFn &fn, int sms);
#endif  // __CUDACC_RTC__

}  // namespace zmc
