// zmc_device.cuh -- device code shared by the sm_103a kernels of multi-function
// direct Monte Carlo (ZMCintegral-v5.1 multi-function mode, arXiv 2104.10073):
// the Philox4x32-10 generator, the uniform -> box map, the per-chunk FP32
// accumulation, and the persistent work-list kernel template.
//
// Each integrand family's sampling path is its own translation unit
// (zmc_fam_<family>.cu): it specialises Eval<FAM, D, G> (the FP32 integrand) and
// dispatch_item / dispatch_eval (variant -> specialised body), then defines its
// FamilyOps from family_ops<FAM>().  Everything here has internal linkage, so a
// kernel is instantiated only in the file of its family.
#pragma once

#include <cstdint>

#include "zmc_internal.h"

// Also compiled at run time by NVRTC for user-defined integrands (zmc_udf.cpp):
// the host-side launch helpers at the end are hidden from it.

namespace zmc {
namespace {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): round multipliers and the
// Weyl increments of the key schedule.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
constexpr unsigned kFullMask = 0xffffffffu;

// Round keys hoisted once per chunk (the key is the integrand's, warp uniform).
struct RoundKeys {
  uint32_t k0[10], k1[10];
};

__device__ __forceinline__ RoundKeys make_round_keys(uint32_t key0, uint32_t key1) {
  RoundKeys rk;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = key0 + static_cast<uint32_t>(r) * kPhiloxW0;
    rk.k1[r] = key1 + static_cast<uint32_t>(r) * kPhiloxW1;
  }
  return rk;
}

// Ten rounds of the 4x32 S-box: two 32x32->64 products, two three-way XORs.
// ZMC_PHILOX_MULHI selects separate high / low multiplies instead of one
// widening multiply per product (same results; a scheduling choice).
#ifndef ZMC_PHILOX_MULHI
#define ZMC_PHILOX_MULHI 0
#endif
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
#if ZMC_PHILOX_MULHI
    const uint32_t hi0 = __umulhi(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
#else
    const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c0;
    const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c2;
    const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
    const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
#endif
    const uint32_t n0 = hi1 ^ c1 ^ rk.k0[r];
    const uint32_t n2 = hi0 ^ c3 ^ rk.k1[r];
    c1 = lo1;
    c3 = lo0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

// The sample stream's counter is (stream_id, block lo, block hi, 0).  Across the
// blocks of one chunk only block lo changes, and it sits in counter word 1, which
// the first round XORs instead of multiplying.  So both products of round 1, the
// second product of round 2 and the first of round 3 are the same for the whole
// chunk: StreamPrefix holds what they contribute, formed once per chunk, and a
// block then costs 16 widening multiplies instead of the 18 that remain when the
// varying word is multiplied in round 1.
struct StreamPrefix {
  uint32_t a;            // round 1: c0' = block lo ^ a
  uint32_t b;            // round 2: c2' = hi(M0 c0) ^ b
  uint32_t c, dk, e;     // round 3: c0' = hi(M1 c2) ^ c, c2' = lo(M0 c0 of round 2) ^ dk, c3' = e
  uint32_t k0[7], k1[7]; // round keys of rounds 4..10
};

__device__ __forceinline__ StreamPrefix make_stream_prefix(const RoundKeys &rk, uint32_t sid,
                                                           uint32_t block_hi) {
  StreamPrefix p;
  const uint64_t r1a = static_cast<uint64_t>(kPhiloxM0) * sid;
  const uint64_t r1b = static_cast<uint64_t>(kPhiloxM1) * block_hi;
  p.a = static_cast<uint32_t>(r1b >> 32) ^ rk.k0[0];
  const uint32_t r2c2 = static_cast<uint32_t>(r1a >> 32) ^ rk.k1[0];  // 0 in counter word 3
  const uint64_t r2b = static_cast<uint64_t>(kPhiloxM1) * r2c2;
  const uint32_t r3c0 = static_cast<uint32_t>(r2b >> 32) ^ static_cast<uint32_t>(r1b) ^ rk.k0[1];
  p.b = static_cast<uint32_t>(r1a) ^ rk.k1[1];
  const uint64_t r3a = static_cast<uint64_t>(kPhiloxM0) * r3c0;
  p.c = static_cast<uint32_t>(r2b) ^ rk.k0[2];
  p.dk = static_cast<uint32_t>(r3a >> 32) ^ rk.k1[2];
  p.e = static_cast<uint32_t>(r3a);
#pragma unroll
  for (int r = 0; r < 7; ++r) {
    p.k0[r] = rk.k0[3 + r];
    p.k1[r] = rk.k1[3 + r];
  }
  return p;
}

// Philox4x32-10 of counter (stream_id, block_lo, block_hi, 0): equal to
// philox(stream_id, block_lo, block_hi, 0, rk) for the prefix made from rk.
__device__ __forceinline__ uint4 philox_block(uint32_t block_lo, const StreamPrefix &p) {
  const uint64_t q0 = static_cast<uint64_t>(kPhiloxM0) * (block_lo ^ p.a);             // round 2
  const uint64_t q1 = static_cast<uint64_t>(kPhiloxM1) * (static_cast<uint32_t>(q0 >> 32) ^ p.b);  // round 3
  uint32_t c0 = static_cast<uint32_t>(q1 >> 32) ^ p.c;
  uint32_t c1 = static_cast<uint32_t>(q1);
  uint32_t c2 = static_cast<uint32_t>(q0) ^ p.dk;
  uint32_t c3 = p.e;
#pragma unroll
  for (int r = 0; r < 7; ++r) {
#if ZMC_PHILOX_MULHI
    const uint32_t hi0 = __umulhi(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
#else
    const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c0;
    const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c2;
    const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
    const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
#endif
    const uint32_t n0 = hi1 ^ c1 ^ p.k0[r];
    const uint32_t n2 = hi0 ^ c3 ^ p.k1[r];
    c1 = lo1;
    c3 = lo0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

// The five 23-bit fields of one Philox block: field k is bits [23k, 23k + 23) of
// the 128-bit output (word 0 least significant), delivered in the low 23 bits
// of f[k]; the bits above are not part of the field, and every consumer masks
// with 0x7FFFFF.  13 of the 128 bits go unused.
__device__ __forceinline__ void block_fields(const uint4 o, uint32_t *f) {
  f[0] = o.x;
  f[1] = __funnelshift_r(o.x, o.y, 23);
  f[2] = __funnelshift_r(o.y, o.z, 14);
  f[3] = o.z >> 5;
  f[4] = __funnelshift_r(o.z, o.w, 28);
}

// The 5*D fields of one quint (5 consecutive samples starting at a multiple of
// 5): sample t, coordinate i is field t*D + i, i.e. field (t*D+i)%5 of Philox
// block quint*D + (t*D+i)/5.
template <int D>
__device__ __forceinline__ void gen_quint(uint64_t quint, uint32_t sid, const RoundKeys &rk,
                                          uint32_t (&r)[5 * D]) {
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const uint64_t b = quint * D + static_cast<uint64_t>(j);
    block_fields(philox(sid, static_cast<uint32_t>(b), static_cast<uint32_t>(b >> 32), 0u, rk),
                 r + 5 * j);
  }
}

// The same fields by way of the chunk prefix, made here for every block (the
// per-sample test path, which thereby checks philox_block for any block hi).
template <int D>
__device__ __forceinline__ void gen_quint_prefixed(uint64_t quint, uint32_t sid,
                                                   const RoundKeys &rk, uint32_t (&r)[5 * D]) {
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const uint64_t b = quint * D + static_cast<uint64_t>(j);
    const StreamPrefix sp = make_stream_prefix(rk, sid, static_cast<uint32_t>(b >> 32));
    block_fields(philox_block(static_cast<uint32_t>(b), sp), r + 5 * j);
  }
}

// The same fields when the caller guarantees that the block index's high word
// is the one the prefix was made for: base_lo is the low word of block quint*D.
template <int D>
__device__ __forceinline__ void gen_quint_fast(uint32_t base_lo, const StreamPrefix &sp,
                                               uint32_t (&r)[5 * D]) {
#pragma unroll
  for (int j = 0; j < D; ++j)
    block_fields(philox_block(base_lo + static_cast<uint32_t>(j), sp), r + 5 * j);
}

// Packed FP32 (sm_100 and later): one instruction issues the operation on both
// halves of a pair, each half rounded exactly as the scalar operation would be.
// The sampling loop is bound by issue slots, so pairs of independent FP32
// operations are issued this way where their operands come in pairs.
#ifndef ZMC_PACKED_F32
#define ZMC_PACKED_F32 1
#endif

__device__ __forceinline__ float unit_v(uint32_t word) {
  // v = 1 + (word & 0x7FFFFF) * 2^-23 in [1, 2), exact: one LOP3.
  return __uint_as_float((word & 0x7FFFFFu) | 0x3F800000u);
}

// ---------------------------------------------------------------- integrands (FP32)
// Eval<FAM, D, G>: load(fn) reads the integrand's FP32 constants from FnDev;
// operator()(r) returns the scaled value f' = S f at the sample whose D 23-bit
// fields are the low 23 bits of r[0..D).  Specialised per family in
// zmc_fam_<family>.cu.  An Eval's last operation is a rounded one (an explicit
// _rn product or an fmaf): a plain product could be contracted into an FMA with
// the sums' f - K, differently in differently unrolled loops, which would make
// the unroll change results.
template <int FAM, int D, int G>
struct Eval;

// An Eval may also provide quint(r, f): the five values of a quint at once (its
// fields r[0 .. 5D)), computed with packed FP32 pairs; equal to f[t] = (*this)(r
// + t D) bit for bit.  eval_quint uses it when present.
template <class T>
struct VoidOf {
  typedef void type;
};
template <class E, class = void>
struct HasQuint {
  static constexpr bool value = false;
};
template <class E>
struct HasQuint<E, typename VoidOf<decltype(&E::quint)>::type> {
  static constexpr bool value = true;
};

template <class E, class = void>
struct PackedSums {
  static constexpr bool value = false;
};
template <class E>
struct PackedSums<E, typename VoidOf<decltype(E::kPackedSums)>::type> {
  static constexpr bool value = E::kPackedSums;
};

template <int D, class E>
__device__ __forceinline__ void eval_quint(const E &ev, const uint32_t (&r)[5 * D],
                                           float (&f)[5]) {
  if constexpr (HasQuint<E>::value && ZMC_PACKED_F32) {
    ev.quint(r, f);
  } else {
#pragma unroll
    for (int t = 0; t < 5; ++t) f[t] = ev(r + t * D);
  }
}

// ---------------------------------------------------------------- one chunk
// One step of Chan's pairwise merge: (n, mean, m2) absorbs (nb, mb, m2b), nb > 0.
// Every operation is an explicit rounded one (no contraction is left to the
// compiler), so the result does not depend on how the code around it is
// unrolled or scheduled.
__device__ __forceinline__ void chan_step(float &n, float &mean, float &m2, float nb, float mb,
                                          float m2b) {
  const float nab = __fadd_rn(n, nb);
  const float delta = __fsub_rn(mb, mean);
  const float wb = __fdiv_rn(nb, nab);
  mean = fmaf(delta, wb, mean);
  m2 = fmaf(__fmul_rn(delta, delta), __fmul_rn(n, wb), __fadd_rn(m2, m2b));
  n = nab;
}

// Chan's pairwise merge of (n, mean, M2) summaries, FP32, down the warp; lane 0
// ends with the warp's summary.
__device__ __forceinline__ void warp_chan_merge(float &n, float &mean, float &m2) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const float nb = __shfl_down_sync(kFullMask, n, off);
    const float mb = __shfl_down_sync(kFullMask, mean, off);
    const float m2b = __shfl_down_sync(kFullMask, m2, off);
    if (nb > 0.0f) {
      chan_step(n, mean, m2, nb, mb, m2b);
    }
  }
}

// FP64 butterfly sum over the warp (every lane ends with the total).
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(kFullMask, v, off);
  return v;
}

// Samples [chunk * 160Q, min(+160Q, N)) of one integrand.  Lane l takes quints
// l, l+32, ..., l+32(Q-1) of the chunk.  Over each block of kBlockQuints of its
// quints it accumulates in FP32
//   s1 = sum f            (each quint summed pairwise first; unshifted, so its
//                          rounding error scales with the values themselves)
//   s2 = sum (f - K)^2    (K = the block's first value, so that s2 does not hold
//                          mean^2 n when the spread is small)
// turns them into (n, mean = s1/n, M2 = s2 - n (mean - K)^2) and merges that into
// the lane's running summary (Chan's pairwise update); the warp then merges the
// 32 lane summaries the same way.
// Quints of one lane unrolled per loop step.  Each family file is compiled once
// per unroll (ZMC_FAM_UNROLL = 1, 2; build.py) into kernels of their own, and the
// autotuner picks one per family.  The loop visits the same samples in the same
// order; results agree within rounding (measured: the unrolled harmonic kernel
// rounds some chunk sums differently, ~1e-7 relative), so a plan's results are
// bit-identical for one choice of unroll.
#ifndef ZMC_FAM_UNROLL
#define ZMC_FAM_UNROLL 1
#endif
template <int FAM>
struct QuintUnroll {
  static constexpr int value = ZMC_FAM_UNROLL;
};
// The exported FamilyOps of a family file, named for its unroll: NAME##U1, NAME##U2.
#define ZMC_PASTE2(a, b) a##b
#define ZMC_PASTE(a, b) ZMC_PASTE2(a, b)
#define ZMC_FAMILY_OPS(name) ZMC_PASTE(name, ZMC_PASTE(U, ZMC_FAM_UNROLL))
// Quints per accumulation block: a lane's shifted sums never span more than
// 5 * kBlockQuints samples, which bounds their rounding error for any chunk length.
constexpr uint32_t kBlockQuints = 13;
template <int FAM, int D, int G, bool FAST>
__device__ __forceinline__ void run_chunk(const FnDev *__restrict__ fn, uint64_t chunk,
                                          uint32_t Q, uint32_t lane) {
  Eval<FAM, D, G> ev;
  ev.load(fn);
  const RoundKeys rk = make_round_keys(fn->key0, fn->key1);
  const uint32_t sid = fn->stream_id;
  const uint64_t chunk_samples = chunk_samples_of(Q);
  const uint64_t s0 = chunk * chunk_samples;
  const uint64_t n_left = fn->n_samples - s0;
  const uint32_t nc = static_cast<uint32_t>(n_left < chunk_samples ? n_left : chunk_samples);
  const uint64_t quint0 = (fn->s_off + s0) / kQuint;  // s_off is a multiple of 5
  const uint64_t block0 = quint0 * D;
  const uint32_t base_lo0 = static_cast<uint32_t>(block0) + lane * D;
  const StreamPrefix sp = make_stream_prefix(rk, sid, static_cast<uint32_t>(block0 >> 32));

  // running (n, mean, M2) of the lane, merged from blocks of kBlockQuints quints
  float n = 0.0f, mean = 0.0f, m2 = 0.0f;
  for (uint32_t jb = 0; jb < Q; jb += kBlockQuints) {
    const uint32_t je = jb + kBlockQuints < Q ? jb + kBlockQuints : Q;
    float K = 0.0f, s1 = 0.0f, s2 = 0.0f;
    // families that ask for it (Eval::kPackedSums) sum full quints in packed
    // pairs: samples (0, 1) and (2, 3) as pairs, 4 alone (the others keep the
    // scalar sums, which need fewer registers)
    constexpr bool kPackedSums = ZMC_PACKED_F32 && PackedSums<Eval<FAM, D, G>>::value;
    float2 s1p = make_float2(0.0f, 0.0f), s2p = make_float2(0.0f, 0.0f), nK2;
    uint32_t cnt = 0;
#pragma unroll QuintUnroll<FAM>::value
    for (uint32_t j = jb; j < je; ++j) {
      const uint32_t ql = lane + 32u * j;
      if (!FAST && kQuint * ql >= nc) break;
      uint32_t r[5 * D];
      if (FAST)
        gen_quint_fast<D>(base_lo0 + 32u * D * j, sp, r);
      else
        gen_quint<D>(quint0 + ql, sid, rk, r);
      float f[5];
      eval_quint<D>(ev, r, f);
      if (j == jb) {
        K = f[0];
        nK2 = make_float2(-K, -K);
      }
      if (FAST && kPackedSums) {
        const float2 f01 = make_float2(f[0], f[1]), f23 = make_float2(f[2], f[3]);
        s1p = __fadd2_rn(s1p, f01);
        s1p = __fadd2_rn(s1p, f23);
        s1 += f[4];
        const float2 d01 = __fadd2_rn(f01, nK2), d23 = __fadd2_rn(f23, nK2);
        s2p = __ffma2_rn(d01, d01, s2p);
        s2p = __ffma2_rn(d23, d23, s2p);
        const float d4 = f[4] - K;
        s2 = fmaf(d4, d4, s2);
      } else if (FAST) {
        s1 += ((f[0] + f[1]) + (f[2] + f[3])) + f[4];
#pragma unroll
        for (int t = 0; t < 5; ++t) {
          const float dlt = f[t] - K;
          s2 = fmaf(dlt, dlt, s2);
        }
      } else {
        float q[5];
#pragma unroll
        for (int t = 0; t < 5; ++t) {
          const bool ok = kQuint * ql + t < nc;
          q[t] = ok ? f[t] : 0.0f;
          const float dlt = ok ? f[t] - K : 0.0f;
          s2 = fmaf(dlt, dlt, s2);
          cnt += ok ? 1u : 0u;
        }
        s1 += ((q[0] + q[1]) + (q[2] + q[3])) + q[4];
      }
    }
    if (FAST && kPackedSums) {
      s1 += s1p.x + s1p.y;
      s2 += s2p.x + s2p.y;
    }
    const float nb = FAST ? static_cast<float>(kQuint * (je - jb)) : static_cast<float>(cnt);
    if (nb > 0.0f) {
      const float mb = __fdiv_rn(s1, nb);
      const float dk = __fsub_rn(mb, K);
      const float m2b = fmaxf(fmaf(__fmul_rn(-nb, dk), dk, s2), 0.0f);
      chan_step(n, mean, m2, nb, mb, m2b);
    }
    if (!FAST && cnt < kQuint * (je - jb)) break;
  }
  warp_chan_merge(n, mean, m2);
  if (lane == 0) fn->rec[chunk] = make_float2(mean, m2);
}

template <int FAM, int D, int G>
__device__ __forceinline__ void run_item(const FnDev *__restrict__ fn, uint64_t chunk,
                                         uint32_t Q, uint32_t lane) {
  const uint64_t chunk_samples = chunk_samples_of(Q);
  const uint64_t s0 = chunk * chunk_samples;
  const bool full = fn->n_samples - s0 >= chunk_samples;
  const uint64_t b_first = ((fn->s_off + s0) / kQuint) * D;
  const uint64_t b_last = b_first + (chunk_samples / kQuint) * D - 1;
  if (full && (b_first >> 32) == (b_last >> 32))
    run_chunk<FAM, D, G, true>(fn, chunk, Q, lane);
  else
    run_chunk<FAM, D, G, false>(fn, chunk, Q, lane);
}

// Variant lists (family, dimension, polynomial degree or Gaussian form).
#define ZMC_VARIANTS_DIM(X, F, G) X(F, 1, G) X(F, 2, G) X(F, 3, G) X(F, 4, G) X(F, 5, G) \
  X(F, 6, G) X(F, 7, G)
#define ZMC_HARMONIC_VARIANTS(X) ZMC_VARIANTS_DIM(X, ZMC_HARMONIC, 0)
// harmonic rows whose dimensions all advance the phase at the same rate (G = 1)
#define ZMC_HARMONIC_EQUAL_VARIANTS(X) X(ZMC_HARMONIC, 2, 1) X(ZMC_HARMONIC, 3, 1) \
  X(ZMC_HARMONIC, 4, 1) X(ZMC_HARMONIC, 5, 1) X(ZMC_HARMONIC, 6, 1) X(ZMC_HARMONIC, 7, 1)
#define ZMC_ABSLIN_VARIANTS(X) ZMC_VARIANTS_DIM(X, ZMC_ABSLIN, 0)
#define ZMC_POLY_VARIANTS(X)                                                         \
  ZMC_VARIANTS_DIM(X, ZMC_POLY, 0) ZMC_VARIANTS_DIM(X, ZMC_POLY, 1)                  \
  ZMC_VARIANTS_DIM(X, ZMC_POLY, 2) ZMC_VARIANTS_DIM(X, ZMC_POLY, 3)                  \
  ZMC_VARIANTS_DIM(X, ZMC_POLY, 4)
#define ZMC_GAUSS_VARIANTS(X) ZMC_VARIANTS_DIM(X, ZMC_GAUSS, 0) ZMC_VARIANTS_DIM(X, ZMC_GAUSS, 1)
// switch cases of dispatch_item / dispatch_eval
#define ZMC_ITEM_CASE(F, D, G) \
  case variant_code(F, D, G): run_item<F, D, G>(fn, chunk, Q, lane); break;
#define ZMC_EVAL_CASE(F, D, G) \
  case variant_code(F, D, G): eval_range<F, D, G>(fn, s_begin, count, out); break;

__device__ __forceinline__ uint32_t find_entry(const Entry *__restrict__ entries, uint32_t ne,
                                               uint64_t item, uint32_t hint) {
  if (hint < ne && entries[hint].item_begin <= item &&
      (hint + 1 == ne || entries[hint + 1].item_begin > item))
    return hint;
  uint32_t lo = 0, hi = ne;  // invariant: entries[lo].item_begin <= item < entries[hi]
  if (hint < ne && entries[hint].item_begin <= item) lo = hint;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (entries[mid].item_begin <= item)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// One work item (chunk) of an integrand of family FAM: switch on its variant to
// the specialised run_item.  Specialised per family.
template <int FAM>
__device__ void dispatch_item(const FnDev *fn, uint64_t chunk, uint32_t Q, uint32_t lane);

// Persistent, one kernel per family (so each gets the register budget of its own
// variants): each warp takes the next work item of its family from a global
// counter until the family's items run out; an item is one chunk of one
// integrand.  Items are grouped by variant so co-resident warps mostly run the
// same code.
// Resident 256-thread blocks per SM each family kernel is compiled for (it caps
// registers at 65536 / (256 * n)); overridable per family at build time.
#ifndef ZMC_MIN_BLOCKS_HARMONIC
#define ZMC_MIN_BLOCKS_HARMONIC 2
#endif
#ifndef ZMC_MIN_BLOCKS_ABSLIN
#define ZMC_MIN_BLOCKS_ABSLIN 2
#endif
#ifndef ZMC_MIN_BLOCKS_GAUSS
#define ZMC_MIN_BLOCKS_GAUSS 2
#endif
#ifndef ZMC_MIN_BLOCKS_POLY
#define ZMC_MIN_BLOCKS_POLY 2
#endif
template <int FAM>
struct MinBlocks {
  static constexpr int value = FAM == ZMC_HARMONIC ? ZMC_MIN_BLOCKS_HARMONIC
                               : FAM == ZMC_ABSLIN ? ZMC_MIN_BLOCKS_ABSLIN
                               : FAM == ZMC_GAUSS  ? ZMC_MIN_BLOCKS_GAUSS
                                                   : ZMC_MIN_BLOCKS_POLY;
};
// Registers per thread each family kernel is capped at (__maxnreg__, which
// cannot be combined with __launch_bounds__; the kernels are launched with 128 or
// 256 threads): by default what ZMC_MIN_BLOCKS_<FAMILY> 256-thread blocks per SM
// leave; overridable per family, e.g. to fit more 128-thread blocks.
#ifndef ZMC_MAXNREG_HARMONIC
#define ZMC_MAXNREG_HARMONIC (65536 / (256 * ZMC_MIN_BLOCKS_HARMONIC))
#endif
#ifndef ZMC_MAXNREG_ABSLIN
#define ZMC_MAXNREG_ABSLIN (65536 / (256 * ZMC_MIN_BLOCKS_ABSLIN))
#endif
#ifndef ZMC_MAXNREG_GAUSS
#define ZMC_MAXNREG_GAUSS (65536 / (256 * ZMC_MIN_BLOCKS_GAUSS))
#endif
#ifndef ZMC_MAXNREG_POLY
#define ZMC_MAXNREG_POLY (65536 / (256 * ZMC_MIN_BLOCKS_POLY))
#endif
template <int FAM>
struct MaxRegs {
  static constexpr int value = FAM == ZMC_HARMONIC ? ZMC_MAXNREG_HARMONIC
                               : FAM == ZMC_ABSLIN ? ZMC_MAXNREG_ABSLIN
                               : FAM == ZMC_GAUSS  ? ZMC_MAXNREG_GAUSS
                                                   : ZMC_MAXNREG_POLY;
};

// The LaunchHdr slot a family's kernel drains: its own for the built-in
// families, slot 0 of a launch of its own for a user-defined integrand.
template <int FAM>
struct HdrSlot {
  static constexpr int value = FAM < 4 ? FAM : 0;
};

template <int FAM>
__device__ __forceinline__ void batched_loop(const Entry *__restrict__ entries,
                                             LaunchHdr *__restrict__ hdr) {
  constexpr int kSlot = HdrSlot<FAM>::value;
  const uint32_t lane = threadIdx.x & 31u;
  const unsigned long long begin = hdr->item_begin[kSlot];
  const unsigned long long count = hdr->item_end[kSlot] - begin;
  const uint32_t ne = hdr->n_entries;
  const uint32_t Q = hdr->quints_per_lane;
  uint32_t e = 0;
  for (;;) {
    unsigned long long k = 0;
    if (lane == 0) k = atomicAdd(&hdr->counter[kSlot], 1ull);
    k = __shfl_sync(kFullMask, k, 0);
    if (k >= count) break;
    const uint64_t item = begin + k;
    e = find_entry(entries, ne, item, e);
    const Entry en = entries[e];
    dispatch_item<FAM>(en.fn, en.chunk_begin + (item - en.item_begin), Q, lane);
  }
}

template <int FAM>
__global__ void __maxnreg__(MaxRegs<FAM>::value)
    zmc_batched_kernel(const Entry *__restrict__ entries, LaunchHdr *__restrict__ hdr) {
  batched_loop<FAM>(entries, hdr);
}

// ---------------------------------------------------------------- per-sample values
// The scaled-back values f of samples [s_begin, s_begin + count) of one integrand,
// from the same generator and Eval as the sampling path (parity tests).
template <int FAM, int D, int G>
__device__ __forceinline__ void eval_range(const FnDev *fn, uint64_t s_begin, uint32_t count,
                                           float *out) {
  Eval<FAM, D, G> ev;
  ev.load(fn);
  const RoundKeys rk = make_round_keys(fn->key0, fn->key1);
  const uint64_t q_first = s_begin / kQuint;
  const uint64_t q_last = (s_begin + count - 1) / kQuint;
  for (uint64_t q = q_first + blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
       q <= q_last; q += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    uint32_t r[5 * D];
    gen_quint_prefixed<D>(q, fn->stream_id, rk, r);
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const uint64_t s = kQuint * q + t;
      if (s >= s_begin && s < s_begin + count)
        out[s - s_begin] = static_cast<float>(static_cast<double>(ev(r + t * D)) * fn->inv_scale);
    }
  }
}

template <int FAM>
__device__ void dispatch_eval(const FnDev *fn, uint64_t s_begin, uint32_t count, float *out);

template <int FAM>
__global__ void zmc_eval_kernel(const FnDev *__restrict__ fn, uint64_t s_begin, uint32_t count,
                                float *__restrict__ out) {
  dispatch_eval<FAM>(fn, s_begin, count, out);
}

#ifndef __CUDACC_RTC__
// ---------------------------------------------------------------- host side of a family
template <int FAM>
cudaError_t launch_batched_family(const Entry *entries, LaunchHdr *hdr, unsigned grid,
                                  unsigned block, cudaStream_t stream) {
  zmc_batched_kernel<FAM><<<grid, block, 0, stream>>>(entries, hdr);
  return cudaGetLastError();
}

template <int FAM>
int max_blocks_family(int block) {
  int n = 0;
  const cudaError_t err =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, zmc_batched_kernel<FAM>, block, 0);
  return err == cudaSuccess ? n : 0;
}

template <int FAM>
int regs_family() {
  cudaFuncAttributes a{};
  return cudaFuncGetAttributes(&a, zmc_batched_kernel<FAM>) == cudaSuccess ? a.numRegs : 0;
}

template <int FAM>
cudaError_t launch_eval_family(const FnDev *fn, uint64_t s_begin, uint32_t count, float *out,
                               cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  const uint64_t quints = (s_begin + count - 1) / kQuint - s_begin / kQuint + 1;
  const uint64_t blocks = (quints + 255) / 256;
  zmc_eval_kernel<FAM><<<static_cast<unsigned>(blocks < 1024 ? blocks : 1024), 256, 0, stream>>>(
      fn, s_begin, count, out);
  return cudaGetLastError();
}

template <int FAM>
constexpr FamilyOps family_ops() {
  return FamilyOps{&launch_batched_family<FAM>, &max_blocks_family<FAM>,
                   &launch_eval_family<FAM>, &regs_family<FAM>};
}

#endif  // __CUDACC_RTC__

}  // namespace
}  // namespace zmc
