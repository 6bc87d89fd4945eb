// zmc_kernels.cu -- sm_103a kernels of multi-function direct Monte Carlo
// (ZMCintegral-v5.1 multi-function mode, arXiv 2104.10073).
//
//   zmc_batched_kernel   persistent work-list launch over (integrand, chunk) items:
//                        Philox4x32-10 -> map onto the box -> FP32 integrand ->
//                        per-lane shifted sums -> warp Chan merge -> one (mean, M2)
//                        record per chunk.  Direct MC per integrand is the paper's
//                        solution method (Sec. "Solution method"); many integrands
//                        of different form, dimension and box share one launch
//                        (Sec. "Summary of revisions", Eq. 1, Eq. 2).
//   zmc_merge_kernel     FP64 k-way Chan merge of an integrand's chunk records in a
//                        fixed order: mean, M2, estimate = V mean,
//                        stderr = V sqrt(M2 / (N (N-1))) (Fig. 1 caption: an estimate
//                        with its spread).
//   zmc_plain_fp64_kernel  one launch per integrand, FP64 map and evaluation with the
//                        CUDA math library, FP64 block reduction (the plain form).
//   zmc_philox_kernel, zmc_eval_kernel   the generator and the per-sample integrand
//                        values of the sampling path, exposed for parity tests.
//
// No tensor cores and no TMA: the path is integer and FP32 arithmetic on the FMA,
// ALU and MUFU pipes, with a few KB of descriptor reads and 8 bytes written per
// 128 * quads_per_lane samples.
#include <cstdint>

#include "zmc_internal.h"
#include "zmc_coeffs.h"

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

// The 4*D words of one quad (4 consecutive samples starting at a multiple of 4):
// sample t, coordinate i is word t*D + i, i.e. lane (t*D+i)%4 of Philox block
// quad*D + (t*D+i)/4.  FAST: the caller guarantees the block index's high word is
// the same for the whole chunk, so only the low word advances.
template <int D, bool FAST>
__device__ __forceinline__ void gen_quad(uint64_t quad, uint32_t base_lo, uint32_t base_hi,
                                         uint32_t sid, const RoundKeys &rk, uint32_t (&r)[4 * D]) {
#pragma unroll
  for (int j = 0; j < D; ++j) {
    uint32_t lo, hi;
    if (FAST) {
      lo = base_lo + static_cast<uint32_t>(j);
      hi = base_hi;
    } else {
      const uint64_t b = quad * D + static_cast<uint64_t>(j);
      lo = static_cast<uint32_t>(b);
      hi = static_cast<uint32_t>(b >> 32);
    }
    const uint4 o = philox(lo, hi, sid, 0u, rk);
    r[4 * j + 0] = o.x;
    r[4 * j + 1] = o.y;
    r[4 * j + 2] = o.z;
    r[4 * j + 3] = o.w;
  }
}

__device__ __forceinline__ float unit_v(uint32_t word) {
  // v = 1 + (word & 0x7FFFFF) * 2^-23 in [1, 2), exact: one LOP3.
  return __uint_as_float((word & 0x7FFFFFu) | 0x3F800000u);
}

// amp 2^-(zh + zl) for zh >= 0, |zl| << 1: the MUFU exponential of the exact
// FP32 input -zh (measured on this part: relative error <= 1.5e-7, mean -5e-8 over
// [-24, 0]), times the first-order correction (1 - ln2 zl).  Values below 2^-126
// flush to zero.
__device__ __forceinline__ float amp_exp2_neg(float amp, float zh, float zl) {
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-zh));
  const float ae = amp * e;
  return fmaf(ae, -0.69314718055994531f * zl, ae);
}

// ---------------------------------------------------------------- integrands (FP32)
template <int FAM, int D, int G>
struct Eval;

// a cos(k.x) + b sin(k.x) (Eq. 1) = R cos(2 pi P), R = sqrt(a^2 + b^2), with the
// phase P in turns = k.x / (2 pi) - atan2(b, a) / (2 pi).  P's fraction is kept
// as a 32-bit fixed-point number (units of 2^-32 turn), formed from the 23-bit
// sample integers m_i: P = P0 + sum_i [T_hi,i m_i + round(T_lo,i m_i / 2^32)],
// where T_i = k_i (hi_i - lo_i) / (2 pi) 2^41 is split into its high and low
// 32-bit words.  The high-word products wrap modulo 1 turn exactly (one 32-bit
// multiply-add each); the low-word contribution (< 2^23 units) is formed by one
// FP32 FMA from v' = 2^23 + m_i, whose rounding and the dropped carries cost at
// most D units of 2^-32 turn.  So |k.x| of any size costs no accuracy.  Then
// cos(2 pi x) = sin(2 pi (1/4 - |x|)), evaluated as t P(t^2) with a degree-5
// polynomial P.
template <int D, int G>
struct Eval<ZMC_HARMONIC, D, G> {
  uint32_t thi[D];
  float tlo[D], kc[D];
  uint32_t p0;
  float R;
  __device__ __forceinline__ void load(const FnDev *fn) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      thi[i] = fn->w[i];
      tlo[i] = __uint_as_float(fn->w[7 + i]);
      kc[i] = __uint_as_float(fn->w[14 + i]);
    }
    p0 = fn->w[21];
    R = __uint_as_float(fn->w[22]);
  }
  __device__ __forceinline__ float operator()(const uint32_t *r) const {
    uint32_t acc = p0, lows = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const uint32_t vb = (r[i] & 0x7FFFFFu) | 0x4B000000u;  // bits of 2^23 + m_i
      const float c = fmaf(tlo[i], __uint_as_float(vb), kc[i]);
      acc = thi[i] * vb + acc;
      lows += __float_as_uint(c);  // the host folds the 0x4B000000 offsets into p0
    }
    acc += lows;
    // x = acc / 2^32 in [-1/2, 1/2) turn; cos(2 pi x) = sin(2 pi y) with
    // y = 1/4 - |x| in [-1/4, 1/4], formed exactly in the integer (two's-complement
    // wrap makes x = -1/2 come out right) and converted with full relative
    // precision, so the value keeps its relative accuracy near the zeros.
    const uint32_t sgn = static_cast<uint32_t>(static_cast<int32_t>(acc) >> 31);
    const uint32_t ax = (acc ^ sgn) - sgn;
    const int32_t y = static_cast<int32_t>(0x40000000u - ax);
    const float t = __int2float_rn(y) * 0x1p-32f;
    const float z = t * t;
    float p = fmaf(ZMC_SINQ_C5, z, ZMC_SINQ_C4);
    p = fmaf(p, z, ZMC_SINQ_C3);
    p = fmaf(p, z, ZMC_SINQ_C2);
    p = fmaf(p, z, ZMC_SINQ_C1);
    p = fmaf(p, z, ZMC_SINQ_C0);
    return (R * t) * p;
  }
};

// a |c.x| (Eq. 2), as a |C + sum g_i v_i|: the g_i are FP32 roundings of FP64
// constants; C carries the FP64 C plus the mean over the box of the dropped
// low parts (sum (g_i - fl(g_i)) * 3/2), which removes their systematic effect.
template <int D, int G>
struct Eval<ZMC_ABSLIN, D, G> {
  float g[D];
  float ch, cl, a;
  __device__ __forceinline__ void load(const FnDev *fn) {
#pragma unroll
    for (int i = 0; i < D; ++i) g[i] = __uint_as_float(fn->w[i]);
    ch = __uint_as_float(fn->w[14]);
    cl = __uint_as_float(fn->w[15]);
    a = __uint_as_float(fn->w[16]);
  }
  __device__ __forceinline__ float operator()(const uint32_t *r) const {
    float sh = ch;
#pragma unroll
    for (int i = 0; i < D; ++i) sh = fmaf(g[i], unit_v(r[i]), sh);
    return a * fabsf(sh + cl);
  }
};

// A exp(-|x-mu|^2 / (2 sigma^2)) = A 2^(-Z), Z = sum_i t_i^2.  FP32 carries a
// relative error of ~2^-24 Z in a plainly summed Z, i.e. ~Z 4e-8 in f, which
// the tails of narrow Gaussians (Z of tens) cannot afford.  So t_i is formed as
// an unevaluated pair th + tl (exact product th = fl(h_hi d), its rounding error,
// and the small terms), t_i^2 as qh + c with qh = th^2 and c = (qh's error) +
// 2 th tl, Z as zh + zl with every addition's rounding error kept (TwoSum), and
// f = A 2^-(zh + zl).  Degree 0 / 1 select how t_i is formed (see FnDev).
template <int D, int G>
struct Eval<ZMC_GAUSS, D, G> {
  float hh[D], hl[D], pa[D], pb[D];
  float A;
  __device__ __forceinline__ void load(const FnDev *fn) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      hh[i] = __uint_as_float(fn->w[i]);
      hl[i] = __uint_as_float(fn->w[7 + i]);
      pa[i] = __uint_as_float(fn->w[14 + i]);
      pb[i] = __uint_as_float(fn->w[21 + i]);
    }
    A = __uint_as_float(fn->w[28]);
  }
  // The products and sums of the error-free transformations use the _rn
  // intrinsics: the compiler never contracts those into an FMA, which would
  // change the rounded value the error terms are computed against.
  __device__ __forceinline__ float operator()(const uint32_t *r) const {
    float zh = 0.0f, zl = 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float th, tl;
      if (G == 0) {
        // d = v - (1 + u0): exact, the result is a multiple of 2^-23 below 2 in size
        const float d = __fsub_rn(unit_v(r[i]), pa[i]);
        th = __fmul_rn(hh[i], d);
        tl = __fadd_rn(fmaf(hh[i], d, -th), fmaf(hl[i], d, pb[i]));
      } else {
        const float u = __fsub_rn(unit_v(r[i]), 1.0f);  // exact
        const float ph = __fmul_rn(hh[i], u);
        const float pl = fmaf(hh[i], u, -ph);
        const float s = __fadd_rn(pa[i], ph);  // TwoSum(e_hi, h_hi u)
        const float bb = __fsub_rn(s, pa[i]);
        const float err = __fadd_rn(__fsub_rn(pa[i], __fsub_rn(s, bb)), __fsub_rn(ph, bb));
        th = s;
        tl = __fadd_rn(__fadd_rn(err, pl), fmaf(hl[i], u, pb[i]));
      }
      const float qh = __fmul_rn(th, th);
      const float c = fmaf(__fadd_rn(th, th), tl, fmaf(th, th, -qh));
      if (i == 0) {
        zh = qh;
        zl = c;
      } else {
        // Fast2Sum on (max, min): both terms are >= 0, so the larger goes first
        const float big = fmaxf(zh, qh), small = fminf(zh, qh);
        const float s = __fadd_rn(big, small);
        const float err = __fsub_rn(small, __fsub_rn(s, big));
        zh = s;
        zl = __fadd_rn(zl, __fadd_rn(err, c));
      }
    }
    return amp_exp2_neg(A, zh, zl);
  }
};

// prod_i q_i(u_i), q_i re-expanded in u_i in [0, 1) on the host; Horner on the
// hi coefficients plus Horner on the lo coefficients (an FP64 coefficient split
// as hi + lo).  The lo terms cannot be replaced by their mean: with few samples
// and cancelling coefficients their fluctuation is visible at 1e-6.
template <int D, int G>
struct Eval<ZMC_POLY, D, G> {
  float ch[D][G + 1], cl[D][G + 1];
  __device__ __forceinline__ void load(const FnDev *fn) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j <= G; ++j) {
        ch[i][j] = __uint_as_float(fn->w[5 * i + j]);
        cl[i][j] = __uint_as_float(fn->w[35 + 5 * i + j]);
      }
  }
  __device__ __forceinline__ float operator()(const uint32_t *r) const {
    float prod = 1.0f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float qi;
      if (G == 0) {
        qi = ch[i][0] + cl[i][0];
      } else {
        const float u = unit_v(r[i]) - 1.0f;
        float ph = ch[i][G], pl = cl[i][G];
#pragma unroll
        for (int j = G - 1; j >= 0; --j) {
          ph = fmaf(ph, u, ch[i][j]);
          pl = fmaf(pl, u, cl[i][j]);
        }
        qi = ph + pl;
      }
      prod = (i == 0) ? qi : prod * qi;
    }
    return prod;
  }
};

// ---------------------------------------------------------------- one chunk
// Chan's pairwise merge of (n, mean, M2) summaries, FP32, down the warp; lane 0
// ends with the warp's summary.
__device__ __forceinline__ void warp_chan_merge(float &n, float &mean, float &m2) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const float nb = __shfl_down_sync(kFullMask, n, off);
    const float mb = __shfl_down_sync(kFullMask, mean, off);
    const float m2b = __shfl_down_sync(kFullMask, m2, off);
    const float nab = n + nb;
    if (nb > 0.0f) {
      const float delta = mb - mean;
      const float wb = __fdiv_rn(nb, nab);
      mean = fmaf(delta, wb, mean);
      m2 = m2 + m2b + delta * delta * (n * wb);
      n = nab;
    }
  }
}

// Samples [chunk * 128Q, min(+128Q, N)) of one integrand.  Lane l takes quads
// l, l+32, ..., l+32(Q-1) of the chunk.  Over each block of kBlockQuads of its
// quads it accumulates in FP32
//   s1 = sum f            (each quad summed pairwise first; unshifted, so its
//                          rounding error scales with the values themselves)
//   s2 = sum (f - K)^2    (K = the block's first value, so that s2 does not hold
//                          mean^2 n when the spread is small)
// turns them into (n, mean = s1/n, M2 = s2 - n (mean - K)^2) and merges that into
// the lane's running summary (Chan's pairwise update); the warp then merges the
// 32 lane summaries the same way.
// Quads of one lane interleaved per loop step, per family (build-time knobs).
#ifndef ZMC_QUAD_UNROLL
#define ZMC_QUAD_UNROLL 1
#endif
#ifndef ZMC_QUAD_UNROLL_HARMONIC
#define ZMC_QUAD_UNROLL_HARMONIC ZMC_QUAD_UNROLL
#endif
template <int FAM>
struct QuadUnroll {
  static constexpr int value = FAM == ZMC_HARMONIC ? ZMC_QUAD_UNROLL_HARMONIC : ZMC_QUAD_UNROLL;
};
// Quads per accumulation block: a lane's shifted sums never span more than
// 4 * kBlockQuads samples, which bounds their rounding error for any chunk length.
constexpr uint32_t kBlockQuads = 16;
template <int FAM, int D, int G, bool FAST>
__device__ __forceinline__ void run_chunk(const FnDev *__restrict__ fn, uint64_t chunk,
                                          uint32_t Q, uint32_t lane) {
  Eval<FAM, D, G> ev;
  ev.load(fn);
  const RoundKeys rk = make_round_keys(fn->key0, fn->key1);
  const uint32_t sid = fn->stream_id;
  const uint64_t chunk_samples = 128ull * Q;
  const uint64_t s0 = chunk * chunk_samples;
  const uint64_t n_left = fn->n_samples - s0;
  const uint32_t nc = static_cast<uint32_t>(n_left < chunk_samples ? n_left : chunk_samples);
  const uint64_t quad0 = (fn->s_off + s0) >> 2;  // s_off is a multiple of 4
  const uint64_t block0 = quad0 * D;
  const uint32_t base_lo0 = static_cast<uint32_t>(block0) + lane * D;
  const uint32_t base_hi = static_cast<uint32_t>(block0 >> 32);

  // running (n, mean, M2) of the lane, merged from blocks of kBlockQuads quads
  float n = 0.0f, mean = 0.0f, m2 = 0.0f;
  for (uint32_t jb = 0; jb < Q; jb += kBlockQuads) {
    const uint32_t je = jb + kBlockQuads < Q ? jb + kBlockQuads : Q;
    float K = 0.0f, s1 = 0.0f, s2 = 0.0f;
    uint32_t cnt = 0;
#pragma unroll QuadUnroll<FAM>::value
    for (uint32_t j = jb; j < je; ++j) {
      const uint32_t ql = lane + 32u * j;
      if (!FAST && 4u * ql >= nc) break;
      uint32_t r[4 * D];
      gen_quad<D, FAST>(quad0 + ql, base_lo0 + 32u * D * j, base_hi, sid, rk, r);
      float f[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) f[t] = ev(r + t * D);
      if (j == jb) K = f[0];
      if (FAST) {
        s1 += (f[0] + f[1]) + (f[2] + f[3]);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float dlt = f[t] - K;
          s2 = fmaf(dlt, dlt, s2);
        }
      } else {
        float q[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const bool ok = 4u * ql + t < nc;
          q[t] = ok ? f[t] : 0.0f;
          const float dlt = ok ? f[t] - K : 0.0f;
          s2 = fmaf(dlt, dlt, s2);
          cnt += ok ? 1u : 0u;
        }
        s1 += (q[0] + q[1]) + (q[2] + q[3]);
      }
    }
    const float nb = FAST ? static_cast<float>(4u * (je - jb)) : static_cast<float>(cnt);
    if (nb > 0.0f) {
      const float mb = __fdiv_rn(s1, nb);
      const float dk = mb - K;
      const float m2b = fmaxf(fmaf(-nb * dk, dk, s2), 0.0f);
      const float nab = n + nb;
      const float delta = mb - mean;
      const float wb = __fdiv_rn(nb, nab);
      mean = fmaf(delta, wb, mean);
      m2 = m2 + m2b + delta * delta * (n * wb);
      n = nab;
    }
    if (!FAST && cnt < 4u * (je - jb)) break;
  }
  warp_chan_merge(n, mean, m2);
  if (lane == 0) fn->rec[chunk] = make_float2(mean, m2);
}

template <int FAM, int D, int G>
__device__ __forceinline__ void run_item(const FnDev *__restrict__ fn, uint64_t chunk,
                                         uint32_t Q, uint32_t lane) {
  const uint64_t chunk_samples = 128ull * Q;
  const uint64_t s0 = chunk * chunk_samples;
  const bool full = fn->n_samples - s0 >= chunk_samples;
  const uint64_t b_first = ((fn->s_off + s0) >> 2) * D;
  const uint64_t b_last = b_first + (chunk_samples >> 2) * D - 1;
  if (full && (b_first >> 32) == (b_last >> 32))
    run_chunk<FAM, D, G, true>(fn, chunk, Q, lane);
  else
    run_chunk<FAM, D, G, false>(fn, chunk, Q, lane);
}

#define ZMC_VARIANTS_DIM(X, F, G) X(F, 1, G) X(F, 2, G) X(F, 3, G) X(F, 4, G) X(F, 5, G) \
  X(F, 6, G) X(F, 7, G)
#define ZMC_POLY_VARIANTS(X)                                                         \
  ZMC_VARIANTS_DIM(X, ZMC_POLY, 0) ZMC_VARIANTS_DIM(X, ZMC_POLY, 1)                  \
  ZMC_VARIANTS_DIM(X, ZMC_POLY, 2) ZMC_VARIANTS_DIM(X, ZMC_POLY, 3)                  \
  ZMC_VARIANTS_DIM(X, ZMC_POLY, 4)
#define ZMC_GAUSS_VARIANTS(X) ZMC_VARIANTS_DIM(X, ZMC_GAUSS, 0) ZMC_VARIANTS_DIM(X, ZMC_GAUSS, 1)
#define ZMC_ALL_VARIANTS(X)                                                          \
  ZMC_VARIANTS_DIM(X, ZMC_HARMONIC, 0) ZMC_VARIANTS_DIM(X, ZMC_ABSLIN, 0)            \
  ZMC_GAUSS_VARIANTS(X) ZMC_POLY_VARIANTS(X)

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

template <int FAM>
__device__ __forceinline__ void dispatch_family(const FnDev *fn, uint64_t chunk, uint32_t Q,
                                                uint32_t lane) {
  switch (fn->variant) {
#define ZMC_CASE(F, D, G) \
  case variant_code(F, D, G): run_item<F, D, G>(fn, chunk, Q, lane); break;
    case 0:  // never a valid code; keeps the switch non-empty for every family
      break;
#define ZMC_FAM_CASES(F) ZMC_VARIANTS_DIM(ZMC_CASE, F, 0)
    default:
      if (FAM == ZMC_HARMONIC) {
        switch (fn->variant) { ZMC_FAM_CASES(ZMC_HARMONIC) default: break; }
      } else if (FAM == ZMC_ABSLIN) {
        switch (fn->variant) { ZMC_FAM_CASES(ZMC_ABSLIN) default: break; }
      } else if (FAM == ZMC_GAUSS) {
        switch (fn->variant) { ZMC_GAUSS_VARIANTS(ZMC_CASE) default: break; }
      } else {
        switch (fn->variant) { ZMC_POLY_VARIANTS(ZMC_CASE) default: break; }
      }
      break;
#undef ZMC_FAM_CASES
#undef ZMC_CASE
  }
}

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

template <int FAM>
__global__ void __launch_bounds__(256, MinBlocks<FAM>::value)
    zmc_batched_kernel(const Entry *__restrict__ entries,
                                                          LaunchHdr *__restrict__ hdr) {
  const uint32_t lane = threadIdx.x & 31u;
  const unsigned long long begin = hdr->item_begin[FAM];
  const unsigned long long count = hdr->item_end[FAM] - begin;
  const uint32_t ne = hdr->n_entries;
  const uint32_t Q = hdr->quads_per_lane;
  uint32_t e = 0;
  for (;;) {
    unsigned long long k = 0;
    if (lane == 0) k = atomicAdd(&hdr->counter[FAM], 1ull);
    k = __shfl_sync(kFullMask, k, 0);
    if (k >= count) break;
    const uint64_t item = begin + k;
    e = find_entry(entries, ne, item, e);
    const Entry en = entries[e];
    dispatch_family<FAM>(en.fn, en.chunk_begin + (item - en.item_begin), Q, lane);
  }
}

// ---------------------------------------------------------------- FP64 merge
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(kFullMask, v, off);
  return v;
}

// One warp per integrand.  With chunk summaries (n_c, m_c, M2_c):
//   mean = sum_c n_c m_c / N,  M2 = sum_c [M2_c + n_c (m_c - mean)^2]
// (Chan et al.'s combination of partial moments, all chunks at once), summed in a
// fixed lane / butterfly order, so the result depends only on the records.
__global__ void __launch_bounds__(256) zmc_merge_kernel(const FnDev *const *__restrict__ fns,
                                                        const LaunchHdr *__restrict__ hdr) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t nm = hdr->n_merge;
  const uint64_t chunk_samples = 128ull * hdr->quads_per_lane;
  for (uint32_t k = warp; k < nm; k += nwarps) {
    const FnDev *fn = fns[k];
    const uint64_t N = fn->n_samples;
    const uint64_t C = (N + chunk_samples - 1) / chunk_samples;
    const float2 *rec = fn->rec;
    double s = 0.0;
    for (uint64_t c = lane; c < C; c += 32) {
      const uint64_t left = N - c * chunk_samples;
      const double nc = static_cast<double>(left < chunk_samples ? left : chunk_samples);
      s = fma(nc, static_cast<double>(rec[c].x), s);
    }
    const double mean = warp_sum_f64(s) / static_cast<double>(N);
    double m = 0.0;
    for (uint64_t c = lane; c < C; c += 32) {
      const uint64_t left = N - c * chunk_samples;
      const double nc = static_cast<double>(left < chunk_samples ? left : chunk_samples);
      const float2 rc = rec[c];
      const double dm = static_cast<double>(rc.x) - mean;
      m += fma(nc * dm, dm, static_cast<double>(rc.y));
    }
    const double inv = fn->inv_scale;
    const double m2 = fmax(warp_sum_f64(m), 0.0) * inv * inv;
    if (lane == 0) {
      const double nd = static_cast<double>(N);
      zmc_result res;
      if (fn->out_mode == 0) {
        res.estimate = fn->volume * (mean * inv);
        res.stderr_ = fn->volume * sqrt(m2 / (nd * (nd - 1.0)));
      } else {  // zmc_moments: unscaled mean and M2 of f over the samples
        res.estimate = mean * inv;
        res.stderr_ = m2;
      }
      res.n = N;
      res.status = ZMC_OK;
      res.reserved = 0;
      *fn->out = res;
    }
  }
}

// ---------------------------------------------------------------- plain FP64 form
template <int FAM>
__device__ __forceinline__ double eval_f64(const PlainFn &fn, const double *x, int d) {
  const double *p = fn.p;
  if (FAM == ZMC_HARMONIC) {
    double ph = 0.0;
    for (int i = 0; i < d; ++i) ph = fma(p[2 + i], x[i], ph);
    double s, c;
    sincos(ph, &s, &c);
    return fma(p[0], c, p[1] * s);
  } else if (FAM == ZMC_ABSLIN) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s = fma(p[1 + i], x[i], s);
    return p[0] * fabs(s);
  } else if (FAM == ZMC_GAUSS) {
    double r2 = 0.0;
    for (int i = 0; i < d; ++i) {
      const double t = x[i] - p[2 + i];
      r2 = fma(t, t, r2);
    }
    return p[0] * exp(-r2 / (2.0 * p[1] * p[1]));
  } else {
    double prod = 1.0;
    for (int i = 0; i < d; ++i) {
      double acc = p[5 * i + fn.deg];
      for (int j = static_cast<int>(fn.deg) - 1; j >= 0; --j) acc = fma(acc, x[i], p[5 * i + j]);
      prod *= acc;
    }
    return prod;
  }
}

// One thread per quad (grid-stride); per-thread FP64 shifted sums; block-level
// Chan merge in shared memory; one (n, mean, M2) record per block.
template <int FAM, int D>
__global__ void __launch_bounds__(256) zmc_plain_fp64_kernel(const PlainFn fn,
                                                             double *__restrict__ rec) {
  const RoundKeys rk = make_round_keys(fn.key0, fn.key1);
  const uint64_t N = fn.n_samples;
  const uint64_t nquads = (N + 3) / 4;
  double K = 0.0, s1 = 0.0, s2 = 0.0, cnt = 0.0;
  for (uint64_t q = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; q < nquads;
       q += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    uint32_t r[4 * D];
    gen_quad<D, false>(q, 0u, 0u, fn.stream_id, rk, r);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (4 * q + t < N) {
        double x[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          const double u = static_cast<double>(r[t * D + i] & 0x7FFFFFu) * 0x1p-23;
          x[i] = fma(fn.w[i], u, fn.lo[i]);
        }
        const double f = eval_f64<FAM>(fn, x, D);
        if (cnt == 0.0) K = f;
        const double dlt = f - K;
        s1 += dlt;
        s2 = fma(dlt, dlt, s2);
        cnt += 1.0;
      }
    }
  }
  __shared__ double sn[256], sm[256], sq[256];
  double mean = 0.0, m2 = 0.0;
  if (cnt > 0.0) {
    mean = K + s1 / cnt;
    m2 = fmax(s2 - s1 * (s1 / cnt), 0.0);
  }
  sn[threadIdx.x] = cnt;
  sm[threadIdx.x] = mean;
  sq[threadIdx.x] = m2;
  __syncthreads();
  for (unsigned half = blockDim.x >> 1; half > 0; half >>= 1) {
    if (threadIdx.x < half) {
      const double na = sn[threadIdx.x], nb = sn[threadIdx.x + half];
      if (nb > 0.0) {
        const double nab = na + nb;
        const double delta = sm[threadIdx.x + half] - sm[threadIdx.x];
        sm[threadIdx.x] += delta * (nb / nab);
        sq[threadIdx.x] += sq[threadIdx.x + half] + delta * delta * (na * nb / nab);
        sn[threadIdx.x] = nab;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    rec[3 * blockIdx.x + 0] = sn[0];
    rec[3 * blockIdx.x + 1] = sm[0];
    rec[3 * blockIdx.x + 2] = sq[0];
  }
}

}  // namespace

namespace {
__global__ void zmc_plain_merge_kernel(const PlainJob *__restrict__ jobs, uint32_t n) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= n) return;
  const PlainJob jb = jobs[warp];
  double nsum = 0.0, s = 0.0;
  for (uint32_t b = lane; b < jb.nblk; b += 32) {
    nsum += jb.rec[3 * b];
    s = fma(jb.rec[3 * b], jb.rec[3 * b + 1], s);
  }
  const double N = warp_sum_f64(nsum);
  const double mean = warp_sum_f64(s) / N;
  double m = 0.0;
  for (uint32_t b = lane; b < jb.nblk; b += 32) {
    const double dm = jb.rec[3 * b + 1] - mean;
    m += fma(jb.rec[3 * b] * dm, dm, jb.rec[3 * b + 2]);
  }
  const double m2 = fmax(warp_sum_f64(m), 0.0);
  if (lane == 0) {
    zmc_result res;
    res.estimate = jb.volume * mean;
    res.stderr_ = jb.volume * sqrt(m2 / (N * (N - 1.0)));
    res.n = static_cast<uint64_t>(N);
    res.status = ZMC_OK;
    res.reserved = 0;
    *jb.out = res;
  }
}

// ---------------------------------------------------------------- test kernels
__global__ void zmc_philox_kernel(const uint32_t *__restrict__ ctr,
                                  const uint32_t *__restrict__ key, uint32_t *__restrict__ out,
                                  size_t n) {
  for (size_t j = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; j < n;
       j += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const RoundKeys rk = make_round_keys(key[2 * j], key[2 * j + 1]);
    const uint4 o = philox(ctr[4 * j], ctr[4 * j + 1], ctr[4 * j + 2], ctr[4 * j + 3], rk);
    out[4 * j + 0] = o.x;
    out[4 * j + 1] = o.y;
    out[4 * j + 2] = o.z;
    out[4 * j + 3] = o.w;
  }
}

template <int FAM, int D, int G>
__device__ __forceinline__ void eval_range(const FnDev *fn, uint64_t s_begin, uint32_t count,
                                           float *out) {
  Eval<FAM, D, G> ev;
  ev.load(fn);
  const RoundKeys rk = make_round_keys(fn->key0, fn->key1);
  const uint64_t q_first = s_begin >> 2;
  const uint64_t q_last = (s_begin + count - 1) >> 2;
  for (uint64_t q = q_first + blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
       q <= q_last; q += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    uint32_t r[4 * D];
    gen_quad<D, false>(q, 0u, 0u, fn->stream_id, rk, r);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint64_t s = 4 * q + t;
      if (s >= s_begin && s < s_begin + count)
        out[s - s_begin] = static_cast<float>(static_cast<double>(ev(r + t * D)) * fn->inv_scale);
    }
  }
}

__global__ void zmc_eval_kernel(const FnDev *__restrict__ fn, uint64_t s_begin, uint32_t count,
                                float *__restrict__ out) {
  switch (fn->variant) {
#define ZMC_CASE(F, D, G) \
  case variant_code(F, D, G): eval_range<F, D, G>(fn, s_begin, count, out); break;
    ZMC_ALL_VARIANTS(ZMC_CASE)
#undef ZMC_CASE
    default:
      break;
  }
}

}  // namespace

// ---------------------------------------------------------------- launch wrappers
cudaError_t launch_batched(int family, const Entry *entries, LaunchHdr *hdr, unsigned grid,
                           unsigned block, cudaStream_t stream) {
  switch (family) {
    case ZMC_HARMONIC:
      zmc_batched_kernel<ZMC_HARMONIC><<<grid, block, 0, stream>>>(entries, hdr);
      break;
    case ZMC_ABSLIN:
      zmc_batched_kernel<ZMC_ABSLIN><<<grid, block, 0, stream>>>(entries, hdr);
      break;
    case ZMC_GAUSS:
      zmc_batched_kernel<ZMC_GAUSS><<<grid, block, 0, stream>>>(entries, hdr);
      break;
    case ZMC_POLY:
      zmc_batched_kernel<ZMC_POLY><<<grid, block, 0, stream>>>(entries, hdr);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_merge(const FnDev *const *fns, const LaunchHdr *hdr, unsigned grid,
                         cudaStream_t stream) {
  zmc_merge_kernel<<<grid, 256, 0, stream>>>(fns, hdr);
  return cudaGetLastError();
}

int batched_max_blocks_per_sm(int family, int block) {
  int n = 0;
  cudaError_t err = cudaErrorInvalidValue;
  switch (family) {
    case ZMC_HARMONIC:
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &n, zmc_batched_kernel<ZMC_HARMONIC>, block, 0);
      break;
    case ZMC_ABSLIN:
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, zmc_batched_kernel<ZMC_ABSLIN>,
                                                          block, 0);
      break;
    case ZMC_GAUSS:
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, zmc_batched_kernel<ZMC_GAUSS>,
                                                          block, 0);
      break;
    case ZMC_POLY:
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, zmc_batched_kernel<ZMC_POLY>,
                                                          block, 0);
      break;
    default:
      break;
  }
  return err == cudaSuccess ? n : 0;
}

unsigned plain_grid(const PlainFn &fn, int sms) {
  const uint64_t nquads = (fn.n_samples + 3) / 4;
  const uint64_t want = (nquads + 255) / 256;
  const uint64_t cap = static_cast<uint64_t>(sms) * 8;
  return static_cast<unsigned>(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_plain(const PlainFn &fn, double *block_rec, unsigned grid,
                         cudaStream_t stream) {
  switch (fn.family * 8 + fn.dim) {
#define ZMC_PCASE(F, D, G) \
  case F * 8 + D: zmc_plain_fp64_kernel<F, D><<<grid, 256, 0, stream>>>(fn, block_rec); break;
    ZMC_VARIANTS_DIM(ZMC_PCASE, ZMC_HARMONIC, 0)
    ZMC_VARIANTS_DIM(ZMC_PCASE, ZMC_ABSLIN, 0)
    ZMC_VARIANTS_DIM(ZMC_PCASE, ZMC_GAUSS, 0)
    ZMC_VARIANTS_DIM(ZMC_PCASE, ZMC_POLY, 0)
#undef ZMC_PCASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_plain_merge(const PlainJob *jobs, uint32_t n, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = (n + 7) / 8;
  zmc_plain_merge_kernel<<<grid, 256, 0, stream>>>(jobs, n);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, size_t n,
                          cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + 255) / 256;
  zmc_philox_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(
      ctr, key, out, n);
  return cudaGetLastError();
}

cudaError_t launch_eval(const FnDev *fn, uint64_t s_begin, uint32_t count, float *out,
                        cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  const uint64_t quads = ((s_begin + count - 1) >> 2) - (s_begin >> 2) + 1;
  const uint64_t blocks = (quads + 255) / 256;
  zmc_eval_kernel<<<static_cast<unsigned>(blocks < 1024 ? blocks : 1024), 256, 0, stream>>>(
      fn, s_begin, count, out);
  return cudaGetLastError();
}

}  // namespace zmc
