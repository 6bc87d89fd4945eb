// zmc_fam_harmonic.cu -- the sampling path of the harmonic family: its FP32
// integrand Eval<ZMC_HARMONIC, D, G>, the persistent kernel zmc_batched_kernel<ZMC_HARMONIC>
// instantiated for its variants, and the per-sample test kernel.
#include "zmc_device.cuh"
#include "zmc_coeffs.h"

namespace zmc {
namespace {

// a cos(k.x) + b sin(k.x) (Eq. 1) = R cos(2 pi P), R = sqrt(a^2 + b^2), with the
// phase P in turns = k.x / (2 pi) - atan2(b, a) / (2 pi).  P's fraction is kept
// as a 32-bit fixed-point number (units of 2^-32 turn), formed from the 23-bit
// sample integers m_i: P = P0 + sum_i [T_hi,i m_i + round(T_lo,i m_i / 2^32)],
// where T_i = k_i (hi_i - lo_i) / (2 pi) 2^41 is split into its high and low
// 32-bit words.  The high-word products wrap modulo 1 turn exactly (one 32-bit
// multiply-add each); the low-word contribution (< 2^23 units) is formed by one
// FP32 FMA from v' = 2^23 + m_i, whose rounding and the dropped carries cost at
// most D units of 2^-32 turn.  So |k.x| of any size costs no accuracy.  Then
// R cos(2 pi x) = R sin(2 pi (1/4 - |x|)), evaluated as t Pr(t^2) with Pr = R P,
// P the degree-4 polynomial of zmc_coeffs.h: the amplitude goes into the
// coefficients once per chunk instead of into every sample.
//
// Variant G = 1 (rows whose dimensions all advance the phase at the same rate,
// T_i = T, as in the paper's Fig. 1 set k = kappa (1, 1, 1, 1) on the unit cube):
// the phase is P0 + T S with S = sum_i m_i < 2^26, formed in integers: T_lo S
// plus the low word of P0 + 1/2 unit by one widening multiply-add, whose high
// word (the carry into whole units) T_hi S + P0_hi adds by one 32-bit
// multiply-add.  So the phase is P0 + T S rounded to the nearest unit of 2^-32
// turn (error <= 1/2 unit, against up to ~D units for the general form), and
// one multiply-add and one widening multiply-add replace D multiply-adds and D
// FMAs.
// How much of the FP32 work is issued as packed pairs (they run on the pipe that
// also takes Philox's widening multiplies, so packing trades issue slots for
// that pipe's time): 0 none, 1 the low-word FMAs, 2 also the sine, 3 also the
// sums (run_chunk).
#ifndef ZMC_HARMONIC_PACK
#define ZMC_HARMONIC_PACK 3
#endif
// 1: |x| of the phase by one abs.s32 instead of the sign-mask form.
#ifndef ZMC_HARMONIC_IABS
#define ZMC_HARMONIC_IABS 0
#endif

template <int D, int G>
struct Eval<ZMC_HARMONIC, D, G> {
  static constexpr bool kPackedSums = ZMC_HARMONIC_PACK >= 3;
  static constexpr int kPairs = D / 2;  // coordinate pairs (2i, 2i + 1) of the low-word FMAs
  uint32_t thi[D];
  float2 tlo2[kPairs + 1], kc2[kPairs + 1];  // (tlo, kc) of coordinates 2i, 2i + 1
  uint32_t p0, p0lo;
  float rc[5];  // R times the coefficients of P
  __device__ __forceinline__ void load(const FnDev *fn) {
    if (G == 1) {  // T_hi at w[0], T_lo (u32) at w[1], the low word of P0 at w[2]
      thi[0] = fn->w[0];
      thi[1] = fn->w[1];
      p0lo = fn->w[2];
    } else {
#pragma unroll
      for (int i = 0; i < D; ++i) thi[i] = fn->w[i];
    }
#pragma unroll
    for (int i = 0; i < D; i += 2) {
      tlo2[i / 2] = make_float2(__uint_as_float(fn->w[7 + i]),
                                i + 1 < D ? __uint_as_float(fn->w[8 + i]) : 0.0f);
      kc2[i / 2] = make_float2(__uint_as_float(fn->w[14 + i]),
                               i + 1 < D ? __uint_as_float(fn->w[15 + i]) : 0.0f);
    }
    p0 = fn->w[21];
    const float R = __uint_as_float(fn->w[22]);
    rc[0] = R * ZMC_SINQ_C0;
    rc[1] = R * ZMC_SINQ_C1;
    rc[2] = R * ZMC_SINQ_C2;
    rc[3] = R * ZMC_SINQ_C3;
    rc[4] = R * ZMC_SINQ_C4;
  }
  // The phase of one sample as the integer y = 2^32 (1/4 - |x|), x the phase in
  // turns reduced to [-1/2, 1/2).  The low-word FMAs of coordinates 2i and 2i + 1
  // run as one packed pair (each half rounded as the scalar FMA).
  // y = 2^32 (1/4 - |x|) of one sample (see fold), as a float.
  __device__ __forceinline__ float phase_y(const uint32_t *r) const {
    if (G == 1) {
      uint32_t sm = 0;
#pragma unroll
      for (int i = 0; i < D; ++i) sm += r[i] & 0x7FFFFFu;
      // T_lo S + (P0 + 1/2 unit) in 64 bits (units of 2^-64 turn); its high
      // word carries the rounded whole units
      const uint64_t lo = static_cast<uint64_t>(thi[1]) * sm +
                          ((static_cast<uint64_t>(p0) << 32) | p0lo);
      return __int2float_rn(fold(thi[0] * sm + static_cast<uint32_t>(lo >> 32)));
    }
    return __int2float_rn(phase(r));
  }
  __device__ __forceinline__ int32_t phase(const uint32_t *r) const {
    uint32_t acc = p0, lows = 0;
    uint32_t vb[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      vb[i] = (r[i] & 0x7FFFFFu) | 0x4B000000u;  // bits of 2^23 + m_i
      acc = thi[i] * vb[i] + acc;
    }
#pragma unroll
    for (int i = 0; i + 1 < D; i += 2) {
#if ZMC_PACKED_F32 && ZMC_HARMONIC_PACK >= 1
      const float2 c = __ffma2_rn(
          tlo2[i / 2], make_float2(__uint_as_float(vb[i]), __uint_as_float(vb[i + 1])),
          kc2[i / 2]);
      lows += __float_as_uint(c.x) + __float_as_uint(c.y);
#else
      lows += __float_as_uint(fmaf(tlo2[i / 2].x, __uint_as_float(vb[i]), kc2[i / 2].x)) +
              __float_as_uint(fmaf(tlo2[i / 2].y, __uint_as_float(vb[i + 1]), kc2[i / 2].y));
#endif
    }
    if (D & 1)  // the host folds the 0x4B000000 offsets into p0
      lows += __float_as_uint(fmaf(tlo2[kPairs].x, __uint_as_float(vb[D - 1]), kc2[kPairs].x));
    return fold(acc + lows);
  }
  // x = acc / 2^32 in [-1/2, 1/2) turn  ->  y = 2^32 (1/4 - |x|)
  __device__ __forceinline__ static int32_t fold(uint32_t acc) {
    // x = acc / 2^32 in [-1/2, 1/2) turn; cos(2 pi x) = sin(2 pi y) with
    // y = 1/4 - |x| in [-1/4, 1/4], formed exactly in the integer (two's-complement
    // wrap makes x = -1/2 come out right) and converted with full relative
    // precision, so the value keeps its relative accuracy near the zeros.
#if ZMC_HARMONIC_IABS
    uint32_t ax;  // abs.s32 maps -2^31 to itself, as the wrap below needs
    asm("abs.s32 %0, %1;" : "=r"(ax) : "r"(acc));
#else
    const uint32_t sgn = static_cast<uint32_t>(static_cast<int32_t>(acc) >> 31);
    const uint32_t ax = (acc ^ sgn) - sgn;
#endif
    return static_cast<int32_t>(0x40000000u - ax);
  }
  // R sin(2 pi t), t = y / 2^32, by the odd polynomial t (R P)(t^2).
  __device__ __forceinline__ float sine(float y) const {
    const float t = y * 0x1p-32f;
    const float z = t * t;
    float p = fmaf(rc[4], z, rc[3]);
    p = fmaf(p, z, rc[2]);
    p = fmaf(p, z, rc[1]);
    p = fmaf(p, z, rc[0]);
    return __fmul_rn(t, p);
  }
  __device__ __forceinline__ float operator()(const uint32_t *r) const { return sine(phase_y(r)); }
  // R sin(2 pi t) of two samples as packed pairs: the same operations as
  // operator(), so the same values bit for bit.
  __device__ __forceinline__ float2 sine2(float ya, float yb) const {
    const float2 t = __fmul2_rn(make_float2(ya, yb), make_float2(0x1p-32f, 0x1p-32f));
    const float2 z = __fmul2_rn(t, t);
    float2 p = __ffma2_rn(make_float2(rc[4], rc[4]), z, make_float2(rc[3], rc[3]));
    p = __ffma2_rn(p, z, make_float2(rc[2], rc[2]));
    p = __ffma2_rn(p, z, make_float2(rc[1], rc[1]));
    p = __ffma2_rn(p, z, make_float2(rc[0], rc[0]));
    return __fmul2_rn(t, p);
  }
  __device__ __forceinline__ void quint(const uint32_t (&r)[5 * D], float (&f)[5]) const {
    float y[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) y[t] = phase_y(r + t * D);
#if ZMC_HARMONIC_PACK < 2
#pragma unroll
    for (int t = 0; t < 5; ++t) f[t] = sine(y[t]);
    return;
#endif
    const float2 a = sine2(y[0], y[1]), b = sine2(y[2], y[3]);
    f[0] = a.x;
    f[1] = a.y;
    f[2] = b.x;
    f[3] = b.y;
    f[4] = sine(y[4]);
  }
};

template <>
__device__ void dispatch_item<ZMC_HARMONIC>(const FnDev *fn, uint64_t chunk, uint32_t Q,
                                      uint32_t lane) {
  switch (fn->variant) {
    ZMC_HARMONIC_VARIANTS(ZMC_ITEM_CASE)
    ZMC_HARMONIC_EQUAL_VARIANTS(ZMC_ITEM_CASE)
    default:
      break;
  }
}

template <>
__device__ void dispatch_eval<ZMC_HARMONIC>(const FnDev *fn, uint64_t s_begin, uint32_t count,
                                      float *out) {
  switch (fn->variant) {
    ZMC_HARMONIC_VARIANTS(ZMC_EVAL_CASE)
    ZMC_HARMONIC_EQUAL_VARIANTS(ZMC_EVAL_CASE)
    default:
      break;
  }
}

}  // namespace

const FamilyOps ZMC_FAMILY_OPS(kFamilyHarmonic) = family_ops<ZMC_HARMONIC>();

}  // namespace zmc
