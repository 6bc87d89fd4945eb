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
template <int D, int G>
struct Eval<ZMC_HARMONIC, D, G> {
  static constexpr int kPairs = D / 2;  // coordinate pairs (2i, 2i + 1) of the low-word FMAs
  uint32_t thi[D];
  float2 tlo2[kPairs + 1], kc2[kPairs + 1];  // (tlo, kc) of coordinates 2i, 2i + 1
  uint32_t p0;
  float rc[5];  // R times the coefficients of P
  __device__ __forceinline__ void load(const FnDev *fn) {
#pragma unroll
    for (int i = 0; i < D; ++i) thi[i] = fn->w[i];
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
#if ZMC_PACKED_F32
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
    acc += lows;
    // x = acc / 2^32 in [-1/2, 1/2) turn; cos(2 pi x) = sin(2 pi y) with
    // y = 1/4 - |x| in [-1/4, 1/4], formed exactly in the integer (two's-complement
    // wrap makes x = -1/2 come out right) and converted with full relative
    // precision, so the value keeps its relative accuracy near the zeros.
    const uint32_t sgn = static_cast<uint32_t>(static_cast<int32_t>(acc) >> 31);
    const uint32_t ax = (acc ^ sgn) - sgn;
    return static_cast<int32_t>(0x40000000u - ax);
  }
  __device__ __forceinline__ float operator()(const uint32_t *r) const {
    const float t = __int2float_rn(phase(r)) * 0x1p-32f;
    const float z = t * t;
    float p = fmaf(rc[4], z, rc[3]);
    p = fmaf(p, z, rc[2]);
    p = fmaf(p, z, rc[1]);
    p = fmaf(p, z, rc[0]);
    return __fmul_rn(t, p);  // never contracted with the sums' f - K
  }
  // R sin(2 pi y) of two samples as packed pairs: the same operations as
  // operator(), so the same values bit for bit.
  __device__ __forceinline__ float2 sine2(int32_t ya, int32_t yb) const {
    const float2 sc = make_float2(0x1p-32f, 0x1p-32f);
    const float2 t = __fmul2_rn(make_float2(__int2float_rn(ya), __int2float_rn(yb)), sc);
    const float2 z = __fmul2_rn(t, t);
    float2 p = __ffma2_rn(make_float2(rc[4], rc[4]), z, make_float2(rc[3], rc[3]));
    p = __ffma2_rn(p, z, make_float2(rc[2], rc[2]));
    p = __ffma2_rn(p, z, make_float2(rc[1], rc[1]));
    p = __ffma2_rn(p, z, make_float2(rc[0], rc[0]));
    return __fmul2_rn(t, p);
  }
  __device__ __forceinline__ void quint(const uint32_t (&r)[5 * D], float (&f)[5]) const {
    int32_t y[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) y[t] = phase(r + t * D);
    const float2 a = sine2(y[0], y[1]), b = sine2(y[2], y[3]);
    f[0] = a.x;
    f[1] = a.y;
    f[2] = b.x;
    f[3] = b.y;
    const float t4 = __int2float_rn(y[4]) * 0x1p-32f;
    const float z4 = t4 * t4;
    float p4 = fmaf(rc[4], z4, rc[3]);
    p4 = fmaf(p4, z4, rc[2]);
    p4 = fmaf(p4, z4, rc[1]);
    p4 = fmaf(p4, z4, rc[0]);
    f[4] = __fmul_rn(t4, p4);
  }
};

template <>
__device__ void dispatch_item<ZMC_HARMONIC>(const FnDev *fn, uint64_t chunk, uint32_t Q,
                                      uint32_t lane) {
  switch (fn->variant) {
    ZMC_HARMONIC_VARIANTS(ZMC_ITEM_CASE)
    default:
      break;
  }
}

template <>
__device__ void dispatch_eval<ZMC_HARMONIC>(const FnDev *fn, uint64_t s_begin, uint32_t count,
                                      float *out) {
  switch (fn->variant) {
    ZMC_HARMONIC_VARIANTS(ZMC_EVAL_CASE)
    default:
      break;
  }
}

}  // namespace

const FamilyOps ZMC_FAMILY_OPS(kFamilyHarmonic) = family_ops<ZMC_HARMONIC>();

}  // namespace zmc
