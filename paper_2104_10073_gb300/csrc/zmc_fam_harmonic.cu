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
  uint32_t thi[D];
  float tlo[D], kc[D];
  uint32_t p0;
  float rc[5];  // R times the coefficients of P
  __device__ __forceinline__ void load(const FnDev *fn) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      thi[i] = fn->w[i];
      tlo[i] = __uint_as_float(fn->w[7 + i]);
      kc[i] = __uint_as_float(fn->w[14 + i]);
    }
    p0 = fn->w[21];
    const float R = __uint_as_float(fn->w[22]);
    rc[0] = R * ZMC_SINQ_C0;
    rc[1] = R * ZMC_SINQ_C1;
    rc[2] = R * ZMC_SINQ_C2;
    rc[3] = R * ZMC_SINQ_C3;
    rc[4] = R * ZMC_SINQ_C4;
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
    float p = fmaf(rc[4], z, rc[3]);
    p = fmaf(p, z, rc[2]);
    p = fmaf(p, z, rc[1]);
    p = fmaf(p, z, rc[0]);
    return t * p;
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

const FamilyOps kFamilyHarmonic = family_ops<ZMC_HARMONIC>();

}  // namespace zmc
