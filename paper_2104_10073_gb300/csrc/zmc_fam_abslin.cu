// zmc_fam_abslin.cu -- the sampling path of the abslin family: its FP32
// integrand Eval<ZMC_ABSLIN, D, G>, the persistent kernel zmc_batched_kernel<ZMC_ABSLIN>
// instantiated for its variants, and the per-sample test kernel.
#include "zmc_device.cuh"

namespace zmc {
namespace {

// a |c.x| (Eq. 2).  Near the hyperplane c.x = 0 the terms of c.x cancel, and a
// sum rounded in FP32 keeps only an absolute accuracy of ~2^-24 of the terms;
// so c.x is summed exactly instead, in units of 2^-F: the integer parts G_i m_i
// (32 x 32 -> 64-bit products) in a 64-bit accumulator, whose modulo-2^64 wrap
// is harmless because the true sum fits, and the sub-unit remainders g_i m_i in
// FP32 (error a few units).  One rounding to FP32 at the end keeps the relative
// accuracy of f down to |c.x| of a few 2^-F.
// Variant G = 1 (rows of many samples): the integer parts summed in 32 bits
// (modulo 2^32; the host's scale keeps the true sum below 2^30), one 32-bit
// multiply-add per coordinate.
template <int D, int G>
struct Eval<ZMC_ABSLIN, D, G> {
  int32_t gi[D];
  float gl[D];
  uint64_t g0;
  float l0, scale;
  __device__ __forceinline__ void load(const FnDev *fn) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      gi[i] = static_cast<int32_t>(fn->w[i]);
      gl[i] = __uint_as_float(fn->w[7 + i]);
    }
    g0 = (static_cast<uint64_t>(fn->w[15]) << 32) | fn->w[14];
    l0 = __uint_as_float(fn->w[16]);
    scale = __uint_as_float(fn->w[17]);
  }
  __device__ __forceinline__ float operator()(const uint32_t *r) const {
    if (G == 1) {
      uint32_t acc = static_cast<uint32_t>(g0);
      float l = l0;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const uint32_t vb = (r[i] & 0x7FFFFFu) | 0x4B000000u;  // bits of 2^23 + m_i
        acc = static_cast<uint32_t>(gi[i]) * vb + acc;
        l = fmaf(gl[i], __uint_as_float(vb), l);
      }
      const float s = __fadd_rn(__int2float_rn(static_cast<int32_t>(acc)), l);
      return __fmul_rn(scale, fabsf(s));
    }
    uint64_t acc = g0;
    float l = l0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const uint32_t vb = (r[i] & 0x7FFFFFu) | 0x4B000000u;  // bits of 2^23 + m_i
      acc += static_cast<uint64_t>(static_cast<int64_t>(gi[i]) *
                                   static_cast<int64_t>(static_cast<int32_t>(vb)));
      l = fmaf(gl[i], __uint_as_float(vb), l);
    }
    const float s = __ll2float_rn(static_cast<long long>(acc)) + l;
    return __fmul_rn(scale, fabsf(s));  // never contracted with the sums' f - K
  }
};

template <>
__device__ void dispatch_item<ZMC_ABSLIN>(const FnDev *fn, uint64_t chunk, uint32_t Q,
                                      uint32_t lane) {
  switch (fn->variant) {
    ZMC_ABSLIN_VARIANTS(ZMC_ITEM_CASE)
    ZMC_VARIANTS_DIM(ZMC_ITEM_CASE, ZMC_ABSLIN, 1)
    default:
      break;
  }
}

template <>
__device__ void dispatch_eval<ZMC_ABSLIN>(const FnDev *fn, uint64_t s_begin, uint32_t count,
                                      float *out) {
  switch (fn->variant) {
    ZMC_ABSLIN_VARIANTS(ZMC_EVAL_CASE)
    ZMC_VARIANTS_DIM(ZMC_EVAL_CASE, ZMC_ABSLIN, 1)
    default:
      break;
  }
}

}  // namespace

const FamilyOps ZMC_FAMILY_OPS(kFamilyAbslin) = family_ops<ZMC_ABSLIN>();

}  // namespace zmc
