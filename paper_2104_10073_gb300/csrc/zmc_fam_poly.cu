// zmc_fam_poly.cu -- the sampling path of the poly family: its FP32
// integrand Eval<ZMC_POLY, D, G>, the persistent kernel zmc_batched_kernel<ZMC_POLY>
// instantiated for its variants, and the per-sample test kernel.
#include <type_traits>

#include "zmc_device.cuh"

namespace zmc {
namespace {

// prod_i q_i(u_i), q_i re-expanded in u_i in [0, 1) on the host.
//
// Coefficient form (variant degree G = 0..4): Horner on the hi coefficients plus
// Horner on the lo coefficients (an FP64 coefficient split as hi + lo).  The lo
// terms cannot be replaced by their mean: with few samples and cancelling
// coefficients their fluctuation is visible at 1e-6.
template <int D, int G>
struct PolyCoeffEval {
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
      prod = (i == 0) ? qi : __fmul_rn(prod, qi);  // never contracted with the sums
    }
    return prod;
  }
};

// Root form (variant degree K + 3 for degree K = 2..4): Horner in FP32 loses
// relative accuracy near a root of a factor inside the box (by the ratio of the
// summed terms to the value).  The host writes each factor as lead times
// "quads" (u - p1)(u - p2) + c -- a real root pair (c = 0) or a complex pair
// (p1 = p2 = a, c = b^2) -- and, for K = 3, a linear term u - r; the kernel
// forms every u - p as (u - p_hi) - p_lo (exact near p by Sterbenz's lemma) and
// a quad with one FMA, so each factor keeps a few ulp of relative accuracy with
// no branch.  The amplitude S prod lead carries the scale.
__device__ __forceinline__ float shifted(float u, float h, float l) {
  return __fsub_rn(__fsub_rn(u, h), l);
}

__device__ __forceinline__ float quad(float u, const float *q) {
  return fmaf(shifted(u, q[0], q[1]), shifted(u, q[2], q[3]), q[4]);
}

template <int D, int K>
struct PolyRootEval {
  static constexpr int kWords = K == 2 ? 5 : K == 3 ? 7 : 10;
  float c[D][kWords];
  float amp;
  __device__ __forceinline__ void load(const FnDev *fn) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = 0; k < kWords; ++k) c[i][k] = __uint_as_float(fn->w[kWords * i + k]);
    amp = __uint_as_float(fn->w[70]);
  }
  __device__ __forceinline__ float operator()(const uint32_t *r) const {
    float prod = amp;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float u = unit_v(r[i]) - 1.0f;  // exact
      float qi;
      if (K == 2)
        qi = quad(u, c[i]);
      else if (K == 3)
        qi = __fmul_rn(shifted(u, c[i][0], c[i][1]), quad(u, c[i] + 2));
      else
        qi = __fmul_rn(quad(u, c[i]), quad(u, c[i] + 5));
      prod = __fmul_rn(prod, qi);
    }
    return prod;
  }
};

template <int D, int G>
struct Eval<ZMC_POLY, D, G>
    : std::conditional_t<(G <= 4), PolyCoeffEval<D, (G <= 4 ? G : 0)>,
                         PolyRootEval<D, (G > 4 ? G - 3 : 1)>> {};

// variants: coefficient form for degrees 0..4 (zmc_device.cuh) and root form
// for degrees 2..4 (variant degree 5..7)
#define ZMC_POLY_ROOT_VARIANTS(X)                                                    \
  ZMC_VARIANTS_DIM(X, ZMC_POLY, 5) ZMC_VARIANTS_DIM(X, ZMC_POLY, 6)                  \
  ZMC_VARIANTS_DIM(X, ZMC_POLY, 7)

template <>
__device__ void dispatch_item<ZMC_POLY>(const FnDev *fn, uint64_t chunk, uint32_t Q,
                                      uint32_t lane) {
  switch (fn->variant) {
    ZMC_POLY_VARIANTS(ZMC_ITEM_CASE)
    ZMC_POLY_ROOT_VARIANTS(ZMC_ITEM_CASE)
    default:
      break;
  }
}

template <>
__device__ void dispatch_eval<ZMC_POLY>(const FnDev *fn, uint64_t s_begin, uint32_t count,
                                      float *out) {
  switch (fn->variant) {
    ZMC_POLY_VARIANTS(ZMC_EVAL_CASE)
    ZMC_POLY_ROOT_VARIANTS(ZMC_EVAL_CASE)
    default:
      break;
  }
}

}  // namespace

const FamilyOps ZMC_FAMILY_OPS(kFamilyPoly) = family_ops<ZMC_POLY>();

}  // namespace zmc
