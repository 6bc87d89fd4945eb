// zmc_fam_poly.cu -- the sampling path of the poly family: its FP32
// integrand Eval<ZMC_POLY, D, G>, the persistent kernel zmc_batched_kernel<ZMC_POLY>
// instantiated for its variants, and the per-sample test kernel.
#include "zmc_device.cuh"

namespace zmc {
namespace {

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

template <>
__device__ void dispatch_item<ZMC_POLY>(const FnDev *fn, uint64_t chunk, uint32_t Q,
                                      uint32_t lane) {
  switch (fn->variant) {
    ZMC_POLY_VARIANTS(ZMC_ITEM_CASE)
    default:
      break;
  }
}

template <>
__device__ void dispatch_eval<ZMC_POLY>(const FnDev *fn, uint64_t s_begin, uint32_t count,
                                      float *out) {
  switch (fn->variant) {
    ZMC_POLY_VARIANTS(ZMC_EVAL_CASE)
    default:
      break;
  }
}

}  // namespace

const FamilyOps kFamilyPoly = family_ops<ZMC_POLY>();

}  // namespace zmc
