// zmc_fam_abslin.cu -- the sampling path of the abslin family: its FP32
// integrand Eval<ZMC_ABSLIN, D, G>, the persistent kernel zmc_batched_kernel<ZMC_ABSLIN>
// instantiated for its variants, and the per-sample test kernel.
#include "zmc_device.cuh"

namespace zmc {
namespace {

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

template <>
__device__ void dispatch_item<ZMC_ABSLIN>(const FnDev *fn, uint64_t chunk, uint32_t Q,
                                      uint32_t lane) {
  switch (fn->variant) {
    ZMC_ABSLIN_VARIANTS(ZMC_ITEM_CASE)
    default:
      break;
  }
}

template <>
__device__ void dispatch_eval<ZMC_ABSLIN>(const FnDev *fn, uint64_t s_begin, uint32_t count,
                                      float *out) {
  switch (fn->variant) {
    ZMC_ABSLIN_VARIANTS(ZMC_EVAL_CASE)
    default:
      break;
  }
}

}  // namespace

const FamilyOps kFamilyAbslin = family_ops<ZMC_ABSLIN>();

}  // namespace zmc
