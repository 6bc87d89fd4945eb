// zmc_udf_kernel.cuh -- the sampling path of a user-defined integrand.  Compiled
// at run time by NVRTC only, after zmc_device.cuh and the user's source (which
// defines zmc_user_f); zmc_udf.cpp assembles the program and defines
// ZMC_UDF_DIM and ZMC_UDF_PRECISION.
//
// The generator, the per-chunk sums and the persistent work-list loop are those
// of the built-in families (zmc_device.cuh); only the evaluation differs:
// Eval<ZMC_USER, ZMC_UDF_DIM, 0> maps the sample onto the box and calls
// zmc_user_f; the FnDev payload words it reads are laid out in zmc_udf_layout.h
// (written by zmc_udf.cpp).  The kernels have C names so that the loader can
// find them.
#include "zmc_udf_layout.h"

namespace zmc {
namespace {

#if ZMC_UDF_PRECISION == 0
template <int D, int G>
struct Eval<ZMC_USER, D, G> {
  float wd[D], lo[D];
  float p[ZMC_NPARAM];
  float S;
  __device__ __forceinline__ void load(const FnDev *fn) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      wd[i] = __uint_as_float(fn->w[kUdfF32W + i]);
      lo[i] = __uint_as_float(fn->w[kUdfF32Lo + i]);
    }
#pragma unroll
    for (int j = 0; j < ZMC_NPARAM; ++j) p[j] = __uint_as_float(fn->w[kUdfF32P + j]);
    S = __uint_as_float(fn->w[kUdfF32S]);
  }
  __device__ __forceinline__ float operator()(const uint32_t *r) const {
    float x[D];
#pragma unroll
    for (int i = 0; i < D; ++i) x[i] = fmaf(wd[i], unit_v(r[i]) - 1.0f, lo[i]);  // u exact
    return S * zmc_user_f(x, p);
  }
};
#else
__device__ __forceinline__ double word_pair_f64(const uint32_t *w) {
  return __hiloint2double(static_cast<int>(w[1]), static_cast<int>(w[0]));
}

template <int D, int G>
struct Eval<ZMC_USER, D, G> {
  double wd[D], lo[D];
  const double *p;
  double S;
  __device__ __forceinline__ void load(const FnDev *fn) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      lo[i] = word_pair_f64(fn->w + kUdfF64Lo + 2 * i);
      wd[i] = word_pair_f64(fn->w + kUdfF64W + 2 * i);
    }
    const unsigned long long addr =
        (static_cast<unsigned long long>(fn->w[kUdfF64P + 1]) << 32) | fn->w[kUdfF64P];
    p = reinterpret_cast<const double *>(addr);
    S = word_pair_f64(fn->w + kUdfF64S);
  }
  __device__ __forceinline__ float operator()(const uint32_t *r) const {
    double x[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const double u = static_cast<double>(r[i] & 0x7FFFFFu) * 0x1p-23;
      x[i] = fma(wd[i], u, lo[i]);
    }
    return static_cast<float>(S * zmc_user_f(x, p));
  }
};
#endif

template <>
__device__ void dispatch_item<ZMC_USER>(const FnDev *fn, uint64_t chunk, uint32_t Q,
                                        uint32_t lane) {
  run_item<ZMC_USER, ZMC_UDF_DIM, 0>(fn, chunk, Q, lane);
}

template <>
__device__ void dispatch_eval<ZMC_USER>(const FnDev *fn, uint64_t s_begin, uint32_t count,
                                        float *out) {
  eval_range<ZMC_USER, ZMC_UDF_DIM, 0>(fn, s_begin, count, out);
}

}  // namespace
}  // namespace zmc

extern "C" __global__ void __launch_bounds__(256, 2)
    zmc_udf_batched(const zmc::Entry *__restrict__ entries, zmc::LaunchHdr *__restrict__ hdr) {
  zmc::batched_loop<ZMC_USER>(entries, hdr);
}

extern "C" __global__ void __launch_bounds__(256)
    zmc_udf_eval(const zmc::FnDev *__restrict__ fn, uint64_t s_begin, uint32_t count,
                 float *__restrict__ out) {
  zmc::dispatch_eval<ZMC_USER>(fn, s_begin, count, out);
}
