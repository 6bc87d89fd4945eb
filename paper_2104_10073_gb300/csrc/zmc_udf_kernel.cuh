// zmc_udf_kernel.cuh -- the sampling path of user-defined integrands.  Compiled
// at run time by NVRTC only; zmc_udf.cpp assembles the program: zmc_device.cuh,
// each user source k in a namespace of its own (zmc_user_<k>, with ZMC_UDF_DIM
// defined to its dimension), this file with ZMC_UDF_PRECISION defined, then the
// generated UserFn<k> thunks and the variant switch udf_dispatch_item /
// udf_dispatch_eval over the (dimension, function) pairs.
//
// The generator, the per-chunk sums and the persistent work-list loop are those
// of the built-in families (zmc_device.cuh); only the evaluation differs:
// Eval<ZMC_USER, D, K> maps the sample onto the box and calls function K; the
// FnDev payload words it reads are laid out in zmc_udf_layout.h (written by
// zmc_udf.cpp).  The kernels have C names so that the loader can find them.
#include "zmc_udf_layout.h"

namespace zmc {
namespace {

#if ZMC_UDF_PRECISION == 0
typedef float UdfReal;
#else
typedef double UdfReal;
#endif

// UserFn<K>::f(x, p) calls user function K (generated after this file).
template <int K>
struct UserFn;

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
    return __fmul_rn(S, UserFn<G>::f(x, p));  // never contracted with the sums' f - K
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
    return static_cast<float>(S * UserFn<G>::f(x, p));
  }
};
#endif

// the (dimension, function) switch, generated after this file
__device__ void udf_dispatch_item(const FnDev *fn, uint64_t chunk, uint32_t Q, uint32_t lane);
__device__ void udf_dispatch_eval(const FnDev *fn, uint64_t s_begin, uint32_t count, float *out);

template <>
__device__ void dispatch_item<ZMC_USER>(const FnDev *fn, uint64_t chunk, uint32_t Q,
                                        uint32_t lane) {
  udf_dispatch_item(fn, chunk, Q, lane);
}

template <>
__device__ void dispatch_eval<ZMC_USER>(const FnDev *fn, uint64_t s_begin, uint32_t count,
                                        float *out) {
  udf_dispatch_eval(fn, s_begin, count, out);
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
