// zmc_fam_gauss.cu -- the sampling path of the gauss family: its FP32
// integrand Eval<ZMC_GAUSS, D, G>, the persistent kernel zmc_batched_kernel<ZMC_GAUSS>
// instantiated for its variants, and the per-sample test kernel.
#include "zmc_device.cuh"

namespace zmc {
namespace {

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

// A exp(-|x-mu|^2 / (2 sigma^2)) = A 2^(-Z), Z = sum_i t_i^2.  FP32 carries a
// relative error of ~2^-24 Z in a plainly summed Z, i.e. ~Z 4e-8 in f, which
// the tails of narrow Gaussians (Z of tens) cannot afford.  So t_i is formed as
// an unevaluated pair th + tl (exact product th = fl(h_hi d), its rounding error,
// and the small terms), t_i^2 as a part on a fixed grid (whose sum is exact)
// plus a small correction, Z as zh + zl, and f = A 2^-(zh + zl).  Degree 0 / 1
// select how t_i is formed (see FnDev).
// 1: the near form (degree 0) of D >= 2 takes its coordinates in packed FP32
// pairs (build knob; measured no faster on the 10^4 mix, 376.5 against 376.9 G
// samples/s: the packed operations occupy the pipe that Philox's multiplies
// bind, so the issue slots they save do not turn into time).
#ifndef ZMC_GAUSS_PACK
#define ZMC_GAUSS_PACK 0
#endif

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
    int i0 = 0;  // coordinates before i0 were taken in packed pairs
#if ZMC_PACKED_F32 && ZMC_GAUSS_PACK
    if (G == 0 && D >= 2) {
      // Coordinates (2k, 2k + 1) as packed FP32 pairs, each half the scalar
      // steps below: th and -th (for the TwoProduct error and the square's
      // rounding, so that no operand needs a negation), the grid square kept
      // negated, -qg, which is what r needs; zh is the sum of the qg, exact.
      const float2 m1 = make_float2(-1.0f, -1.0f), m256 = make_float2(-256.0f, -256.0f);
      const float2 p256 = make_float2(256.0f, 256.0f);
      float2 nzh2 = make_float2(0.0f, 0.0f), zl2 = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k + 1 < D; k += 2) {
        const float2 hh2 = make_float2(hh[k], hh[k + 1]), hl2 = make_float2(hl[k], hl[k + 1]);
        const float2 pb2 = make_float2(pb[k], pb[k + 1]);
        const float2 d = __fadd2_rn(make_float2(unit_v(r[k]), unit_v(r[k + 1])),
                                    make_float2(-pa[k], -pa[k + 1]));  // exact
        const float2 th = __fmul2_rn(hh2, d);
        const float2 nth = __fmul2_rn(th, m1);
        const float2 tl = __fadd2_rn(__ffma2_rn(hh2, d, nth), __ffma2_rn(hl2, d, pb2));
        const float2 nqg = __fadd2_rn(__ffma2_rn(nth, th, m256), p256);  // -qg
        const float2 rr = __ffma2_rn(th, th, nqg);
        const float2 c = __ffma2_rn(th, tl, __ffma2_rn(th, tl, rr));
        nzh2 = __fadd2_rn(nzh2, nqg);
        zl2 = __fadd2_rn(zl2, c);
      }
      zh = -__fadd_rn(nzh2.x, nzh2.y);
      zl = __fadd_rn(zl2.x, zl2.y);
      i0 = D & ~1;
    }
#endif
#pragma unroll
    for (int i = i0; i < D; ++i) {
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
      if (D == 1) {
        zh = __fmul_rn(th, th);
        zl = fmaf(__fadd_rn(th, th), tl, fmaf(th, th, -zh));
      } else {
        // t_i^2 = qg + c with qg on the grid of 2^-15: fl(th^2 + 256) has that
        // spacing while th^2 < 256 and removing the 256 is exact (Sterbenz), so
        // qg is th^2 rounded once to a multiple of 2^-15, r = th^2 - qg
        // (|r| <= 2^-16, exact to 2^-40), and c adds 2 th tl.  Multiples of
        // 2^-15 add exactly in FP32 while the sum stays below 512, so zh needs
        // no error term; beyond that (or th^2 >= 256) f is below 2^-256 and
        // flushes to zero anyway.
        const float qg = __fsub_rn(fmaf(th, th, 256.0f), 256.0f);
        const float r = fmaf(th, th, -qg);
        const float c = fmaf(th, tl, fmaf(th, tl, r));
        zh = (i == 0) ? qg : __fadd_rn(zh, qg);
        zl = (i == 0) ? c : __fadd_rn(zl, c);  // i > 0 whenever pairs came first
      }
    }
    return amp_exp2_neg(A, zh, zl);
  }
};

template <>
__device__ void dispatch_item<ZMC_GAUSS>(const FnDev *fn, uint64_t chunk, uint32_t Q,
                                      uint32_t lane) {
  switch (fn->variant) {
    ZMC_GAUSS_VARIANTS(ZMC_ITEM_CASE)
    default:
      break;
  }
}

template <>
__device__ void dispatch_eval<ZMC_GAUSS>(const FnDev *fn, uint64_t s_begin, uint32_t count,
                                      float *out) {
  switch (fn->variant) {
    ZMC_GAUSS_VARIANTS(ZMC_EVAL_CASE)
    default:
      break;
  }
}

}  // namespace

const FamilyOps ZMC_FAMILY_OPS(kFamilyGauss) = family_ops<ZMC_GAUSS>();

}  // namespace zmc
