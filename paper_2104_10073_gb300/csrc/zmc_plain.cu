// zmc_plain.cu -- the plain FP64 form: one direct-MC launch per integrand
// (FP64 map and evaluation with the CUDA math library, FP64 block reductions of
// (n, mean, M2)), then one merge launch for all integrands.  The baseline the
// batched FP32 path is measured against; same generator and field layout.
#include "zmc_device.cuh"

namespace zmc {
namespace {

template <int FAM>
__device__ __forceinline__ double eval_f64(const PlainFn &fn, const double *x, int d) {
  const double *p = fn.p;
  if (FAM == ZMC_HARMONIC) {
    double ph = 0.0;
    for (int i = 0; i < d; ++i) ph = fma(p[2 + i], x[i], ph);
    double s, c;
    sincos(ph, &s, &c);
    return fma(p[0], c, p[1] * s);
  } else if (FAM == ZMC_ABSLIN) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s = fma(p[1 + i], x[i], s);
    return p[0] * fabs(s);
  } else if (FAM == ZMC_GAUSS) {
    double r2 = 0.0;
    for (int i = 0; i < d; ++i) {
      const double t = x[i] - p[2 + i];
      r2 = fma(t, t, r2);
    }
    return p[0] * exp(-r2 / (2.0 * p[1] * p[1]));
  } else {
    double prod = 1.0;
    for (int i = 0; i < d; ++i) {
      double acc = p[5 * i + fn.deg];
      for (int j = static_cast<int>(fn.deg) - 1; j >= 0; --j) acc = fma(acc, x[i], p[5 * i + j]);
      prod *= acc;
    }
    return prod;
  }
}

// One thread per quint (grid-stride); per-thread FP64 shifted sums; block-level
// Chan merge in shared memory; one (n, mean, M2) record per block.
template <int FAM, int D>
__global__ void __launch_bounds__(256) zmc_plain_fp64_kernel(const PlainFn fn,
                                                             double *__restrict__ rec) {
  const RoundKeys rk = make_round_keys(fn.key0, fn.key1);
  const uint64_t N = fn.n_samples;
  const uint64_t nquints = (N + kQuint - 1) / kQuint;
  double K = 0.0, s1 = 0.0, s2 = 0.0, cnt = 0.0;
  for (uint64_t q = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; q < nquints;
       q += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    uint32_t r[5 * D];
    gen_quint<D>(q, fn.stream_id, rk, r);
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      if (kQuint * q + t < N) {
        double x[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          const double u = static_cast<double>(r[t * D + i] & 0x7FFFFFu) * 0x1p-23;
          x[i] = fma(fn.w[i], u, fn.lo[i]);
        }
        const double f = eval_f64<FAM>(fn, x, D);
        if (cnt == 0.0) K = f;
        const double dlt = f - K;
        s1 += dlt;
        s2 = fma(dlt, dlt, s2);
        cnt += 1.0;
      }
    }
  }
  __shared__ double sn[256], sm[256], sq[256];
  double mean = 0.0, m2 = 0.0;
  if (cnt > 0.0) {
    mean = K + s1 / cnt;
    m2 = fmax(s2 - s1 * (s1 / cnt), 0.0);
  }
  sn[threadIdx.x] = cnt;
  sm[threadIdx.x] = mean;
  sq[threadIdx.x] = m2;
  __syncthreads();
  for (unsigned half = blockDim.x >> 1; half > 0; half >>= 1) {
    if (threadIdx.x < half) {
      const double na = sn[threadIdx.x], nb = sn[threadIdx.x + half];
      if (nb > 0.0) {
        const double nab = na + nb;
        const double delta = sm[threadIdx.x + half] - sm[threadIdx.x];
        sm[threadIdx.x] += delta * (nb / nab);
        sq[threadIdx.x] += sq[threadIdx.x + half] + delta * delta * (na * nb / nab);
        sn[threadIdx.x] = nab;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    rec[3 * blockIdx.x + 0] = sn[0];
    rec[3 * blockIdx.x + 1] = sm[0];
    rec[3 * blockIdx.x + 2] = sq[0];
  }
}

// One warp per integrand: Chan's combination of the block records, fixed order.
__global__ void zmc_plain_merge_kernel(const PlainJob *__restrict__ jobs, uint32_t n) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= n) return;
  const PlainJob jb = jobs[warp];
  double nsum = 0.0, s = 0.0;
  for (uint32_t b = lane; b < jb.nblk; b += 32) {
    nsum += jb.rec[3 * b];
    s = fma(jb.rec[3 * b], jb.rec[3 * b + 1], s);
  }
  const double N = warp_sum_f64(nsum);
  const double mean = warp_sum_f64(s) / N;
  double m = 0.0;
  for (uint32_t b = lane; b < jb.nblk; b += 32) {
    const double dm = jb.rec[3 * b + 1] - mean;
    m += fma(jb.rec[3 * b] * dm, dm, jb.rec[3 * b + 2]);
  }
  const double m2 = fmax(warp_sum_f64(m), 0.0);
  if (lane == 0) {
    zmc_result res;
    res.estimate = jb.volume * mean;
    res.stderr_ = jb.volume * sqrt(m2 / (N * (N - 1.0)));
    res.n = static_cast<uint64_t>(N);
    res.status = ZMC_OK;
    res.reserved = 0;
    *jb.out = res;
  }
}

}  // namespace

unsigned plain_grid(const PlainFn &fn, int sms) {
  const uint64_t nquints = (fn.n_samples + kQuint - 1) / kQuint;
  const uint64_t want = (nquints + 255) / 256;
  const uint64_t cap = static_cast<uint64_t>(sms) * 8;
  return static_cast<unsigned>(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_plain(const PlainFn &fn, double *block_rec, unsigned grid,
                         cudaStream_t stream) {
  switch (fn.family * 8 + fn.dim) {
#define ZMC_PCASE(F, D, G) \
  case F * 8 + D: zmc_plain_fp64_kernel<F, D><<<grid, 256, 0, stream>>>(fn, block_rec); break;
    ZMC_HARMONIC_VARIANTS(ZMC_PCASE)
    ZMC_ABSLIN_VARIANTS(ZMC_PCASE)
    ZMC_VARIANTS_DIM(ZMC_PCASE, ZMC_GAUSS, 0)
    ZMC_VARIANTS_DIM(ZMC_PCASE, ZMC_POLY, 0)
#undef ZMC_PCASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_plain_merge(const PlainJob *jobs, uint32_t n, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = (n + 7) / 8;
  zmc_plain_merge_kernel<<<grid, 256, 0, stream>>>(jobs, n);
  return cudaGetLastError();
}

}  // namespace zmc
