// zmc_kernels.cu -- the kernels shared by every integrand family, and the
// host-side dispatch to the per-family sampling paths (zmc_fam_<family>.cu).
//
//   zmc_batched_kernel<FAM>  (one file per family) persistent work-list launch over
//                        (integrand, chunk) items: Philox4x32-10 -> map onto the
//                        box -> FP32 integrand -> per-lane shifted sums -> warp
//                        Chan merge -> one (mean, M2) record per chunk.  Direct MC
//                        per integrand is the paper's solution method (Sec.
//                        "Solution method"); many integrands of different form,
//                        dimension and box share one launch (Sec. "Summary of
//                        revisions", Eq. 1, Eq. 2).
//   zmc_merge_kernel     FP64 k-way Chan merge of an integrand's chunk records in a
//                        fixed order: mean, M2, estimate = V mean,
//                        stderr = V sqrt(M2 / (N (N-1))) (Fig. 1 caption: an estimate
//                        with its spread).
//   zmc_plain_fp64_kernel  (zmc_plain.cu) the plain form, one launch per integrand.
//   zmc_philox_rate_kernel  the generator alone (its throughput: the ceiling of
//                        any sampling kernel, which draws d / 5 blocks per sample).
//   zmc_philox_kernel, zmc_eval_kernel<FAM>   the generator and the per-sample
//                        integrand values of the sampling path, for parity tests.
//
// No tensor cores and no TMA: the path is integer and FP32 arithmetic on the FMA,
// ALU and MUFU pipes, with a few KB of descriptor reads and 8 bytes written per
// 160 * quints_per_lane samples.
#include "zmc_device.cuh"

namespace zmc {
namespace {

// ---------------------------------------------------------------- FP64 merge
// One warp per integrand.  With chunk summaries (n_c, m_c, M2_c):
//   mean = sum_c n_c m_c / N,  M2 = sum_c [M2_c + n_c (m_c - mean)^2]
// (Chan et al.'s combination of partial moments, all chunks at once), summed in a
// fixed lane / butterfly order, so the result depends only on the records.  Moments
// of earlier samples of the stream (prior_n > 0) are combined in last with the
// pairwise update, n = n_a + n_b, mean = mean_a + d n_b / n,
// M2 = M2_a + M2_b + d^2 n_a n_b / n, d = mean_b - mean_a.
__global__ void __launch_bounds__(256) zmc_merge_kernel(const FnDev *const *__restrict__ fns,
                                                        const LaunchHdr *__restrict__ hdr) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t nm = hdr->n_merge;
  const uint64_t chunk_samples = chunk_samples_of(hdr->quints_per_lane);
  for (uint32_t k = warp; k < nm; k += nwarps) {
    const FnDev *fn = fns[k];
    const uint64_t N = fn->n_samples;
    const uint64_t C = (N + chunk_samples - 1) / chunk_samples;
    const float2 *rec = fn->rec;
    double s = 0.0;
    for (uint64_t c = lane; c < C; c += 32) {
      const uint64_t left = N - c * chunk_samples;
      const double nc = static_cast<double>(left < chunk_samples ? left : chunk_samples);
      s = fma(nc, static_cast<double>(rec[c].x), s);
    }
    const double mean = N ? warp_sum_f64(s) / static_cast<double>(N) : 0.0;
    double m = 0.0;
    for (uint64_t c = lane; c < C; c += 32) {
      const uint64_t left = N - c * chunk_samples;
      const double nc = static_cast<double>(left < chunk_samples ? left : chunk_samples);
      const float2 rc = rec[c];
      const double dm = static_cast<double>(rc.x) - mean;
      m += fma(nc * dm, dm, static_cast<double>(rc.y));
    }
    const double inv = fn->inv_scale;
    double mu = mean * inv;
    double m2 = fmax(warp_sum_f64(m), 0.0) * inv * inv;
    uint64_t n_all = N;
    if (fn->prior_n > 0) {
      const double na = static_cast<double>(fn->prior_n), nb = static_cast<double>(N);
      const double nab = na + nb;
      const double d = mu - fn->prior_mean;
      mu = fn->prior_mean + d * (nb / nab);
      m2 = fn->prior_m2 + m2 + d * d * (na * nb / nab);
      n_all = fn->prior_n + N;
    }
    if (lane == 0) {
      const double nd = static_cast<double>(n_all);
      zmc_result res;
      if (fn->out_mode == 0) {
        res.estimate = fn->volume * mu;
        res.stderr_ = fn->volume * sqrt(m2 / (nd * (nd - 1.0)));
      } else {  // zmc_moments: unscaled mean and M2 of f over the samples
        res.estimate = mu;
        res.stderr_ = m2;
      }
      res.n = n_all;
      res.status = ZMC_OK;
      res.reserved = 0;
      *fn->out = res;
    }
  }
}

// ---------------------------------------------------------------- test kernels
__global__ void zmc_philox_kernel(const uint32_t *__restrict__ ctr,
                                  const uint32_t *__restrict__ key, uint32_t *__restrict__ out,
                                  size_t n) {
  for (size_t j = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; j < n;
       j += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const RoundKeys rk = make_round_keys(key[2 * j], key[2 * j + 1]);
    const uint4 o = philox(ctr[4 * j], ctr[4 * j + 1], ctr[4 * j + 2], ctr[4 * j + 3], rk);
    out[4 * j + 0] = o.x;
    out[4 * j + 1] = o.y;
    out[4 * j + 2] = o.z;
    out[4 * j + 3] = o.w;
  }
}

// Generator rate: every thread draws per_thread Philox4x32-10 blocks, four
// independent calls at a time, with the sampling kernels' counter layout and
// chunk prefix (block lo advancing; stream word, block hi and key the same for
// the whole warp) and their launch bound, and folds the words into one so that
// none is dead.
__global__ void __launch_bounds__(256, 2) zmc_philox_rate_kernel(uint32_t key0, uint32_t key1,
                                                                 uint32_t sid,
                                                                 uint32_t per_thread,
                                                                 uint32_t *__restrict__ out) {
  const StreamPrefix sp = make_stream_prefix(make_round_keys(key0, key1), sid, 0u);
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t base = t * per_thread;  // wraps on huge grids: a rate needs no distinct counters
  uint32_t acc = 0;
  for (uint32_t q = 0; q < per_thread; q += 4) {
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
      const uint4 o = philox_block(base + q + j, sp);
      acc ^= o.x ^ o.y ^ o.z ^ o.w;
    }
  }
  out[t] = acc;
}

const FamilyOps *ops_of(int family, int unroll = 1) {
  static const FamilyOps *const kOps[kMaxUnroll][4] = {
      {&kFamilyHarmonicU1, &kFamilyAbslinU1, &kFamilyGaussU1, &kFamilyPolyU1},
      {&kFamilyHarmonicU2, &kFamilyAbslinU2, &kFamilyGaussU2, &kFamilyPolyU2}};
  if (family < 0 || family > ZMC_POLY || unroll < 1 || unroll > kMaxUnroll) return nullptr;
  return kOps[unroll - 1][family];
}

}  // namespace

// ---------------------------------------------------------------- launch wrappers
cudaError_t launch_batched(int family, const Entry *entries, LaunchHdr *hdr, unsigned grid,
                           unsigned block, cudaStream_t stream, int unroll) {
  const FamilyOps *ops = ops_of(family, unroll);
  return ops ? ops->launch_batched(entries, hdr, grid, block, stream) : cudaErrorInvalidValue;
}

cudaError_t launch_merge(const FnDev *const *fns, const LaunchHdr *hdr, unsigned grid,
                         cudaStream_t stream) {
  zmc_merge_kernel<<<grid, 256, 0, stream>>>(fns, hdr);
  return cudaGetLastError();
}

int batched_max_blocks_per_sm(int family, int block, int unroll) {
  const FamilyOps *ops = ops_of(family, unroll);
  return ops ? ops->max_blocks_per_sm(block) : 0;
}

int batched_regs_per_thread(int family, int unroll) {
  const FamilyOps *ops = ops_of(family, unroll);
  return ops ? ops->regs_per_thread() : 0;
}

cudaError_t launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, size_t n,
                          cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + 255) / 256;
  zmc_philox_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(
      ctr, key, out, n);
  return cudaGetLastError();
}

cudaError_t launch_philox_rate(uint32_t per_thread, unsigned grid, uint32_t *out,
                               cudaStream_t stream) {
  zmc_philox_rate_kernel<<<grid, 256, 0, stream>>>(0x2104u, 0x10073u, 7u, per_thread, out);
  return cudaGetLastError();
}

cudaError_t launch_eval(int family, const FnDev *fn, uint64_t s_begin, uint32_t count,
                        float *out, cudaStream_t stream) {
  const FamilyOps *ops = ops_of(family);
  return ops ? ops->launch_eval(fn, s_begin, count, out, stream) : cudaErrorInvalidValue;
}

}  // namespace zmc
