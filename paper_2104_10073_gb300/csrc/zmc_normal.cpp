// zmc_normal.cpp -- stratified sampling with a heuristic tree search, the
// paper's ZMCintegral_normal use case (Sec. "Solution method" and "Additional
// comments": the integration domain is stratified and the strata are refined by
// a heuristic tree search, for integrands of higher dimension, 8 to 12).
//
// The paper names the two techniques but gives none of their steps; this file
// implements the following reading, which the CPU oracle (oracle/normal.py)
// restates step by step:
//   1. Level 0: the box is cut into k^d equal cells (k = divisions per
//      dimension; cell j has grid index (j / k^i) mod k in dimension i).
//   2. Every cell is integrated by direct Monte Carlo with samples_per_cell
//      samples on its own Philox stream (the j-th cell created uses stream
//      stream_base + j, key = seed): cell estimate e_c = V_c mean_c and its
//      standard error s_c = V_c sqrt(M2_c / (N_c (N_c - 1))).  All new cells of
//      a round are one batched launch of the sampling kernels.
//   3. A refinement round takes the leaves (cells not split) in order,
//      threshold tau = sigma_mult * (sum of leaf s_c) / (number of leaves), and
//      splits every leaf with s_c > tau into its 2^d halves (child b takes the
//      upper half of dimension i when bit i of b is set), as long as the leaf
//      count stays within max_leaves; the children replace their parent in the
//      leaf order and are evaluated as in step 2.  At most `depth` rounds; a
//      round that splits nothing ends the search.
//   4. Estimate = sum over leaves of e_c, stderr = sqrt(sum of s_c^2) (strata
//      are independent), both summed in leaf order in FP64.
// Steps 1, 3 and 4 are host bookkeeping over the per-cell results; step 2 runs
// on the GPU (the built-in families through the batched plan path, user
// integrands through the run-time compiled kernel).
#include <cmath>
#include <cstring>
#include <vector>

#include "zmc_runtime.h"

using namespace zmc;

namespace {

struct Tree {
  uint32_t dim = 0;
  std::vector<double> lo, hi;   // cell boxes, dim values each
  std::vector<uint32_t> stream;
  std::vector<double> est, err;  // per cell, once evaluated
  size_t n_cells() const { return stream.size(); }
  void add(const double *l, const double *h, uint32_t s) {
    lo.insert(lo.end(), l, l + dim);
    hi.insert(hi.end(), h, h + dim);
    stream.push_back(s);
    est.push_back(0.0);
    err.push_back(0.0);
  }
};

// Evaluates cells [first, tree.n_cells()) of the tree.
using EvalFn = zmc_status (*)(void *user, Tree &tree, size_t first);

struct BuiltinCtx {
  zmc_ctx *ctx;
  zmc_desc base;
  uint64_t n, seed;
};

zmc_status eval_builtin(void *user, Tree &t, size_t first) {
  auto *b = static_cast<BuiltinCtx *>(user);
  const size_t m = t.n_cells() - first;
  std::vector<zmc_desc> tab(m, b->base);
  for (size_t q = 0; q < m; ++q) {
    zmc_desc &d = tab[q];
    const size_t c = first + q;
    for (uint32_t i = 0; i < t.dim; ++i) {
      d.lo[i] = t.lo[c * t.dim + i];
      d.hi[i] = t.hi[c * t.dim + i];
    }
    d.n_samples = b->n;
    d.seed = b->seed;
    d.stream_id = t.stream[c];
  }
  std::vector<zmc_result> res(m);
  const zmc_status st = zmc_integrate(b->ctx, tab.data(), m, res.data());
  if (st != ZMC_OK) return st;
  for (size_t q = 0; q < m; ++q) {
    t.est[first + q] = res[q].estimate;
    t.err[first + q] = res[q].stderr_;
  }
  return ZMC_OK;
}

struct UdfCtx {
  zmc_ctx *ctx;
  const zmc_udf *udf;
  const double *p;
  uint64_t n, seed;
};

zmc_status eval_udf(void *user, Tree &t, size_t first) {
  auto *u = static_cast<UdfCtx *>(user);
  const size_t m = t.n_cells() - first;
  std::vector<UdfRow> rows(m);
  for (size_t q = 0; q < m; ++q) {
    const size_t c = first + q;
    rows[q].dim = t.dim;
    rows[q].stream_id = t.stream[c];
    rows[q].n_samples = u->n;
    rows[q].seed = u->seed;
    rows[q].lo = &t.lo[c * t.dim];
    rows[q].hi = &t.hi[c * t.dim];
    rows[q].p = u->p;
  }
  std::vector<zmc_result> res(m);
  const zmc_status st = udf_run(u->ctx, u->udf, rows.data(), m, res.data());
  if (st != ZMC_OK) return st;
  for (size_t q = 0; q < m; ++q) {
    t.est[first + q] = res[q].estimate;
    t.err[first + q] = res[q].stderr_;
  }
  return ZMC_OK;
}

zmc_status run_tree(uint32_t dim, const double *lo, const double *hi, const zmc_normal_opts &o,
                    EvalFn eval, void *user, zmc_normal_result *out) {
  const uint32_t k = o.divisions;
  if (k < 1) return set_error(ZMC_EINVAL, "divisions must be >= 1");
  if (o.samples_per_cell < 2 || o.samples_per_cell > (1ull << 40))
    return set_error(ZMC_EINVAL, "samples_per_cell must be in 2..2^40");
  if (!(o.sigma_mult > 0.0) || !std::isfinite(o.sigma_mult))
    return set_error(ZMC_EINVAL, "sigma_mult must be finite and > 0");
  const uint64_t max_leaves = o.max_leaves ? o.max_leaves : (1ull << 20);
  if (max_leaves > (1ull << 22)) return set_error(ZMC_EINVAL, "max_leaves above 2^22");
  uint64_t n0 = 1;
  for (uint32_t i = 0; i < dim; ++i) {
    n0 *= k;
    if (n0 > (1ull << 20)) return set_error(ZMC_EINVAL, "divisions^dim above 2^20 cells");
    if (!std::isfinite(lo[i]) || !std::isfinite(hi[i]) || !(lo[i] < hi[i]))
      return set_error(ZMC_EINVAL, "box dimension %u needs finite lo < hi", i);
  }
  const uint64_t n_children = 1ull << dim;
  uint64_t next_stream = o.stream_base;
  auto take_stream = [&](uint32_t *s) {
    if (next_stream > 0xffffffffull) return false;
    *s = static_cast<uint32_t>(next_stream++);
    return true;
  };

  Tree t;
  t.dim = dim;
  std::vector<double> cl(dim), ch(dim);
  for (uint64_t j = 0; j < n0; ++j) {
    uint64_t r = j;
    for (uint32_t i = 0; i < dim; ++i) {
      const uint64_t idx = r % k;
      r /= k;
      const double w = hi[i] - lo[i];
      cl[i] = lo[i] + (w * static_cast<double>(idx)) / static_cast<double>(k);
      ch[i] = idx + 1 == k ? hi[i] : lo[i] + (w * static_cast<double>(idx + 1)) / static_cast<double>(k);
    }
    uint32_t s;
    if (!take_stream(&s)) return set_error(ZMC_EINVAL, "stream ids exceed 32 bits");
    t.add(cl.data(), ch.data(), s);
  }
  zmc_status st = eval(user, t, 0);
  if (st != ZMC_OK) return st;
  std::vector<size_t> leaves(n0);
  for (uint64_t j = 0; j < n0; ++j) leaves[j] = j;

  uint32_t rounds = 0;
  for (uint32_t r = 0; r < o.depth; ++r) {
    double sum = 0.0;
    for (size_t c : leaves) sum += t.err[c];
    const double tau = o.sigma_mult * (sum / static_cast<double>(leaves.size()));
    std::vector<size_t> next;
    next.reserve(leaves.size());
    const size_t first_new = t.n_cells();
    uint64_t n_leaves = leaves.size();
    bool split_any = false;
    for (size_t c : leaves) {
      const bool want = t.err[c] > tau && n_leaves + n_children - 1 <= max_leaves;
      if (!want) {
        next.push_back(c);
        continue;
      }
      split_any = true;
      n_leaves += n_children - 1;
      for (uint64_t b = 0; b < n_children; ++b) {
        for (uint32_t i = 0; i < dim; ++i) {
          const double l = t.lo[c * dim + i], h = t.hi[c * dim + i];
          const double mid = l + (h - l) * 0.5;
          const bool upper = (b >> i) & 1u;
          cl[i] = upper ? mid : l;
          ch[i] = upper ? h : mid;
        }
        uint32_t s;
        if (!take_stream(&s)) return set_error(ZMC_EINVAL, "stream ids exceed 32 bits");
        t.add(cl.data(), ch.data(), s);
        next.push_back(t.n_cells() - 1);
      }
    }
    if (!split_any) break;
    st = eval(user, t, first_new);
    if (st != ZMC_OK) return st;
    leaves.swap(next);
    ++rounds;
  }
  double est = 0.0, var = 0.0;
  for (size_t c : leaves) {
    est += t.est[c];
    var += t.err[c] * t.err[c];
  }
  out->estimate = est;
  out->stderr_ = std::sqrt(var);
  out->n_samples = static_cast<uint64_t>(t.n_cells()) * o.samples_per_cell;
  out->n_cells = t.n_cells();
  out->n_leaves = leaves.size();
  out->rounds = rounds;
  out->status = ZMC_OK;
  return ZMC_OK;
}

}  // namespace

extern "C" {

zmc_status zmc_normal_default_options(zmc_normal_opts *opt) {
  if (!opt) return set_error(ZMC_EINVAL, "null options");
  std::memset(opt, 0, sizeof *opt);
  opt->divisions = 2;
  opt->depth = 2;
  opt->samples_per_cell = 1u << 14;
  opt->sigma_mult = 2.0;
  opt->max_leaves = 1u << 20;
  return ZMC_OK;
}

zmc_status zmc_normal_integrate(zmc_ctx *ctx, const zmc_desc *base, const zmc_normal_opts *opt,
                                zmc_normal_result *out) {
  if (!ctx || !base || !opt || !out) return set_error(ZMC_EINVAL, "null argument");
  if (base->dim < 1 || base->dim > ZMC_MAX_DIM)
    return set_error(ZMC_EINVAL, "dim %u not in 1..%d", base->dim, ZMC_MAX_DIM);
  std::memset(out, 0, sizeof *out);
  zmc_desc check = *base;
  check.n_samples = 2;
  zmc_status st = zmc_validate(&check, 1, nullptr);
  if (st != ZMC_OK) return st;
  BuiltinCtx b{ctx, *base, opt->samples_per_cell, opt->seed};
  return run_tree(base->dim, base->lo, base->hi, *opt, eval_builtin, &b, out);
}

zmc_status zmc_normal_integrate_udf(zmc_ctx *ctx, const zmc_udf *udf, const double *lo,
                                    const double *hi, const double *p,
                                    const zmc_normal_opts *opt, zmc_normal_result *out) {
  if (!ctx || !udf || !lo || !hi || !p || !opt || !out)
    return set_error(ZMC_EINVAL, "null argument");
  std::memset(out, 0, sizeof *out);
  UdfCtx u{ctx, udf, p, opt->samples_per_cell, opt->seed};
  return run_tree(udf_dim(udf), lo, hi, *opt, eval_udf, &u, out);
}

}  // extern "C"
