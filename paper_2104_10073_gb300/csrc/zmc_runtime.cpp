// zmc_runtime.cpp -- host runtime of the GB300 multi-function Monte Carlo
// library: descriptor validation and FP64 precompute, the device arena, plans
// (device-resident tables replayed as CUDA graphs), and the C ABI entry points
// other than serving (zmc_serving.cpp).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <numeric>
#include <sstream>

#include "zmc_runtime.h"

namespace zmc {

namespace {
thread_local std::string g_last_error;
}

zmc_status set_error(zmc_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

zmc_status ctx_cuda_fail(zmc_ctx *ctx, cudaError_t err, const char *what) {
  if (ctx) ctx->poisoned = true;
  return set_error(ZMC_ECUDA, "%s: %s", what, cudaGetErrorString(err));
}

#define ZMC_CUDA(ctx, call)                                              \
  do {                                                                   \
    cudaError_t zmc_err_ = (call);                                       \
    if (zmc_err_ != cudaSuccess) return ctx_cuda_fail(ctx, zmc_err_, #call); \
  } while (0)

// ---------------------------------------------------------------- arena
void Arena::init(char *base, size_t bytes) {
  std::lock_guard<std::mutex> g(mu_);
  base_ = base;
  size_ = bytes & ~static_cast<size_t>(255);
  used_ = 0;
  free_.clear();
  allocated_.clear();
  if (size_) free_[0] = size_;
}

void *Arena::alloc(size_t bytes) {
  std::lock_guard<std::mutex> g(mu_);
  bytes = (std::max<size_t>(bytes, 1) + 255) & ~static_cast<size_t>(255);
  for (auto it = free_.begin(); it != free_.end(); ++it) {
    if (it->second < bytes) continue;
    const size_t off = it->first, len = it->second;
    free_.erase(it);
    if (len > bytes) free_[off + bytes] = len - bytes;
    allocated_[off] = bytes;
    used_ += bytes;
    return base_ + off;
  }
  return nullptr;
}

void Arena::release(void *p) {
  if (!p) return;
  std::lock_guard<std::mutex> g(mu_);
  const size_t off = static_cast<size_t>(static_cast<char *>(p) - base_);
  auto a = allocated_.find(off);
  if (a == allocated_.end()) return;
  size_t len = a->second;
  allocated_.erase(a);
  used_ -= len;
  size_t start = off;
  auto next = free_.lower_bound(off);
  if (next != free_.end() && next->first == off + len) {
    len += next->second;
    next = free_.erase(next);
  }
  if (next != free_.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == start) {
      start = prev->first;
      len += prev->second;
      free_.erase(prev);
    }
  }
  free_[start] = len;
}

size_t Arena::largest_free() const {
  std::lock_guard<std::mutex> g(mu_);
  size_t m = 0;
  for (auto &kv : free_) m = std::max(m, kv.second);
  return m;
}

// ---------------------------------------------------------------- precompute
namespace {
constexpr double kTwoPi = 6.283185307179586476925286766559;

void split(double v, uint32_t *hi, uint32_t *lo) {
  const float h = static_cast<float>(v);
  const float l = static_cast<float>(v - static_cast<double>(h));
  std::memcpy(hi, &h, 4);
  std::memcpy(lo, &l, 4);
}

void put_f32(uint32_t *dst, double v) {
  const float f = static_cast<float>(v);
  std::memcpy(dst, &f, 4);
}

bool finite_f32(double v) {
  return std::isfinite(v) && std::fabs(v) <= static_cast<double>(std::numeric_limits<float>::max());
}

double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
}  // namespace

// Product polynomial of degree g >= 2 in root form (variant degree g + 3).  Each
// factor is lead * (its roots grouped into "quads" and, for g = 3, one linear
// term): a quad is (u - p1)(u - p2) + c, either a pair of real roots (p1, p2,
// c = 0) or a complex pair a +- ib (p1 = p2 = a, c = b^2); the linear term is
// u - r.  Words per dimension i: g = 2: quad (p1 hi, p1 lo, p2 hi, p2 lo, c) at
// w[5i..]; g = 3: linear (r hi, r lo) then quad at w[7i..]; g = 4: two quads at
// w[10i..]; the amplitude S prod_i lead_i at w[70].  False (keep the
// coefficient form) when a factor has no reliable root form or a lower degree
// than g, a leading coefficient below 1e-6 of its factor's coefficient sum, or
// a root beyond 2^10 in size.
static bool poly_roots_payload(const double (*e)[5], int dim, int g, double S, FnDev *fn) {
  const int words = g == 2 ? 5 : g == 3 ? 7 : 10;
  double amp = S;
  uint32_t w[kMaxDim * 10];
  for (int i = 0; i < dim; ++i) {
    RootForm rf;
    if (!poly_root_form(e[i], g, &rf) || rf.n != g) return false;
    double sum = 0.0;
    for (int k = 0; k <= g; ++k) sum += std::fabs(e[i][k]);
    if (!(std::fabs(rf.lead) >= 1e-6 * sum)) return false;
    double reals[4], ca[2], cb2[2];
    int nr = 0, nc = 0;
    for (int s = 0; s < rf.n; ++s) {
      if (!(std::fabs(rf.v[s]) <= 1024.0)) return false;
      if (rf.type[s] == 1) reals[nr++] = rf.v[s];
      if (rf.type[s] == 2) {
        ca[nc] = rf.v[s];
        cb2[nc++] = rf.v[s + 1];
      }
    }
    uint32_t *o = w + words * i;
    auto quad = [&](uint32_t *q, double p1, double p2, double c) {
      split(p1, &q[0], &q[1]);
      split(p2, &q[2], &q[3]);
      put_f32(&q[4], c);
    };
    int ri = 0, ci = 0;
    if (g == 3) {  // the linear term takes a real root (a cubic has at least one)
      split(reals[ri], &o[0], &o[1]);
      ++ri;
      o += 2;
    }
    for (int qd = 0; qd < (g == 3 ? 1 : g / 2); ++qd, o += 5) {
      if (ci < nc) {
        quad(o, ca[ci], ca[ci], cb2[ci]);
        ++ci;
      } else if (ri + 1 < nr) {
        quad(o, reals[ri], reals[ri + 1], 0.0);
        ri += 2;
      } else {
        return false;
      }
    }
    amp *= rf.lead;
  }
  if (!finite_f32(amp)) return false;
  std::memcpy(fn->w, w, sizeof(uint32_t) * words * dim);
  put_f32(&fn->w[70], amp);
  fn->variant = variant_code(ZMC_POLY, static_cast<uint32_t>(dim), static_cast<uint32_t>(g + 3));
  return true;
}

// Abs-linear rows with at least this many samples use the 32-bit sum of c.x.
constexpr uint64_t kAbsLinNarrowMinSamples = 256;

zmc_status precompute(const zmc_desc &d, FnDev *fn, PlainFn *plain, double *volume) {
  if (d.family > ZMC_POLY) return set_error(ZMC_EINVAL, "unknown family %u", d.family);
  if (d.dim < 1 || d.dim > kMaxDim) return set_error(ZMC_EINVAL, "dim %u not in 1..7", d.dim);
  if (d.n_samples == 0) return set_error(ZMC_EINVAL, "n_samples must be >= 1");
  if (d.n_samples > (1ull << 62)) return set_error(ZMC_EINVAL, "n_samples too large");
  if (d.family == ZMC_POLY && d.deg > 4) return set_error(ZMC_EINVAL, "poly degree %u > 4", d.deg);
  const int dim = static_cast<int>(d.dim);
  double w[kMaxDim] = {0};
  double vol = 1.0;
  for (int i = 0; i < dim; ++i) {
    if (!std::isfinite(d.lo[i]) || !std::isfinite(d.hi[i]) || !(d.lo[i] < d.hi[i]))
      return set_error(ZMC_EINVAL, "box dimension %d: need finite lo < hi", i);
    w[i] = d.hi[i] - d.lo[i];
    vol *= w[i];
  }
  for (int j = 0; j < ZMC_NPARAM; ++j)
    if (!std::isfinite(d.p[j])) return set_error(ZMC_EINVAL, "parameter p[%d] not finite", j);

  std::memset(fn, 0, sizeof(FnDev));
  const double *p = d.p;
  // An upper bound of |f| over the box; the kernel works on S f with
  // S = 2^(48 - ceil(log2 bound)) (clamped), undone exactly in the merge.
  double fsup = 0.0;
  double poly_e[kMaxDim][5] = {{0}};
  switch (d.family) {
    case ZMC_HARMONIC:
      fsup = std::fabs(p[0]) + std::fabs(p[1]);
      break;
    case ZMC_ABSLIN: {
      double up = 0.0, dn = 0.0;
      for (int i = 0; i < dim; ++i) {
        const double c = p[1 + i];
        up += c * (c > 0 ? d.hi[i] : d.lo[i]);
        dn += c * (c > 0 ? d.lo[i] : d.hi[i]);
      }
      fsup = std::fabs(p[0]) * std::max(std::fabs(up), std::fabs(dn));
      break;
    }
    case ZMC_GAUSS:
      fsup = std::fabs(p[0]);
      break;
    default: {  // POLY: q_i(u) = sum_j c_ij (lo_i + w_i u)^j = sum_k e_ik u^k
      const int g = static_cast<int>(d.deg);
      fsup = 1.0;
      for (int i = 0; i < dim; ++i) {
        double bound = 0.0;
        for (int k = 0; k <= g; ++k) {
          double e = 0.0;
          for (int j = k; j <= g; ++j)
            e += p[5 * i + j] * binom(j, k) * std::pow(d.lo[i], j - k) * std::pow(w[i], k);
          poly_e[i][k] = e;
          bound += std::fabs(e);
        }
        fsup *= bound;
      }
      break;
    }
  }
  int sexp = 0;
  if (fsup > 0.0 && std::isfinite(fsup)) {
    sexp = 48 - static_cast<int>(std::ceil(std::log2(fsup)));
    sexp = std::max(-100, std::min(100, sexp));
  }
  const double S = std::ldexp(1.0, sexp);
  fn->variant = variant_code(d.family, d.dim, d.family == ZMC_POLY ? d.deg : 0);
  fn->stream_id = d.stream_id;
  fn->key0 = static_cast<uint32_t>(d.seed);
  fn->key1 = static_cast<uint32_t>(d.seed >> 32);
  fn->n_samples = d.n_samples;
  fn->volume = vol;
  fn->inv_scale = std::ldexp(1.0, -sexp);
  bool ok = true;
  switch (d.family) {
    case ZMC_HARMONIC: {
      // f = R cos(2 pi P): R = S sqrt(a^2+b^2), P = k.x/(2 pi) - atan2(b,a)/(2 pi)
      // in turns; k.x/(2 pi) = k.lo/(2 pi) + sum_i [k_i w_i / (2 pi)] m_i 2^-23.
      double phi = -std::atan2(p[1], p[0]) / kTwoPi;
      uint32_t fold = 0;  // the 2^23 offsets the kernel adds, removed from P0
      uint64_t T0 = 0;
      bool equal_rates = dim >= 2;  // every T_i the same: variant G = 1
      for (int i = 0; i < dim; ++i) {
        const double tau = p[2 + i] * w[i] / kTwoPi;
        if (!(std::fabs(tau) <= 1048576.0))
          return set_error(ZMC_EINVAL, "harmonic |k_i (hi_i-lo_i)| / 2pi above 2^20 turns");
        const uint64_t T = static_cast<uint64_t>(std::llround(std::ldexp(tau, 41)));
        if (i == 0) T0 = T;
        equal_rates = equal_rates && T == T0;
        const uint32_t thi = static_cast<uint32_t>(T >> 32);
        const double tlo = std::ldexp(static_cast<double>(static_cast<uint32_t>(T)), -32);
        const float tlo_f = static_cast<float>(tlo);
        const float kc = static_cast<float>(8388608.0 - static_cast<double>(tlo_f) * 8388608.0);
        fn->w[i] = thi;
        std::memcpy(&fn->w[7 + i], &tlo_f, 4);
        std::memcpy(&fn->w[14 + i], &kc, 4);
        fold += (thi + 1u) * 0x4B000000u;
        phi += p[2 + i] * d.lo[i] / kTwoPi;
      }
      if (!(std::fabs(phi) < 4.0e15)) return set_error(ZMC_EINVAL, "harmonic phase too large");
      const double fr = phi - std::floor(phi);  // exact, in [0, 1)
      const uint64_t p0_64 = static_cast<uint64_t>(std::ldexp(fr, 64));  // exact
      const uint32_t p0 = static_cast<uint32_t>((p0_64 + 0x80000000ull) >> 32);  // nearest
      fn->w[21] = p0 - fold;
      if (equal_rates) {
        // phase = P0 + T S (units of 2^-64 turn), S = sum_i m_i (no offsets),
        // plus half a unit of 2^-32 turn so that the kernel's carry rounds it
        const uint64_t p0r = p0_64 + 0x80000000ull;  // modulo one turn
        fn->variant = variant_code(ZMC_HARMONIC, d.dim, 1);
        fn->w[0] = static_cast<uint32_t>(T0 >> 32);
        fn->w[1] = static_cast<uint32_t>(T0);
        fn->w[2] = static_cast<uint32_t>(p0r);
        fn->w[21] = static_cast<uint32_t>(p0r >> 32);
      }
      const double R = S * std::hypot(p[0], p[1]);
      ok = finite_f32(R);
      put_f32(&fn->w[22], R);
      break;
    }
    case ZMC_ABSLIN: {
      // s = c.x = S0 + sum_i T_i m_i, S0 = c.lo, T_i = c_i w_i 2^-23, in units of
      // 2^-F: G_i = round(T_i 2^F) fits 32 bits and |s| 2^F fits 63, so the kernel
      // sums G_i m_i exactly in 64-bit integers (modulo 2^64; the true value fits)
      // and the remainders g_i = T_i 2^F - G_i (|g_i| <= 1/2) in FP32.  It multiplies
      // G_i by vb_i = 0x4B000000 + m_i, whose bits are also the float 2^23 + m_i,
      // so the offsets G_i 0x4B000000 and 2^23 g_i are taken out of the constants.
      //
      // Rows of at least kAbsLinNarrowMinSamples samples (variant degree 1) take a
      // 32-bit integer sum instead: units of 2^-F with |c.x| 2^F <= 2^29 over the
      // box, one 32-bit multiply-add per coordinate.  Its error, a few units of
      // the FP32 remainder sum (<= D^2 / 4), stays below ~2e-8 of max|c.x|, i.e.
      // below 2e-7 of mean|c.x| (at least a tenth of the maximum for a box of up
      // to 7 dimensions): far inside 1e-6 of the estimate's mean|f| once the row
      // has enough samples for its sample mean of |f| to be near the true one.
      // Rows with fewer samples, down to a single one next to the hyperplane,
      // keep the 64-bit sum.
      double s0 = 0.0, tmax = 0.0, smax = 0.0, up = 0.0, dn = 0.0;
      for (int i = 0; i < dim; ++i) {
        const double c = p[1 + i];
        s0 += c * d.lo[i];
        tmax = std::max(tmax, std::fabs(c * w[i]) * 0x1p-23);
        smax += std::fabs(c) * std::max(std::fabs(d.lo[i]), std::fabs(d.hi[i]));
        up += c * (c > 0 ? d.hi[i] : d.lo[i]);
        dn += c * (c > 0 ? d.lo[i] : d.hi[i]);
      }
      if (!std::isfinite(s0) || !std::isfinite(smax) || !std::isfinite(tmax))
        return set_error(ZMC_EINVAL, "abs-linear constants not finite");
      const bool narrow = d.n_samples >= kAbsLinNarrowMinSamples;
      const double srange = std::max(std::fabs(up), std::fabs(dn));  // max |c.x| on the box
      int F = 1000;
      if (tmax > 0.0) F = std::min(F, static_cast<int>(std::floor(std::log2(2147483647.0 / tmax))));
      if (narrow && srange > 0.0)
        F = std::min(F, 29 - static_cast<int>(std::ceil(std::log2(srange))));
      if (!narrow && smax > 0.0) F = std::min(F, 61 - static_cast<int>(std::ceil(std::log2(smax))));
      if (F == 1000) F = 0;
      F = std::max(-900, F);
      // log2 rounding can overshoot by one at a power of two: step down until
      // every G_i fits 32 bits
      for (int i = 0; i < dim; ++i)
        while (std::fabs(std::ldexp(p[1 + i] * w[i] * 0x1p-23, F)) > 2147483647.0) --F;
      uint64_t g0 = static_cast<uint64_t>(std::llround(std::ldexp(s0, F)));
      float l0 = 0.0f;
      double l0d = 0.0;
      for (int i = 0; i < dim; ++i) {
        const double t = std::ldexp(p[1 + i] * w[i] * 0x1p-23, F);
        const int64_t G = std::llround(t);
        const float gl = static_cast<float>(t - static_cast<double>(G));
        fn->w[i] = static_cast<uint32_t>(static_cast<int32_t>(G));
        std::memcpy(&fn->w[7 + i], &gl, 4);
        g0 -= static_cast<uint64_t>(G) * 0x4B000000ull;
        l0d -= static_cast<double>(gl) * 8388608.0;
      }
      l0 = static_cast<float>(l0d);
      fn->w[14] = static_cast<uint32_t>(g0);
      fn->w[15] = static_cast<uint32_t>(g0 >> 32);
      std::memcpy(&fn->w[16], &l0, 4);
      if (narrow) fn->variant = variant_code(ZMC_ABSLIN, d.dim, 1);
      const double sc = S * p[0] * std::ldexp(1.0, -F);
      ok = finite_f32(sc) && (sc == 0.0 || std::fabs(sc) >= 0x1p-126);
      put_f32(&fn->w[17], sc);
      break;
    }
    case ZMC_GAUSS: {
      const double sigma = p[1];
      if (!(sigma > 0.0)) return set_error(ZMC_EINVAL, "gauss sigma must be > 0");
      const double beta = std::sqrt(1.4426950408889634073599246810019 / 2.0) / sigma;
      bool near = true;
      double pos[kMaxDim];
      for (int i = 0; i < dim; ++i) {
        pos[i] = (p[2 + i] - d.lo[i]) / w[i];  // mu_i in units of the box width from lo_i
        if (!(pos[i] >= -1.0 && pos[i] <= 2.0)) near = false;
      }
      for (int i = 0; i < dim; ++i) {
        const double h = w[i] * beta;
        ok = ok && finite_f32(h);
        split(h, &fn->w[i], &fn->w[7 + i]);
        if (near) {
          // 1 + mu's position rounded to 2^-22: exact in FP32 over [0, 3]
          const double u0 = std::ldexp(std::nearbyint(std::ldexp(pos[i], 22)), -22);
          put_f32(&fn->w[14 + i], 1.0 + u0);                  // exact
          put_f32(&fn->w[21 + i], -h * (pos[i] - u0));        // |.| <= h 2^-23
        } else {
          const double e = (d.lo[i] - p[2 + i]) * beta;
          ok = ok && finite_f32(e);
          split(e, &fn->w[14 + i], &fn->w[21 + i]);
        }
      }
      fn->variant = variant_code(ZMC_GAUSS, d.dim, near ? 0 : 1);
      ok = ok && finite_f32(S * p[0]);
      put_f32(&fn->w[28], S * p[0]);
      break;
    }
    default: {
      const int g = static_cast<int>(d.deg);
      if (g >= 2 && poly_roots_payload(poly_e, dim, g, S, fn)) break;
      for (int i = 0; i < dim; ++i) {
        for (int k = 0; k <= g; ++k) {
          const double e = (i == 0 ? S : 1.0) * poly_e[i][k];
          ok = ok && finite_f32(e);
          split(e, &fn->w[5 * i + k], &fn->w[35 + 5 * i + k]);
        }
      }
      break;
    }
  }
  if (!ok) return set_error(ZMC_EINVAL, "parameters out of FP32 range");
  if (plain) {
    std::memset(plain, 0, sizeof(PlainFn));
    plain->family = d.family;
    plain->dim = d.dim;
    plain->stream_id = d.stream_id;
    plain->deg = d.family == ZMC_POLY ? d.deg : 0;
    plain->key0 = fn->key0;
    plain->key1 = fn->key1;
    plain->n_samples = d.n_samples;
    for (int i = 0; i < dim; ++i) {
      plain->lo[i] = d.lo[i];
      plain->w[i] = w[i];
    }
    std::memcpy(plain->p, d.p, sizeof(d.p));
  }
  if (volume) *volume = vol;
  return ZMC_OK;
}

zmc_status ensure_stage(zmc_ctx *ctx, size_t bytes) {
  if (ctx->stage_bytes >= bytes) return ZMC_OK;
  if (ctx->stage) {
    ZMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFreeHost(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
  }
  size_t want = std::max<size_t>(bytes, 1 << 20);
  ZMC_CUDA(ctx, cudaHostAlloc(&ctx->stage, want, cudaHostAllocDefault));
  ctx->stage_bytes = want;
  return ZMC_OK;
}

unsigned grid_for(const zmc_ctx *ctx, int family, unsigned block, unsigned bps, uint64_t items,
                  int unroll) {
  const unsigned warps_per_block = block / 32;
  const int maxb = batched_max_blocks_per_sm(family, static_cast<int>(block), unroll);
  if (bps == 0 || bps > static_cast<unsigned>(std::max(maxb, 1)))
    bps = static_cast<unsigned>(std::max(maxb, 1));
  const uint64_t full = static_cast<uint64_t>(ctx->sms) * bps;
  const uint64_t need = (items + warps_per_block - 1) / warps_per_block;
  return static_cast<unsigned>(std::max<uint64_t>(1, std::min(full, need)));
}

unsigned family_grid(const zmc_ctx *ctx, int family, uint64_t items, int unroll) {
  return grid_for(ctx, family, ctx->shape.block, ctx->shape.blocks_per_sm[family], items, unroll);
}

cudaError_t FamilyFork::init() {
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming);
  }
  return e;
}

void FamilyFork::destroy() {
  for (int k = 0; k < 3; ++k) {
    if (side[k]) cudaStreamDestroy(side[k]);
    if (join[k]) cudaEventDestroy(join[k]);
    side[k] = nullptr;
    join[k] = nullptr;
  }
  if (fork) cudaEventDestroy(fork);
  fork = nullptr;
}

cudaError_t launch_families(FamilyFork &ff, const Entry *entries, LaunchHdr *hdr,
                            const unsigned *grid, const unsigned *block, const bool *present,
                            cudaStream_t main, const unsigned *unroll) {
  int fams[4], n = 0;
  for (int f = 0; f < 4; ++f)
    if (present[f]) fams[n++] = f;
  auto launch = [&](int f, cudaStream_t s) {
    return launch_batched(f, entries, hdr, grid[f], block[f], s,
                          unroll ? static_cast<int>(unroll[f]) : 1);
  };
  if (n == 0) return cudaSuccess;
  if (n == 1 || !ff.fork) return launch(fams[0], main);
  cudaError_t e = cudaEventRecord(ff.fork, main);
  for (int k = 1; k < n && e == cudaSuccess; ++k) {
    e = cudaStreamWaitEvent(ff.side[k - 1], ff.fork, 0);
    if (e == cudaSuccess) e = launch(fams[k], ff.side[k - 1]);
    if (e == cudaSuccess) e = cudaEventRecord(ff.join[k - 1], ff.side[k - 1]);
  }
  if (e == cudaSuccess) e = launch(fams[0], main);
  for (int k = 1; k < n && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(main, ff.join[k - 1], 0);
  return e;
}

}  // namespace zmc

using namespace zmc;

// ---------------------------------------------------------------- plans
struct zmc_plan {
  zmc_ctx *ctx = nullptr;
  size_t n = 0;
  FnDev *d_fns = nullptr;
  float2 *d_rec = nullptr;
  zmc_result *d_out = nullptr;
  Entry *d_entries = nullptr;
  LaunchHdr *d_hdr = nullptr;
  const FnDev **d_merge = nullptr;
  std::vector<PlainFn> plain;
  std::vector<double> volume;
  double *d_prec = nullptr;
  PlainJob *d_pjobs = nullptr;
  std::vector<unsigned> pgrid;
  std::vector<size_t> poff;
  LaunchHdr h_hdr{};
  uint64_t n_chunks = 0, n_samples = 0;
  uint64_t fam_items[4] = {0, 0, 0, 0};
  bool ranged = false;  // built by zmc_integrate_moments (no plain form)
  uint32_t quints = 0;  // chunk = 160 * quints samples
  unsigned unroll[4] = {1, 1, 1, 1};  // quint-loop unroll of each family kernel
  int chunk_source = 0;  // chunk length and unroll: 0 default, 1 measured, 2 cached
  unsigned grid[4] = {0, 0, 0, 0};
  unsigned block[4] = {256, 256, 256, 256};
  int tune_source[4] = {0, 0, 0, 0};  // 0 default, 1 measured, 2 from the cache
  int dominant_dim[4] = {0, 0, 0, 0};
  cudaGraphExec_t graph = nullptr;
  std::vector<void *> blocks;

  void *alloc(size_t bytes) {
    void *p = ctx->arena.alloc(bytes);
    if (p) blocks.push_back(p);
    return p;
  }
  void release_all() {
    for (void *p : blocks) ctx->arena.release(p);
    blocks.clear();
  }
};

namespace {

zmc_status check_ctx(zmc_ctx *ctx) {
  if (!ctx) return set_error(ZMC_EINVAL, "null context");
  if (ctx->poisoned) return set_error(ZMC_ECUDA, "context poisoned by an earlier CUDA error");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaSetDevice");
  return ZMC_OK;
}

// Autotuner: for each family kernel of the plan, the geometry (threads per
// block, resident blocks per SM) that runs a bounded slice of the plan's own
// items fastest, or the cached choice for the same key.  Geometry never changes
// results; the slice's records are recomputed identically by the real launch.
zmc_status plan_autotune(zmc_plan *plan) {
  zmc_ctx *ctx = plan->ctx;
  cudaStream_t str = ctx->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;  // created at the first cache miss
  zmc_status st = ZMC_OK;
  for (int f = 0; f < 4 && st == ZMC_OK; ++f) {
    if (plan->fam_items[f] == 0) continue;
    const int U = static_cast<int>(plan->unroll[f]);
    const std::string key = tune_key(ctx, f, plan->dominant_dim[f], plan->quints, U);
    auto hit = ctx->tune_cache.find(key);
    if (hit != ctx->tune_cache.end()) {
      plan->block[f] = hit->second.block;
      plan->grid[f] = grid_for(ctx, f, hit->second.block, hit->second.blocks_per_sm,
                               plan->fam_items[f], U);
      plan->tune_source[f] = 2;
      continue;
    }
    if (!e0) {
      cudaError_t ce = cudaEventCreate(&e0);
      if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
      if (ce != cudaSuccess) {
        st = ctx_cuda_fail(ctx, ce, "autotune events");
        break;
      }
    }
    // a slice of about 32 items per resident warp at the largest geometry
    LaunchHdr th = plan->h_hdr;
    const uint64_t slice = std::min<uint64_t>(plan->fam_items[f],
                                              static_cast<uint64_t>(ctx->sms) * 64 * 32);
    for (int g = 0; g < 4; ++g) th.item_end[g] = th.item_begin[g];
    th.item_end[f] = th.item_begin[f] + slice;
    TuneChoice best;
    best.ms = 1e30f;
    for (unsigned block : {128u, 256u}) {
      const int maxb = batched_max_blocks_per_sm(f, static_cast<int>(block), U);
      for (int bps = 1; bps <= maxb && st == ZMC_OK; ++bps) {
        const unsigned grid = grid_for(ctx, f, block, static_cast<unsigned>(bps), slice, U);
        float ms_best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          cudaError_t e = cudaMemcpyAsync(plan->d_hdr, &th, sizeof th, cudaMemcpyHostToDevice, str);
          if (e == cudaSuccess) e = cudaEventRecord(e0, str);
          if (e == cudaSuccess)
            e = launch_batched(f, plan->d_entries, plan->d_hdr, grid, block, str, U);
          if (e == cudaSuccess) e = cudaEventRecord(e1, str);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.0f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e != cudaSuccess) {
            st = ctx_cuda_fail(ctx, e, "autotune");
            break;
          }
          if (rep > 0) ms_best = std::min(ms_best, ms);  // rep 0 warms up
        }
        if (ms_best < best.ms) {
          best.ms = ms_best;
          best.block = block;
          best.blocks_per_sm = static_cast<unsigned>(bps);
        }
      }
    }
    if (st != ZMC_OK) break;
    plan->block[f] = best.block;
    plan->grid[f] = grid_for(ctx, f, best.block, best.blocks_per_sm, plan->fam_items[f], U);
    plan->tune_source[f] = 1;
    tune_cache_store(ctx, key, best);
  }
  const bool timed = e0 != nullptr;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != ZMC_OK) return st;
  if (!timed) return ZMC_OK;  // every family from the cache: nothing ran
  // put the real header back (the slices overwrote it)
  ZMC_CUDA(ctx, cudaMemcpyAsync(plan->d_hdr, &plan->h_hdr, sizeof plan->h_hdr,
                                cudaMemcpyHostToDevice, str));
  ZMC_CUDA(ctx, cudaStreamSynchronize(str));
  return ZMC_OK;
}

// A fixed chunk length and unroll for plan_build (the chunk tuner's trial plans).
struct PlanChoice {
  uint32_t quints;
  unsigned unroll[4];
};

zmc_status plan_build(zmc_ctx *ctx, const zmc_desc *desc, size_t n, zmc_plan **out,
                      const uint64_t *s_begin = nullptr, const uint64_t *s_end = nullptr,
                      const PlanChoice *force = nullptr, bool wait_upload = true);
void plan_free(zmc_plan *plan);
zmc_status plan_enqueue(zmc_plan *plan, uint32_t stages);

// The key of a table's shape class for the chunk tuner: the GPU, the families
// present with their dominant dimension and kernels' registers, and the
// table's size (log2 of the rows and of the mean samples per row).
std::string chunk_tune_key(const zmc_ctx *ctx, const zmc_desc *desc, size_t n) {
  double dim_samples[4][kMaxDim + 1] = {{0}};
  double total = 0.0;
  for (size_t i = 0; i < n; ++i) {
    dim_samples[desc[i].family][desc[i].dim] += static_cast<double>(desc[i].n_samples);
    total += static_cast<double>(desc[i].n_samples);
  }
  std::ostringstream k;
  k << "chunk|" << ctx->gpu_name << '|' << ctx->sms;
  for (int f = 0; f < 4; ++f) {
    int best = 0;
    for (int d = 1; d <= kMaxDim; ++d)
      if (dim_samples[f][d] > dim_samples[f][best]) best = d;
    if (best == 0) continue;
    k << "|f" << f << 'd' << best << 'r' << ctx->kernel_regs[0][f] << '/'
      << ctx->kernel_regs[1][f];
  }
  k << "|n" << static_cast<int>(std::floor(std::log2(static_cast<double>(n)))) << "|s"
    << static_cast<int>(std::floor(std::log2(std::max(1.0, total / static_cast<double>(n)))));
  return k.str();
}

// Device time of one family kernel of a plan draining all of its items: the
// best of two launches after a warm-up (milliseconds).
zmc_status time_family(zmc_plan *plan, int f, int unroll, cudaEvent_t e0, cudaEvent_t e1,
                       float *ms_out) {
  zmc_ctx *ctx = plan->ctx;
  cudaStream_t str = ctx->stream;
  const unsigned grid = grid_for(ctx, f, ctx->shape.block, ctx->shape.blocks_per_sm[f],
                                 plan->fam_items[f], unroll);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaError_t e = cudaMemsetAsync(plan->d_hdr, 0, sizeof(plan->d_hdr->counter), str);
    if (e == cudaSuccess) e = cudaEventRecord(e0, str);
    if (e == cudaSuccess)
      e = launch_batched(f, plan->d_entries, plan->d_hdr, grid, ctx->shape.block, str, unroll);
    if (e == cudaSuccess) e = cudaEventRecord(e1, str);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "chunk autotune");
    if (rep > 0) best = std::min(best, ms);
  }
  *ms_out = best;
  return ZMC_OK;
}

// Device time of a plan's sampling stage as a plan runs it (the family kernels
// concurrently): the best of two launches after a warm-up (milliseconds).
zmc_status time_plan_sample(zmc_plan *plan, cudaEvent_t e0, cudaEvent_t e1, float *ms_out) {
  zmc_ctx *ctx = plan->ctx;
  cudaStream_t str = ctx->stream;
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaError_t e = cudaEventRecord(e0, str);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "chunk autotune");
    const zmc_status st = plan_enqueue(plan, ZMC_STAGE_SAMPLE);
    if (st != ZMC_OK) return st;
    e = cudaEventRecord(e1, str);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "chunk autotune");
    if (rep > 0) best = std::min(best, ms);
  }
  *ms_out = best;
  return ZMC_OK;
}

// Samples and rows of the table subset the chunk tuner times each candidate on.
constexpr double kTrialSamples = 2147483648.0;
constexpr size_t kTrialRows = 1u << 16;

// Chunk tuner: the chunk length (kTuneQuints) and per-family unroll for a
// table, or the cached choice for the table's shape class.  The candidates are
// timed on a bounded subset of the table's rows (every k-th row, whole rows; at
// most ~2^31 samples and 2^16 rows), as a plan runs it (every family kernel at
// once, unroll 1).  When the subset is not the whole table, its time is carried
// over to the table by a straight line through two subsets, every 2k-th and
// every k-th row: T(samples) = O + b * samples, predicted = O + b *
// samples(table).  The fixed part O (the kernels draining their last chunks at
// each change of family and at the end; on the 10^4-integrand mix 1.4 to 7
// chunk times, growing with the chunk length) weighs several times more in a
// subset than in the table, and scaling the subset's time alone picked chunks
// of 52 quints where 208 ran the table 1.8% faster.  Then, at the chosen length,
// each family kernel present is timed alone at both unrolls (their fixed parts
// are alike).  *source: 1 measured, 2 cached, 0 left at the defaults (no trial
// plan fitted the arena).
zmc_status choose_chunk(zmc_ctx *ctx, const zmc_desc *desc, size_t n, PlanChoice *choice,
                        int *source) {
  const std::string key = chunk_tune_key(ctx, desc, n);
  auto hit = ctx->tune_cache.find(key);
  if (hit != ctx->tune_cache.end()) {
    choice->quints = hit->second.quints;
    for (int f = 0; f < 4; ++f) choice->unroll[f] = hit->second.unroll[f];
    *source = 2;
    return ZMC_OK;
  }
  double total = 0.0;
  for (size_t i = 0; i < n; ++i) total += static_cast<double>(desc[i].n_samples);
  const size_t stride = std::max<size_t>(
      total <= kTrialSamples ? 1 : static_cast<size_t>(std::ceil(total / kTrialSamples)),
      (n + kTrialRows - 1) / kTrialRows);
  std::vector<zmc_desc> sub, half;  // every stride-th row; every 2 stride-th row
  double sub_total = 0.0, half_total = 0.0;
  for (size_t i = 0; i < n; i += stride) {
    sub.push_back(desc[i]);
    sub_total += static_cast<double>(desc[i].n_samples);
    if ((i / stride) % 2 == 0) {
      half.push_back(desc[i]);
      half_total += static_cast<double>(desc[i].n_samples);
    }
  }
  // a line needs two subsets of different size, and is not needed when the
  // subset is the table
  const bool extrapolate = stride > 1 && half_total < sub_total;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ZMC_CUDA(ctx, cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return ctx_cuda_fail(ctx, ce, "chunk autotune");
  }
  zmc_status st = ZMC_OK;
  double best_pred = 1e300;
  TuneChoice best;
  zmc_plan *best_trial = nullptr;
  for (uint32_t q : kTuneQuints) {
    PlanChoice trial_choice{q, {1, 1, 1, 1}};
    zmc_plan *trial = nullptr;
    st = plan_build(ctx, sub.data(), sub.size(), &trial, nullptr, nullptr, &trial_choice);
    if (st == ZMC_ENOMEM) {  // the arena cannot hold this trial: skip the candidate
      st = ZMC_OK;
      continue;
    }
    if (st != ZMC_OK) break;
    float ms = 0.0f;
    st = time_plan_sample(trial, e0, e1, &ms);
    double pred = ms;
    if (st == ZMC_OK && extrapolate) {
      zmc_plan *trial_half = nullptr;
      st = plan_build(ctx, half.data(), half.size(), &trial_half, nullptr, nullptr,
                      &trial_choice);
      float ms_half = 0.0f;
      if (st == ZMC_OK) {
        st = time_plan_sample(trial_half, e0, e1, &ms_half);
        plan_free(trial_half);
        const double b = (static_cast<double>(ms) - ms_half) / (sub_total - half_total);
        pred = ms + b * (total - sub_total);
      } else if (st == ZMC_ENOMEM) {  // no room for the second subset: scale the first
        st = ZMC_OK;
        pred = ms * total / sub_total;
      }
    }
    if (st != ZMC_OK) {
      plan_free(trial);
      break;
    }
    if (pred < best_pred) {
      best_pred = pred;
      best.quints = q;
      best.ms = static_cast<float>(pred);
      if (best_trial) plan_free(best_trial);
      best_trial = trial;
    } else {
      plan_free(trial);
    }
  }
  // the unroll of each family kernel at the chosen chunk length
  for (int f = 0; f < 4 && st == ZMC_OK && best_trial; ++f) {
    if (best_trial->fam_items[f] == 0) continue;
    float t_best = 1e30f;
    for (int u = 1; u <= kMaxUnroll && st == ZMC_OK; ++u) {
      float ms = 0.0f;
      st = time_family(best_trial, f, u, e0, e1, &ms);
      if (ms < t_best) {
        t_best = ms;
        best.unroll[f] = static_cast<unsigned>(u);
      }
    }
  }
  if (best_trial) plan_free(best_trial);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ZMC_OK) return st;
  if (best.quints == 0) {  // no candidate fitted
    *source = 0;
    return ZMC_OK;
  }
  tune_cache_store(ctx, key, best);
  choice->quints = best.quints;
  for (int f = 0; f < 4; ++f) choice->unroll[f] = best.unroll[f];
  *source = 1;
  return ZMC_OK;
}

// ranges: optional [s_begin[i], s_end[i]) sample ranges (moments output).
// force: a fixed chunk length and unroll, no autotuning (trial plans).
// wait_upload = false: the caller's next use of the staging buffer is
// stream-ordered after the upload (a device-to-host copy of results), so the
// host need not wait for the upload here.
zmc_status plan_build(zmc_ctx *ctx, const zmc_desc *desc, size_t n, zmc_plan **out,
                      const uint64_t *s_begin, const uint64_t *s_end, const PlanChoice *force,
                      bool wait_upload) {
  if (!desc || !out || n == 0) return set_error(ZMC_EINVAL, "need n >= 1 descriptors");
  if (n >= (1u << 31)) return set_error(ZMC_EINVAL, "too many descriptors");
  auto plan = std::make_unique<zmc_plan>();
  plan->ctx = ctx;
  plan->n = n;
  plan->ranged = s_begin != nullptr;
  std::vector<FnDev> fns(n);
  std::vector<uint64_t> len(n);
  plan->plain.resize(n);
  plan->volume.resize(n);
  // per-descriptor validation and FP64 precompute, in parallel for large tables;
  // the first failing row is redone on this thread for its message
  std::vector<uint8_t> ok(n, 1);
  host_parallel_for(n, 64, [&](size_t b, size_t e) {
    for (size_t i = b; i < e; ++i)
      ok[i] = precompute(desc[i], &fns[i], &plan->plain[i], &plan->volume[i]) == ZMC_OK;
  });
  for (size_t i = 0; i < n; ++i) {
    if (!ok[i]) {
      const zmc_status st = precompute(desc[i], &fns[i], &plan->plain[i], &plan->volume[i]);
      return set_error(st, "descriptor %zu: %s", i, zmc_last_error(nullptr));
    }
    len[i] = desc[i].n_samples;
    if (s_begin) {
      if (s_begin[i] % kQuint != 0 || !(s_end[i] > s_begin[i]) ||
          s_end[i] - s_begin[i] > (1ull << 62))
        return set_error(ZMC_EINVAL,
                         "range %zu: need s_begin a multiple of 5 and s_begin < s_end", i);
      if (s_end[i] > ~0ull / kMaxDim)
        return set_error(ZMC_EINVAL, "range %zu: sample index too large", i);
      fns[i].s_off = s_begin[i];
      len[i] = s_end[i] - s_begin[i];
      fns[i].n_samples = len[i];
      fns[i].out_mode = 1;
    }
  }
  // chunk length and unroll: fixed by the caller, chosen by the chunk tuner, or
  // the context's chunk length with unroll 1
  PlanChoice choice{ctx->quints_per_lane, {1, 1, 1, 1}};
  if (force) {
    choice = *force;
  } else if ((ctx->autotune & ZMC_TUNE_CHUNK) && !s_begin) {
    const zmc_status cs = choose_chunk(ctx, desc, n, &choice, &plan->chunk_source);
    if (cs != ZMC_OK) return cs;
  }
  plan->quints = choice.quints;
  for (int f = 0; f < 4; ++f) plan->unroll[f] = choice.unroll[f];
  const uint64_t chunk = chunk_samples_of(plan->quints);
  std::vector<uint64_t> nchunk(n), rec_off(n);
  uint64_t total = 0, samples = 0;
  for (size_t i = 0; i < n; ++i) {
    nchunk[i] = (len[i] + chunk - 1) / chunk;
    rec_off[i] = total;
    total += nchunk[i];
    samples += len[i];
  }
  plan->n_chunks = total;
  plan->n_samples = samples;

  const size_t fn_bytes = n * sizeof(FnDev);
  const size_t ent_bytes = n * sizeof(Entry);
  const size_t mrg_bytes = n * sizeof(FnDev *);
  plan->d_fns = static_cast<FnDev *>(plan->alloc(fn_bytes));
  plan->d_rec = static_cast<float2 *>(plan->alloc(total * sizeof(float2)));
  plan->d_out = static_cast<zmc_result *>(plan->alloc(n * sizeof(zmc_result)));
  plan->d_entries = static_cast<Entry *>(plan->alloc(ent_bytes));
  plan->d_merge = static_cast<const FnDev **>(plan->alloc(mrg_bytes));
  plan->d_hdr = static_cast<LaunchHdr *>(plan->alloc(sizeof(LaunchHdr)));
  if (!plan->d_fns || !plan->d_rec || !plan->d_out || !plan->d_entries || !plan->d_merge ||
      !plan->d_hdr) {
    plan->release_all();
    return set_error(ZMC_ENOMEM, "plan needs %.1f MB of device memory; arena has %.1f MB free",
                     (fn_bytes + total * 8.0 + n * 64.0) / 1e6,
                     ctx->arena.largest_free() / 1e6);
  }
  for (size_t i = 0; i < n; ++i) {
    fns[i].rec = plan->d_rec + rec_off[i];
    fns[i].out = plan->d_out + i;
  }
  // item order: by family, then variant, then table order
  std::vector<uint32_t> order(n);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
    const uint32_t fa = desc[a].family, fb = desc[b].family;
    if (fa != fb) return fa < fb;
    return fns[a].variant < fns[b].variant;
  });
  std::vector<Entry> ents(n);
  LaunchHdr &h = plan->h_hdr;
  std::memset(&h, 0, sizeof h);
  uint64_t item = 0;
  for (int f = 0; f < 4; ++f) h.item_begin[f] = h.item_end[f] = 0;
  int cur_f = -1;
  for (size_t k = 0; k < n; ++k) {
    const uint32_t i = order[k];
    const int f = static_cast<int>(desc[i].family);
    while (cur_f < f) {
      ++cur_f;
      h.item_begin[cur_f] = item;
      h.item_end[cur_f] = item;
    }
    ents[k].item_begin = item;
    ents[k].fn = plan->d_fns + i;
    ents[k].chunk_begin = 0;
    item += nchunk[i];
    h.item_end[f] = item;
  }
  while (cur_f < 3) {
    ++cur_f;
    h.item_begin[cur_f] = item;
    h.item_end[cur_f] = item;
  }
  h.n_entries = static_cast<uint32_t>(n);
  h.n_merge = static_cast<uint32_t>(n);
  h.quints_per_lane = plan->quints;
  for (int f = 0; f < 4; ++f) {
    plan->fam_items[f] = h.item_end[f] - h.item_begin[f];
    plan->block[f] = ctx->shape.block;
    plan->grid[f] = family_grid(ctx, f, plan->fam_items[f], static_cast<int>(plan->unroll[f]));
  }
  {
    double dim_samples[4][kMaxDim + 1] = {{0}};
    for (size_t i = 0; i < n; ++i)
      dim_samples[desc[i].family][desc[i].dim] += static_cast<double>(len[i]);
    for (int f = 0; f < 4; ++f) {
      int best = 0;
      for (int dd = 1; dd <= kMaxDim; ++dd)
        if (dim_samples[f][dd] > dim_samples[f][best]) best = dd;
      plan->dominant_dim[f] = best;
    }
  }
  std::vector<const FnDev *> merge(n);
  for (size_t i = 0; i < n; ++i) merge[i] = plan->d_fns + i;

  const size_t stage = fn_bytes + ent_bytes + mrg_bytes + sizeof(LaunchHdr);
  zmc_status st = ensure_stage(ctx, stage);
  if (st != ZMC_OK) {
    plan->release_all();
    return st;
  }
  // the staging buffer is reused by the next call, so the copies are waited for
  // (unless the caller's next use of it is stream-ordered: wait_upload)
  char *s = static_cast<char *>(ctx->stage);
  std::memcpy(s, fns.data(), fn_bytes);
  std::memcpy(s + fn_bytes, ents.data(), ent_bytes);
  std::memcpy(s + fn_bytes + ent_bytes, merge.data(), mrg_bytes);
  std::memcpy(s + fn_bytes + ent_bytes + mrg_bytes, &h, sizeof h);
  cudaStream_t str = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(plan->d_fns, s, fn_bytes, cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(plan->d_entries, s + fn_bytes, ent_bytes, cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(plan->d_merge, s + fn_bytes + ent_bytes, mrg_bytes,
                        cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(plan->d_hdr, s + fn_bytes + ent_bytes + mrg_bytes, sizeof h,
                        cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess && wait_upload) e = cudaStreamSynchronize(str);
  if (e != cudaSuccess) {
    plan->release_all();
    return ctx_cuda_fail(ctx, e, "plan upload");
  }
  if ((ctx->autotune & ZMC_TUNE_GEOMETRY) && !force) {
    zmc_status ts = plan_autotune(plan.get());
    if (ts != ZMC_OK) {
      plan->release_all();
      return ts;
    }
  }
  *out = plan.release();
  return ZMC_OK;
}

zmc_status plan_enqueue(zmc_plan *plan, uint32_t stages) {
  zmc_ctx *ctx = plan->ctx;
  cudaStream_t str = ctx->stream;
  if (stages & ZMC_STAGE_SAMPLE) {
    ZMC_CUDA(ctx, cudaMemsetAsync(plan->d_hdr, 0, sizeof(plan->d_hdr->counter), str));
    bool present[4];
    for (int f = 0; f < 4; ++f) present[f] = plan->fam_items[f] > 0;
    ZMC_CUDA(ctx, launch_families(ctx->fork, plan->d_entries, plan->d_hdr, plan->grid,
                                  plan->block, present, str, plan->unroll));
  }
  if (stages & ZMC_STAGE_MERGE) {
    const unsigned grid = static_cast<unsigned>(
        std::min<size_t>((plan->n + 7) / 8, static_cast<size_t>(ctx->sms) * 16));
    ZMC_CUDA(ctx, launch_merge(plan->d_merge, plan->d_hdr, grid, str));
  }
  return ZMC_OK;
}

zmc_status plan_results_to(zmc_plan *plan, zmc_result *out) {
  zmc_ctx *ctx = plan->ctx;
  const size_t bytes = plan->n * sizeof(zmc_result);
  zmc_status st = ensure_stage(ctx, bytes);
  if (st != ZMC_OK) return st;
  ZMC_CUDA(ctx, cudaMemcpyAsync(ctx->stage, plan->d_out, bytes, cudaMemcpyDeviceToHost,
                                ctx->stream));
  ZMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::memcpy(out, ctx->stage, bytes);
  return ZMC_OK;
}

void plan_free(zmc_plan *plan) {
  if (!plan) return;
  if (plan->graph) cudaGraphExecDestroy(plan->graph);
  // stream order makes reuse of the released ranges safe for later work on this
  // stream; wait anyway so no kernel of this plan can outlive the plan object.
  cudaStreamSynchronize(plan->ctx->stream);
  plan->release_all();
  delete plan;
}

zmc_status plain_prepare(zmc_plan *plan) {
  if (plan->d_pjobs) return ZMC_OK;
  zmc_ctx *ctx = plan->ctx;
  const size_t n = plan->n;
  plan->pgrid.resize(n);
  plan->poff.resize(n);
  size_t total = 0;
  for (size_t i = 0; i < n; ++i) {
    plan->pgrid[i] = plain_grid(plan->plain[i], ctx->sms);
    plan->poff[i] = total;
    total += 3 * static_cast<size_t>(plan->pgrid[i]);
  }
  plan->d_prec = static_cast<double *>(plan->alloc(total * sizeof(double)));
  PlainJob *jobs_dev = static_cast<PlainJob *>(plan->alloc(n * sizeof(PlainJob)));
  if (!plan->d_prec || !jobs_dev) return set_error(ZMC_ENOMEM, "plain form: arena full");
  std::vector<PlainJob> jobs(n);
  for (size_t i = 0; i < n; ++i) {
    jobs[i].rec = plan->d_prec + plan->poff[i];
    jobs[i].nblk = plan->pgrid[i];
    jobs[i].volume = plan->volume[i];
    jobs[i].out = plan->d_out + i;
  }
  zmc_status st = ensure_stage(ctx, n * sizeof(PlainJob));
  if (st != ZMC_OK) return st;
  std::memcpy(ctx->stage, jobs.data(), n * sizeof(PlainJob));
  ZMC_CUDA(ctx, cudaMemcpyAsync(jobs_dev, ctx->stage, n * sizeof(PlainJob),
                                cudaMemcpyHostToDevice, ctx->stream));
  ZMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  plan->d_pjobs = jobs_dev;
  return ZMC_OK;
}

zmc_status plain_enqueue(zmc_plan *plan) {
  zmc_ctx *ctx = plan->ctx;
  if (plan->ranged) return set_error(ZMC_EINVAL, "the plain form runs whole descriptors only");
  zmc_status st = plain_prepare(plan);
  if (st != ZMC_OK) return st;
  for (size_t i = 0; i < plan->n; ++i)
    ZMC_CUDA(ctx, launch_plain(plan->plain[i], plan->d_prec + plan->poff[i], plan->pgrid[i],
                               ctx->stream));
  ZMC_CUDA(ctx, launch_plain_merge(plan->d_pjobs, static_cast<uint32_t>(plan->n), ctx->stream));
  return ZMC_OK;
}

}  // namespace

// ---------------------------------------------------------------- C ABI
extern "C" {

zmc_status zmc_default_options(zmc_options *opt) {
  if (!opt) return set_error(ZMC_EINVAL, "null options");
  std::memset(opt, 0, sizeof *opt);
  opt->mem_budget_bytes = 1ull << 30;
  opt->quints_per_lane = 0;  // chosen at zmc_create
  return ZMC_OK;
}

const char *zmc_last_error(zmc_ctx *) { return g_last_error.c_str(); }

size_t zmc_desc_size(void) { return sizeof(zmc_desc); }

zmc_status zmc_validate(const zmc_desc *desc, size_t n, size_t *bad_index) {
  if (!desc && n) return set_error(ZMC_EINVAL, "null descriptor table");
  std::vector<uint8_t> ok(n, 1);
  host_parallel_for(n, 64, [&](size_t b, size_t e) {
    FnDev fn;
    for (size_t i = b; i < e; ++i) ok[i] = precompute(desc[i], &fn, nullptr, nullptr) == ZMC_OK;
  });
  for (size_t i = 0; i < n; ++i) {
    if (ok[i]) continue;
    FnDev fn;
    const zmc_status st = precompute(desc[i], &fn, nullptr, nullptr);
    if (bad_index) *bad_index = i;
    return set_error(st, "descriptor %zu: %s", i, zmc_last_error(nullptr));
  }
  return ZMC_OK;
}
size_t zmc_result_size(void) { return sizeof(zmc_result); }

zmc_status zmc_variant_of(const zmc_desc *desc, size_t n, uint32_t *forms, size_t *bad_index) {
  if ((!desc || !forms) && n) return set_error(ZMC_EINVAL, "null argument");
  for (size_t i = 0; i < n; ++i) {
    FnDev fn;
    const zmc_status st = precompute(desc[i], &fn, nullptr, nullptr);
    if (st != ZMC_OK) {
      if (bad_index) *bad_index = i;
      return set_error(st, "descriptor %zu: %s", i, zmc_last_error(nullptr));
    }
    forms[i] = fn.variant;
  }
  return ZMC_OK;
}

zmc_status zmc_create(const zmc_options *opt_in, zmc_ctx **out) {
  if (!out) return set_error(ZMC_EINVAL, "null output pointer");
  *out = nullptr;
  zmc_options opt;
  zmc_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.mem_budget_bytes == 0) opt.mem_budget_bytes = 1ull << 30;
  // longer chunks amortise the per-chunk work (keys, descriptor loads, warp
  // merge: 8192 samples measured fastest for whole tables); serving keeps them
  // at 4096, which measured lower job latency under load
  if (opt.quints_per_lane == 0) opt.quints_per_lane = opt.serving ? 26 : 104;
  if (opt.quints_per_lane > 1024) return set_error(ZMC_EINVAL, "quints_per_lane above 1024");
  if (opt.autotune & ~(ZMC_TUNE_GEOMETRY | ZMC_TUNE_CHUNK))
    return set_error(ZMC_EINVAL, "unknown autotune flags 0x%x", opt.autotune);
  if (opt.arena && (reinterpret_cast<uintptr_t>(opt.arena) & 255))
    return set_error(ZMC_EINVAL, "arena must be 256-byte aligned");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0)
    return set_error(ZMC_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
  if (opt.device < 0 || opt.device >= ndev)
    return set_error(ZMC_EINVAL, "device %d not present", opt.device);
  auto ctx = std::make_unique<zmc_ctx>();
  ctx->device = opt.device;
  e = cudaSetDevice(opt.device);
  if (e != cudaSuccess) return set_error(ZMC_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, opt.device);
  if (e != cudaSuccess) return set_error(ZMC_ECUDA, "device query: %s", cudaGetErrorString(e));
  ctx->sms = prop.multiProcessorCount;
  ctx->gpu_name = prop.name;
  if (opt.stream) {
    ctx->stream = static_cast<cudaStream_t>(opt.stream);
  } else {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return set_error(ZMC_ECUDA, "stream: %s", cudaGetErrorString(e));
    ctx->own_stream = true;
  }
  if (opt.arena) {
    ctx->arena_base = static_cast<char *>(opt.arena);
  } else {
    e = cudaMalloc(reinterpret_cast<void **>(&ctx->arena_base), opt.mem_budget_bytes);
    if (e != cudaSuccess) {
      if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
      return set_error(ZMC_ENOMEM, "arena of %llu bytes: %s",
                       static_cast<unsigned long long>(opt.mem_budget_bytes),
                       cudaGetErrorString(e));
    }
    ctx->own_arena = true;
  }
  ctx->arena.init(ctx->arena_base, opt.mem_budget_bytes);
  ctx->quints_per_lane = opt.quints_per_lane;
  ctx->max_chunks_per_iter = opt.max_chunks_per_iter;
  ctx->serving_share = opt.serving_share;
  ctx->serving_cut_backlog = opt.serving_cut_backlog ? opt.serving_cut_backlog : (1ull << 34);
  ctx->autotune = opt.autotune;
  if (opt.tune_cache_path) ctx->tune_cache_path = opt.tune_cache_path;
  tune_cache_load(ctx.get());
  for (int f = 0; f < 4; ++f) {
    ctx->max_blocks_per_sm[f] = batched_max_blocks_per_sm(f, 256);
    for (int u = 1; u <= kMaxUnroll; ++u) ctx->kernel_regs[u - 1][f] = batched_regs_per_thread(f, u);
  }
  e = ctx->fork.init();
  if (e != cudaSuccess) {
    ctx->fork.destroy();
    if (ctx->own_arena) cudaFree(ctx->arena_base);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    return set_error(ZMC_ECUDA, "side streams: %s", cudaGetErrorString(e));
  }
  zmc_ctx *raw = ctx.release();
  if (opt.serving) {
    raw->serving = true;
    zmc_status st = serving_start(raw);
    if (st != ZMC_OK) {
      zmc_destroy(raw);
      return st;
    }
  }
  *out = raw;
  return ZMC_OK;
}

zmc_status zmc_destroy(zmc_ctx *ctx) {
  if (!ctx) return ZMC_OK;
  cudaSetDevice(ctx->device);
  if (ctx->serving) serving_stop(ctx);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->stage) cudaFreeHost(ctx->stage);
  for (cudaStream_t sd : ctx->fork.side)
    if (sd) cudaStreamSynchronize(sd);
  ctx->fork.destroy();
  if (ctx->own_arena && ctx->arena_base) cudaFree(ctx->arena_base);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return ZMC_OK;
}

zmc_status zmc_plan_create(zmc_ctx *ctx, const zmc_desc *desc, size_t n, zmc_plan **out) {
  zmc_status st = check_ctx(ctx);
  if (st != ZMC_OK) return st;
  std::lock_guard<std::recursive_mutex> g(ctx->api_mu);
  return plan_build(ctx, desc, n, out);
}

zmc_status zmc_plan_run(zmc_plan *plan, uint32_t stages) {
  if (!plan) return set_error(ZMC_EINVAL, "null plan");
  zmc_ctx *ctx = plan->ctx;
  zmc_status st = check_ctx(ctx);
  if (st != ZMC_OK) return st;
  if ((stages & ZMC_STAGE_ALL) == 0 || (stages & ~ZMC_STAGE_ALL))
    return set_error(ZMC_EINVAL, "stages must be a non-empty subset of ZMC_STAGE_ALL");
  std::lock_guard<std::recursive_mutex> g(ctx->api_mu);
  if (stages != ZMC_STAGE_ALL) return plan_enqueue(plan, stages);
  if (!plan->graph) {
    cudaGraph_t graph = nullptr;
    ZMC_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    zmc_status est = plan_enqueue(plan, ZMC_STAGE_ALL);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (est != ZMC_OK) {
      if (graph) cudaGraphDestroy(graph);
      return est;
    }
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "graph capture");
    e = cudaGraphInstantiate(&plan->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "graph instantiate");
  }
  ZMC_CUDA(ctx, cudaGraphLaunch(plan->graph, ctx->stream));
  return ZMC_OK;
}

zmc_status zmc_plan_run_plain(zmc_plan *plan) {
  if (!plan) return set_error(ZMC_EINVAL, "null plan");
  zmc_status st = check_ctx(plan->ctx);
  if (st != ZMC_OK) return st;
  std::lock_guard<std::recursive_mutex> g(plan->ctx->api_mu);
  return plain_enqueue(plan);
}

zmc_status zmc_plan_results(zmc_plan *plan, zmc_result *out) {
  if (!plan || !out) return set_error(ZMC_EINVAL, "null argument");
  zmc_status st = check_ctx(plan->ctx);
  if (st != ZMC_OK) return st;
  std::lock_guard<std::recursive_mutex> g(plan->ctx->api_mu);
  return plan_results_to(plan, out);
}

zmc_status zmc_plan_device_results(zmc_plan *plan, void **device_ptr) {
  if (!plan || !device_ptr) return set_error(ZMC_EINVAL, "null argument");
  *device_ptr = plan->d_out;
  return ZMC_OK;
}

zmc_status zmc_plan_info_get(const zmc_plan *plan, zmc_plan_info *out) {
  if (!plan || !out) return set_error(ZMC_EINVAL, "null argument");
  out->n_fn = plan->n;
  out->n_chunks = plan->n_chunks;
  out->n_samples = plan->n_samples;
  unsigned g = 0;
  for (int f = 0; f < 4; ++f) g = std::max(g, plan->grid[f]);
  out->grid = g;
  out->block = plan->ctx->shape.block;
  for (int f = 0; f < 4; ++f) {
    out->family_grid[f] = plan->grid[f];
    out->family_block[f] = plan->fam_items[f] ? plan->block[f] : 0;
    out->tune_source[f] = plan->tune_source[f];
  }
  out->quints_per_lane = plan->quints;
  out->sms = static_cast<uint32_t>(plan->ctx->sms);
  for (int f = 0; f < 4; ++f) out->family_unroll[f] = plan->unroll[f];
  out->chunk_tune_source = plan->chunk_source;
  out->reserved = 0;
  return ZMC_OK;
}

zmc_status zmc_plan_destroy(zmc_plan *plan) {
  if (!plan) return ZMC_OK;
  std::lock_guard<std::recursive_mutex> g(plan->ctx->api_mu);
  cudaSetDevice(plan->ctx->device);
  plan_free(plan);
  return ZMC_OK;
}

zmc_status zmc_integrate(zmc_ctx *ctx, const zmc_desc *desc, size_t n, zmc_result *out) {
  zmc_status st = check_ctx(ctx);
  if (st != ZMC_OK) return st;
  if (!out) return set_error(ZMC_EINVAL, "null output");
  std::lock_guard<std::recursive_mutex> g(ctx->api_mu);
  zmc_plan *plan = nullptr;
  // the results copy below is the next use of the staging buffer, stream-ordered
  st = plan_build(ctx, desc, n, &plan, nullptr, nullptr, nullptr, false);
  if (st != ZMC_OK) return st;
  st = plan_enqueue(plan, ZMC_STAGE_ALL);
  if (st == ZMC_OK) st = plan_results_to(plan, out);
  plan_free(plan);
  return st;
}

zmc_status zmc_integrate_plain(zmc_ctx *ctx, const zmc_desc *desc, size_t n, zmc_result *out) {
  zmc_status st = check_ctx(ctx);
  if (st != ZMC_OK) return st;
  if (!out) return set_error(ZMC_EINVAL, "null output");
  std::lock_guard<std::recursive_mutex> g(ctx->api_mu);
  zmc_plan *plan = nullptr;
  st = plan_build(ctx, desc, n, &plan);
  if (st != ZMC_OK) return st;
  st = plain_enqueue(plan);
  if (st == ZMC_OK) st = plan_results_to(plan, out);
  plan_free(plan);
  return st;
}

zmc_status zmc_integrate_moments(zmc_ctx *ctx, const zmc_desc *desc, const uint64_t *s_begin,
                                 const uint64_t *s_end, size_t n, zmc_moments *out) {
  zmc_status st = check_ctx(ctx);
  if (st != ZMC_OK) return st;
  if (!out || !s_begin || !s_end) return set_error(ZMC_EINVAL, "null argument");
  static_assert(sizeof(zmc_moments) == sizeof(zmc_result), "moments share the result slot");
  std::lock_guard<std::recursive_mutex> g(ctx->api_mu);
  zmc_plan *plan = nullptr;
  st = plan_build(ctx, desc, n, &plan, s_begin, s_end, nullptr, false);
  if (st != ZMC_OK) return st;
  st = plan_enqueue(plan, ZMC_STAGE_ALL);
  if (st == ZMC_OK) st = plan_results_to(plan, reinterpret_cast<zmc_result *>(out));
  plan_free(plan);
  return st;
}

zmc_status zmc_integrate_functional(zmc_ctx *ctx, const zmc_desc *base, const uint32_t *slots,
                                    uint32_t n_slots, const double *values, size_t n_points,
                                    uint32_t independent_streams, zmc_result *out) {
  zmc_status st = check_ctx(ctx);
  if (st != ZMC_OK) return st;
  if (!base || !out || (n_slots && (!slots || !values)) || n_points == 0)
    return set_error(ZMC_EINVAL, "bad functional arguments");
  for (uint32_t k = 0; k < n_slots; ++k)
    if (slots[k] >= ZMC_SLOT_HI(ZMC_MAX_DIM))
      return set_error(ZMC_EINVAL, "slot %u out of range", slots[k]);
  if (independent_streams && static_cast<uint64_t>(base->stream_id) + n_points > (1ull << 32))
    return set_error(ZMC_EINVAL, "stream ids would exceed 32 bits");
  std::vector<zmc_desc> table(n_points, *base);
  for (size_t q = 0; q < n_points; ++q) {
    zmc_desc &d = table[q];
    for (uint32_t k = 0; k < n_slots; ++k) {
      const uint32_t slot = slots[k];
      const double v = values[q * n_slots + k];
      if (slot < ZMC_NPARAM)
        d.p[slot] = v;
      else if (slot < ZMC_SLOT_HI(0))
        d.lo[slot - ZMC_SLOT_LO(0)] = v;
      else
        d.hi[slot - ZMC_SLOT_HI(0)] = v;
    }
    if (independent_streams) d.stream_id = base->stream_id + static_cast<uint32_t>(q);
  }
  std::lock_guard<std::recursive_mutex> g(ctx->api_mu);
  zmc_plan *plan = nullptr;
  st = plan_build(ctx, table.data(), n_points, &plan, nullptr, nullptr, nullptr, false);
  if (st != ZMC_OK) return st;
  st = plan_enqueue(plan, ZMC_STAGE_ALL);
  if (st == ZMC_OK) st = plan_results_to(plan, out);
  plan_free(plan);
  return st;
}

zmc_status zmc_philox4x32_10(zmc_ctx *ctx, const uint32_t *ctr, const uint32_t *key,
                             uint32_t *out, size_t n) {
  zmc_status st = check_ctx(ctx);
  if (st != ZMC_OK) return st;
  if (n == 0) return ZMC_OK;
  if (!ctr || !key || !out) return set_error(ZMC_EINVAL, "null argument");
  std::lock_guard<std::recursive_mutex> g(ctx->api_mu);
  const size_t bytes = n * 40;  // 16 ctr + 8 key + 16 out
  char *d = static_cast<char *>(ctx->arena.alloc(bytes));
  if (!d) return set_error(ZMC_ENOMEM, "arena full");
  st = ensure_stage(ctx, bytes);
  if (st == ZMC_OK) {
    char *s = static_cast<char *>(ctx->stage);
    std::memcpy(s, ctr, n * 16);
    std::memcpy(s + n * 16, key, n * 8);
    cudaError_t e = cudaMemcpyAsync(d, s, n * 24, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = launch_philox(reinterpret_cast<uint32_t *>(d), reinterpret_cast<uint32_t *>(d + n * 16),
                        reinterpret_cast<uint32_t *>(d + n * 24), n, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s, d + n * 24, n * 16, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
      st = ctx_cuda_fail(ctx, e, "philox");
    else
      std::memcpy(out, s, n * 16);
  }
  ctx->arena.release(d);
  return st;
}

zmc_status zmc_philox_rate(zmc_ctx *ctx, uint64_t n_blocks, double *blocks_per_second) {
  zmc_status st = check_ctx(ctx);
  if (st != ZMC_OK) return st;
  if (!blocks_per_second) return set_error(ZMC_EINVAL, "null argument");
  if (n_blocks == 0 || n_blocks > (1ull << 40))
    return set_error(ZMC_EINVAL, "n_blocks must be in 1..2^40");
  std::lock_guard<std::recursive_mutex> g(ctx->api_mu);
  // one wave: 2 x 256-thread blocks per SM, every thread a whole number of groups of 4
  const unsigned grid = static_cast<unsigned>(ctx->sms) * 2u;
  const uint64_t threads = static_cast<uint64_t>(grid) * 256u;
  const uint64_t per = std::max<uint64_t>(4, (n_blocks + threads * 4 - 1) / (threads * 4) * 4);
  if (per > 0xFFFFFFF0ull) return set_error(ZMC_EINVAL, "n_blocks too large for one wave");
  const uint32_t per_thread = static_cast<uint32_t>(per);
  uint32_t *d = static_cast<uint32_t *>(ctx->arena.alloc(threads * sizeof(uint32_t)));
  if (!d) return set_error(ZMC_ENOMEM, "arena full");
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  // one untimed launch (clocks up, code loaded), then the timed one
  if (e == cudaSuccess) e = launch_philox_rate(per_thread, grid, d, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], ctx->stream);
  if (e == cudaSuccess) e = launch_philox_rate(per_thread, grid, d, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], ctx->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  ctx->arena.release(d);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "philox rate");
  if (!(ms > 0.0f)) return set_error(ZMC_ECUDA, "philox rate: zero elapsed time");
  *blocks_per_second = static_cast<double>(threads) * per_thread / (1e-3 * ms);
  return ZMC_OK;
}

zmc_status zmc_eval_samples(zmc_ctx *ctx, const zmc_desc *desc, uint64_t s_begin,
                            uint32_t count, float *out) {
  zmc_status st = check_ctx(ctx);
  if (st != ZMC_OK) return st;
  if (!desc || !out) return set_error(ZMC_EINVAL, "null argument");
  if (count == 0) return ZMC_OK;
  if (s_begin + count > desc->n_samples)
    return set_error(ZMC_EINVAL, "sample range beyond n_samples");
  FnDev fn;
  st = precompute(*desc, &fn, nullptr, nullptr);
  if (st != ZMC_OK) return st;
  std::lock_guard<std::recursive_mutex> g(ctx->api_mu);
  const size_t bytes = sizeof(FnDev) + static_cast<size_t>(count) * 4;
  char *d = static_cast<char *>(ctx->arena.alloc(bytes));
  if (!d) return set_error(ZMC_ENOMEM, "arena full");
  st = ensure_stage(ctx, bytes);
  if (st == ZMC_OK) {
    char *s = static_cast<char *>(ctx->stage);
    std::memcpy(s, &fn, sizeof fn);
    cudaError_t e = cudaMemcpyAsync(d, s, sizeof fn, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = launch_eval(static_cast<int>(desc->family), reinterpret_cast<FnDev *>(d), s_begin, count,
                      reinterpret_cast<float *>(d + sizeof(FnDev)), ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s, d + sizeof(FnDev), static_cast<size_t>(count) * 4,
                          cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
      st = ctx_cuda_fail(ctx, e, "eval_samples");
    else
      std::memcpy(out, s, static_cast<size_t>(count) * 4);
  }
  ctx->arena.release(d);
  return st;
}

}  // extern "C"
