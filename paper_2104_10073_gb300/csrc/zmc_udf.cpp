// zmc_udf.cpp -- user-defined integrands compiled at run time with NVRTC.
//
// The paper's integrators take the integrand as user code that is compiled for
// the GPU.  Here the user writes zmc_user_f in CUDA C++; zmc_udf_create compiles
// it together with the library's own device code (zmc_device.cuh: Philox4x32-10,
// the box map, the per-chunk FP32 sums, the persistent work-list loop) and
// zmc_udf_kernel.cuh, for sm_103a, into a cubin kept in the handle.  The texts of
// those headers are compiled into this library (zmc_jit_sources.h, generated by
// the build), so the user-defined path runs exactly the sampling code of the
// built-in families.  NVRTC is opened with dlopen at first use; without it
// zmc_udf_create returns ZMC_ENOSYS and nothing else is affected.
//
// zmc_udf_integrate loads the cubin (cudaLibraryLoadData, once per handle),
// builds the same FnDev / Entry / LaunchHdr tables as a plan, launches the
// compiled zmc_udf_batched kernel and then the library's zmc_merge_kernel.
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvrtc.h>  // types and prototypes only: the library is opened with dlopen

#include "zmc_jit_sources.h"
#include "zmc_runtime.h"
#include "zmc_udf_layout.h"

using namespace zmc;

struct zmc_udf {
  std::vector<uint32_t> dims;   // per function
  std::vector<double> scales;   // per function: the kernel sums S f
  uint32_t precision = 0;
  std::vector<char> cubin;
  std::string log;
  mutable std::mutex mu;
  mutable cudaLibrary_t lib = nullptr;
  mutable cudaKernel_t k_batched = nullptr;
  mutable cudaKernel_t k_eval = nullptr;
  mutable int max_blocks = 0;  // resident 256-thread blocks per SM of k_batched
};

namespace {

struct Nvrtc {
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&nvrtcGetErrorString) error_string = nullptr;
  bool ok = false;
  std::string why;
};

const Nvrtc &nvrtc() {
  static Nvrtc api;
  static std::once_flag once;
  std::call_once(once, [] {
    const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void *h = nullptr;
    for (const char *n : names)
      if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) {
      api.why = "libnvrtc.so.13 not found";
      return;
    }
    api.create = reinterpret_cast<decltype(api.create)>(dlsym(h, "nvrtcCreateProgram"));
    api.compile = reinterpret_cast<decltype(api.compile)>(dlsym(h, "nvrtcCompileProgram"));
    api.log_size = reinterpret_cast<decltype(api.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
    api.log = reinterpret_cast<decltype(api.log)>(dlsym(h, "nvrtcGetProgramLog"));
    api.cubin_size = reinterpret_cast<decltype(api.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
    api.cubin = reinterpret_cast<decltype(api.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
    api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
    api.error_string =
        reinterpret_cast<decltype(api.error_string)>(dlsym(h, "nvrtcGetErrorString"));
    api.ok = api.create && api.compile && api.log_size && api.log && api.cubin_size &&
             api.cubin && api.destroy && api.error_string;
    if (!api.ok) api.why = "libnvrtc lacks an expected entry point";
  });
  return api;
}

// Minimal standard headers for the run-time compilation (NVRTC has none).
const char kStdint[] =
    "#pragma once\n"
    "typedef signed char int8_t; typedef short int16_t; typedef int int32_t;\n"
    "typedef long long int64_t; typedef unsigned char uint8_t;\n"
    "typedef unsigned short uint16_t; typedef unsigned int uint32_t;\n"
    "typedef unsigned long long uint64_t;\n";
const char kCstdint[] =
    "#pragma once\n#include \"stdint.h\"\n"
    "namespace std { using ::int8_t; using ::int16_t; using ::int32_t; using ::int64_t;\n"
    "using ::uint8_t; using ::uint16_t; using ::uint32_t; using ::uint64_t; }\n";
const char kStddef[] =
    "#pragma once\ntypedef decltype(sizeof(0)) size_t;\n"
    "typedef decltype((char *)0 - (char *)0) ptrdiff_t;\n";
const char kCstddef[] =
    "#pragma once\n#include \"stddef.h\"\nnamespace std { using ::size_t; using ::ptrdiff_t; }\n";
const char kCudaRuntime[] = "#pragma once\n";

bool finite_f32(double v) { return std::isfinite(v) && std::fabs(v) <= 3.0e38; }

void put_f32(uint32_t *w, double v) {
  const float f = static_cast<float>(v);
  std::memcpy(w, &f, 4);
}

void put_f64(uint32_t *w, double v) { std::memcpy(w, &v, 8); }

size_t round256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

// FnDev of one user integrand (validated).  For ZMC_UDF_F64 the address of its
// FP64 parameters is filled in by udf_run.
zmc_status udf_fn(const zmc_udf *u, const UdfRow &d, size_t i, FnDev *fn) {
  if (d.func >= u->dims.size())
    return set_error(ZMC_EINVAL, "row %zu: function %u, the udf has %zu", i, d.func,
                     u->dims.size());
  if (d.dim != u->dims[d.func])
    return set_error(ZMC_EINVAL, "row %zu: dim %u, function %u was compiled for %u", i, d.dim,
                     d.func, u->dims[d.func]);
  const double scale = u->scales[d.func];
  if (d.n_samples == 0 || d.n_samples > (1ull << 62))
    return set_error(ZMC_EINVAL, "row %zu: n_samples must be in 1..2^62", i);
  std::memset(fn, 0, sizeof *fn);
  double vol = 1.0;
  const bool f32 = u->precision == ZMC_UDF_F32;
  for (uint32_t k = 0; k < d.dim; ++k) {
    if (!std::isfinite(d.lo[k]) || !std::isfinite(d.hi[k]) || !(d.lo[k] < d.hi[k]))
      return set_error(ZMC_EINVAL, "row %zu: box dimension %u needs finite lo < hi", i, k);
    const double w = d.hi[k] - d.lo[k];
    vol *= w;
    if (f32) {
      if (!finite_f32(w) || !finite_f32(d.lo[k]))
        return set_error(ZMC_EINVAL, "row %zu: box out of FP32 range", i);
      put_f32(&fn->w[kUdfF32W + k], w);
      put_f32(&fn->w[kUdfF32Lo + k], d.lo[k]);
    } else {
      put_f64(&fn->w[kUdfF64Lo + 2 * k], d.lo[k]);
      put_f64(&fn->w[kUdfF64W + 2 * k], w);
    }
  }
  for (int j = 0; j < ZMC_NPARAM; ++j) {
    if (!std::isfinite(d.p[j]) || (f32 && !finite_f32(d.p[j])))
      return set_error(ZMC_EINVAL, "row %zu: parameter p[%d] not finite%s", i, j,
                       f32 ? " in FP32" : "");
    if (f32) put_f32(&fn->w[kUdfF32P + j], d.p[j]);
  }
  if (f32)
    put_f32(&fn->w[kUdfF32S], scale);
  else
    put_f64(&fn->w[kUdfF64S], scale);
  fn->variant = variant_code(ZMC_USER, d.dim, d.func);
  fn->stream_id = d.stream_id;
  fn->key0 = static_cast<uint32_t>(d.seed);
  fn->key1 = static_cast<uint32_t>(d.seed >> 32);
  fn->n_samples = d.n_samples;
  fn->volume = vol;
  fn->inv_scale = 1.0 / scale;  // a power of two: exact
  return ZMC_OK;
}

UdfRow row_of(const zmc_desc &d) {
  UdfRow r;
  r.dim = d.dim;
  r.func = d.deg;
  r.stream_id = d.stream_id;
  r.n_samples = d.n_samples;
  r.seed = d.seed;
  r.lo = d.lo;
  r.hi = d.hi;
  r.p = d.p;
  return r;
}

// Load the cubin (once per handle; the library is context independent).
zmc_status udf_load(zmc_ctx *ctx, const zmc_udf *u) {
  std::lock_guard<std::mutex> g(u->mu);
  if (u->lib) return ZMC_OK;
  cudaLibrary_t lib = nullptr;
  cudaError_t e = cudaLibraryLoadData(&lib, u->cubin.data(), nullptr, nullptr, 0, nullptr,
                                      nullptr, 0);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "udf cudaLibraryLoadData");
  cudaKernel_t kb = nullptr, ke = nullptr;
  e = cudaLibraryGetKernel(&kb, lib, "zmc_udf_batched");
  if (e == cudaSuccess) e = cudaLibraryGetKernel(&ke, lib, "zmc_udf_eval");
  int nb = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, reinterpret_cast<const void *>(kb),
                                                      256, 0);
  if (e != cudaSuccess) {
    cudaLibraryUnload(lib);
    return ctx_cuda_fail(ctx, e, "udf kernel lookup");
  }
  u->k_batched = kb;
  u->k_eval = ke;
  u->max_blocks = nb > 0 ? nb : 1;
  u->lib = lib;
  return ZMC_OK;
}

// Device blocks of one call, taken from the context's arena.
struct ArenaBlocks {
  zmc_ctx *ctx;
  std::vector<void *> held;
  void *get(size_t bytes) {
    void *p = ctx->arena.alloc(bytes);
    if (p) held.push_back(p);
    return p;
  }
  ~ArenaBlocks() {
    for (void *p : held) ctx->arena.release(p);
  }
};

void set_param_address(FnDev *fn, const double *d_p) {
  const uint64_t a = reinterpret_cast<uint64_t>(d_p);
  fn->w[kUdfF64P] = static_cast<uint32_t>(a);
  fn->w[kUdfF64P + 1] = static_cast<uint32_t>(a >> 32);
}

}  // namespace

namespace zmc {

// Integrate n user rows: the same FnDev / Entry / LaunchHdr tables as a plan,
// the compiled persistent kernel, then the library's FP64 merge.  FP64
// parameters are uploaded once per distinct parameter array.
zmc_status udf_run(zmc_ctx *ctx, const zmc_udf *udf, const UdfRow *rows, size_t n,
                   zmc_result *out) {
  if (!ctx) return set_error(ZMC_EINVAL, "null context");
  if (!udf || !rows || !out || n == 0) return set_error(ZMC_EINVAL, "bad udf arguments");
  if (n >= (1u << 31)) return set_error(ZMC_EINVAL, "too many rows");
  if (ctx->poisoned) return set_error(ZMC_ECUDA, "context poisoned by an earlier CUDA error");
  std::lock_guard<std::recursive_mutex> g(ctx->api_mu);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaSetDevice");
  zmc_status st = udf_load(ctx, udf);
  if (st != ZMC_OK) return st;

  const bool f64 = udf->precision == ZMC_UDF_F64;
  const uint64_t chunk = chunk_samples_of(ctx->quints_per_lane);
  std::vector<FnDev> tab(n);
  std::vector<uint64_t> rec_off(n);
  std::vector<uint32_t> prow(n);        // FP64: index of the row's parameter block
  std::vector<const double *> params;   // distinct parameter arrays, in first-use order
  uint64_t total = 0;
  for (size_t i = 0; i < n; ++i) {
    st = udf_fn(udf, rows[i], i, &tab[i]);  // validates
    if (st != ZMC_OK) return st;
    rec_off[i] = total;
    total += (rows[i].n_samples + chunk - 1) / chunk;
    if (f64) {
      if (params.empty() || params.back() != rows[i].p) {
        if (params.size() >= (1u << 24)) return set_error(ZMC_EINVAL, "too many parameter rows");
        params.push_back(rows[i].p);
      }
      prow[i] = static_cast<uint32_t>(params.size() - 1);
    }
  }
  ArenaBlocks ab{ctx, {}};
  const size_t fn_b = n * sizeof(FnDev), ent_b = n * sizeof(Entry), mrg_b = n * sizeof(FnDev *),
               p_b = params.size() * ZMC_NPARAM * sizeof(double);
  auto *d_fns = static_cast<FnDev *>(ab.get(fn_b));
  auto *d_rec = static_cast<float2 *>(ab.get(total * sizeof(float2)));
  auto *d_out = static_cast<zmc_result *>(ab.get(n * sizeof(zmc_result)));
  auto *d_ent = static_cast<Entry *>(ab.get(ent_b));
  auto *d_mrg = static_cast<const FnDev **>(ab.get(mrg_b));
  auto *d_hdr = static_cast<LaunchHdr *>(ab.get(sizeof(LaunchHdr)));
  auto *d_p = static_cast<double *>(p_b ? ab.get(p_b) : nullptr);
  if (!d_fns || !d_rec || !d_out || !d_ent || !d_mrg || !d_hdr || (p_b && !d_p))
    return set_error(ZMC_ENOMEM, "udf call needs %.1f MB of device memory",
                     (fn_b + total * 8.0 + n * 64.0 + p_b) / 1e6);

  // host tables in the pinned staging buffer: fns | entries | merge list | hdr | params
  const size_t o_ent = round256(fn_b), o_mrg = o_ent + round256(ent_b),
               o_hdr = o_mrg + round256(mrg_b), o_p = o_hdr + round256(sizeof(LaunchHdr)),
               o_end = o_p + round256(p_b);
  st = ensure_stage(ctx, std::max(o_end, n * sizeof(zmc_result)));
  if (st != ZMC_OK) return st;
  char *s = static_cast<char *>(ctx->stage);
  auto *fns = reinterpret_cast<FnDev *>(s);
  auto *ents = reinterpret_cast<Entry *>(s + o_ent);
  auto *mrg = reinterpret_cast<const FnDev **>(s + o_mrg);
  auto *hdr = reinterpret_cast<LaunchHdr *>(s + o_hdr);
  auto *ps = reinterpret_cast<double *>(s + o_p);
  for (size_t q = 0; q < params.size(); ++q)
    std::memcpy(ps + q * ZMC_NPARAM, params[q], ZMC_NPARAM * sizeof(double));
  for (size_t i = 0; i < n; ++i) {
    fns[i] = tab[i];
    if (f64) set_param_address(&fns[i], d_p + static_cast<size_t>(prow[i]) * ZMC_NPARAM);
    fns[i].rec = d_rec + rec_off[i];
    fns[i].out = d_out + i;
    mrg[i] = d_fns + i;
  }
  // the work list runs the rows grouped by variant (dimension and user function),
  // so that consecutive work items, which co-resident warps take, use the same
  // specialised code; records and results stay in row order, so the order
  // changes no result
  std::vector<uint32_t> order(n);
  for (size_t i = 0; i < n; ++i) order[i] = static_cast<uint32_t>(i);
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t a, uint32_t b) { return tab[a].variant < tab[b].variant; });
  uint64_t item = 0;
  for (size_t k = 0; k < n; ++k) {
    const uint32_t i = order[k];
    ents[k].item_begin = item;
    ents[k].fn = d_fns + i;
    ents[k].chunk_begin = 0;
    item += (rows[i].n_samples + chunk - 1) / chunk;
  }
  std::memset(hdr, 0, sizeof *hdr);
  hdr->item_end[0] = item;
  hdr->n_entries = static_cast<uint32_t>(n);
  hdr->n_merge = static_cast<uint32_t>(n);
  hdr->quints_per_lane = ctx->quints_per_lane;

  cudaStream_t str = ctx->stream;
  e = cudaMemcpyAsync(d_fns, fns, fn_b, cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ent, ents, ent_b, cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_mrg, mrg, mrg_b, cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_hdr, hdr, sizeof *hdr, cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess && p_b) e = cudaMemcpyAsync(d_p, ps, p_b, cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess) {
    // persistent grid: the kernel's occupancy, no more warps than work items
    const uint64_t want = (item + 7) / 8;
    const uint64_t cap = static_cast<uint64_t>(ctx->sms) * udf->max_blocks;
    const unsigned grid = static_cast<unsigned>(std::max<uint64_t>(1, std::min(want, cap)));
    const Entry *a0 = d_ent;
    LaunchHdr *a1 = d_hdr;
    void *args[] = {&a0, &a1};
    e = cudaLaunchKernel(reinterpret_cast<const void *>(udf->k_batched), dim3(grid), dim3(256),
                         args, 0, str);
  }
  if (e == cudaSuccess) {
    const unsigned mg = static_cast<unsigned>(
        std::min<uint64_t>((n + 7) / 8, static_cast<uint64_t>(ctx->sms) * 16));
    e = launch_merge(d_mrg, d_hdr, mg, str);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s, d_out, n * sizeof(zmc_result), cudaMemcpyDeviceToHost, str);
  if (e == cudaSuccess) e = cudaStreamSynchronize(str);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "udf integrate");
  std::memcpy(out, s, n * sizeof(zmc_result));
  return ZMC_OK;
}

uint32_t udf_dim(const zmc_udf *udf) { return udf && !udf->dims.empty() ? udf->dims[0] : 0; }

}  // namespace zmc

extern "C" {

zmc_status zmc_udf_create_multi(const char *const *sources, const uint32_t *dims,
                                uint32_t n_funcs, uint32_t precision, const double *amplitudes,
                                zmc_udf **out) {
  if (!sources || !dims || !out) return set_error(ZMC_EINVAL, "null argument");
  *out = nullptr;
  if (n_funcs < 1 || n_funcs > 64) return set_error(ZMC_EINVAL, "n_funcs must be in 1..64");
  if (precision != ZMC_UDF_F32 && precision != ZMC_UDF_F64)
    return set_error(ZMC_EINVAL, "precision must be ZMC_UDF_F32 or ZMC_UDF_F64");
  std::vector<double> scales(n_funcs, 1.0);
  for (uint32_t k = 0; k < n_funcs; ++k) {
    if (!sources[k]) return set_error(ZMC_EINVAL, "source %u is null", k);
    if (dims[k] < 1 || dims[k] > static_cast<uint32_t>(kUdfMaxDim))
      return set_error(ZMC_EINVAL, "function %u: dim %u not in 1..%d", k, dims[k], kUdfMaxDim);
    const double a = amplitudes ? amplitudes[k] : 0.0;
    if (!(a >= 0.0) || !std::isfinite(a))
      return set_error(ZMC_EINVAL, "function %u: amplitude must be finite and >= 0", k);
    if (a > 0.0) {
      int sexp = 48 - static_cast<int>(std::ceil(std::log2(a)));
      sexp = std::max(-100, std::min(100, sexp));
      scales[k] = std::ldexp(1.0, sexp);
    }
  }
  const Nvrtc &api = nvrtc();
  if (!api.ok) return set_error(ZMC_ENOSYS, "NVRTC unavailable: %s", api.why.c_str());

  // each source in a namespace of its own, then the sampling path, then the
  // thunks and the (dimension, function) switch
  std::string prog = "#define ZMC_UDF_PRECISION " + std::to_string(precision) + "\n" +
                     "#include \"zmc_device.cuh\"\n";
  for (uint32_t k = 0; k < n_funcs; ++k) {
    const std::string ks = std::to_string(k);
    prog += "namespace zmc_user_" + ks + " {\n#define ZMC_UDF_DIM " + std::to_string(dims[k]) +
            "\n#line 1 \"zmc_user_source_" + ks + "\"\n" + sources[k] +
            "\n#undef ZMC_UDF_DIM\n}\n";
  }
  prog += "#include \"zmc_udf_kernel.cuh\"\nnamespace zmc {\nnamespace {\n";
  for (uint32_t k = 0; k < n_funcs; ++k) {
    const std::string ks = std::to_string(k);
    prog += "template <> struct UserFn<" + ks +
            "> { __device__ __forceinline__ static UdfReal f(const UdfReal *x, const UdfReal *p) "
            "{ return ::zmc_user_" + ks + "::zmc_user_f(x, p); } };\n";
  }
  std::string item_cases, eval_cases;
  for (uint32_t k = 0; k < n_funcs; ++k) {
    const std::string v = "variant_code(ZMC_USER, " + std::to_string(dims[k]) + ", " +
                          std::to_string(k) + ")";
    const std::string targs = "<ZMC_USER, " + std::to_string(dims[k]) + ", " + std::to_string(k) + ">";
    item_cases += "    case " + v + ": run_item" + targs + "(fn, chunk, Q, lane); break;\n";
    eval_cases += "    case " + v + ": eval_range" + targs + "(fn, s_begin, count, out); break;\n";
  }
  prog += "__device__ void udf_dispatch_item(const FnDev *fn, uint64_t chunk, uint32_t Q, "
          "uint32_t lane) {\n  switch (fn->variant) {\n" + item_cases +
          "    default: break;\n  }\n}\n"
          "__device__ void udf_dispatch_eval(const FnDev *fn, uint64_t s_begin, uint32_t count, "
          "float *out) {\n  switch (fn->variant) {\n" + eval_cases +
          "    default: break;\n  }\n}\n}  // namespace\n}  // namespace zmc\n";

  const char *hdr_text[] = {kJitZmcH,   kJitZmcInternalH, kJitZmcDeviceCuh, kJitZmcUdfKernelCuh,
                            kJitZmcUdfLayoutH, kStdint, kCstdint, kStddef, kCstddef,
                            kCudaRuntime};
  const char *hdr_name[] = {"zmc.h",    "zmc_internal.h", "zmc_device.cuh", "zmc_udf_kernel.cuh",
                            "zmc_udf_layout.h", "stdint.h", "cstdint", "stddef.h", "cstddef",
                            "cuda_runtime.h"};
  const int n_hdr = static_cast<int>(sizeof hdr_name / sizeof hdr_name[0]);
  nvrtcProgram p = nullptr;
  nvrtcResult r = api.create(&p, prog.c_str(), "zmc_udf.cu", n_hdr, hdr_text, hdr_name);
  if (r != NVRTC_SUCCESS)
    return set_error(ZMC_EINVAL, "nvrtcCreateProgram: %s", api.error_string(r));
  // -default-device: the library headers' host prototypes (and unannotated user
  // functions) are taken as device declarations
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo",
                        "-default-device", "-diag-suppress=177", "--split-compile=0"};
  r = api.compile(p, static_cast<int>(sizeof opts / sizeof opts[0]), opts);
  size_t log_n = 0;
  api.log_size(p, &log_n);
  std::string log(log_n, '\0');
  if (log_n) api.log(p, &log[0]);
  while (!log.empty() && (log.back() == '\0' || log.back() == '\n')) log.pop_back();
  if (r != NVRTC_SUCCESS) {
    api.destroy(&p);
    return set_error(ZMC_EINVAL, "udf source does not compile: %.440s", log.c_str());
  }
  size_t cb = 0;
  api.cubin_size(p, &cb);
  auto u = new zmc_udf;
  u->cubin.resize(cb);
  api.cubin(p, u->cubin.data());
  api.destroy(&p);
  u->dims.assign(dims, dims + n_funcs);
  u->scales = scales;
  u->precision = precision;
  u->log = log;
  *out = u;
  return ZMC_OK;
}

zmc_status zmc_udf_create(const char *source, uint32_t dim, uint32_t precision,
                          double amplitude, zmc_udf **out) {
  if (!source || !out) return set_error(ZMC_EINVAL, "null argument");
  return zmc_udf_create_multi(&source, &dim, 1, precision, &amplitude, out);
}

const char *zmc_udf_log(const zmc_udf *udf) { return udf ? udf->log.c_str() : ""; }

zmc_status zmc_udf_destroy(zmc_udf *udf) {
  if (!udf) return ZMC_OK;
  if (udf->lib) cudaLibraryUnload(udf->lib);
  delete udf;
  return ZMC_OK;
}

zmc_status zmc_udf_integrate(zmc_ctx *ctx, const zmc_udf *udf, const zmc_desc *desc, size_t n,
                             zmc_result *out) {
  if (!ctx) return set_error(ZMC_EINVAL, "null context");
  if (!udf || !desc || !out || n == 0) return set_error(ZMC_EINVAL, "bad udf_integrate arguments");
  std::vector<UdfRow> rows(n);
  for (size_t i = 0; i < n; ++i) {
    if (desc[i].family != ZMC_USER)
      return set_error(ZMC_EINVAL, "descriptor %zu: family must be ZMC_USER", i);
    if (desc[i].dim > ZMC_MAX_DIM)
      return set_error(ZMC_EINVAL,
                       "descriptor %zu: a descriptor holds at most %d dimensions; integrands "
                       "of more integrate through zmc_normal_integrate_udf", i, ZMC_MAX_DIM);
    rows[i] = row_of(desc[i]);
  }
  return udf_run(ctx, udf, rows.data(), n, out);
}

zmc_status zmc_udf_eval_samples(zmc_ctx *ctx, const zmc_udf *udf, const zmc_desc *desc,
                                uint64_t s_begin, uint32_t count, float *out) {
  if (!ctx) return set_error(ZMC_EINVAL, "null context");
  if (!udf || !desc || !out) return set_error(ZMC_EINVAL, "null argument");
  if (ctx->poisoned) return set_error(ZMC_ECUDA, "context poisoned by an earlier CUDA error");
  if (desc->family != ZMC_USER) return set_error(ZMC_EINVAL, "family must be ZMC_USER");
  if (desc->dim > ZMC_MAX_DIM) return set_error(ZMC_EINVAL, "a descriptor holds at most 7 dimensions");
  if (count == 0) return ZMC_OK;
  if (s_begin + count > desc->n_samples)
    return set_error(ZMC_EINVAL, "sample range beyond n_samples");
  std::lock_guard<std::recursive_mutex> g(ctx->api_mu);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "cudaSetDevice");
  zmc_status st = udf_load(ctx, udf);
  if (st != ZMC_OK) return st;
  const bool f64 = udf->precision == ZMC_UDF_F64;
  ArenaBlocks ab{ctx, {}};
  auto *d_fn = static_cast<FnDev *>(ab.get(sizeof(FnDev)));
  auto *d_p = static_cast<double *>(ab.get(ZMC_NPARAM * sizeof(double)));
  auto *d_v = static_cast<float *>(ab.get(static_cast<size_t>(count) * 4));
  if (!d_fn || !d_p || !d_v) return set_error(ZMC_ENOMEM, "arena full");
  const size_t o_p = round256(sizeof(FnDev));
  st = ensure_stage(ctx, std::max<size_t>(o_p + ZMC_NPARAM * 8, static_cast<size_t>(count) * 4));
  if (st != ZMC_OK) return st;
  char *s = static_cast<char *>(ctx->stage);
  FnDev *fn = reinterpret_cast<FnDev *>(s);
  st = udf_fn(udf, row_of(*desc), 0, fn);
  if (st != ZMC_OK) return st;
  if (f64) set_param_address(fn, d_p);
  std::memcpy(s + o_p, desc->p, ZMC_NPARAM * sizeof(double));
  cudaStream_t str = ctx->stream;
  e = cudaMemcpyAsync(d_fn, fn, sizeof(FnDev), cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_p, s + o_p, ZMC_NPARAM * sizeof(double), cudaMemcpyHostToDevice, str);
  if (e == cudaSuccess) {
    const uint64_t quints = (s_begin + count - 1) / kQuint - s_begin / kQuint + 1;
    const unsigned grid = static_cast<unsigned>(std::min<uint64_t>((quints + 255) / 256, 1024));
    const FnDev *a0 = d_fn;
    uint64_t a1 = s_begin;
    uint32_t a2 = count;
    float *a3 = d_v;
    void *args[] = {&a0, &a1, &a2, &a3};
    e = cudaLaunchKernel(reinterpret_cast<const void *>(udf->k_eval), dim3(grid), dim3(256), args,
                         0, str);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s, d_v, static_cast<size_t>(count) * 4, cudaMemcpyDeviceToHost, str);
  if (e == cudaSuccess) e = cudaStreamSynchronize(str);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "udf eval_samples");
  std::memcpy(out, s, static_cast<size_t>(count) * 4);
  return ZMC_OK;
}

}  // extern "C"
