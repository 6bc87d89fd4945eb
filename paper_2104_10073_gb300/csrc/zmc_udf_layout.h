// zmc_udf_layout.h -- where a user-defined integrand's constants sit in the
// FnDev payload words w[] (shared by the host, zmc_udf.cpp, and the run-time
// compiled device code, zmc_udf_kernel.cuh).  Dimensions up to kUdfMaxDim.
#pragma once

namespace zmc {

constexpr int kUdfMaxDim = 12;

// ZMC_UDF_F32: FP32 words
constexpr int kUdfF32W = 0;    // hi_i - lo_i, kUdfMaxDim words
constexpr int kUdfF32Lo = 12;  // lo_i, kUdfMaxDim words
constexpr int kUdfF32P = 24;   // p_j, 40 words
constexpr int kUdfF32S = 64;   // the scale S
// ZMC_UDF_F64: FP64 values, two words each (low word first)
constexpr int kUdfF64Lo = 0;   // lo_i, 2 kUdfMaxDim words
constexpr int kUdfF64W = 24;   // hi_i - lo_i, 2 kUdfMaxDim words
constexpr int kUdfF64P = 48;   // device address of the 40 FP64 parameters
constexpr int kUdfF64S = 50;   // the scale S

static_assert(kUdfF32S < 72 && kUdfF64S + 2 <= 72, "FnDev payload holds 72 words");

}  // namespace zmc
