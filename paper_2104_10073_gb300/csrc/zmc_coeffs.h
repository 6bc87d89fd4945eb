// Generated by gen_coeffs.py: Remez fits rounded to binary32.  Max error of the
// rounded polynomials in exact arithmetic:
//   sin(2 pi t), |t| <= 1/8 (in t^2): 2.99e-08 absolute
//   cos(2 pi t), |t| <= 1/8 (in t^2): 6.68e-09 absolute
//   2^x, |x| <= 0.51, degree 6:       2.01e-08 relative
#pragma once
#define ZMC_SIN_C0 0x1.921fb40000000p+2f  // 6.283185005e+00
#define ZMC_SIN_C1 -0x1.4abba80000000p+5f  // -4.134162903e+01
#define ZMC_SIN_C2 0x1.465a3e0000000p+6f  // 8.158812714e+01
#define ZMC_SIN_C3 -0x1.2cf5d40000000p+6f  // -7.524006653e+01
#define ZMC_COS_C0 0x1.0000000000000p+0f  // 1.000000000e+00
#define ZMC_COS_C1 -0x1.3bd3cc0000000p+4f  // -1.973920822e+01
#define ZMC_COS_C2 0x1.03c1dc0000000p+6f  // 6.493931580e+01
#define ZMC_COS_C3 -0x1.55c57c0000000p+6f  // -8.544285583e+01
#define ZMC_COS_C4 0x1.d9c3640000000p+5f  // 5.922040558e+01
#define ZMC_EXP2_C0 0x1.0000000000000p+0f  // 1.000000000e+00
#define ZMC_EXP2_C1 0x1.62e4300000000p-1f  // 6.931471825e-01
#define ZMC_EXP2_C2 0x1.ebfbda0000000p-3f  // 2.402264625e-01
#define ZMC_EXP2_C3 0x1.c6aeb00000000p-5f  // 5.550321937e-02
#define ZMC_EXP2_C4 0x1.3b2dfc0000000p-7f  // 9.618518874e-03
#define ZMC_EXP2_C5 0x1.5f57500000000p-10f  // 1.340259798e-03
#define ZMC_EXP2_C6 0x1.41c6b40000000p-13f  // 1.534348412e-04
