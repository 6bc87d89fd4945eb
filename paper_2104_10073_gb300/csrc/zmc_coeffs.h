// Generated by gen_coeffs.py: Remez fits rounded to binary32.  Max error of the
// rounded polynomials in exact arithmetic:
//   cos(2 pi t), 0 <= t <= 1/4 (degree 5 in t^2): 1.84e-08 absolute
//   2^x, |x| <= 0.51, degree 6:       2.01e-08 relative
#pragma once
#define ZMC_COSQ_C0 0x1.0000000000000p+0f  // 1.000000000e+00
#define ZMC_COSQ_C1 -0x1.3bd3cc0000000p+4f  // -1.973920822e+01
#define ZMC_COSQ_C2 0x1.03c1e40000000p+6f  // 6.493934631e+01
#define ZMC_COSQ_C3 -0x1.55d0760000000p+6f  // -8.545357513e+01
#define ZMC_COSQ_C4 0x1.e126f20000000p+5f  // 6.014401627e+01
#define ZMC_COSQ_C5 -0x1.8fb73e0000000p+4f  // -2.498223686e+01
#define ZMC_EXP2_C0 0x1.0000000000000p+0f  // 1.000000000e+00
#define ZMC_EXP2_C1 0x1.62e4300000000p-1f  // 6.931471825e-01
#define ZMC_EXP2_C2 0x1.ebfbda0000000p-3f  // 2.402264625e-01
#define ZMC_EXP2_C3 0x1.c6aeb00000000p-5f  // 5.550321937e-02
#define ZMC_EXP2_C4 0x1.3b2dfc0000000p-7f  // 9.618518874e-03
#define ZMC_EXP2_C5 0x1.5f57500000000p-10f  // 1.340259798e-03
#define ZMC_EXP2_C6 0x1.41c6b40000000p-13f  // 1.534348412e-04
