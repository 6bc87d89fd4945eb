// Generated by gen_sincos.py: Remez fits of sin(2 pi t)/t and cos(2 pi t) in
// z = t^2 on |t| <= 1/8 turn, rounded to binary32.  Max error of the rounded
// polynomials in exact arithmetic: sin 2.99e-08, cos 6.68e-09.
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
