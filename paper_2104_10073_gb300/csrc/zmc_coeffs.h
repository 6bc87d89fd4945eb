// Generated by gen_coeffs.py: Remez fits rounded to binary32.  Max error of the
// rounded polynomials in exact arithmetic:
//   sin(2 pi t), |t| <= 1/4 (t times degree 5 in t^2): 5.38e-08 relative
#pragma once
#define ZMC_SINQ_C0 0x1.921fb60000000p+2f  // 6.283185482e+00
#define ZMC_SINQ_C1 -0x1.4abbce0000000p+5f  // -4.134170151e+01
#define ZMC_SINQ_C2 0x1.466bc00000000p+6f  // 8.160522461e+01
#define ZMC_SINQ_C3 -0x1.32d1120000000p+6f  // -7.670417023e+01
#define ZMC_SINQ_C4 0x1.500ff80000000p+5f  // 4.200779724e+01
#define ZMC_SINQ_C5 -0x1.cc345a0000000p+3f  // -1.438139057e+01
