// Generated by gen_coeffs.py: Remez fits rounded to binary32.  Max error of the
// rounded polynomials in exact arithmetic:
//   sin(2 pi t), |t| <= 1/4 (t times degree 4 in t^2): 4.23e-08 relative
#pragma once
#define ZMC_SINQ_C0 0x1.921fb60000000p+2f  // 6.283185482e+00
#define ZMC_SINQ_C1 -0x1.4abbc20000000p+5f  // -4.134167862e+01
#define ZMC_SINQ_C2 0x1.4668b00000000p+6f  // 8.160223389e+01
#define ZMC_SINQ_C3 -0x1.324cca0000000p+6f  // -7.657498932e+01
#define ZMC_SINQ_C4 0x1.3daff60000000p+5f  // 3.971091843e+01
