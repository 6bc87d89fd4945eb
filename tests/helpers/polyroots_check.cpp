// Host-only check of the root form of degree-2..4 polynomials: for each input
// line "g e_0 ... e_g" prints "ok rel abs" where ok says whether a root form was
// found, rel is the largest |rootform(u) - q(u)| / |q(u)| over the points where
// q is well determined by its FP64 coefficients (|q(u)| >= 1e-10 sum_k |e_k u^k|)
// and abs the largest |rootform(u) - q(u)| / sum_k |e_k u^k| over all points;
// 2001 points u in [0, 1], both forms evaluated in long double (the root form
// from the FP64 roots it returns); "0 -1 -1" when no form was found.
#include <cmath>
#include <cstdio>

#include "zmc_runtime.h"

int main() {
  int g;
  while (std::scanf("%d", &g) == 1) {
    double e[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k <= g; ++k)
      if (std::scanf("%lf", &e[k]) != 1) return 2;
    zmc::RootForm rf;
    const bool ok = zmc::poly_root_form(e, g, &rf);
    if (!ok) {
      std::printf("0 -1 -1\n");
      continue;
    }
    long double worst = 0.0L, worst_abs = 0.0L;
    for (int t = 0; t <= 2000; ++t) {
      const long double u = t / 2000.0L;
      long double q = 0.0L, sa = 0.0L, up = 1.0L;
      for (int k = 0; k <= g; ++k) {
        q += e[k] * up;
        sa += std::fabs(e[k]) * up;
        up *= u;
      }
      long double r = rf.lead;
      for (int s = 0; s < rf.n; ++s) {
        if (rf.type[s] == 1) r *= u - static_cast<long double>(rf.v[s]);
        if (rf.type[s] == 2) {
          const long double d = u - static_cast<long double>(rf.v[s]);
          r *= d * d + static_cast<long double>(rf.v[s + 1]);
        }
      }
      if (std::fabs(q) >= 1e-10L * sa && std::fabs(r - q) / std::fabs(q) > worst)
        worst = std::fabs(r - q) / std::fabs(q);
      if (std::fabs(r - q) / sa > worst_abs) worst_abs = std::fabs(r - q) / sa;
    }
    std::printf("1 %.3Le %.3Le\n", worst, worst_abs);
  }
  return 0;
}
