// Host evaluation of the free-smoothness Matern correlation (matern_nu, the
// same source the kernels compile): reads "nu h" pairs from stdin and prints
// rho, d rho / d h and d rho / d nu for each.
#include <cstdio>
#include "../paper_1507_04789_gb300/csrc/mra_device.cuh"

int main() {
  double nu, h;
  while (scanf("%lf %lf", &nu, &h) == 2) {
    const mra::Cov c = mra::make_cov(1.0, 1.0, 2, 0, nu);
    const mra::MaternNu m = mra::matern_nu(c, h);
    printf("%.17g %.17g %.17g\n", m.rho, m.dh, m.dnu);
  }
  return 0;
}
