// Host check of the covariance exponential exp_neg_tab (table-driven, Tang 1989)
// against long double expl: prints the largest relative error over a sweep.
#include <cmath>
#include <cstdio>
#include "../paper_1507_04789_gb300/csrc/mra_device.cuh"

int main() {
  double worst = 0.0, worst_a = 0.0;
  long n = 0;
  // dense sweep of [0, 40], a log sweep up to 700, and the reduction boundaries
  for (long i = 0; i <= 2000000; ++i) {
    const double a = 40.0 * (double)i / 2000000.0;
    const long double ref = expl(-(long double)a);
    const double v = mra::exp_neg_tab(a, mra::k_exp2_tab_host);
    const double rel = (double)fabsl(((long double)v - ref) / ref);
    if (rel > worst) { worst = rel; worst_a = a; }
    ++n;
  }
  for (double a = 1e-300; a < 700.0; a *= 1.001) {
    const long double ref = expl(-(long double)a);
    const double v = mra::exp_neg_tab(a, mra::k_exp2_tab_host);
    const double rel = (double)fabsl(((long double)v - ref) / ref);
    if (rel > worst) { worst = rel; worst_a = a; }
    ++n;
  }
  for (int k = 0; k < 64 * 600; ++k) {
    const double a0 = (double)k * (double)(mra::MRA_LN2L / 128.0L);
    for (double d : {-1e-12, 0.0, 1e-12}) {
      const double a = a0 + d;
      if (a < 0.0) continue;
      const long double ref = expl(-(long double)a);
      const double v = mra::exp_neg_tab(a, mra::k_exp2_tab_host);
      const double rel = (double)fabsl(((long double)v - ref) / ref);
      if (rel > worst) { worst = rel; worst_a = a; }
      ++n;
    }
  }
  const int zero_ok = mra::exp_neg_tab(709.0, mra::k_exp2_tab_host) == 0.0 && mra::exp_neg_tab(0.0, mra::k_exp2_tab_host) == 1.0;
  printf("points %ld max_rel %.3e at a=%.17g edges_ok %d\n", n, worst, worst_a, zero_ok);
  return 0;
}
