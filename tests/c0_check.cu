// Host evaluation of the covariance kernels' few-FP64-operation C0 (c0_fast,
// the same source the kernels compile): reads "family u sc" lines from stdin
// (u the squared scaled distance as a hexadecimal double) and prints the
// value as a hexadecimal double.
#include <cstdio>
#include "../paper_1507_04789_gb300/csrc/mra_device.cuh"

int main() {
  int family;
  double u, sc;
  while (scanf("%d %la %la", &family, &u, &sc) == 3) printf("%a\n", mra::c0_fast(family, u, sc));
  return 0;
}
