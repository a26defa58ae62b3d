// Host driver for tests/test_double_float.py: applies the library's double-float sum,
// product and fused multiply-add (paper_2301_05985_gb300/csrc/df32.cuh) to the operands read
// from stdin ("a_hi a_lo b_hi b_lo c_hi c_lo" per line, C99 hex floats) and prints
// "sum_hi sum_lo prod_hi prod_lo fma_hi fma_lo" per line, again as hex floats.
#include <cstdio>

#include "df32.cuh"

int main() {
  float v[6];
  while (std::scanf("%a %a %a %a %a %a", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) == 6) {
    const df a(v[0], v[1]), b(v[2], v[3]), c(v[4], v[5]);
    const df s = a + b, p = a * b, f = fma(a, b, c);
    std::printf("%a %a %a %a %a %a\n", s.hi, s.lo, p.hi, p.lo, f.hi, f.lo);
  }
  return 0;
}
