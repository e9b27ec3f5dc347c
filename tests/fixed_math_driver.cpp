// Host driver for tests/test_fixed_math.py: reads cases from stdin and prints
// the fixed-point helpers' results (the same header the CUDA kernels use).
//   mode s: "x k"          -> fx_scale_round(x, k)
//   mode e: "y"            -> fx_exponent(y)
//   mode p: "q"            -> fx_split29(q): hi lo
//   mode r: "a0 a1 a2 a3 e" -> fx_round(a, e) as a hex float
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "fx_math.h"

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const char mode = argv[1][0];
  if (mode == 's') {
    double x;
    int k;
    while (scanf("%la %d", &x, &k) == 2) printf("%lld\n", (long long)irkmg::fx_scale_round(x, k));
  } else if (mode == 'e') {
    double y;
    while (scanf("%la", &y) == 1) printf("%d\n", irkmg::fx_exponent(y));
  } else if (mode == 'p') {
    long long q;
    while (scanf("%lld", &q) == 1) {
      int32_t hi, lo;
      irkmg::fx_split29((int64_t)q, &hi, &lo);
      printf("%d %d\n", hi, lo);
    }
  } else if (mode == 'r') {
    long long a[4];
    int e;
    while (scanf("%lld %lld %lld %lld %d", &a[0], &a[1], &a[2], &a[3], &e) == 5) {
      const int64_t b[4] = {a[0], a[1], a[2], a[3]};
      printf("%a\n", irkmg::fx_round(b, e));
    }
  } else {
    return 2;
  }
  return 0;
}
