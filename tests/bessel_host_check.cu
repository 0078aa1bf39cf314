// Host build of the library's Bessel routines (bessel.cuh is host-and-device code) for the CPU test
// tests/test_bessel_host.py.  Reads x values (one per line) from stdin and prints, per x, the double-float
// path the assembly kernels use (J0, Y0, J1, Y1 as hi + lo), the FP64 path (self terms, near field) and the
// FP64 routines that build the Taylor table, in hexadecimal floating point so that no digits are lost.  No
// CUDA call is made.
#include <cstdio>

#include "bessel.cuh"

int main() {
  double x;
  while (std::scanf("%lf", &x) == 1) {
    bem::Bessel01F2 f;
    bem::bessel01_f2(x, bem::f2_from(x), f);
    bem::Bessel01 d;
    bem::bessel01(x, d);
    // the FP64 routines the host uses to build the Taylor table (series below 2, as everywhere)
    bem::Bessel01 t;
    if (x < bem::BEM_X_SERIES) bem::bessel01_series(x, t);
    else if (x < bem::BEM_X_ASYMP) bem::bessel01_miller(x, t);
    else bem::bessel01_asymp(x, t);
    std::printf("%a %a %a %a %a %a %a %a %a %a %a %a %a\n", x, bem::f2_to(f.j0), bem::f2_to(f.y0),
                bem::f2_to(f.j1), bem::f2_to(f.y1), d.j0, d.y0, d.j1, d.y1, t.j0, t.y0, t.j1, t.y1);
  }
  return 0;
}
