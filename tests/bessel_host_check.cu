// Host build of the library's Bessel routines (bessel.cuh is host-and-device code) for the CPU test
// tests/test_bessel_host.py.  Reads x values (one per line) from stdin and prints, per x, the double-float
// path the assembly kernels use (J0, Y0, J1, Y1 as hi + lo), the FP64 path (self terms, near field) and the
// FP64 routines that build the Taylor table, and the double-float path with the argument split into an FP64
// base and a double-float offset, in hexadecimal floating point so that no digits are lost.  No
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
    // the assembly's form of the argument: an FP64 base plus a double-float offset whose sum is exactly x: for
    // x >= 2 a base about 3/64 below and one about 3/16 above x (base and node on different table grid points);
    // below 2, where the offset of neighbouring elements is comparable to x itself, x/2 and 2x.  The offset is
    // x - base, exact in FP64 (Sterbenz) and held exactly in double-float.
    bem::Bessel01F2 s1, s2;
    {
      bem::BesselArg a;
      const bool small = x < 2.0;
      const double b1 = small ? 0.5 * x : x - 0.046875, b2 = small ? 2.0 * x : x + 0.1875;
      bem::bessel_arg_base(b1, a);
      bem::bessel01_f2_at(a, bem::f2_from(x - b1), bem::f2_from(x), s1);
      bem::bessel_arg_base(b2, a);
      bem::bessel01_f2_at(a, bem::f2_from(x - b2), bem::f2_from(x), s2);
    }
    std::printf("%a %a %a %a %a %a %a %a %a %a %a %a %a %a %a %a %a %a %a %a %a\n", x, bem::f2_to(f.j0),
                bem::f2_to(f.y0), bem::f2_to(f.j1), bem::f2_to(f.y1), d.j0, d.y0, d.j1, d.y1, t.j0, t.y0, t.j1, t.y1,
                bem::f2_to(s1.j0), bem::f2_to(s1.y0), bem::f2_to(s1.j1), bem::f2_to(s1.y1), bem::f2_to(s2.j0),
                bem::f2_to(s2.y0), bem::f2_to(s2.j1), bem::f2_to(s2.y1));
  }
  return 0;
}
