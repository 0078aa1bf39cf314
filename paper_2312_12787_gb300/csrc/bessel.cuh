// Bessel functions J0, J1, Y0, Y1 of real positive argument, giving the Hankel functions
// H0^(1) = J0 + i Y0 and H1^(1) = J1 + i Y1 that make up the kernels of the single-, double-, adjoint
// double- and hypersingular operators (paper Sec. 3.3, eq. fundamental_sol: G = (i/4) H0^(1)(k r)).
//
// Written from the published mathematics (NIST DLMF), not from any library's internals:
//   * x < BEM_X_SERIES:   ascending power series, DLMF 10.2.2 (J_n) and 10.8.1 (Y_n, n = 0, 1).  (The
//                         double-float path of the kernels takes the series only below 1 and Taylor steps from a
//                         table on 1 <= x < 128, below.)
//   * x < BEM_X_ASYMP:    Miller's backward recurrence for J_n (DLMF 3.6(vi), 10.74(iv)), normalised by
//                         1 = J0 + 2 sum J_2k (DLMF 10.12.4), and the Neumann expansions
//                         Y0 = (2/pi)(ln(x/2)+gamma) J0 - (4/pi) sum_k (-1)^k J_2k / k  (a Neumann expansion, DLMF 10.23(ii))
//                         Y1 = -Y0' = (2/pi)[(ln(x/2)+gamma) J1 - J0/x]
//                              + (2/pi) sum_k (-1)^k (J_{2k-1} - J_{2k+1}) / k.
//   * otherwise:          Hankel's asymptotic expansion, DLMF 10.17.5 with a_k(nu) from 10.17.1.
// Double precision throughout; the accuracy target is ~1e-15 relative to |H|.
#pragma once

#include <cstring>
#include <vector>

#if defined(__CUDACC__)
#define BEM_HD __host__ __device__ __forceinline__
#else
#define BEM_HD inline
#include <cmath>
#endif

namespace bem {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double kTwoOverPi = 0.636619772367581343075535053490057448;
constexpr double kEulerGamma = 0.577215664901532860606512090082402431;
constexpr double kInvSqrt2 = 0.707106781186547524400844362104849039;

constexpr double BEM_X_SERIES = 2.0;   // below: ascending series
constexpr double BEM_X_ASYMP = 18.0;   // at and above: Hankel asymptotic expansion
constexpr int BEM_MILLER_START = 56;   // fixed (even) starting order of the backward recurrence
constexpr int BEM_ASYMP_TERMS = 22;    // terms k = 0 .. BEM_ASYMP_TERMS-1 of DLMF 10.17.5

struct Bessel01 {
  double j0, y0, j1, y1;
};

// a_k(nu) of DLMF 10.17.1: a_0 = 1, a_k = a_{k-1} (4 nu^2 - (2k-1)^2) / (8k), for nu = 0 and nu = 1,
// multiplied by i^k and split into the real (even k) and imaginary (odd k) parts of sum i^k a_k x^-k.
struct AsympCoef {
  double p0[BEM_ASYMP_TERMS], q0[BEM_ASYMP_TERMS], p1[BEM_ASYMP_TERMS], q1[BEM_ASYMP_TERMS];
};
constexpr AsympCoef make_asymp_coef() {
  AsympCoef c{};
  double a0 = 1.0, a1 = 1.0;
  for (int k = 0; k < BEM_ASYMP_TERMS; ++k) {
    if (k > 0) {
      const double m = 2.0 * k - 1.0;
      a0 = a0 * (-(m * m)) / (8.0 * k);
      a1 = a1 * (4.0 - m * m) / (8.0 * k);
    }
    const int r = k & 3;   // i^k = 1, i, -1, -i
    c.p0[k] = r == 0 ? a0 : (r == 2 ? -a0 : 0.0);
    c.q0[k] = r == 1 ? a0 : (r == 3 ? -a0 : 0.0);
    c.p1[k] = r == 0 ? a1 : (r == 2 ? -a1 : 0.0);
    c.q1[k] = r == 1 ? a1 : (r == 3 ? -a1 : 0.0);
  }
  return c;
}

BEM_HD void bessel01_series(double x, Bessel01& b) {
  const double t = 0.25 * x * x;
  double e0 = 1.0;          // (-t)^m / (m!)^2
  double e1 = 1.0;          // (-t)^m / (m! (m+1)!)
  double sj0 = 1.0, sj1 = 1.0;
  double hm = 0.0;          // harmonic number H_m
  double sy0 = 0.0;         // sum_{m>=1} -(-t)^m H_m / (m!)^2
  double sy1 = 1.0;         // sum_{m>=0} (H_m + H_{m+1}) (-t)^m / (m!(m+1)!), m = 0 term is H_1 = 1
  for (int m = 1; m < 40; ++m) {
    const double dm = (double)m;
    e0 *= -t / (dm * dm);
    e1 *= -t / (dm * (dm + 1.0));
    const double hm1 = hm + 1.0 / dm;           // H_m
    const double hm2 = hm1 + 1.0 / (dm + 1.0);  // H_{m+1}
    sj0 += e0;
    sj1 += e1;
    sy0 -= e0 * hm1;
    sy1 += e1 * (hm1 + hm2);
    hm = hm1;
    if (fabs(e0) * (hm2 + 1.0) < 1e-18 * fabs(sj0) && fabs(e1) * (hm2 + 1.0) < 1e-18 * fabs(sj1)) break;
  }
  const double lg = log(0.5 * x) + kEulerGamma;
  b.j0 = sj0;
  b.j1 = 0.5 * x * sj1;
  b.y0 = kTwoOverPi * (lg * b.j0 + sy0);
  b.y1 = -kTwoOverPi / x + kTwoOverPi * lg * b.j1 - (0.5 * x / kPi) * sy1;
}

// Valid for BEM_X_SERIES <= x < BEM_X_ASYMP: the fixed start order keeps f_n within range there.
BEM_HD void bessel01_miller(double x, Bessel01& b) {
  const double two_over_x = 2.0 / x;
  double fp = 0.0;        // f_{n+1}
  double f = 1e-200;      // f_n, n = BEM_MILLER_START
  double norm = 0.0;      // sum over even n >= 2 of f_n
  double sy0 = 0.0;       // sum_k (-1)^k f_{2k}/k
  double sy1 = 0.0;       // sum_k (-1)^k (f_{2k-1} - f_{2k+1})/k
  double f_odd_above = 0.0;
#pragma unroll
  for (int n = BEM_MILLER_START; n >= 1; --n) {
    if ((n & 1) == 0) {
      const int kk = n >> 1;
      const double c = ((kk & 1) ? -1.0 : 1.0) / (double)kk;
      norm += f;
      sy0 += c * f;
      f_odd_above = fp;
    } else {
      const int kk = (n + 1) >> 1;
      const double c = ((kk & 1) ? -1.0 : 1.0) / (double)kk;
      sy1 += c * (f - f_odd_above);
    }
    const double fm = ((double)n * two_over_x) * f - fp;   // f_{n-1}
    fp = f;
    f = fm;
  }
  const double s = 1.0 / (f + 2.0 * norm);
  const double j0 = f * s, j1 = fp * s;
  const double lg = log(0.5 * x) + kEulerGamma;
  b.j0 = j0;
  b.j1 = j1;
  b.y0 = kTwoOverPi * (lg * j0) - 2.0 * kTwoOverPi * sy0 * s;
  b.y1 = kTwoOverPi * (lg * j1 - j0 / x) + kTwoOverPi * sy1 * s;
}

// ---- double-float arithmetic (a value is hi + lo, two FP32 numbers; ~48-bit significand) ----------
// Error-free transformations of Knuth (two-sum), Dekker (fast two-sum) and the FMA-based exact product.
// GB300 executes FP32 at many times its FP64 rate, so recurrences that need more than FP32 accuracy run
// faster in this form than in native FP64.
struct F2 {
  float h, l;
};
BEM_HD F2 f2_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return F2{s, (a - (s - bb)) + (b - bb)};
}
BEM_HD F2 f2_fast_two_sum(float a, float b) {   // requires |a| >= |b| or a == 0
  const float s = a + b;
  return F2{s, b - (s - a)};
}
BEM_HD F2 f2_add(F2 a, F2 b) {
  const F2 s = f2_two_sum(a.h, b.h);
  return f2_fast_two_sum(s.h, s.l + (a.l + b.l));
}
BEM_HD F2 f2_neg(F2 a) { return F2{-a.h, -a.l}; }
BEM_HD F2 f2_mul(F2 a, F2 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return f2_fast_two_sum(p, e);
}
BEM_HD F2 f2_mulf(F2 a, float b) {
  const float p = a.h * b;
  const float e = fmaf(a.l, b, fmaf(a.h, b, -p));
  return f2_fast_two_sum(p, e);
}
BEM_HD F2 f2_from(double d) {
  const float h = (float)d;
  return F2{h, (float)(d - (double)h)};
}
BEM_HD double f2_to(F2 a) { return (double)a.h + (double)a.l; }

// The split of f2_from done with integer operations only: hi = d truncated to a float's 24 significant bits,
// lo = the remaining 29 mantissa bits rounded to a float (|d - hi - lo| <= 2^-47 |d|).  On GB300 the
// conversions of f2_from run on the FP64 pipe; this form keeps them off it.  For |d| < 2^-126 the result is
// (0, 0) and for |d| < 2^-74 lo is 0 (an absolute error below 2^-97); |d| must be below 2^128.
BEM_HD F2 f2_from_bits(double d) {
#if defined(__CUDA_ARCH__)
  const unsigned hi32 = (unsigned)__double2hiint(d), lo32 = (unsigned)__double2loint(d);
#else
  unsigned long long b;
  memcpy(&b, &d, sizeof b);
  const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
#endif
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  if (e < 897) return F2{0.f, 0.f};
  const unsigned sign = hi32 & 0x80000000u;
  const unsigned hb = sign | ((unsigned)(e - 896) << 23) | ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
  const unsigned sb = e >= 949 ? (sign | ((unsigned)(e - 948) << 23)) : sign;   // +-2^(e-1075), or +-0
  const float rem = (float)(lo32 & 0x1fffffffu);
#if defined(__CUDA_ARCH__)
  return F2{__uint_as_float(hb), rem * __uint_as_float(sb)};
#else
  float hf, sf;
  memcpy(&hf, &hb, sizeof hf);
  memcpy(&sf, &sb, sizeof sf);
  return F2{hf, rem * sf};
#endif
}

// +-1/k for the Neumann sums, as double-float constants folded at compile time
struct MillerCoefF2 {
  float h[BEM_MILLER_START / 2 + 1], l[BEM_MILLER_START / 2 + 1];
};
constexpr MillerCoefF2 make_miller_coef_f2() {
  MillerCoefF2 c{};
  for (int k = 1; k <= BEM_MILLER_START / 2; ++k) {
    const double v = ((k & 1) ? -1.0 : 1.0) / (double)k;
    const float h = (float)v;
    c.h[k] = h;
    c.l[k] = (float)(v - (double)h);
  }
  return c;
}

// Miller's algorithm exactly as bessel01_miller, with the recurrence and the three sums in double-float
// arithmetic on the FP32 pipe (start value 2^-30, rescaled by 2^-40 whenever it grows past 2^40 so that it
// stays inside the FP32 exponent range); the normalisation and the logarithmic terms are FP64.
BEM_HD void bessel01_miller_f2(double x, Bessel01& b) {
  constexpr MillerCoefF2 C = make_miller_coef_f2();
  const double tox_d = 2.0 / x;
  const F2 tox = f2_from(tox_d);
  F2 fp{0.f, 0.f}, f{0x1p-30f, 0.f}, norm{0.f, 0.f}, sy0{0.f, 0.f}, sy1{0.f, 0.f}, fodd{0.f, 0.f};
#pragma unroll
  for (int n = BEM_MILLER_START; n >= 1; --n) {
    if ((n & 1) == 0) {
      const int kk = n >> 1;
      norm = f2_add(norm, f);
      sy0 = f2_add(sy0, f2_mul(f, F2{C.h[kk], C.l[kk]}));
      fodd = fp;
    } else {
      const int kk = (n + 1) >> 1;
      sy1 = f2_add(sy1, f2_mul(f2_add(f, f2_neg(fodd)), F2{C.h[kk], C.l[kk]}));
    }
    const F2 cn = f2_mulf(tox, (float)n);
    const F2 fm = f2_add(f2_mul(cn, f), f2_neg(fp));
    fp = f;
    f = fm;
    if ((n & 3) == 1 && fabsf(f.h) > 0x1p40f) {
      const float sc = 0x1p-40f;
      f = F2{f.h * sc, f.l * sc}; fp = F2{fp.h * sc, fp.l * sc};
      norm = F2{norm.h * sc, norm.l * sc}; sy0 = F2{sy0.h * sc, sy0.l * sc};
      sy1 = F2{sy1.h * sc, sy1.l * sc}; fodd = F2{fodd.h * sc, fodd.l * sc};
    }
  }
  const double f0 = f2_to(f), f1 = f2_to(fp);
  const double s = 1.0 / (f0 + 2.0 * f2_to(norm));
  const double j0 = f0 * s, j1 = f1 * s;
  const double lg = log(0.5 * x) + kEulerGamma;
  b.j0 = j0;
  b.j1 = j1;
  b.y0 = kTwoOverPi * (lg * j0) - 2.0 * kTwoOverPi * f2_to(sy0) * s;
  b.y1 = kTwoOverPi * (lg * j1 - 0.5 * tox_d * j0) + kTwoOverPi * f2_to(sy1) * s;
}

BEM_HD void bessel01_asymp(double x, Bessel01& b) {
  constexpr AsympCoef C = make_asymp_coef();
  const double y = 1.0 / x;
  double p0 = 0.0, q0 = 0.0, p1 = 0.0, q1 = 0.0;
#pragma unroll
  for (int k = BEM_ASYMP_TERMS - 1; k >= 0; --k) {
    // Horner in y; the zero coefficients fold away
    p0 = C.p0[k] + y * p0; q0 = C.q0[k] + y * q0;
    p1 = C.p1[k] + y * p1; q1 = C.q1[k] + y * q1;
  }
  double sn, cs;
#if defined(__CUDA_ARCH__)
  sincos(x, &sn, &cs);
#else
  sn = sin(x); cs = cos(x);
#endif
  const double amp = sqrt(kTwoOverPi * y) * kInvSqrt2;
  // e^{i(x - pi/4)} = ((cos x + sin x) + i (sin x - cos x)) / sqrt 2
  const double er = (cs + sn) * amp, ei = (sn - cs) * amp;
  // H0 = (p0 + i q0) e^{i(x - pi/4)};  H1 = (p1 + i q1) e^{i(x - 3pi/4)} = -i (p1 + i q1) e^{i(x - pi/4)}
  b.j0 = p0 * er - q0 * ei;
  b.y0 = p0 * ei + q0 * er;
  const double hr = p1 * er - q1 * ei, hi = p1 * ei + q1 * er;
  b.j1 = hi;
  b.y1 = -hr;
}

// The expansion's P0, Q0, P1, Q1 as polynomials in u = 1/x^2 (Horner in u halves the multiply-adds).
struct AsympCoefU {
  double p0[BEM_ASYMP_TERMS / 2], q0[BEM_ASYMP_TERMS / 2], p1[BEM_ASYMP_TERMS / 2], q1[BEM_ASYMP_TERMS / 2];
};
constexpr AsympCoefU make_asymp_coef_u() {
  AsympCoef c = make_asymp_coef();
  AsympCoefU u{};
  for (int m = 0; m < BEM_ASYMP_TERMS / 2; ++m) {
    u.p0[m] = c.p0[2 * m];
    u.p1[m] = c.p1[2 * m];
    u.q0[m] = c.q0[2 * m + 1];
    u.q1[m] = c.q1[2 * m + 1];
  }
  return u;
}

// ---- the expansion evaluated in double-float ------------------------------------------------------
// Hankel's expansion (DLMF 10.17.5) with each of P0, Q0, P1, Q1 written as a polynomial in u = 1/x^2,
// arranged so that almost all of the arithmetic runs on the FP32 pipe: cos x and sin x come from a
// Cody-Waite reduction of x by pi/2 in FP64 (three-part split of pi/2; exact for x < 2^20) followed by
// Taylor series of the reduced argument |r| <= pi/4 in double-float (terms through r^17 and r^18); P0, Q0,
// P1, Q1 are Horner sums in u = 1/x^2 with double-float coefficients; the final products too.  Only the reduction, the reciprocal square root and the
// conversions stay in FP64.
struct F2Coef {
  float h[BEM_ASYMP_TERMS / 2], l[BEM_ASYMP_TERMS / 2];
};
struct AsympCoefF2 {
  F2Coef p0, q0, p1, q1;
  float sh[9], sl[9];    // (-1)^k / (2k+1)!, k = 0..8
  float ch[10], cl[10];  // (-1)^k / (2k)!,   k = 0..9
};
constexpr void f2_split(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}
constexpr AsympCoefF2 make_asymp_coef_f2() {
  AsympCoefU u = make_asymp_coef_u();
  AsympCoefF2 c{};
  for (int m = 0; m < BEM_ASYMP_TERMS / 2; ++m) {
    f2_split(u.p0[m], c.p0.h[m], c.p0.l[m]);
    f2_split(u.q0[m], c.q0.h[m], c.q0.l[m]);
    f2_split(u.p1[m], c.p1.h[m], c.p1.l[m]);
    f2_split(u.q1[m], c.q1.h[m], c.q1.l[m]);
  }
  double f = 1.0;   // (2k+1)! running
  for (int k = 0; k < 9; ++k) {
    if (k > 0) f *= (2.0 * k) * (2.0 * k + 1.0);
    f2_split(((k & 1) ? -1.0 : 1.0) / f, c.sh[k], c.sl[k]);
  }
  f = 1.0;          // (2k)! running
  for (int k = 0; k < 10; ++k) {
    if (k > 0) f *= (2.0 * k - 1.0) * (2.0 * k);
    f2_split(((k & 1) ? -1.0 : 1.0) / f, c.ch[k], c.cl[k]);
  }
  return c;
}

// Horner sum of the first T coefficients (T <= BEM_ASYMP_TERMS / 2)
template <int T = BEM_ASYMP_TERMS / 2>
BEM_HD F2 f2_horner(const F2Coef& c, F2 u) {
  F2 acc{c.h[T - 1], c.l[T - 1]};
#pragma unroll
  for (int m = T - 2; m >= 0; --m) acc = f2_add(f2_mul(acc, u), F2{c.h[m], c.l[m]});
  return acc;
}

BEM_HD void bessel01_asymp_f2(double x, Bessel01& b) {
  constexpr AsympCoefF2 C = make_asymp_coef_f2();
  constexpr double kPio2_1 = 0x1.921fb54400000p+0;    // pi/2 = kPio2_1 + kPio2_2 + kPio2_3 + O(1e-37)
  constexpr double kPio2_2 = 0x1.0b4611a600000p-34;
  constexpr double kPio2_3 = 0x1.3198a2e037073p-69;
#if defined(__CUDA_ARCH__)
  const double rs = rsqrt(x);
#else
  const double rs = 1.0 / sqrt(x);
#endif
  const double y = rs * rs;
  // argument reduction x = kq pi/2 + r, |r| <= pi/4
  const double kq = rint(x * kTwoOverPi);
  double r = fma(-kq, kPio2_1, x);
  r = fma(-kq, kPio2_2, r);
  r = fma(-kq, kPio2_3, r);
  const int quad = (int)((long long)kq & 3);
  const F2 R = f2_from(r);
  const F2 R2 = f2_mul(R, R);
  F2 sp{C.sh[8], C.sl[8]};
#pragma unroll
  for (int k = 7; k >= 0; --k) sp = f2_add(f2_mul(sp, R2), F2{C.sh[k], C.sl[k]});
  const F2 sr = f2_mul(sp, R);
  F2 cr{C.ch[9], C.cl[9]};
#pragma unroll
  for (int k = 8; k >= 0; --k) cr = f2_add(f2_mul(cr, R2), F2{C.ch[k], C.cl[k]});
  // rotate by quad * pi/2: (sin x, cos x)
  F2 sn, cs;
  if (quad == 0) { sn = sr; cs = cr; }
  else if (quad == 1) { sn = cr; cs = f2_neg(sr); }
  else if (quad == 2) { sn = f2_neg(sr); cs = f2_neg(cr); }
  else { sn = f2_neg(cr); cs = sr; }
  // asymptotic sums
  const F2 U = f2_from(y * y);
  const F2 Y = f2_from(y);
  const F2 p0 = f2_horner(C.p0, U), p1 = f2_horner(C.p1, U);
  const F2 q0 = f2_mul(f2_horner(C.q0, U), Y), q1 = f2_mul(f2_horner(C.q1, U), Y);
  // e^{i(x - pi/4)} sqrt(2/(pi x)) = (cos x + sin x, sin x - cos x) * rs / sqrt(pi)
  const F2 A = f2_from(rs * 0.564189583547756286948079451560772586);   // 1/sqrt(pi)
  const F2 er = f2_mul(f2_add(cs, sn), A), ei = f2_mul(f2_add(sn, f2_neg(cs)), A);
  b.j0 = f2_to(f2_add(f2_mul(p0, er), f2_neg(f2_mul(q0, ei))));
  b.y0 = f2_to(f2_add(f2_mul(p0, ei), f2_mul(q0, er)));
  b.j1 = f2_to(f2_add(f2_mul(p1, ei), f2_mul(q1, er)));
  b.y1 = -f2_to(f2_add(f2_mul(p1, er), f2_neg(f2_mul(q1, ei))));
}

BEM_HD void bessel01(double x, Bessel01& b) {
  if (x < BEM_X_SERIES) bessel01_series(x, b);
  else if (x < BEM_X_ASYMP) bessel01_miller_f2(x, b);
  else bessel01_asymp_f2(x, b);
}

// ---- results in double-float ----------------------------------------------------------------------
// The assembly accumulates its Gauss sums in double-float, so the three branches below hand their results
// over in that form and skip the conversions back to FP64.  x (FP64) selects the branch and, in the
// expansion, fixes the phase (the reduction of x by pi/2 needs all of FP64's bits when k r reaches ~100);
// X = x in double-float carries everything that only needs relative accuracy (amplitudes, 1/x).
struct Bessel01F2 {
  F2 j0, y0, j1, y1;
};

BEM_HD F2 f2_sub(F2 a, F2 b) { return f2_add(a, f2_neg(b)); }
BEM_HD F2 f2_pow2(F2 a, float s) { return F2{a.h * s, a.l * s}; }   // s a power of two: exact

BEM_HD float f32_rsqrt_seed(float v) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(v);
#else
  return 1.0f / sqrtf(v);
#endif
}
BEM_HD float f32_rcp_seed(float v) {
#if defined(__CUDA_ARCH__)
  return __frcp_rn(v);
#else
  return 1.0f / v;
#endif
}
// a / b for b != 0: the FP32 quotient of the leading parts, corrected once by the double-float remainder
// a - b q (a Newton step on the quotient; relative error ~2^-46).
BEM_HD F2 f2_div(F2 a, F2 b) {
  const float y = f32_rcp_seed(b.h);
  const float q1 = a.h * y;
  const F2 rem = f2_sub(a, f2_mulf(b, q1));
  const float q2 = rem.h * y;
  return f2_fast_two_sum(q1, q2);
}

// 1/sqrt(a), a > 0: an FP32 estimate refined by two Newton steps y <- y + y (1 - a y^2) / 2 in double-float
// (each step squares the relative error: ~1e-7 -> ~1e-14 -> double-float rounding).
BEM_HD F2 f2_rsqrt(F2 a) {
  F2 y{f32_rsqrt_seed(a.h), 0.f};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const F2 e = f2_sub(F2{1.f, 0.f}, f2_mul(a, f2_mul(y, y)));
    y = f2_add(y, f2_mul(y, f2_pow2(e, 0.5f)));
  }
  return y;
}

// Coefficient tables of the ascending series (DLMF 10.2.2, 10.8.1): 1/m^2, 1/(m(m+1)) and the harmonic
// numbers H_m, so that the loop multiplies instead of dividing.
constexpr int kSeriesTerms = 14;   // x < 2: t = x^2/4 < 1, so the last term t^13/(13!)^2 < 3e-20
struct SeriesCoef {
  double inv_mm[kSeriesTerms], inv_mm1[kSeriesTerms], hm[kSeriesTerms + 1];
};
constexpr SeriesCoef make_series_coef() {
  SeriesCoef c{};
  c.hm[0] = 0.0;
  for (int m = 1; m < kSeriesTerms; ++m) {
    c.inv_mm[m] = 1.0 / ((double)m * (double)m);
    c.inv_mm1[m] = 1.0 / ((double)m * (double)(m + 1));
  }
  for (int m = 1; m <= kSeriesTerms; ++m) c.hm[m] = c.hm[m - 1] + 1.0 / (double)m;
  return c;
}

// The ascending series of bessel01_series with tabulated coefficients, in FP64, converted to double-float (only
// for the arguments below the table: a few neighbouring elements of each collocation point).
// The double-float path takes the series only below kTabXMin = 1/4 (the table serves 1/4 <= x < 128):
// t = x^2/4 <= 1/64, so terms m = 0 .. 6 suffice (the first one left out, t^7/(7!)^2 H_7, is below 2e-20).
constexpr int kSeriesTermsF2 = 7;
BEM_HD void bessel01_series_f2(double x, Bessel01F2& b) {
  constexpr SeriesCoef C = make_series_coef();
  const double t = 0.25 * x * x;
  double e0 = 1.0, e1 = 1.0, sj0 = 1.0, sj1 = 1.0, sy0 = 0.0, sy1 = 1.0;
#pragma unroll   // a fixed count: constant indices make the coefficients immediates (no table in memory)
  for (int m = 1; m < kSeriesTermsF2; ++m) {
    e0 *= -t * C.inv_mm[m];
    e1 *= -t * C.inv_mm1[m];
    sj0 += e0;
    sj1 += e1;
    sy0 -= e0 * C.hm[m];
    sy1 += e1 * (C.hm[m] + C.hm[m + 1]);
  }
  const double lg = log(0.5 * x) + kEulerGamma;
  const double j1 = 0.5 * x * sj1;
  b.j0 = f2_from(sj0);
  b.j1 = f2_from(j1);
  b.y0 = f2_from(kTwoOverPi * (lg * sj0 + sy0));
  b.y1 = f2_from(-kTwoOverPi / x + kTwoOverPi * lg * j1 - (0.5 * x / kPi) * sy1);
}

constexpr F2 f2_const(double v) { return F2{(float)v, (float)(v - (double)(float)v)}; }

// The expansion's coefficients for a rolled Horner loop: which = 0..3 selects P0, Q0, P1, Q1 (constant memory
// on the device: the index is uniform over a warp, so reads are broadcasts; a constexpr table on the host).
#if defined(__CUDACC__)
static __constant__ AsympCoefF2 kAsympCoefDev = make_asymp_coef_f2();
#endif
static constexpr AsympCoefF2 kAsympCoefHost = make_asymp_coef_f2();
#if defined(__CUDA_ARCH__)
#define BEM_ASYMP_TAB kAsympCoefDev
#else
#define BEM_ASYMP_TAB kAsympCoefHost
#endif
BEM_HD F2 bem_asymp_coef(int which, int m) {
  switch (which) {
    case 0: return F2{BEM_ASYMP_TAB.p0.h[m], BEM_ASYMP_TAB.p0.l[m]};
    case 1: return F2{BEM_ASYMP_TAB.q0.h[m], BEM_ASYMP_TAB.q0.l[m]};
    case 2: return F2{BEM_ASYMP_TAB.p1.h[m], BEM_ASYMP_TAB.p1.l[m]};
    default: return F2{BEM_ASYMP_TAB.q1.h[m], BEM_ASYMP_TAB.q1.l[m]};
  }
}
#undef BEM_ASYMP_TAB

// Hankel's expansion as bessel01_asymp_f2, with 1/sqrt(x) and 1/x from X in double-float, given the phase
// reduced by pi/2: x = quad pi/2 + R (mod 2 pi), |R| <= pi/4 (up to ~0.9 the sine and cosine sums below keep
// their accuracy).
BEM_HD void bessel01_asymp_f2r(F2 X, F2 R, int quad, Bessel01F2& b) {
  constexpr AsympCoefF2 C = make_asymp_coef_f2();
  const F2 rs = f2_rsqrt(X);
  const F2 Y = f2_mul(rs, rs);
  const F2 U = f2_mul(Y, Y);
  const F2 R2 = f2_mul(R, R);
  F2 sp{C.sh[8], C.sl[8]};
#pragma unroll
  for (int k = 7; k >= 0; --k) sp = f2_add(f2_mul(sp, R2), F2{C.sh[k], C.sl[k]});
  const F2 sr = f2_mul(sp, R);
  F2 cr{C.ch[9], C.cl[9]};
#pragma unroll
  for (int k = 8; k >= 0; --k) cr = f2_add(f2_mul(cr, R2), F2{C.ch[k], C.cl[k]});
  F2 sn, cs;
  if (quad == 0) { sn = sr; cs = cr; }
  else if (quad == 1) { sn = cr; cs = f2_neg(sr); }
  else if (quad == 2) { sn = f2_neg(sr); cs = f2_neg(cr); }
  else { sn = f2_neg(cr); cs = sr; }
  // terms of the expansion: 22 below x = 25, 16 up to 35, 12 beyond (each keeps the truncation below
  // 1e-15 of |H|); the tier is the one the smallest x of the warp's active lanes needs
  float xmin = X.h;
#if defined(__CUDA_ARCH__)
  xmin = __int_as_float(__reduce_min_sync(__activemask(), __float_as_int(xmin)));   // x > 0: int order = float order
#endif
  const int T = xmin >= 35.f ? 6 : (xmin >= 25.f ? 8 : BEM_ASYMP_TERMS / 2);
  F2 p0 = bem_asymp_coef(0, T - 1), q0 = bem_asymp_coef(1, T - 1);
  F2 p1 = bem_asymp_coef(2, T - 1), q1 = bem_asymp_coef(3, T - 1);
#pragma unroll 1
  for (int m = T - 2; m >= 0; --m) {   // four independent Horner sums in u = 1/x^2
    p0 = f2_add(f2_mul(p0, U), bem_asymp_coef(0, m));
    q0 = f2_add(f2_mul(q0, U), bem_asymp_coef(1, m));
    p1 = f2_add(f2_mul(p1, U), bem_asymp_coef(2, m));
    q1 = f2_add(f2_mul(q1, U), bem_asymp_coef(3, m));
  }
  q0 = f2_mul(q0, Y);
  q1 = f2_mul(q1, Y);
  constexpr F2 kInvSqrtPi = f2_const(0.564189583547756286948079451560772586);
  const F2 A = f2_mul(rs, kInvSqrtPi);
  const F2 er = f2_mul(f2_add(cs, sn), A), ei = f2_mul(f2_sub(sn, cs), A);
  b.j0 = f2_sub(f2_mul(p0, er), f2_mul(q0, ei));
  b.y0 = f2_add(f2_mul(p0, ei), f2_mul(q0, er));
  b.j1 = f2_add(f2_mul(p1, ei), f2_mul(q1, er));
  b.y1 = f2_neg(f2_sub(f2_mul(p1, er), f2_mul(q1, ei)));
}

// pi/2 = kPio2_1 + kPio2_2 + kPio2_3 + O(1e-37) (three-part split for Cody-Waite reduction in FP64)
constexpr double kPio2_1 = 0x1.921fb54400000p+0;
constexpr double kPio2_2 = 0x1.0b4611a600000p-34;
constexpr double kPio2_3 = 0x1.3198a2e037073p-69;

// x = quad pi/2 + r with |r| <= pi/4 for 0 < x < 2^50 (Cody-Waite: kq = x 2/pi rounded to an integer by adding
// 1.5 * 2^52, which leaves it in the low bits of t).
BEM_HD double reduce_pio2(double x, int& quad) {
  const double t = fma(x, kTwoOverPi, 0x1.8p52);
  const double kq = t - 0x1.8p52;
  double r = fma(-kq, kPio2_1, x);
  r = fma(-kq, kPio2_2, r);
  r = fma(-kq, kPio2_3, r);
#if defined(__CUDA_ARCH__)
  quad = __double2loint(t) & 3;
#else
  unsigned long long tb;
  memcpy(&tb, &t, sizeof tb);
  quad = (int)(tb & 3u);
#endif
  return r;
}

// Hankel's expansion with the phase reduced from the FP64 argument x.
BEM_HD void bessel01_asymp_f2x(double x, F2 X, Bessel01F2& b) {
  int quad;
  const double r = reduce_pio2(x, quad);
  bessel01_asymp_f2r(X, f2_from_bits(r), quad, b);
}

// ---- tabulated values and Taylor steps on 1/4 <= x < 128 -----------------------------------------------
// J0, Y0, J1, Y1 at the grid points (computed once on the host with the FP64 routines above, error ~1e-15 of
// |H|), stored in double-float with 1/x_k: x = 1/4 + k/128 for entries k = 0 .. 95 and x = 1 + (k - 96)/32 from
// entry 96 on, so that every step |h| <= half a grid spacing keeps |h| / x <= 1/64.  All grid points are
// multiples of 1/128.  Between grid points both pairs obey the same first-order system
// Z0' = -Z1, Z1' = Z0 - Z1/x (DLMF 10.6.2), so with Z0(x_k + h) = sum a_n h^n and Z1(x_k + h) = sum b_n h^n the
// Taylor coefficients follow from
//   a_{n+1} = -b_n / (n+1),   b_{n+1} = (a_n - c_n) / (n+1),   c_n = (b_n - c_{n-1}) / x_k,
// where c_n are the coefficients of Z1/(x_k + h).  Eight orders leave a remainder below 1e-16 from x = 2 on and
// below ~4e-15 where |h| / x reaches 1/64 (the derivatives of Y_n grow like n!/x^n toward the origin:
// (h/x)^8 = 64^-8); orders 0-3 run in double-float, orders 4-7 (below 3e-9 of the value from x = 2 on, ~1e-7 at
// |h| / x = 1/64) in FP32.  This replaces the
// recurrence of Miller's algorithm (56 steps) and Hankel's expansion up to x = 128 by about a fifth of the
// arithmetic of the expansion (whose double-float sine, cosine and four Horner sums take ~1000 FP32 operations
// per evaluation); the table costs 128 bytes per grid point, read through the L1 cache (the lanes of a warp
// take neighbouring elements, so their arguments share a few grid points).
constexpr double kTabStep = 1.0 / 32.0;   // spacing from x = 1 on
constexpr double kTabX0 = 1.0;            // where the 1/32 spacing starts (entry kTabFine)
constexpr int kTabFine = 96;              // entries of the 1/128 spacing on [1/4, 1)
constexpr int kTabN = kTabFine + 4065;    // then x = 1 + k / 32, k = 0 .. 4064: [1, 128]
constexpr float kTabXMin = 0.25f;         // the table serves 1/4 <= x < 128 (532 KB of device memory); the series
constexpr float kTabXMax = 128.0f;        // below, Hankel's expansion above
// Grid point of entry k in units of 1/128 (an integer).
BEM_HD int tab_g128(int k) { return k < kTabFine ? 32 + k : 128 + 4 * (k - kTabFine); }
BEM_HD double tab_x(int k) { return (double)tab_g128(k) * (1.0 / 128.0); }
// One grid point x_k: for each pair (J0, J1) and (Y0, Y1) the Taylor coefficients of orders 0..3 of Z0 (a_n)
// and Z1 (b_n) as double-float (a_1 = -b_0 is not stored), c_3 (FP32, the start of the FP32 orders) and
// 1/x_k (FP32).  The coefficients depend on x_k only, so they are made once on the host in FP64.
struct alignas(16) BesselTabPair {
  float a0h, a0l, b0h, b0l;
  float b1h, b1l, a2h, a2l;
  float b2h, b2l, a3h, a3l;
  float b3h, b3l, c3, inv;   // inv = 1/x_k (both pairs)
};
struct alignas(16) BesselTabEntry {
  BesselTabPair j, y;   // 128 bytes: eight 16-byte loads
};

#if defined(__CUDACC__)
static __device__ BesselTabEntry g_bessel_tab[kTabN];
#endif

// Taylor coefficients at x of a solution pair of Z0' = -Z1, Z1' = Z0 - Z1/x (DLMF 10.6.2) with values z0, z1:
// with Z0 = sum a_n h^n, Z1 = sum b_n h^n and Z1/x = sum c_n h^n (x c_n + c_{n-1} = b_n),
// a_{n+1} = -b_n/(n+1), b_{n+1} = (a_n - c_n)/(n+1).
inline void taylor_coefs_host(double x, double z0, double z1, BesselTabPair& t) {
  auto put = [](double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
  };
  const double a0 = z0, b0 = z1, c0 = b0 / x;
  const double a1 = -b0, b1 = a0 - c0, c1 = (b1 - c0) / x;
  const double a2 = -b1 / 2, b2 = (a1 - c1) / 2, c2 = (b2 - c1) / x;
  const double a3 = -b2 / 3, b3 = (a2 - c2) / 3, c3 = (b3 - c2) / x;
  put(a0, t.a0h, t.a0l);
  put(b0, t.b0h, t.b0l);
  put(b1, t.b1h, t.b1l);
  put(a2, t.a2h, t.a2l);
  put(b2, t.b2h, t.b2l);
  put(a3, t.a3h, t.a3l);
  put(b3, t.b3h, t.b3l);
  t.c3 = (float)c3;
  t.inv = (float)(1.0 / x);
}

// Host copy of the table (built on first use, thread-safe).
inline const BesselTabEntry* bessel_tab_host() {
  static const std::vector<BesselTabEntry> tab = [] {
    std::vector<BesselTabEntry> t(kTabN);
    for (int k = 0; k < kTabN; ++k) {
      const double x = tab_x(k);
      Bessel01 b;
      if (x < BEM_X_SERIES) bessel01_series(x, b);
      else if (x < BEM_X_ASYMP) bessel01_miller(x, b);
      else bessel01_asymp(x, b);
      taylor_coefs_host(x, b.j0, b.j1, t[k].j);
      taylor_coefs_host(x, b.y0, b.y1, t[k].y);
    }
    return t;
  }();
  return tab.data();
}

// Taylor sums for one pair from the stored coefficients: orders 0..3 in double-float, orders 4..7 by the
// same recurrence in FP32 (their terms are below 2^-24 of the sum for |h| <= 1/64); H = h.
BEM_HD void taylor_pair(float4 q0, float4 q1, float4 q2, float4 q3, F2 H, F2& out0, F2& out1) {
  const F2 a0{q0.x, q0.y}, b0{q0.z, q0.w}, b1{q1.x, q1.y}, a2{q1.z, q1.w};
  const F2 b2{q2.x, q2.y}, a3{q2.z, q2.w}, b3{q3.x, q3.y};
  const F2 a1 = f2_neg(b0);
  const float c3 = q3.z, iv = q3.w, hf = H.h;
  float an = -b3.h * 0.25f, bn = (a3.h - c3) * 0.25f, cn = (bn - c3) * iv;
  float a[4], bq[4];
  a[0] = an; bq[0] = bn;
#pragma unroll
  for (int n = 4; n < 7; ++n) {
    const float r = 1.f / (float)(n + 1);
    const float an1 = -bn * r, bn1 = (an - cn) * r;
    an = an1; bn = bn1;
    cn = (bn - cn) * iv;
    a[n - 3] = an; bq[n - 3] = bn;
  }
  float pa = a[3], pb = bq[3];
#pragma unroll
  for (int n = 2; n >= 0; --n) {
    pa = fmaf(pa, hf, a[n]);
    pb = fmaf(pb, hf, bq[n]);
  }
  // double-float Horner over orders 3..0 with the FP32 tail
  F2 s0 = f2_add(a3, f2_mulf(H, pa));
  F2 s1 = f2_add(b3, f2_mulf(H, pb));
  s0 = f2_add(a2, f2_mul(s0, H));
  s1 = f2_add(b2, f2_mul(s1, H));
  s0 = f2_add(a1, f2_mul(s0, H));
  s1 = f2_add(b1, f2_mul(s1, H));
  out0 = f2_add(a0, f2_mul(s0, H));
  out1 = f2_add(b0, f2_mul(s1, H));
}

// Nearest grid entry of x (kTabXMin <= xh < kTabXMax).
BEM_HD int tab_index(float xh) {
#if defined(__CUDA_ARCH__)
  return xh < (float)kTabX0 ? __float2int_rn((xh - kTabXMin) * 128.f)
                            : kTabFine + __float2int_rn((xh - (float)kTabX0) * 32.f);
#else
  return xh < (float)kTabX0 ? (int)lrintf((xh - kTabXMin) * 128.f)
                            : kTabFine + (int)lrintf((xh - (float)kTabX0) * 32.f);
#endif
}

// The Taylor sums at x = x_k + H from grid point k (|H| <= 1/64 up to rounding).
BEM_HD void bessel01_taylor_f2h(int k, F2 H, Bessel01F2& b) {
#if defined(__CUDA_ARCH__)
  const float4* ep = reinterpret_cast<const float4*>(&g_bessel_tab[k]);
  const float4 e0 = __ldg(ep), e1 = __ldg(ep + 1), e2 = __ldg(ep + 2), e3 = __ldg(ep + 3);
  const float4 e4 = __ldg(ep + 4), e5 = __ldg(ep + 5), e6 = __ldg(ep + 6), e7 = __ldg(ep + 7);
#else
  const float4* ep = reinterpret_cast<const float4*>(&bessel_tab_host()[k]);
  const float4 e0 = ep[0], e1 = ep[1], e2 = ep[2], e3 = ep[3], e4 = ep[4], e5 = ep[5], e6 = ep[6], e7 = ep[7];
#endif
  taylor_pair(e0, e1, e2, e3, H, b.j0, b.j1);
  taylor_pair(e4, e5, e6, e7, H, b.y0, b.y1);
}

BEM_HD void bessel01_taylor_f2(double x, F2 X, Bessel01F2& b) {
  const int k = tab_index(X.h);
  const double h = x - tab_x(k);   // exact: x and the grid point agree to within 1/64 of x
  bessel01_taylor_f2h(k, f2_from_bits(h), b);
}

// ---- arguments given as an FP64 base plus a small double-float offset -----------------------------------
// The assembly evaluates x = k r at the Gauss nodes of element j as x = x_b + x_c: x_b = k |d| with d the
// vector from element j's centre to the collocation point (FP64, once per element pair), and x_c = k c_m with
// c_m = r_m - |d| (double-float, |c_m| <= h_j / 2).  The FP64 work (the table offset and the reduction by pi/2 of
// x_b) is then done once per pair; per node only x_c is added in double-float, with an absolute error of
// ~2^-46 |x_c|, so the argument keeps FP64's absolute accuracy.
struct BesselArg {
  double xb;   // x_b
  int kb;      // grid point of x_b: x_kb = 1 + kb / 32
  F2 hb;       // x_b - x_kb
  int qb;      // x_b = qb pi/2 + rb (mod 2 pi)
  F2 rb;
};

// asym = false: the caller knows that no argument x_b + x_c reaches Hankel's expansion (x >= kTabXMax), so the
// reduction by pi/2 (five FP64 operations) is skipped and rb, qb are zero.
BEM_HD void bessel_arg_base(double xb, BesselArg& a, bool asym = true) {
  a.xb = xb;
  // kb = (xb - 1) 32 rounded to an integer (magic-number rounding; |kb| < 2^31 for the arguments that occur)
  const double t = fma(xb - kTabX0, 32.0, 0x1.8p52);
  const double kd = t - 0x1.8p52;
#if defined(__CUDA_ARCH__)
  a.kb = __double2loint(t);
#else
  a.kb = (int)kd;
#endif
  a.hb = f2_from_bits(xb - fma(kd, kTabStep, kTabX0));   // exact: x_kb is a multiple of 1/32
  if (asym) {
    a.rb = f2_from_bits(reduce_pio2(xb, a.qb));
  } else {
    a.rb = F2{0.f, 0.f};
    a.qb = 0;
  }
}

// J0, Y0, J1, Y1 at x = a.xb + XC (XC small), X = x in double-float (branch choice and amplitudes).
BEM_HD void bessel01_f2_at(const BesselArg& a, F2 XC, F2 X, Bessel01F2& b) {
  if (X.h < kTabXMin) {
    bessel01_series_f2(a.xb + ((double)XC.h + (double)XC.l), b);
  } else if (X.h < kTabXMax) {
    // x - x_k = (x_b - x_kb) + x_c - (x_k - x_kb) (the last step by a two-sum: when the difference crosses a
    // power of two its rounding is not exact); x_k - x_kb is a multiple of 1/128, exact in FP32
    const int k = tab_index(X.h);
    const F2 Hp = f2_add(a.hb, XC);
    const float dk = (float)(tab_g128(k) - (128 + 4 * a.kb)) * (1.f / 128.f);
    const F2 t = f2_two_sum(Hp.h, -dk);
    const F2 H = f2_fast_two_sum(t.h, t.l + Hp.l);
    bessel01_taylor_f2h(k, H, b);
  } else {
    // the phase x_b reduced by pi/2 plus x_c, reduced once more if x_c carried it past pi/4
    F2 R = f2_add(a.rb, XC);
    int quad = a.qb;
    const float q = rintf(R.h * (float)kTwoOverPi);
    if (q != 0.f) {
      constexpr F2 kPio2F2{(float)kPio2_1, (float)(kPio2_1 - (double)(float)kPio2_1 + kPio2_2)};
      R = f2_sub(R, f2_mulf(kPio2F2, q));
      quad = (quad + (int)q) & 3;
    }
    bessel01_asymp_f2r(X, R, quad, b);
  }
}

BEM_HD void bessel01_f2(double x, F2 X, Bessel01F2& b) {
  if (X.h < kTabXMin) {
    bessel01_series_f2(x, b);
  } else if (X.h < kTabXMax) {
    bessel01_taylor_f2(x, X, b);
  } else {
    bessel01_asymp_f2x(x, X, b);
  }
}

// integral_0^x J0(t) dt and integral_0^x Y0(t) dt for the weakly singular self-element integral,
// by termwise integration of the ascending series DLMF 10.2.2 / 10.8.1 (x is small: x = k h / 2),
// with Y0 = (2/pi)(ln(t/2)+gamma) J0(t) + (2/pi) sum_{m>=1} (-1)^{m+1} H_m (t^2/4)^m/(m!)^2 and
//   int_0^x t^{2m} ln(t/2) dt = x^{2m+1}/(2m+1) (ln(x/2) - 1/(2m+1)).
// Only valid for moderate x; elements are always far below a wavelength in practice (x < ~10).
BEM_HD void int_j0_y0(double x, double& ij0, double& iy0) {
  const double t = 0.25 * x * x;
  double c = 1.0;             // (-t)^m/(m!)^2
  double hm = 0.0;
  const double lg = log(0.5 * x) + kEulerGamma;
  double sj = 0.0, sy = 0.0;
  for (int m = 0; m < 60; ++m) {
    const double dm = (double)m;
    if (m > 0) {
      c *= -t / (dm * dm);
      hm += 1.0 / dm;
    }
    const double inv = 1.0 / (2.0 * dm + 1.0);
    const double term_j = c * inv;                       // integral of c t^0 scaled: x * c/(2m+1)
    sj += term_j;
    // (2/pi) [ (ln(x/2)+gamma) c/(2m+1) - c/(2m+1)^2 ] - (2/pi) c H_m/(2m+1)
    sy += c * inv * (lg - inv - hm);
    if (m > 3 && fabs(c) * (hm + 2.0) < 1e-19 * (fabs(sj) + 1e-300)) break;
  }
  ij0 = x * sj;
  iy0 = kTwoOverPi * x * sy;
}

}  // namespace bem
