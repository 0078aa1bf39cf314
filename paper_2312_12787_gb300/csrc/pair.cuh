// The four matrix entries of one element pair (i, j): operators S, D, D*, N of Sec. 3.3 (eqs. stmp-ddtmp)
// with G = (i/4) H0^(1)(k r) (eq. fundamental_sol), constant elements collocated at their centres,
// Gauss-Legendre quadrature off the diagonal and exact self-element integrals on it (Sec. 7 opening
// paragraph), rows placed by the Sec. 6 recipe (eq. calderon_bieb with beta = -alpha, eq. 3dom_calderon_bie
// with gamma = alpha/eps) or one of the comparison forms.
//
// Precision plan (GB300 issues FP64 at 2 operations per clock per SM against 128 for FP32): FP64 forms, once
// per element pair, the centre-to-centre vector, its length and projections (the cosines of nearly tangent
// pairs cancel there, so they keep FP64's extra bits) and the FP64 part of each Bessel argument (an error of
// k r is an error of the Hankel function's phase, and k r reaches ~100).  The node distances and direction
// cosines relative to that vector, the node offsets of the Bessel arguments, the Bessel values, Gauss weights,
// the four sums and their combination into entries are double-float arithmetic on the FP32 pipe.  Accuracy against the FP64 definition: ~1e-14 of the largest
// entry of a block, a few 1e-12 relative on entries above 1e-6 of it.
#pragma once

#include "bessel.cuh"
#include "internal.cuh"

namespace bem {

BEM_HD double2 mul_i(double2 z) { return make_double2(-z.y, z.x); }

struct RowEq {
  int dom;        // domain whose equation this row carries
  int bm;         // 1: Burton-Miller (standard + gamma * normal derivative), 0: standard
  int ia;         // 1: the row is multiplied by -alpha = i/k_1, 0: by 1
  double2 scale;  // row multiplier (1 or i/k_1)
};

// Row plan of Sec. 5-6 for an element with (P, M); half 0 = upper row, 1 = lower row.
BEM_HD RowEq row_eq(int form, int half, int P, int M, double k1) {
  RowEq e;
  int ia;
  if (form == BEM_FORM_CONV) {
    if (half == 0) { e.dom = P; e.bm = (P == 0); ia = 0; }
    else { e.dom = M; e.bm = 0; ia = 0; }
  } else if (half == 0) {
    e.dom = M; e.bm = 0; ia = (form == BEM_FORM_BETA1) ? 0 : 1;
  } else {
    e.dom = P;
    if (form == BEM_FORM_ORIG && P != 0) { e.bm = 0; ia = 1; }
    else { e.bm = 1; ia = 0; }
  }
  e.ia = ia;
  e.scale = ia ? make_double2(0.0, 1.0 / k1) : make_double2(1.0, 0.0);
  return e;
}

// complex double-float
struct C2 {
  F2 x, y;
};
BEM_HD C2 c2_add(C2 a, C2 b) { return C2{f2_add(a.x, b.x), f2_add(a.y, b.y)}; }
BEM_HD C2 c2_sub(C2 a, C2 b) { return C2{f2_sub(a.x, b.x), f2_sub(a.y, b.y)}; }
BEM_HD C2 c2_neg(C2 a) { return C2{f2_neg(a.x), f2_neg(a.y)}; }
BEM_HD C2 c2_mul_i(C2 a) { return C2{f2_neg(a.y), a.x}; }
BEM_HD C2 c2_real(C2 a, F2 s) { return C2{f2_mul(a.x, s), f2_mul(a.y, s)}; }
BEM_HD C2 c2_pow2(C2 a, float s) { return C2{f2_pow2(a.x, s), f2_pow2(a.y, s)}; }
BEM_HD C2 c2_zero() { return C2{F2{0.f, 0.f}, F2{0.f, 0.f}}; }
BEM_HD C2 c2_from(double2 v) { return C2{f2_from(v.x), f2_from(v.y)}; }
BEM_HD double2 c2_to(C2 v) { return make_double2(f2_to(v.x), f2_to(v.y)); }
// acc += s a without renormalising: the product's leading part enters acc.h by a two-sum, its error terms
// and the two-sum's error join acc.l plainly (12 FP32 operations instead of 18 for a product and a sum).
// Over the Q nodes of a Gauss sum acc.l stays within a few units of 2^-24 |acc|, so its own roundings are
// ~2^-48 |acc|; c2_norm renormalises once the sum is complete.
BEM_HD void f2_acc_mul(F2& acc, F2 s, F2 a) {
  const float p = s.h * a.h;
  const float e = fmaf(s.l, a.h, fmaf(s.h, a.l, fmaf(s.h, a.h, -p)));
  const F2 t = f2_two_sum(acc.h, p);
  acc.h = t.h;
  acc.l += t.l + e;
}
// acc += s (a + i b) for real double-float s and Bessel pair (a, b); read acc through c2_norm
BEM_HD void c2_acc(C2& acc, F2 s, F2 a, F2 b) {
  f2_acc_mul(acc.x, s, a);
  f2_acc_mul(acc.y, s, b);
}
BEM_HD C2 c2_norm(C2 a) {
  const F2 x = f2_two_sum(a.x.h, a.x.l), y = f2_two_sum(a.y.h, a.y.l);
  return C2{x, y};
}

// Diagonal pair (i, i): exact self terms in FP64 (N of the N^2 pairs).
//   S_ii = (i/(2k)) [int J0 + i int Y0] over (0, k h/2),  N_ii = k^2 S_ii - (ik/2) H1(k h/2),  D = D* = 0.
BEM_HD void self_pair(const ElemDev& e, const DomTab& dom, int form, int i, C2 (&out)[2][2]) {
  const int Pi = e.P[i], Mi = e.M[i];
  const double k1 = dom.k[0], hj = e.h[i];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const RowEq eq = row_eq(form, half, Pi, Mi, k1);
    const int d = eq.dom;
    const double sg = (Pi == d) ? 1.0 : ((Mi == d) ? -1.0 : 0.0);
    const double k = dom.k[d], eps = dom.eps[d];
    const double gim = -1.0 / (k1 * eps);   // gamma = alpha/eps_d = i * gim
    const double ka = 0.5 * k * hj;
    double ij0, iy0;
    int_j0_y0(ka, ij0, iy0);
    const double2 S = make_double2(-iy0 / (2.0 * k), ij0 / (2.0 * k));
    Bessel01 b;
    bessel01(ka, b);
    // -(ik/2) H1 = -(ik/2)(j1 + i y1) = (k/2) y1 - i (k/2) j1
    const double2 N = make_double2(k * k * S.x + 0.5 * k * b.y1, k * k * S.y - 0.5 * k * b.j1);
    double2 cu = make_double2(0.5, 0.0);
    double2 cw = make_double2(-sg * eps * S.x, -sg * eps * S.y);
    if (eq.bm) {
      const double2 gN = make_double2(-gim * N.y, gim * N.x);
      cu.x += sg * gN.x; cu.y += sg * gN.y;
      cw.y += 0.5 * gim * eps;
    }
    out[half][0] = c2_from(cmul(eq.scale, cu));
    out[half][1] = c2_from(cmul(eq.scale, cw));
  }
}

// Coefficients of one equation row at column j: cu multiplies u_j, cw multiplies w_j.
//   standard:        cu = 1/2 d_ij + s D,                  cw = -s eps S
//   Burton-Miller:   cu = 1/2 d_ij + s (D + gamma N),      cw = gamma eps/2 d_ij - s eps (S + gamma D*)
// with s = sigma_{d,j}, gamma = alpha/eps_d, alpha = -i/k_1, and
//   S = (i/4) sS,  D = (ik/4) sD,  D* = -(ik/4) sDs,  N = (ik/4) sN,
// where sS, sD, sDs, sN are the Gauss sums of H0, (zh.n_j) H1, (zh.n_i) H1 and
// H1/r (n_i.n_j - 2 (zh.n_i)(zh.n_j)) + k H0 (zh.n_i)(zh.n_j) over the element j (zh = (x_i - y)/r).
// out[half][0] multiplies u_j, out[half][1] multiplies w_j in row half*N + i.
// kAsym = false: the caller guarantees that no argument k r of the launch reaches Hankel's expansion
// (k (|d| + h_j / 2) < kTabXMax - 1 for every pair), so the reduction of the arguments by pi/2 is left out.
template <bool kAsym = true>
BEM_HD void assemble_pair_f2(const ElemDev& e, const DomTab& dom, const Quad& q, int form, int i, int j,
                             C2 (&out)[2][2]) {
  if (i == j) {
    self_pair(e, dom, form, i, out);
    return;
  }
  const double xi = e.mx[i], yi = e.my[i];
  const int Pi = e.P[i], Mi = e.M[i];
  const double mxj = e.mx[j], myj = e.my[j], txj = e.tx[j], tyj = e.ty[j];
  const int Pj = e.P[j], Mj = e.M[j];
  const double nxi = -e.ty[i], nyi = e.tx[i], nxj = -tyj, nyj = txj;
  const F2 HH{e.hhh[j], e.hhl[j]};
  const F2 NN = f2_from_bits(nxi * nxj + nyi * nyj);   // n_i . n_j
  // Node geometry.  Once per pair in FP64: the vector d = x_i - m_j from element j's centre to the collocation
  // point, |d| and its projections on tau_j, n_i and n_j.  The node y_m = m_j + s_m tau_j (s_m = t_m h_j / 2)
  // then has z_m = x_i - y_m = d - s_m tau_j, so per node, in double-float:
  //   r_m^2 - |d|^2 = s_m (s_m - 2 d.tau_j),   z_m.n_j = d.n_j (tau_j is orthogonal to n_j),
  //   z_m.n_i = d.n_i - s_m tau_j.n_i.
  // The phase k r_m needs r_m to FP64's absolute accuracy (k r reaches ~100, and Gauss sums of oscillating
  // kernels can cancel by three decades): r_m = |d| + c_m with |d| in FP64 and the node's offset
  // c_m = (r_m^2 - |d|^2) / (r_m + |d|), |c_m| <= h_j / 2, in double-float, so the only error beyond FP64's is
  // that of c_m, ~2^-46 h_j.  The Bessel routines take k r_m as k |d| (FP64, reduced once per pair) plus k c_m
  // (double-float), so no FP64 operation is left per node.
  const double dx = xi - mxj, dy = yi - myj;
  const double dd = dx * dx + dy * dy;
  const double dn = sqrt(dd);
  const F2 DD = f2_from_bits(dd), DN = f2_from_bits(dn);
  const F2 DP2 = f2_from_bits(2.0 * (dx * txj + dy * tyj));
  const F2 DNJ = f2_from_bits(dx * nxj + dy * nyj);

  RowEq eq[2];
  float sg[2];
  double kk[2];
  F2 K[2];
  bool any_bm = false;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    eq[half] = row_eq(form, half, Pi, Mi, dom.k[0]);
    const int d = eq[half].dom;
    sg[half] = (Pj == d) ? 1.f : ((Mj == d) ? -1.f : 0.f);
    kk[half] = dom.k[d];
    K[half] = F2{dom.kh[d], dom.kl[d]};
    any_bm = any_bm || (eq[half].bm && sg[half] != 0.f);
  }
  F2 DNI{0.f, 0.f}, TNI{0.f, 0.f};
  if (any_bm) {
    DNI = f2_from_bits(dx * nxi + dy * nyi);
    TNI = f2_from_bits(txj * nxi + tyj * nyi);
  }
  // the Bessel arguments' FP64 part k |d| (table offset and, where the expansion can be reached, reduction by
  // pi/2, once per pair and domain)
  BesselArg arg0{}, arg1{};
  if (sg[0] != 0.f) bessel_arg_base(kk[0] * dn, arg0, kAsym);
  if (sg[1] != 0.f) bessel_arg_base(kk[1] * dn, arg1, kAsym);

  C2 sS[2], sD[2], sDs[2], sN[2];
#pragma unroll
  for (int half = 0; half < 2; ++half) sS[half] = sD[half] = sDs[half] = sN[half] = c2_zero();
  for (int m = 0; m < q.Q; ++m) {
    const F2 S = f2_mul(HH, F2{q.th[m], q.tl[m]});
    const F2 NUM = f2_mul(S, f2_sub(S, DP2));           // r_m^2 - |d|^2
    const F2 R2 = f2_add(DD, NUM);
    const F2 IR = f2_rsqrt(R2);
    const F2 R = f2_mul(R2, IR);
    const F2 CM = f2_div(NUM, f2_add(R, DN));         // c_m = r_m - |d|
    const F2 CJ = f2_mul(DNJ, IR);
    const F2 WD = f2_mul(HH, F2{q.wh[m], q.wl[m]});
    const F2 WCJ = f2_mul(WD, CJ);
    F2 WCI{0.f, 0.f}, A1{0.f, 0.f}, A0{0.f, 0.f};
    if (any_bm) {
      const F2 CI = f2_mul(f2_sub(DNI, f2_mul(S, TNI)), IR);
      const F2 CC = f2_mul(CI, CJ);
      WCI = f2_mul(WD, CI);
      A1 = f2_mul(f2_mul(WD, IR), f2_sub(NN, f2_pow2(CC, 2.f)));
      A0 = f2_mul(WD, CC);
    }
    // The Hankel values of both row domains.  One call site in a rolled loop: the Bessel code is long,
    // and two inlined copies overflow the instruction cache.
    Bessel01F2 bh[2];
    {
      Bessel01F2 b0{}, b1{};
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        if ((h ? sg[1] : sg[0]) == 0.f) continue;
        const F2 Kh = h ? K[1] : K[0];
        Bessel01F2 b;
        bessel01_f2_at(h ? arg1 : arg0, f2_mul(Kh, CM), f2_mul(Kh, R), b);
        if (h) b1 = b; else b0 = b;
      }
      bh[0] = b0;
      bh[1] = b1;
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      if (sg[half] == 0.f) continue;
      const Bessel01F2& b = bh[half];
      c2_acc(sS[half], WD, b.j0, b.y0);
      c2_acc(sD[half], WCJ, b.j1, b.y1);
      if (eq[half].bm) {
        c2_acc(sDs[half], WCI, b.j1, b.y1);
        c2_acc(sN[half], A1, b.j1, b.y1);
        c2_acc(sN[half], f2_mul(A0, K[half]), b.j0, b.y0);
      }
    }
  }
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    C2 cu = c2_zero(), cw = c2_zero();
    if (sg[half] != 0.f) {
      const int d = eq[half].dom;
      const F2 K4 = f2_pow2(K[half], 0.25f);
      const F2 EPS{dom.eh[d], dom.el[d]};
      const C2 S = c2_pow2(c2_mul_i(c2_norm(sS[half])), 0.25f);
      const C2 D = c2_real(c2_mul_i(c2_norm(sD[half])), K4);
      cu = D;
      cw = c2_neg(c2_real(S, EPS));
      if (eq[half].bm) {
        const F2 GIM{dom.gh[d], dom.gl[d]};   // gamma = i * GIM
        const C2 Ds = c2_neg(c2_real(c2_mul_i(c2_norm(sDs[half])), K4));
        const C2 N = c2_real(c2_mul_i(c2_norm(sN[half])), K4);
        cu = c2_add(cu, c2_mul_i(c2_real(N, GIM)));
        cw = c2_sub(cw, c2_real(c2_mul_i(c2_real(Ds, GIM)), EPS));
      }
      if (sg[half] < 0.f) {
        cu = c2_neg(cu);
        cw = c2_neg(cw);
      }
    }
    if (eq[half].ia) {
      const F2 IK1{dom.ik1h, dom.ik1l};
      cu = c2_mul_i(c2_real(cu, IK1));
      cw = c2_mul_i(c2_real(cw, IK1));
    }
    out[half][0] = cu;
    out[half][1] = cw;
  }
}

}  // namespace bem
