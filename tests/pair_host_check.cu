// Host build of the library's entry formulas (pair.cuh: the four entries of one element pair, the code the
// assembly kernels run) for the CPU test tests/test_pair_host.py.  No CUDA call is made.
//
// stdin: n Q form n_dom, then k[n_dom], eps[n_dom], the Gauss-Legendre nodes t[Q] and weights w[Q] on
// [-1, 1], then one line per element: ax ay bx by P M (start and end vertex, the domain the normal points out
// of and the domain it points into), optionally followed by a pair count and that many "i j" lines.  stdout: the
// 2n x 2n matrix row by row, "re im" per entry in hexadecimal floating point, or, with a pair list, the four
// entries (i, j), (i, N+j), (N+i, j), (N+i, N+j) of each listed pair on one line.  The element geometry below is the per-element step of the element kernel, restated.
#include <cstdio>
#include <vector>

#include "internal.cuh"
#include "bessel.cuh"
#include "pair.cuh"

using namespace bem;

static void split(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

int main() {
  int n = 0, Q = 0, form = 0, nd = 0;
  if (std::scanf("%d %d %d %d", &n, &Q, &form, &nd) != 4 || n < 1 || Q < 1 || Q > kMaxQuad || nd < 2 ||
      nd > kMaxDomains)
    return 2;
  DomTab dom{};
  dom.n = nd;
  for (int d = 0; d < nd; ++d)
    if (std::scanf("%lf", &dom.k[d]) != 1) return 2;
  for (int d = 0; d < nd; ++d)
    if (std::scanf("%lf", &dom.eps[d]) != 1) return 2;
  for (int d = 0; d < nd; ++d) {
    split(dom.k[d], dom.kh[d], dom.kl[d]);
    split(dom.eps[d], dom.eh[d], dom.el[d]);
    split(-1.0 / (dom.k[0] * dom.eps[d]), dom.gh[d], dom.gl[d]);
  }
  split(1.0 / dom.k[0], dom.ik1h, dom.ik1l);
  Quad q{};
  q.Q = Q;
  for (int m = 0; m < Q; ++m) {
    if (std::scanf("%lf", &q.t[m]) != 1) return 2;
    split(q.t[m], q.th[m], q.tl[m]);
  }
  for (int m = 0; m < Q; ++m) {
    if (std::scanf("%lf", &q.w[m]) != 1) return 2;
    split(q.w[m], q.wh[m], q.wl[m]);
  }
  std::vector<double> ax(n), ay(n), bx(n), by(n), mx(n), my(n), tx(n), ty(n), h(n);
  std::vector<int> P(n), M(n);
  std::vector<float> txh(n), txl(n), tyh(n), tyl(n), hhh(n), hhl(n);
  for (int i = 0; i < n; ++i) {
    if (std::scanf("%lf %lf %lf %lf %d %d", &ax[i], &ay[i], &bx[i], &by[i], &P[i], &M[i]) != 6) return 2;
    const double dx = bx[i] - ax[i], dy = by[i] - ay[i];
    h[i] = std::sqrt(dx * dx + dy * dy);
    tx[i] = dx / h[i];
    ty[i] = dy / h[i];
    mx[i] = 0.5 * (ax[i] + bx[i]);
    my[i] = 0.5 * (ay[i] + by[i]);
    const F2 t1 = f2_from(dx / h[i]), t2 = f2_from(dy / h[i]), hh = f2_from(0.5 * h[i]);
    txh[i] = t1.h; txl[i] = t1.l;
    tyh[i] = t2.h; tyl[i] = t2.l;
    hhh[i] = hh.h; hhl[i] = hh.l;
  }
  const ElemDev e{ax.data(), ay.data(), bx.data(), by.data(), mx.data(), my.data(), tx.data(), ty.data(),
                  h.data(), P.data(), M.data(), txh.data(), txl.data(), tyh.data(), tyl.data(), hhh.data(),
                  hhl.data()};
  // optional: a list of pairs (count, then i j per pair) -> the four entries of each pair, one pair per line
  int npairs = 0;
  if (std::scanf("%d", &npairs) == 1) {
    for (int k = 0; k < npairs; ++k) {
      int i = 0, j = 0;
      if (std::scanf("%d %d", &i, &j) != 2 || i < 0 || j < 0 || i >= n || j >= n) return 2;
      C2 out[2][2];
      assemble_pair_f2(e, dom, q, form, i, j, out);
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const double2 v = c2_to(out[a][b]);
          std::printf("%a %a%c", v.x, v.y, (a == 1 && b == 1) ? '\n' : ' ');
        }
    }
    return 0;
  }
  const size_t n2 = 2 * (size_t)n;
  std::vector<double2> A(n2 * n2);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      C2 out[2][2];
      assemble_pair_f2(e, dom, q, form, i, j, out);
      A[(size_t)i * n2 + j] = c2_to(out[0][0]);
      A[(size_t)i * n2 + n + j] = c2_to(out[0][1]);
      A[(size_t)(n + i) * n2 + j] = c2_to(out[1][0]);
      A[(size_t)(n + i) * n2 + n + j] = c2_to(out[1][1]);
    }
  for (size_t r = 0; r < n2; ++r)
    for (size_t c = 0; c < n2; ++c) std::printf("%a %a%c", A[r * n2 + c].x, A[r * n2 + c].y, c + 1 == n2 ? '\n' : ' ');
  return 0;
}
