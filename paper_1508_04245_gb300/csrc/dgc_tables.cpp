// Reference tables of the dgconv library, built on the host in long double.
//
// * Gauss-Jacobi rules by Newton iteration with deflation on the Jacobi
//   polynomial (weights from the closed-form Christoffel numbers), collapsed
//   into tensor rules on the unit simplex (Duffy map).  The paper leaves the
//   quadrature open; exact rules (volume degree 3k-1, facet degree 3k) make
//   the discrete operator unique (Sec. 2.3).
// * The L2-orthonormal element basis of Sec. 2.3 (Dubiner's collapsed
//   Jacobi products, cited in Sec. 2.2.3), evaluated through division-free
//   homogenised Jacobi recurrences in forward-mode dual numbers, so values
//   and gradients come from one pass.
// * The BDM_k space of Sec. 2.1.1 as the inverse of its degree-of-freedom
//   matrix on the vector Dubiner basis; facet moments against the facet
//   Dubiner basis in the facet's sorted-vertex parametrisation, interior
//   moments against the first-kind Nedelec space N_{k-1} scaled to unit
//   L2 norm.
#include <cmath>
#include <map>
#include <mutex>
#include <stdexcept>
#include <utility>

#include "dgc_internal.h"

namespace dgc {
namespace {

typedef long double LD;

// ---------------------------------------------------------------------------
// Jacobi polynomials and Gauss-Jacobi rules
// ---------------------------------------------------------------------------
LD jacobi_value(int n, LD a, LD b, LD x) {
  if (n == 0) return 1;
  LD p0 = 1, p1 = (a + 1) + (a + b + 2) * (x - 1) / 2;
  for (int m = 2; m <= n; ++m) {
    LD c1 = 2 * m * (m + a + b) * (2 * m + a + b - 2);
    LD c2 = (2 * m + a + b - 1) * (a * a - b * b);
    LD c3 = (2 * m + a + b - 1) * (2 * m + a + b) * (2 * m + a + b - 2);
    LD c4 = 2 * (m + a - 1) * (m + b - 1) * (2 * m + a + b);
    LD p2 = ((c2 + c3 * x) * p1 - c4 * p0) / c1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

LD jacobi_deriv(int n, LD a, LD b, LD x) {
  if (n == 0) return 0;
  return (n + a + b + 1) / 2 * jacobi_value(n - 1, a + 1, b + 1, x);
}

// n-point Gauss-Jacobi rule on [-1, 1], weight (1-x)^a (1+x)^b.
void gauss_jacobi(int n, LD a, LD b, std::vector<LD>& x, std::vector<LD>& w) {
  x.assign(n, 0);
  w.assign(n, 0);
  const LD pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    LD r = -cosl((2 * i + 1) * pi / (2 * n));
    if (i > 0) r = (r + x[i - 1]) / 2;
    for (int it = 0; it < 200; ++it) {
      LD p = jacobi_value(n, a, b, r);
      LD dp = jacobi_deriv(n, a, b, r);
      LD defl = 0;
      for (int j = 0; j < i; ++j) defl += 1 / (r - x[j]);
      LD delta = p / (dp - defl * p);
      r -= delta;
      if (fabsl(delta) < 1e-21L) break;
    }
    x[i] = r;
  }
  LD logc = (a + b + 1) * logl(2.0L) + lgammal(n + a + 1) + lgammal(n + b + 1) -
            lgammal(n + a + b + 1) - lgammal((LD)n + 1);
  LD c = expl(logc);
  for (int i = 0; i < n; ++i) {
    LD dp = jacobi_deriv(n, a, b, x[i]);
    w[i] = c / ((1 - x[i] * x[i]) * dp * dp);
  }
}

int points_for_degree(int degree) { return (degree < 0 ? 0 : degree) / 2 + 1; }

// Collapsed rule on the unit simplex of dimension dim (weights sum to 1/dim!).
void simplex_rule(int dim, int degree, std::vector<LD>& pts, std::vector<LD>& wts) {
  int n = points_for_degree(degree);
  std::vector<LD> t0, w0, t1, w1, t2, w2;
  gauss_jacobi(n, 0, 0, t0, w0);
  pts.clear();
  wts.clear();
  if (dim == 1) {
    for (int i = 0; i < n; ++i) {
      pts.push_back((1 + t0[i]) / 2);
      wts.push_back(w0[i] / 2);
    }
    return;
  }
  gauss_jacobi(n, 1, 0, t1, w1);
  if (dim == 2) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        LD s0 = (1 + t0[i]) / 2, s1 = (1 + t1[j]) / 2;
        pts.push_back(s0 * (1 - s1));
        pts.push_back(s1);
        wts.push_back(w0[i] / 2 * w1[j] / 4);
      }
    return;
  }
  gauss_jacobi(n, 2, 0, t2, w2);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int l = 0; l < n; ++l) {
        LD s0 = (1 + t0[i]) / 2, s1 = (1 + t1[j]) / 2, s2 = (1 + t2[l]) / 2;
        pts.push_back(s0 * (1 - s1) * (1 - s2));
        pts.push_back(s1 * (1 - s2));
        pts.push_back(s2);
        wts.push_back(w0[i] / 2 * w1[j] / 4 * w2[l] / 8);
      }
}

// ---------------------------------------------------------------------------
// forward-mode dual numbers (value + gradient in up to 3 variables)
// ---------------------------------------------------------------------------
struct Dual {
  LD v;
  LD g[3];
};
Dual dconst(LD c) { return Dual{c, {0, 0, 0}}; }
Dual dvar(LD x, int axis) {
  Dual d{x, {0, 0, 0}};
  d.g[axis] = 1;
  return d;
}
Dual operator+(const Dual& a, const Dual& b) {
  return Dual{a.v + b.v, {a.g[0] + b.g[0], a.g[1] + b.g[1], a.g[2] + b.g[2]}};
}
Dual operator-(const Dual& a, const Dual& b) {
  return Dual{a.v - b.v, {a.g[0] - b.g[0], a.g[1] - b.g[1], a.g[2] - b.g[2]}};
}
Dual operator*(const Dual& a, const Dual& b) {
  return Dual{a.v * b.v,
              {a.g[0] * b.v + a.v * b.g[0], a.g[1] * b.v + a.v * b.g[1], a.g[2] * b.v + a.v * b.g[2]}};
}
Dual operator*(LD s, const Dual& a) { return Dual{s * a.v, {s * a.g[0], s * a.g[1], s * a.g[2]}}; }

// v^n P_n^{(alpha,0)}(u/v), by the Jacobi recurrence multiplied through by v^n.
Dual hjacobi(int n, LD alpha, const Dual& u, const Dual& v) {
  if (n == 0) return dconst(1);
  LD a = alpha, b = 0;
  Dual p0 = dconst(1);
  Dual p1 = (a + 1) * v + ((a + b + 2) / 2) * (u - v);
  Dual v2 = v * v;
  for (int m = 2; m <= n; ++m) {
    LD c1 = 2 * m * (m + a + b) * (2 * m + a + b - 2);
    LD c2 = (2 * m + a + b - 1) * (a * a - b * b);
    LD c3 = (2 * m + a + b - 1) * (2 * m + a + b) * (2 * m + a + b - 2);
    LD c4 = 2 * (m + a - 1) * (m + b - 1) * (2 * m + a + b);
    Dual p2 = (1 / c1) * ((c2 * v + c3 * u) * p1 - c4 * (v2 * p0));
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Dubiner index list: by total degree, then (2D) q ascending; (3D) r, then q ascending.
struct Idx {
  int p, q, r;
};
std::vector<Idx> dubiner_indices(int dim, int k) {
  std::vector<Idx> out;
  for (int n = 0; n <= k; ++n) {
    if (dim == 1) {
      out.push_back({n, 0, 0});
    } else if (dim == 2) {
      for (int q = 0; q <= n; ++q) out.push_back({n - q, q, 0});
    } else {
      for (int r = 0; r <= n; ++r)
        for (int q = 0; q <= n - r; ++q) out.push_back({n - q - r, q, r});
    }
  }
  return out;
}

int dim_pk(int dim, int k) {
  if (k < 0) return 0;
  if (dim == 1) return k + 1;
  if (dim == 2) return (k + 1) * (k + 2) / 2;
  return (k + 1) * (k + 2) * (k + 3) / 6;
}

// Orthonormal Dubiner basis (values + gradients) of P^k at one point.
void dubiner(int dim, int k, const LD* x, std::vector<Dual>& out) {
  std::vector<Idx> idx = dubiner_indices(dim, k);
  out.resize(idx.size());
  Dual X = dvar(x[0], 0);
  Dual Y = dim > 1 ? dvar(x[1], 1) : dconst(0);
  Dual Z = dim > 2 ? dvar(x[2], 2) : dconst(0);
  Dual one = dconst(1);
  for (size_t j = 0; j < idx.size(); ++j) {
    int p = idx[j].p, q = idx[j].q, r = idx[j].r;
    if (dim == 1) {
      out[j] = sqrtl((LD)(2 * p + 1)) * hjacobi(p, 0, 2 * X - one, one);
    } else if (dim == 2) {
      Dual A = hjacobi(p, 0, 2 * X - one + Y, one - Y);
      Dual B = hjacobi(q, 2 * p + 1, 2 * Y - one, one);
      out[j] = sqrtl((LD)(2 * p + 1) * 2 * (p + q + 1)) * (A * B);
    } else {
      Dual A = hjacobi(p, 0, 2 * X - one + Y + Z, one - Y - Z);
      Dual B = hjacobi(q, 2 * p + 1, 2 * Y - one + Z, one - Z);
      Dual C = hjacobi(r, 2 * p + 2 * q + 2, 2 * Z - one, one);
      out[j] = sqrtl((LD)(2 * p + 1) * 2 * (p + q + 1) * (2 * (p + q + r) + 3)) * (A * B * C);
    }
  }
}

// ---------------------------------------------------------------------------
// reference simplex
// ---------------------------------------------------------------------------
void ref_vertex(int dim, int v, LD* out) {
  for (int a = 0; a < dim; ++a) out[a] = (v > 0 && a == v - 1) ? 1 : 0;
}
// -grad lambda_f: (1,..,1) for f = 0, -e_{f-1} otherwise
LD mgl(int f, int a) { return f == 0 ? 1 : (a == f - 1 ? -1 : 0); }

void facet_point(int dim, int f, const LD* s, LD* xi) {
  int fv[3], n = 0;
  for (int v = 0; v <= dim; ++v)
    if (v != f) fv[n++] = v;
  LD v0[3], vj[3];
  ref_vertex(dim, fv[0], v0);
  for (int a = 0; a < dim; ++a) xi[a] = v0[a];
  for (int j = 0; j < dim - 1; ++j) {
    ref_vertex(dim, fv[j + 1], vj);
    for (int a = 0; a < dim; ++a) xi[a] += s[j] * (vj[a] - v0[a]);
  }
}

// Gauss-Jordan elimination with partial pivoting: returns A^{-1}.
std::vector<LD> invert(std::vector<LD> A, int n) {
  std::vector<LD> B(n * n, 0);
  for (int i = 0; i < n; ++i) B[i * n + i] = 1;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r * n + c]) > fabsl(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0) throw std::runtime_error("singular matrix in table build");
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(A[c * n + j], A[piv * n + j]);
        std::swap(B[c * n + j], B[piv * n + j]);
      }
    LD inv = 1 / A[c * n + c];
    for (int j = 0; j < n; ++j) {
      A[c * n + j] *= inv;
      B[c * n + j] *= inv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c || A[r * n + c] == 0) continue;
      LD f = A[r * n + c];
      for (int j = 0; j < n; ++j) {
        A[r * n + j] -= f * A[c * n + j];
        B[r * n + j] -= f * B[c * n + j];
      }
    }
  }
  return B;
}

// ---------------------------------------------------------------------------
// Nedelec interior test fields N_{k-1} (unnormalised), value at one point
// ---------------------------------------------------------------------------
struct Nedelec {
  int dim, k, n_vec, count;
  std::vector<int> mono;      // S-part: exponents (a, b, c) and cross index e, 4 ints each
  std::vector<LD> inv_norm;   // scaling to unit L2 norm
  Nedelec(int dim_, int k_) : dim(dim_), k(k_) {
    n_vec = k >= 2 ? dim * dim_pk(dim, k - 2) : 0;
    int deg = k - 2;
    if (k >= 2) {
      if (dim == 2) {
        for (int a = 0; a <= deg; ++a) mono.insert(mono.end(), {a, deg - a, 0, 0});
      } else {
        for (int c3 = 0; c3 <= deg; ++c3)
          for (int b = 0; b <= deg - c3; ++b) {
            int a = deg - c3 - b;
            for (int e = 0; e < 3; ++e) {
              if (e == 2 && c3 > 0) continue;
              mono.insert(mono.end(), {a, b, c3, e});
            }
          }
      }
    }
    count = n_vec + (int)mono.size() / 4;
    inv_norm.assign(count, 1);
    std::vector<LD> pts, wts;
    simplex_rule(dim, 2 * k, pts, wts);
    std::vector<LD> nrm(count, 0);
    LD val[3];
    for (size_t q = 0; q < wts.size(); ++q)
      for (int m = 0; m < count; ++m) {
        eval_raw(m, &pts[q * dim], val);
        for (int a = 0; a < dim; ++a) nrm[m] += wts[q] * val[a] * val[a];
      }
    for (int m = 0; m < count; ++m) inv_norm[m] = 1 / sqrtl(nrm[m]);
  }
  void eval_raw(int m, const LD* x, LD* out) const {
    for (int a = 0; a < 3; ++a) out[a] = 0;
    if (m < n_vec) {
      int nb = dim_pk(dim, k - 2);
      int c = m / nb, j = m % nb;
      std::vector<Dual> psi;
      dubiner(dim, k, x, psi);
      out[c] = psi[j].v;
      return;
    }
    const int* e = &mono[(m - n_vec) * 4];
    LD mv = powl(x[0], e[0]) * powl(x[1], e[1]) * (dim == 3 ? powl(x[2], e[2]) : 1);
    if (dim == 2) {                 // (-y, x) m
      out[0] = -x[1] * mv;
      out[1] = x[0] * mv;
    } else if (e[3] == 0) {         // x cross e_0 = (0, z, -y)
      out[1] = x[2] * mv;
      out[2] = -x[1] * mv;
    } else if (e[3] == 1) {         // x cross e_1 = (-z, 0, x)
      out[0] = -x[2] * mv;
      out[2] = x[0] * mv;
    } else {                        // x cross e_2 = (y, -x, 0)
      out[0] = x[1] * mv;
      out[1] = -x[0] * mv;
    }
  }
  void eval(int m, const LD* x, LD* out) const {
    eval_raw(m, x, out);
    for (int a = 0; a < 3; ++a) out[a] *= inv_norm[m];
  }
};

std::vector<LD> lagrange_nodes(int dim, int order) {
  std::vector<LD> out;
  if (dim == 2) {
    for (int j = 0; j <= order; ++j)
      for (int i = 0; i <= order - j; ++i) out.insert(out.end(), {(LD)i / order, (LD)j / order});
  } else {
    for (int l = 0; l <= order; ++l)
      for (int j = 0; j <= order - l; ++j)
        for (int i = 0; i <= order - l - j; ++i)
          out.insert(out.end(), {(LD)i / order, (LD)j / order, (LD)l / order});
  }
  return out;
}

Tables build(int D, int K) {
  Tables t;
  t.s = make_sizes(D, K);
  const Sizes& s = t.s;
  const int N = s.N, NF = s.NF, NFM = s.NFM, NW = s.NW, NINT = s.NINT;
  std::vector<Dual> psi, qb;

  // ---- volume rule and stage tables ---------------------------------------
  std::vector<LD> xv, wv;
  simplex_rule(D, 3 * K - 1, xv, wv);
  if ((int)wv.size() != s.QV) throw std::runtime_error("volume rule size");
  t.Bv.resize(s.QV * N);
  t.Gv.resize(s.QV * N * D);
  t.wv.resize(s.QV);
  t.xv.resize(s.QV * D);
  for (int j = 0; j < s.QV * D; ++j) t.xv[j] = (double)xv[j];
  for (int q = 0; q < s.QV; ++q) {
    dubiner(D, K, &xv[q * D], psi);
    t.wv[q] = (double)wv[q];
    for (int i = 0; i < N; ++i) {
      t.Bv[q * N + i] = (double)psi[i].v;
      for (int a = 0; a < D; ++a) t.Gv[(q * N + i) * D + a] = (double)psi[i].g[a];
    }
  }
  // ---- facet rule (degree 3k) ----------------------------------------------
  std::vector<LD> sf, wf;
  simplex_rule(D - 1, 3 * K, sf, wf);
  if ((int)wf.size() != s.QF) throw std::runtime_error("facet rule size");
  t.wf.resize(s.QF);
  t.sf.resize(s.QF * (D - 1));
  for (int j = 0; j < s.QF * (D - 1); ++j) t.sf[j] = (double)sf[j];
  t.Qt.resize(s.QF * NFM);
  t.Bf.resize(NF * s.QF * N);
  for (int q = 0; q < s.QF; ++q) {
    t.wf[q] = (double)wf[q];
    dubiner(D - 1, K, &sf[q * (D - 1)], qb);
    for (int m = 0; m < NFM; ++m) t.Qt[q * NFM + m] = (double)qb[m].v;
    for (int f = 0; f < NF; ++f) {
      LD xi[3];
      facet_point(D, f, &sf[q * (D - 1)], xi);
      dubiner(D, K, xi, psi);
      for (int i = 0; i < N; ++i) t.Bf[(f * s.QF + q) * N + i] = (double)psi[i].v;
    }
  }
  // ---- facet restriction on the facet basis (exact, degree 2k) -------------
  std::vector<LD> sd, wd;
  simplex_rule(D - 1, 2 * K + 2, sd, wd);
  if ((int)wd.size() != s.QFD) throw std::runtime_error("facet DOF rule size");
  std::vector<LD> Ef(NF * NFM * N, 0);
  std::vector<LD> V(NW * NW, 0);
  t.wfd.resize(s.QFD);
  t.Qfd.resize(s.QFD * NFM);
  for (int q = 0; q < s.QFD; ++q) {
    t.wfd[q] = (double)wd[q];
    dubiner(D - 1, K, &sd[q * (D - 1)], qb);
    for (int m = 0; m < NFM; ++m) t.Qfd[q * NFM + m] = (double)qb[m].v;
    for (int f = 0; f < NF; ++f) {
      LD xi[3];
      facet_point(D, f, &sd[q * (D - 1)], xi);
      dubiner(D, K, xi, psi);
      for (int m = 0; m < NFM; ++m)
        for (int i = 0; i < N; ++i) {
          LD c = wd[q] * qb[m].v * psi[i].v;
          Ef[(f * NFM + m) * N + i] += c;
          for (int a = 0; a < D; ++a) V[(f * NFM + m) * NW + a * N + i] += mgl(f, a) * c;
        }
    }
  }
  t.Ef.resize(Ef.size());
  for (size_t j = 0; j < Ef.size(); ++j) t.Ef[j] = (double)Ef[j];
  // ---- interior moments ----------------------------------------------------
  Nedelec ned(D, K);
  if (ned.count != NINT) throw std::runtime_error("Nedelec count");
  std::vector<LD> xd, wdd;
  simplex_rule(D, 2 * K + 2, xd, wdd);
  if ((int)wdd.size() != s.QD) throw std::runtime_error("interior DOF rule size");
  t.wd.resize(s.QD);
  t.xd.resize(s.QD * D);
  t.Bd.resize(s.QD * N);
  t.Tint.resize(s.QD * NINT * D);
  for (int q = 0; q < s.QD; ++q) {
    t.wd[q] = (double)wdd[q];
    for (int a = 0; a < D; ++a) t.xd[q * D + a] = (double)xd[q * D + a];
    dubiner(D, K, &xd[q * D], psi);
    for (int i = 0; i < N; ++i) t.Bd[q * N + i] = (double)psi[i].v;
    for (int m = 0; m < NINT; ++m) {
      LD tv[3];
      ned.eval(m, &xd[q * D], tv);
      for (int a = 0; a < D; ++a) {
        t.Tint[(q * NINT + m) * D + a] = (double)tv[a];
        for (int i = 0; i < N; ++i) V[(NF * NFM + m) * NW + a * N + i] += wdd[q] * tv[a] * psi[i].v;
      }
    }
  }
  // ---- BDM basis = inverse of the DOF matrix --------------------------------
  std::vector<LD> Cb = invert(V, NW);
  t.Cb.resize(NW * NW);
  for (int j = 0; j < NW * NW; ++j) t.Cb[j] = (double)Cb[j];
  // ---- Lagrange P^{k+1} gradients for curls of potentials ------------------
  std::vector<LD> nodes = lagrange_nodes(D, K + 1);
  const int NL = s.NLAG;
  if ((int)nodes.size() != NL * D) throw std::runtime_error("Lagrange node count");
  t.lag_nodes.resize(NL * D);
  for (int j = 0; j < NL * D; ++j) t.lag_nodes[j] = (double)nodes[j];
  std::vector<LD> VL(NL * NL);
  for (int n = 0; n < NL; ++n) {
    dubiner(D, K + 1, &nodes[n * D], psi);
    for (int j = 0; j < NL; ++j) VL[n * NL + j] = psi[j].v;
  }
  std::vector<LD> VLi = invert(VL, NL);   // L_n = sum_j VLi[j][n] psi_j
  auto lag_grad = [&](const LD* x, double* out /*[NL][D]*/) {
    dubiner(D, K + 1, x, psi);
    for (int n = 0; n < NL; ++n)
      for (int a = 0; a < D; ++a) {
        LD g = 0;
        for (int j = 0; j < NL; ++j) g += VLi[j * NL + n] * psi[j].g[a];
        out[n * D + a] = (double)g;
      }
  };
  t.Lg_int.resize(s.QD * NL * D);
  for (int q = 0; q < s.QD; ++q) lag_grad(&xd[q * D], &t.Lg_int[q * NL * D]);
  t.Lg_fac.resize(NF * s.QFD * NL * D);
  t.xfd.resize(NF * s.QFD * D);
  for (int f = 0; f < NF; ++f)
    for (int q = 0; q < s.QFD; ++q) {
      LD xi[3];
      facet_point(D, f, &sd[q * (D - 1)], xi);
      for (int a = 0; a < D; ++a) t.xfd[(f * s.QFD + q) * D + a] = (double)xi[a];
      lag_grad(xi, &t.Lg_fac[(f * s.QFD + q) * NL * D]);
    }
  return t;
}

}  // namespace

void gauss_legendre01(int n, std::vector<long double>& x, std::vector<long double>& w) {
  gauss_jacobi(n, 0, 0, x, w);
  for (int i = 0; i < n; ++i) {
    x[i] = (x[i] + 1) / 2;
    w[i] /= 2;
  }
}

std::vector<long double> invert_matrix(const std::vector<long double>& A, int n) { return invert(A, n); }

Sizes make_sizes(int D, int K) {
  Sizes s;
  s.D = D;
  s.K = K;
  s.N = dim_pk(D, K);
  s.NF = D + 1;
  s.NFM = dim_pk(D - 1, K);
  s.NW = D * s.N;
  s.NINT = s.NW - s.NF * s.NFM;
  int nv = points_for_degree(3 * K - 1), nf = points_for_degree(3 * K), nd = points_for_degree(2 * K + 2);
  s.QV = D == 2 ? nv * nv : nv * nv * nv;
  s.QF = D == 2 ? nf : nf * nf;
  s.NLAG = dim_pk(D, K + 1);
  s.QD = D == 2 ? nd * nd : nd * nd * nd;
  s.QFD = D == 2 ? nd : nd * nd;
  return s;
}

bool supported(int D, int K) { return (D == 2 && K >= 1 && K <= 6) || (D == 3 && K >= 1 && K <= 5); }

const Tables& tables(int D, int K) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, Tables> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(D, K);
  auto it = cache.find(key);
  if (it == cache.end()) it = cache.emplace(key, build(D, K)).first;
  return it->second;
}

}  // namespace dgc
