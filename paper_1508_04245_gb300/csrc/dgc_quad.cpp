// Reference tables and facet connectivity for parallelograms, the uncurved
// quadrilaterals of Sec. 2 ("Preliminaries"), built on the host in long double.
//
// Reference square [0,1]^2, x = X_0 + J xi with J[:, 0] = X_1 - X_0 and
// J[:, 1] = X_3 - X_0 for the vertices in cyclic order.
//
// * V_h = [Q^k]^2 with the L2-orthonormal tensor basis
//   psi_{ab}(xi, eta) = l_a(xi) l_b(eta), i = a (k+1) + b, where
//   l_a(t) = sqrt(2a+1) P_a(2t-1) (Legendre three-term recurrence), so the
//   mass matrix is |det J| Id as on simplices (Sec. 2.3).
// * W_h = the H(div)-conforming subspace of the Piola images of [Q^k]^2, which
//   keeps W_h inside V_h so that I is an embedding (Sec. 2.4).  Local DOFs:
//   facet moments int_0^1 u^ . n^_f l_m(s) ds in the local facet parameter s
//   (m = 0..k, facets in the order eta = 0, xi = 1, eta = 1, xi = 0), then
//   interior moments of u^ against (l_a l_b, 0), a <= k-2, b <= k, and
//   (0, l_a l_b), a <= k, b <= k-2.  The basis is the inverse of that DOF
//   matrix on the vector tensor basis.
// * Exact Gauss-Legendre rules, m = floor(3k/2) + 1 points per direction in
//   volumes and on facets (degree 3k per variable).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <stdexcept>

#include "dgc_internal.h"

namespace dgc {
namespace {

typedef long double LD;

constexpr LD kNref[4][2] = {{0, -1}, {1, 0}, {0, 1}, {-1, 0}};   // reference outward normals

// l_a(t) and l_a'(t), a < n: P_{j+1} = ((2j+1) x P_j - j P_{j-1}) / (j+1) and
// P'_{j+1} = P'_{j-1} + (2j+1) P_j at x = 2t - 1.
void legendre01(int n, LD t, LD* v, LD* d) {
  LD P[16], dP[16];
  const LD x = 2 * t - 1;
  P[0] = 1;
  dP[0] = 0;
  if (n > 1) {
    P[1] = x;
    dP[1] = 1;
  }
  for (int j = 1; j + 1 < n; ++j) {
    P[j + 1] = ((2 * j + 1) * x * P[j] - j * P[j - 1]) / (j + 1);
    dP[j + 1] = dP[j - 1] + (2 * j + 1) * P[j];
  }
  for (int a = 0; a < n; ++a) {
    const LD c = sqrtl((LD)(2 * a + 1));
    v[a] = c * P[a];
    d[a] = 2 * c * dP[a];
  }
}

// 1D Lagrange basis at the equispaced nodes j/K and its derivative
void lagrange01(int K, LD t, LD* v, LD* d) {
  for (int j = 0; j <= K; ++j) {
    LD val = 1, der = 0;
    for (int l = 0; l <= K; ++l) {
      if (l == j) continue;
      const LD den = (LD)(j - l) / K;
      LD prod = 1 / den;
      for (int r = 0; r <= K; ++r)
        if (r != j && r != l) prod *= (t - (LD)r / K) / ((LD)(j - r) / K);
      der += prod;
      val *= (t - (LD)l / K) / den;
    }
    v[j] = val;
    d[j] = der;
  }
}

void facet_point(int f, LD s, LD* xi) {
  const LD pts[4][2] = {{s, 0}, {1, s}, {s, 1}, {0, s}};
  xi[0] = pts[f][0];
  xi[1] = pts[f][1];
}

// psi_i and its reference gradient at xi
void tensor_basis(int K, const LD* xi, LD* val, LD* gx, LD* gy) {
  const int n = K + 1;
  LD lx[16], dx[16], ly[16], dy[16];
  legendre01(n, xi[0], lx, dx);
  legendre01(n, xi[1], ly, dy);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      val[a * n + b] = lx[a] * ly[b];
      if (gx) gx[a * n + b] = dx[a] * ly[b];
      if (gy) gy[a * n + b] = lx[a] * dy[b];
    }
}

// interior test field j at xi: component and value
void interior_test(int K, int j, const LD* xi, LD* t) {
  const int n = K + 1;
  LD lx[16], dx[16], ly[16], dy[16];
  legendre01(n, xi[0], lx, dx);
  legendre01(n, xi[1], ly, dy);
  const int nx = (K - 1) * n;
  if (j < nx) {
    t[0] = lx[j / n] * ly[j % n];
    t[1] = 0;
  } else {
    const int jj = j - nx;
    t[0] = 0;
    t[1] = lx[jj / (K - 1)] * ly[jj % (K - 1)];
  }
}

Tables build_quad(int K) {
  Tables t;
  const Sizes s = make_quad_sizes(K);
  t.s = s;
  const int n = K + 1, N = s.N, NW = s.NW, NFM = s.NFM, NINT = s.NINT;
  const int m = s.QF, nd = s.QFD;
  std::vector<LD> g, w, gd, wdl;
  gauss_legendre01(m, g, w);
  gauss_legendre01(nd, gd, wdl);
  std::vector<LD> val(N), gx(N), gy(N);
  // ---- volume and facet points of the stage ------------------------------------
  t.Bv.resize((size_t)s.QV * N);
  t.Gv.resize((size_t)s.QV * N * 2);
  t.wv.resize(s.QV);
  t.xv.resize((size_t)s.QV * 2);
  for (int q1 = 0; q1 < m; ++q1)
    for (int q2 = 0; q2 < m; ++q2) {
      const int q = q1 * m + q2;
      const LD xi[2] = {g[q1], g[q2]};
      tensor_basis(K, xi, val.data(), gx.data(), gy.data());
      for (int i = 0; i < N; ++i) {
        t.Bv[(size_t)q * N + i] = (double)val[i];
        t.Gv[((size_t)q * N + i) * 2 + 0] = (double)gx[i];
        t.Gv[((size_t)q * N + i) * 2 + 1] = (double)gy[i];
      }
      t.wv[q] = (double)(w[q1] * w[q2]);
      t.xv[2 * q] = (double)xi[0];
      t.xv[2 * q + 1] = (double)xi[1];
    }
  t.wf.resize(m);
  t.sf.resize(m);
  t.Bf.resize((size_t)4 * m * N);
  for (int q = 0; q < m; ++q) {
    t.wf[q] = (double)w[q];
    t.sf[q] = (double)g[q];
  }
  for (int f = 0; f < 4; ++f)
    for (int q = 0; q < m; ++q) {
      LD xi[2];
      facet_point(f, g[q], xi);
      tensor_basis(K, xi, val.data(), nullptr, nullptr);
      for (int i = 0; i < N; ++i) t.Bf[((size_t)f * m + q) * N + i] = (double)val[i];
    }
  // ---- 1D tables of the sum-factorised kernel ------------------------------------
  {
    LD v[16], d[16];
    t.q1L.resize((size_t)m * n);
    t.q1D.resize((size_t)m * n);
    for (int q = 0; q < m; ++q) {
      legendre01(n, g[q], v, d);
      for (int a = 0; a < n; ++a) {
        t.q1L[(size_t)q * n + a] = (double)v[a];
        t.q1D[(size_t)q * n + a] = (double)d[a];
      }
    }
    t.q1E.resize((size_t)2 * n);
    for (int e = 0; e < 2; ++e) {
      legendre01(n, (LD)e, v, d);
      for (int a = 0; a < n; ++a) t.q1E[(size_t)e * n + a] = (double)v[a];
    }
  }
  // ---- W_h: DOF matrix on the vector tensor basis, inverted ---------------------
  std::vector<LD> Dm((size_t)NW * NW, 0);
  for (int f = 0; f < 4; ++f)
    for (int q = 0; q < nd; ++q) {
      LD xi[2], lv[16], ld[16];
      facet_point(f, gd[q], xi);
      tensor_basis(K, xi, val.data(), nullptr, nullptr);
      legendre01(n, gd[q], lv, ld);
      for (int mm = 0; mm < NFM; ++mm)
        for (int c = 0; c < 2; ++c)
          for (int i = 0; i < N; ++i)
            Dm[(size_t)(f * NFM + mm) * NW + c * N + i] += wdl[q] * kNref[f][c] * val[i] * lv[mm];
    }
  for (int q1 = 0; q1 < nd; ++q1)
    for (int q2 = 0; q2 < nd; ++q2) {
      const LD xi[2] = {gd[q1], gd[q2]};
      const LD wq = wdl[q1] * wdl[q2];
      tensor_basis(K, xi, val.data(), nullptr, nullptr);
      for (int j = 0; j < NINT; ++j) {
        LD tt[2];
        interior_test(K, j, xi, tt);
        for (int c = 0; c < 2; ++c)
          if (tt[c] != 0)
            for (int i = 0; i < N; ++i) Dm[(size_t)(4 * NFM + j) * NW + c * N + i] += wq * tt[c] * val[i];
      }
    }
  const std::vector<LD> Cinv = invert_matrix(Dm, NW);   // coefficient b of local basis function j: Cinv[b][j]
  t.Cb.resize((size_t)NW * NW);
  for (size_t j = 0; j < Cinv.size(); ++j) t.Cb[j] = (double)Cinv[j];
  // ---- DOF rules: facets (nd points), interior (nd x nd) ------------------------
  t.wfd.resize(nd);
  t.Qfd.resize((size_t)nd * NFM);
  t.xfd.resize((size_t)4 * nd * 2);
  for (int q = 0; q < nd; ++q) {
    LD lv[16], ld[16];
    legendre01(n, gd[q], lv, ld);
    t.wfd[q] = (double)wdl[q];
    for (int mm = 0; mm < NFM; ++mm) t.Qfd[(size_t)q * NFM + mm] = (double)lv[mm];
  }
  for (int f = 0; f < 4; ++f)
    for (int q = 0; q < nd; ++q) {
      LD xi[2];
      facet_point(f, gd[q], xi);
      t.xfd[((size_t)f * nd + q) * 2] = (double)xi[0];
      t.xfd[((size_t)f * nd + q) * 2 + 1] = (double)xi[1];
    }
  t.wd.resize(s.QD);
  t.xd.resize((size_t)s.QD * 2);
  t.Bd.resize((size_t)s.QD * N);
  t.Tint.resize((size_t)s.QD * NINT * 2);
  for (int q1 = 0; q1 < nd; ++q1)
    for (int q2 = 0; q2 < nd; ++q2) {
      const int q = q1 * nd + q2;
      const LD xi[2] = {gd[q1], gd[q2]};
      t.wd[q] = (double)(wdl[q1] * wdl[q2]);
      t.xd[2 * q] = (double)xi[0];
      t.xd[2 * q + 1] = (double)xi[1];
      tensor_basis(K, xi, val.data(), nullptr, nullptr);
      for (int i = 0; i < N; ++i) t.Bd[(size_t)q * N + i] = (double)val[i];
      for (int j = 0; j < NINT; ++j) {
        LD tt[2];
        interior_test(K, j, xi, tt);
        t.Tint[((size_t)q * NINT + j) * 2] = (double)tt[0];
        t.Tint[((size_t)q * NINT + j) * 2 + 1] = (double)tt[1];
      }
    }
  // ---- stream functions: Q^k Lagrange interpolation at the nodes (a/k, b/k) ------
  t.lag_nodes.resize((size_t)s.NLAG * 2);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      t.lag_nodes[(size_t)(a * n + b) * 2] = (double)a / K;
      t.lag_nodes[(size_t)(a * n + b) * 2 + 1] = (double)b / K;
    }
  auto lag_grad = [&](const LD* xi, double* out) {   // [NLAG][2]
    LD vx[16], dx[16], vy[16], dy[16];
    lagrange01(K, xi[0], vx, dx);
    lagrange01(K, xi[1], vy, dy);
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        out[(a * n + b) * 2] = (double)(dx[a] * vy[b]);
        out[(a * n + b) * 2 + 1] = (double)(vx[a] * dy[b]);
      }
  };
  t.Lg_int.resize((size_t)s.QD * s.NLAG * 2);
  for (int q = 0; q < s.QD; ++q) {
    const LD xi[2] = {gd[q / nd], gd[q % nd]};
    lag_grad(xi, &t.Lg_int[(size_t)q * s.NLAG * 2]);
  }
  t.Lg_fac.resize((size_t)4 * nd * s.NLAG * 2);
  for (int f = 0; f < 4; ++f)
    for (int q = 0; q < nd; ++q) {
      LD xi[2];
      facet_point(f, gd[q], xi);
      lag_grad(xi, &t.Lg_fac[((size_t)f * nd + q) * s.NLAG * 2]);
    }
  return t;
}

// ---- parallelepipeds ----------------------------------------------------------------
constexpr LD kNref3[6][3] = {{0, 0, -1}, {0, -1, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, 0, 1}};
constexpr int kFaceAxis[6] = {2, 1, 0, 1, 0, 2};
constexpr int kFaceSide[6] = {0, 0, 1, 1, 0, 1};

void hex_face_point(int f, LD s1, LD s2, LD* xi) {
  int t[2], n = 0;
  for (int a = 0; a < 3; ++a)
    if (a != kFaceAxis[f]) t[n++] = a;
  xi[kFaceAxis[f]] = kFaceSide[f];
  xi[t[0]] = s1;
  xi[t[1]] = s2;
}

void tensor3_basis(int K, const LD* xi, LD* val, LD* g0, LD* g1, LD* g2) {
  const int n = K + 1;
  LD l[3][16], d[3][16];
  for (int a = 0; a < 3; ++a) legendre01(n, xi[a], l[a], d[a]);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c) {
        const int i = (a * n + b) * n + c;
        val[i] = l[0][a] * l[1][b] * l[2][c];
        if (g0) {
          g0[i] = d[0][a] * l[1][b] * l[2][c];
          g1[i] = l[0][a] * d[1][b] * l[2][c];
          g2[i] = l[0][a] * l[1][b] * d[2][c];
        }
      }
}

// interior test fields: component d against l_a l_b l_c with the d-th degree <= k-2
struct HexTest {
  int d, a, b, c;
};
std::vector<HexTest> hex_tests(int K) {
  std::vector<HexTest> out;
  const int n = K + 1;
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b)
        for (int c = 0; c < n; ++c) {
          const int deg[3] = {a, b, c};
          if (deg[d] <= K - 2) out.push_back({d, a, b, c});
        }
  return out;
}

Tables build_hex(int K) {
  Tables t;
  const Sizes s = make_hex_sizes(K);
  t.s = s;
  const int n = K + 1, N = s.N, NW = s.NW, NFM = s.NFM, NINT = s.NINT;
  const int m = (3 * K) / 2 + 1, nd = K + 2;
  std::vector<LD> g, w, gd, wdl;
  gauss_legendre01(m, g, w);
  gauss_legendre01(nd, gd, wdl);
  std::vector<LD> val(N), v0(N), v1(N), v2(N);
  t.Bv.resize((size_t)s.QV * N);
  t.wv.resize(s.QV);
  t.xv.resize((size_t)s.QV * 3);
  for (int q1 = 0; q1 < m; ++q1)
    for (int q2 = 0; q2 < m; ++q2)
      for (int q3 = 0; q3 < m; ++q3) {
        const int q = (q1 * m + q2) * m + q3;
        const LD xi[3] = {g[q1], g[q2], g[q3]};
        tensor3_basis(K, xi, val.data(), nullptr, nullptr, nullptr);
        for (int i = 0; i < N; ++i) t.Bv[(size_t)q * N + i] = (double)val[i];
        t.wv[q] = (double)(w[q1] * w[q2] * w[q3]);
        for (int a = 0; a < 3; ++a) t.xv[3 * q + a] = (double)xi[a];
      }
  t.wf.resize((size_t)m * m);
  t.sf.resize((size_t)m * m * 2);
  t.Bf.resize((size_t)6 * m * m * N);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      t.wf[a * m + b] = (double)(w[a] * w[b]);
      t.sf[2 * (a * m + b)] = (double)g[a];
      t.sf[2 * (a * m + b) + 1] = (double)g[b];
    }
  for (int f = 0; f < 6; ++f)
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        LD xi[3];
        hex_face_point(f, g[a], g[b], xi);
        tensor3_basis(K, xi, val.data(), nullptr, nullptr, nullptr);
        for (int i = 0; i < N; ++i) t.Bf[((size_t)f * m * m + a * m + b) * N + i] = (double)val[i];
      }
  {
    LD lv[16], ld[16];
    t.q1L.resize((size_t)m * n);
    t.q1D.resize((size_t)m * n);
    for (int q = 0; q < m; ++q) {
      legendre01(n, g[q], lv, ld);
      for (int a = 0; a < n; ++a) {
        t.q1L[(size_t)q * n + a] = (double)lv[a];
        t.q1D[(size_t)q * n + a] = (double)ld[a];
      }
    }
    t.q1E.resize((size_t)2 * n);
    for (int e = 0; e < 2; ++e) {
      legendre01(n, (LD)e, lv, ld);
      for (int a = 0; a < n; ++a) t.q1E[(size_t)e * n + a] = (double)lv[a];
    }
  }
  // ---- W_h: DOF matrix on the vector tensor basis, inverted ---------------------------
  const std::vector<HexTest> tests = hex_tests(K);
  std::vector<LD> Dm((size_t)NW * NW, 0);
  for (int f = 0; f < 6; ++f)
    for (int a = 0; a < nd; ++a)
      for (int b = 0; b < nd; ++b) {
        LD xi[3], l1[16], l2[16], d1[16], d2[16];
        hex_face_point(f, gd[a], gd[b], xi);
        tensor3_basis(K, xi, val.data(), nullptr, nullptr, nullptr);
        legendre01(n, gd[a], l1, d1);
        legendre01(n, gd[b], l2, d2);
        const LD wq = wdl[a] * wdl[b];
        for (int al = 0; al < n; ++al)
          for (int be = 0; be < n; ++be)
            for (int c = 0; c < 3; ++c)
              if (kNref3[f][c] != 0)
                for (int i = 0; i < N; ++i)
                  Dm[(size_t)(f * NFM + al * n + be) * NW + c * N + i] += wq * kNref3[f][c] * val[i] * l1[al] * l2[be];
      }
  std::vector<LD> lx(16), dx(16), ly(16), dy(16), lz(16), dz(16);
  for (int q1 = 0; q1 < nd; ++q1)
    for (int q2 = 0; q2 < nd; ++q2)
      for (int q3 = 0; q3 < nd; ++q3) {
        const LD xi[3] = {gd[q1], gd[q2], gd[q3]};
        const LD wq = wdl[q1] * wdl[q2] * wdl[q3];
        tensor3_basis(K, xi, val.data(), nullptr, nullptr, nullptr);
        legendre01(n, xi[0], lx.data(), dx.data());
        legendre01(n, xi[1], ly.data(), dy.data());
        legendre01(n, xi[2], lz.data(), dz.data());
        for (int j = 0; j < NINT; ++j) {
          const HexTest& h = tests[j];
          const LD tv = lx[h.a] * ly[h.b] * lz[h.c];
          for (int i = 0; i < N; ++i) Dm[(size_t)(6 * NFM + j) * NW + h.d * N + i] += wq * tv * val[i];
        }
      }
  const std::vector<LD> Cinv = invert_matrix(Dm, NW);
  t.Cb.resize((size_t)NW * NW);
  for (size_t j = 0; j < Cinv.size(); ++j) t.Cb[j] = (double)Cinv[j];
  // ---- DOF rules --------------------------------------------------------------------
  t.wfd.resize((size_t)nd * nd);
  t.Qfd.resize((size_t)nd * nd * NFM);
  t.xfd.resize((size_t)6 * nd * nd * 3);
  for (int a = 0; a < nd; ++a)
    for (int b = 0; b < nd; ++b) {
      LD l1[16], l2[16], d1[16], d2[16];
      legendre01(n, gd[a], l1, d1);
      legendre01(n, gd[b], l2, d2);
      t.wfd[a * nd + b] = (double)(wdl[a] * wdl[b]);
      for (int al = 0; al < n; ++al)
        for (int be = 0; be < n; ++be) t.Qfd[(size_t)(a * nd + b) * NFM + al * n + be] = (double)(l1[al] * l2[be]);
      for (int f = 0; f < 6; ++f) {
        LD xi[3];
        hex_face_point(f, gd[a], gd[b], xi);
        for (int c = 0; c < 3; ++c) t.xfd[((size_t)f * nd * nd + a * nd + b) * 3 + c] = (double)xi[c];
      }
    }
  t.wd.resize(s.QD);
  t.xd.resize((size_t)s.QD * 3);
  t.Bd.resize((size_t)s.QD * N);
  t.Tint.resize((size_t)s.QD * NINT * 3, 0.0);
  for (int q1 = 0; q1 < nd; ++q1)
    for (int q2 = 0; q2 < nd; ++q2)
      for (int q3 = 0; q3 < nd; ++q3) {
        const int q = (q1 * nd + q2) * nd + q3;
        const LD xi[3] = {gd[q1], gd[q2], gd[q3]};
        t.wd[q] = (double)(wdl[q1] * wdl[q2] * wdl[q3]);
        for (int c = 0; c < 3; ++c) t.xd[3 * q + c] = (double)xi[c];
        tensor3_basis(K, xi, val.data(), nullptr, nullptr, nullptr);
        for (int i = 0; i < N; ++i) t.Bd[(size_t)q * N + i] = (double)val[i];
        legendre01(n, xi[0], lx.data(), dx.data());
        legendre01(n, xi[1], ly.data(), dy.data());
        legendre01(n, xi[2], lz.data(), dz.data());
        for (int j = 0; j < NINT; ++j) {
          const HexTest& h = tests[j];
          t.Tint[((size_t)q * NINT + j) * 3 + h.d] = (double)(lx[h.a] * ly[h.b] * lz[h.c]);
        }
      }
  // ---- vector potentials: [Q^k]^3 Lagrange interpolation at the nodes (a/k, b/k, c/k) ----
  t.lag_nodes.resize((size_t)s.NLAG * 3);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c) {
        const int i = (a * n + b) * n + c;
        t.lag_nodes[3 * i] = (double)a / K;
        t.lag_nodes[3 * i + 1] = (double)b / K;
        t.lag_nodes[3 * i + 2] = (double)c / K;
      }
  auto lag_grad = [&](const LD* xi, double* out) {   // [NLAG][3]
    LD v[3][16], d[3][16];
    for (int a = 0; a < 3; ++a) lagrange01(K, xi[a], v[a], d[a]);
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b)
        for (int c = 0; c < n; ++c) {
          const int i = (a * n + b) * n + c;
          out[i * 3] = (double)(d[0][a] * v[1][b] * v[2][c]);
          out[i * 3 + 1] = (double)(v[0][a] * d[1][b] * v[2][c]);
          out[i * 3 + 2] = (double)(v[0][a] * v[1][b] * d[2][c]);
        }
  };
  t.Lg_int.resize((size_t)s.QD * s.NLAG * 3);
  for (int q = 0; q < s.QD; ++q) {
    const LD xg[3] = {gd[q / (nd * nd)], gd[(q / nd) % nd], gd[q % nd]};   // the interior point q
    lag_grad(xg, &t.Lg_int[(size_t)q * s.NLAG * 3]);
  }
  t.Lg_fac.resize((size_t)6 * s.QFD * s.NLAG * 3);
  for (int f = 0; f < 6; ++f)
    for (int a = 0; a < nd; ++a)
      for (int b = 0; b < nd; ++b) {
        LD xi[3];
        hex_face_point(f, gd[a], gd[b], xi);
        lag_grad(xi, &t.Lg_fac[((size_t)f * s.QFD + a * nd + b) * s.NLAG * 3]);
      }
  return t;
}

}  // namespace

Sizes make_quad_sizes(int K) {
  Sizes s;
  s.D = 2;
  s.K = K;
  s.N = (K + 1) * (K + 1);
  s.NF = 4;
  s.NFM = K + 1;
  s.NW = 2 * s.N;
  s.NINT = 2 * (K + 1) * (K - 1);
  const int m = (3 * K) / 2 + 1;
  s.QV = m * m;
  s.QF = m;
  s.NLAG = (K + 1) * (K + 1);
  s.QFD = K + 2;
  s.QD = (K + 2) * (K + 2);
  return s;
}

bool quad_supported(int K) { return K >= 1 && K <= 6; }

const Tables& quad_tables(int K) {
  static std::mutex mu;
  static std::map<int, Tables> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(K);
  if (it == cache.end()) it = cache.emplace(K, build_quad(K)).first;
  return it->second;
}

Sizes make_hex_sizes(int K) {
  Sizes s;
  const int n = K + 1, m = (3 * K) / 2 + 1, nd = K + 2;
  s.D = 3;
  s.K = K;
  s.N = n * n * n;
  s.NF = 6;
  s.NFM = n * n;
  s.NW = 3 * s.N;
  s.NINT = 3 * n * n * (n - 2);
  s.QV = m * m * m;
  s.QF = m * m;
  s.NLAG = n * n * n;
  s.QFD = nd * nd;
  s.QD = nd * nd * nd;
  return s;
}

bool hex_supported(int K) { return K >= 1 && K <= 3; }

const Tables& hex_tables(int K) {
  static std::mutex mu;
  static std::map<int, Tables> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(K);
  if (it == cache.end()) it = cache.emplace(K, build_hex(K)).first;
  return it->second;
}

std::string build_hex_connectivity(int n_vert, int n_elem, const std::vector<int>& elems, Connectivity& out,
                                   std::vector<signed char>& fcode, std::vector<int>& qnbr) {
  for (int e = 0; e < n_elem; ++e) {
    const int* v = &elems[(size_t)e * 8];
    for (int a = 0; a < 8; ++a) {
      if (v[a] < 0 || v[a] >= n_vert)
        return "element " + std::to_string(e) + " references vertex " + std::to_string(v[a]) + " out of range";
      for (int b = 0; b < a; ++b)
        if (v[a] == v[b]) return "element " + std::to_string(e) + " repeats a vertex";
    }
  }
  struct FK {
    std::array<int, 4> v;
    int e, f;
  };
  const int loc[4][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}};
  std::vector<FK> keys((size_t)n_elem * 6);
  fcode.assign((size_t)n_elem * 6, 0);
  for (int e = 0; e < n_elem; ++e)
    for (int f = 0; f < 6; ++f) {
      int ids[4];
      for (int c = 0; c < 4; ++c) ids[c] = elems[(size_t)e * 8 + kHexFace[f][c]];
      FK k{{ids[0], ids[1], ids[2], ids[3]}, e, f};
      std::sort(k.v.begin(), k.v.end());
      keys[(size_t)e * 6 + f] = k;
      int o = 0;
      for (int c = 1; c < 4; ++c)
        if (ids[c] < ids[o]) o = c;
      int g1 = -1;
      for (int c = 0; c < 4; ++c) {
        const bool d1 = loc[c][0] != loc[o][0], d2 = loc[c][1] != loc[o][1];
        if (d1 != d2 && (g1 < 0 || ids[c] < ids[g1])) g1 = c;
      }
      const int T = loc[g1][0] != loc[o][0] ? 0 : 1;
      fcode[(size_t)e * 6 + f] = (signed char)(T | (loc[o][0] << 1) | (loc[o][1] << 2));
    }
  std::sort(keys.begin(), keys.end(), [](const FK& a, const FK& b) {
    if (a.v != b.v) return a.v < b.v;
    return a.e < b.e;
  });
  out.nbr.assign((size_t)n_elem * 6, -1);
  out.facet_id.assign((size_t)n_elem * 6, -1);
  out.orient.assign((size_t)n_elem * 6, 1);
  out.sides.clear();
  qnbr.assign((size_t)n_elem * 6, -1);
  int nF = 0;
  for (size_t j = 0; j < keys.size();) {
    size_t l = j + 1;
    while (l < keys.size() && keys[l].v == keys[j].v) ++l;
    if (l - j > 2) return "a face is shared by " + std::to_string(l - j) + " elements: mesh is not conforming";
    const FK& a = keys[j];
    out.facet_id[(size_t)a.e * 6 + a.f] = nF;
    out.sides.push_back((a.e << 3) | a.f);
    if (l - j == 2) {
      const FK& b = keys[j + 1];
      if (b.e == a.e) return "element " + std::to_string(a.e) + " uses one face twice";
      out.facet_id[(size_t)b.e * 6 + b.f] = nF;
      out.nbr[(size_t)a.e * 6 + a.f] = (b.e << 3) | b.f;
      out.nbr[(size_t)b.e * 6 + b.f] = (a.e << 3) | a.f;
      out.orient[(size_t)b.e * 6 + b.f] = -1;
      qnbr[(size_t)a.e * 6 + a.f] = (b.e << 3) | b.f;
      qnbr[(size_t)b.e * 6 + b.f] = (a.e << 3) | a.f;
      out.sides.push_back((b.e << 3) | b.f);
    } else {
      out.sides.push_back(-1);
    }
    ++nF;
    j = l;
  }
  out.n_facets = nF;
  return std::string();
}

std::string build_quad_connectivity(int n_vert, int n_elem, const std::vector<int>& elems, Connectivity& out,
                                    std::vector<signed char>& flip, std::vector<int>& qnbr) {
  for (int e = 0; e < n_elem; ++e) {
    const int* v = &elems[(size_t)e * 4];
    for (int a = 0; a < 4; ++a) {
      if (v[a] < 0 || v[a] >= n_vert)
        return "element " + std::to_string(e) + " references vertex " + std::to_string(v[a]) + " out of range";
      for (int b = 0; b < a; ++b)
        if (v[a] == v[b]) return "element " + std::to_string(e) + " repeats a vertex";
    }
  }
  struct FK {
    std::array<int, 2> v;
    int e, f;
  };
  std::vector<FK> keys((size_t)n_elem * 4);
  flip.assign((size_t)n_elem * 4, 0);
  for (int e = 0; e < n_elem; ++e)
    for (int f = 0; f < 4; ++f) {
      const int A = elems[(size_t)e * 4 + kQuadFacet[f][0]], B = elems[(size_t)e * 4 + kQuadFacet[f][1]];
      keys[(size_t)e * 4 + f] = FK{{std::min(A, B), std::max(A, B)}, e, f};
      flip[(size_t)e * 4 + f] = A > B ? 1 : 0;
    }
  std::sort(keys.begin(), keys.end(), [](const FK& a, const FK& b) {
    if (a.v != b.v) return a.v < b.v;
    return a.e < b.e;
  });
  out.nbr.assign((size_t)n_elem * 4, -1);
  out.facet_id.assign((size_t)n_elem * 4, -1);
  out.orient.assign((size_t)n_elem * 4, 1);
  out.sides.clear();
  qnbr.assign((size_t)n_elem * 4, -1);
  int nF = 0;
  for (size_t j = 0; j < keys.size();) {
    size_t l = j + 1;
    while (l < keys.size() && keys[l].v == keys[j].v) ++l;
    if (l - j > 2) return "a facet is shared by " + std::to_string(l - j) + " elements: mesh is not conforming";
    const FK& a = keys[j];
    out.facet_id[(size_t)a.e * 4 + a.f] = nF;
    out.sides.push_back((a.e << 2) | a.f);
    if (l - j == 2) {
      const FK& b = keys[j + 1];
      if (b.e == a.e) return "element " + std::to_string(a.e) + " uses one edge twice";
      out.facet_id[(size_t)b.e * 4 + b.f] = nF;
      out.nbr[(size_t)a.e * 4 + a.f] = (b.e << 2) | b.f;
      out.nbr[(size_t)b.e * 4 + b.f] = (a.e << 2) | a.f;
      out.orient[(size_t)b.e * 4 + b.f] = -1;
      const int rev = flip[(size_t)a.e * 4 + a.f] != flip[(size_t)b.e * 4 + b.f] ? 1 : 0;
      qnbr[(size_t)a.e * 4 + a.f] = (b.e << 3) | (rev << 2) | b.f;
      qnbr[(size_t)b.e * 4 + b.f] = (a.e << 3) | (rev << 2) | a.f;
      out.sides.push_back((b.e << 2) | b.f);
    } else {
      out.sides.push_back(-1);
    }
    ++nF;
    j = l;
  }
  out.n_facets = nF;
  return std::string();
}

}  // namespace dgc
