// Internal declarations of the dgconv library (not part of the C-ABI).
//
// Discretisation (Lehrenfeld & Schoeberl, arXiv:1508.04245):
//   V_h  = [P^k(T)]^d per affine simplex, L2-orthonormal (Dubiner) basis, so
//          the DG mass matrix is |det J_T| Id            (Sec. 2.3)
//   W_h  = BDM_k, facet normal moments + Nedelec interior moments (Sec. 2.1.1)
//   C_h  = upwind DG trilinear form                      (Sec. 2.3)
//
// Everything a kernel needs is expressed on the reference simplex: with the
// contravariant Piola map u = J u^/det J the volume term u . grad psi_i
// |det J| becomes sign(det J) u^ . grad^ psi^_i and the facet flux
// (u . n) dS becomes sign(det J) (u^ . (-grad lambda_f)) ds on the facet
// parameter simplex, so the stage kernels see one scalar 1/det J per element,
// folded into the frozen wind data, and no Jacobian.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace dgc {

constexpr int cpow(int b, int e) { return e == 0 ? 1 : b * cpow(b, e - 1); }

// Compile-time sizes of one (dimension, order) pair.
template <int D, int K>
struct Dims {
  static constexpr int N = D == 2 ? (K + 1) * (K + 2) / 2 : (K + 1) * (K + 2) * (K + 3) / 6;
  static constexpr int NF = D + 1;                                    // facets per element
  static constexpr int NFM = D == 2 ? K + 1 : (K + 1) * (K + 2) / 2;  // dim P^k(facet)
  static constexpr int NW = D * N;                                    // dim BDM_k
  static constexpr int NINT = NW - NF * NFM;                          // interior moments
  static constexpr int NQ1V = (3 * K - 1) / 2 + 1;                    // volume rule, degree 3k-1
  static constexpr int QV = cpow(NQ1V, D);
  static constexpr int NQ1F = (3 * K) / 2 + 1;                        // facet rule, degree 3k
  static constexpr int QF = cpow(NQ1F, D - 1);
};

// Runtime copy of the same sizes.
struct Sizes {
  int D, K, N, NF, NFM, NW, NINT, QV, QF;
  int NLAG;      // Lagrange nodes of P^{k+1} (potential interpolation)
  int QD;        // interior rule of the DOF / projection computations
  int QFD;       // facet rule of the DOF computations
};
Sizes make_sizes(int D, int K);

// Reference tables of one (D, K), built on the host in long double and
// stored as double.  Layouts are row-major in the order of the index list.
struct Tables {
  Sizes s;
  // stage-kernel tables
  std::vector<double> Bv;    // [QV][N]        psi^_i(xi_q)
  std::vector<double> Gv;    // [QV][N][D]     d_a psi^_i(xi_q)
  std::vector<double> Ef;    // [NF][NFM][N]   psi^_i restricted to facet f, on the facet basis
  std::vector<double> Qt;    // [QF][NFM]      facet basis at the facet points
  // wind preparation
  std::vector<double> wv;    // [QV]           volume weights (sum 1/D!)
  std::vector<double> wf;    // [QF]           facet-parameter weights (sum 1/(D-1)!)
  std::vector<double> Bf;    // [NF][QF][N]    psi^_i at the facet points of facet f
  std::vector<double> Cb;    // [NW][NW]       BDM basis on the vector Dubiner basis, [b][j]
  // DOFs of curls of potentials (Lagrange P^{k+1})
  std::vector<double> lag_nodes;  // [NLAG][D]
  std::vector<double> Lg_int;     // [QD][NLAG][D]     grad^ of Lagrange fns at interior points
  std::vector<double> Lg_fac;     // [NF][QFD][NLAG][D] at the facet DOF points
  std::vector<double> Tint;       // [QD][NINT][D]     interior test fields (unit L2 norm)
  std::vector<double> wd;         // [QD]
  std::vector<double> wfd;        // [QFD]
  std::vector<double> Qfd;        // [QFD][NFM]        facet basis at facet DOF points
  // projection of point values onto V_h
  std::vector<double> xd;         // [QD][D]  interior DOF / projection points
  std::vector<double> Bd;         // [QD][N]
  // rule points (for introspection)
  std::vector<double> xfd;        // [NF][QFD][D]  facet DOF points on each local facet
  std::vector<double> xv;         // [QV][D]
  std::vector<double> sf;         // [QF][D-1]
  // parallelograms only: 1D tables of the sum-factorised stage kernel
  std::vector<double> q1L, q1D, q1E;
};

const Tables& tables(int D, int K);   // cached, thread-safe build
bool supported(int D, int K);

// Shared long-double helpers of the table builders.
void gauss_legendre01(int n, std::vector<long double>& x, std::vector<long double>& w);   // n-point rule on [0,1]
std::vector<long double> invert_matrix(const std::vector<long double>& A, int n);         // row-major n x n

// Parallelograms (uncurved quadrilaterals, Sec. 2 "Preliminaries"): the same
// table fields with the meaning they have on the reference square [0,1]^2
// (basis psi_{ab} = l_a(xi) l_b(eta), i = a (k+1) + b, W_h = the H(div)
// subspace of [Q^k]^2, see dgc_quad.cpp), plus the 1D tables of the
// sum-factorised stage kernel: q1L [m][k+1] = l_a at the m Gauss points,
// q1D the same for l_a', q1E [2][k+1] = l_a(0), l_a(1).
Sizes make_quad_sizes(int K);
const Tables& quad_tables(int K);
bool quad_supported(int K);

// Parallelepipeds (uncurved hexahedra): the same fields on [0,1]^3 with
// psi_{abc} = l_a(xi) l_b(eta) l_c(zeta), i = (a (k+1) + b)(k+1) + c, six faces
// (zeta = 0, eta = 0, xi = 1, eta = 1, xi = 0, zeta = 1), face modes
// l_alpha(s1) l_beta(s2), j = alpha (k+1) + beta, in the local face parameter
// (the tangential reference coordinates in increasing axis order).
Sizes make_hex_sizes(int K);
const Tables& hex_tables(int K);
bool hex_supported(int K);

// Facet connectivity of a conforming simplicial mesh (elements' vertex ids
// sorted in place).  Returns an empty string on success, else the reason.
struct Connectivity {
  int n_facets = 0;
  std::vector<int> facet_id, nbr, sides;
  std::vector<signed char> orient;
};
std::string build_connectivity(int D, int n_vert, int n_elem, std::vector<int>& elems, Connectivity& out);

// Facet connectivity of a conforming parallelogram mesh, vertices of every
// element in cyclic order (not reordered).  Local facet f runs from local
// vertex kQuadFacet[f][0] to kQuadFacet[f][1]; flip[e][f] = 1 when that runs
// from the higher to the lower global vertex id; qnbr[e][f] =
// (e' << 3) | (rev << 2) | f' with rev = 1 when the neighbour's local facet
// parameter runs the other way, -1 on the boundary.  Facets are numbered by
// sorting their sorted vertex pairs; the lower-index element owns a facet.
constexpr int kQuadFacet[4][2] = {{0, 1}, {1, 2}, {3, 2}, {0, 3}};
std::string build_quad_connectivity(int n_vert, int n_elem, const std::vector<int>& elems, Connectivity& out,
                                    std::vector<signed char>& flip, std::vector<int>& qnbr);

// Face connectivity of a conforming parallelepiped mesh, local vertex order
// (0,0,0), (1,0,0), (1,1,0), (0,1,0), (0,0,1), (1,0,1), (1,1,1), (0,1,1) (kept).
// kHexFace[f] = local vertices at the face corners (s1, s2) = (0,0), (1,0),
// (0,1), (1,1).  fcode[e][f] = T | o1 << 1 | o2 << 2 relates the local face
// parameter to the global one (origin at the lowest global vertex id, s1
// towards the lower-id of its two face neighbours): (o1, o2) is the local corner
// of the origin and T = 1 when the global s1 runs along the local s2.
// qnbr[e][f] = (e' << 3) | f', -1 on the boundary.  Faces are numbered by their
// sorted vertex quadruples; the lower-index element owns a face.
constexpr int kHexFace[6][4] = {{0, 1, 3, 2}, {0, 1, 4, 5}, {1, 2, 5, 6}, {3, 2, 7, 6}, {0, 3, 4, 7}, {4, 5, 7, 6}};
std::string build_hex_connectivity(int n_vert, int n_elem, const std::vector<int>& elems, Connectivity& out,
                                   std::vector<signed char>& fcode, std::vector<int>& qnbr);

}  // namespace dgc
