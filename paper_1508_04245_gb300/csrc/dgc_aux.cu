// Per-element FP64 kernels around the stage kernel: geometry (step a1),
// frozen-wind preparation, the transfer I (a2) and its transpose I^T (a8),
// the diagonal mass, and input construction (curl-of-potential winds,
// L2 projection, wind speed for the CFL rule).
//
// These run once per call (not once per RK stage), so they use runtime sizes
// and per-thread scratch arrays sized for the largest supported order.
#include <cuda_runtime.h>

#include <cmath>

#include "dgc_kernels.h"
#include "dgc_tc3_layout.h"

namespace dgc {
namespace {

constexpr int MAXW = 192;   // W_h of parallelepipeds, k = 3 (BDM_5 on tetrahedra: 168)
constexpr int MAXF = 21;    // dim P^5 on a triangle
constexpr int MAXI = 96;    // interior moments of parallelepipeds, k = 3 (BDM_5 on tetrahedra: 84)
constexpr int MAXL = 84;    // dim P^6 in 3D (Lagrange nodes of P^{k+1})
constexpr int MAXN = 28;    // dim P^6 on a triangle (curved elements)
constexpr int BLOCK = 128;

inline int grid_for(long n) { return (int)((n + BLOCK - 1) / BLOCK); }

// Direction of the reference facet flux: on the simplex -grad lambda_f ((1, .., 1)
// for f = 0, -e_{f-1} otherwise; its length carries the facet measure), on the
// square the outward unit normal of facet f (eta = 0, xi = 1, eta = 1, xi = 0),
// on the cube that of face f (zeta = 0, eta = 0, xi = 1, eta = 1, xi = 0, zeta = 1).
__device__ __forceinline__ double ref_dir(const DevMesh& m, int f, int a) {
  if (m.quad) {
    const double nq[4][2] = {{0.0, -1.0}, {1.0, 0.0}, {0.0, 1.0}, {-1.0, 0.0}};
    return nq[f][a];
  }
  if (m.hex) {
    const double nh[6][3] = {{0, 0, -1}, {0, -1, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, 0, 1}};
    return nh[f][a];
  }
  return f == 0 ? 1.0 : (a == f - 1 ? -1.0 : 0.0);
}

// Local facet mode j of element e's facet f against the global facet modes: returns
// the factor and sets *jg to the global mode.  Simplices sort their vertices (identity);
// parallelograms flip (-1)^j where the local parameter runs against the global one;
// parallelepipeds map (alpha, beta) to (beta, alpha) when transposed, with the factor
// (-1)^(alpha o1 + beta o2).
__device__ __forceinline__ double facet_mode(const DevMesh& m, int e, int f, int j, int* jg) {
  *jg = j;
  if (m.flip) return (m.flip[(long)e * 4 + f] && (j & 1)) ? -1.0 : 1.0;
  if (m.fcode) {
    const int n = m.s.K + 1, al = j / n, be = j % n, c = m.fcode[(long)e * 6 + f];
    const int o1 = (c >> 1) & 1, o2 = (c >> 2) & 1;
    if (c & 1) *jg = be * n + al;
    return ((al * o1 + be * o2) & 1) ? -1.0 : 1.0;
  }
  return 1.0;
}

__global__ void geometry_kernel(DevMesh m) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const int D = m.s.D;
  const int* v = m.elems + (long)e * (m.hex ? 8 : m.s.NF);   // vertices per element
  double X0[3], J[9];
  for (int a = 0; a < D; ++a) X0[a] = m.verts[(long)v[0] * D + a];
  // simplex: J[:, c] = X_{c+1} - X_0; parallelogram: [X_1, X_3] - X_0; parallelepiped: [X_1, X_3, X_4] - X_0
  const int cols[3] = {1, (m.quad || m.hex) ? 3 : 2, m.hex ? 4 : 3};
  for (int c = 0; c < D; ++c)
    for (int r = 0; r < D; ++r) J[r * D + c] = m.verts[(long)v[cols[c]] * D + r] - X0[r];
  double det;
  if (D == 2) {
    det = J[0] * J[3] - J[1] * J[2];
  } else {
    det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
          J[2] * (J[3] * J[7] - J[4] * J[6]);
  }
  for (int j = 0; j < D * D; ++j) m.J[(long)e * D * D + j] = J[j];
  m.detJ[e] = det;
}

// local BDM DOFs of element e, signs applied: facet moments of local facet f
// carry orient(e, f) * sign(det J), interior moments are element-owned.
__device__ void gather_local(const DevMesh& m, int e, const double* __restrict__ u, double* ut) {
  const Sizes& s = m.s;
  const double sg = m.detJ[e] > 0 ? 1.0 : -1.0;
  for (int f = 0; f < s.NF; ++f) {
    const long g = m.facet_id[(long)e * s.NF + f] + (DGC_CHECKED && m.inject_bad_facet && e == 0 ? m.nF : 0);
    const double sf = sg * (double)m.orient[(long)e * s.NF + f];
    const bool ok = gather_ok(g, m.nF, m.status);
    for (int j = 0; j < s.NFM; ++j) {
      int jg;
      const double fm = facet_mode(m, e, f, j, &jg);
      ut[f * s.NFM + j] = ok ? sf * fm * u[g * s.NFM + jg] : 0.0;
    }
  }
  const long base = (long)m.nF * s.NFM + (long)e * s.NINT;
  for (int j = 0; j < s.NINT; ++j) ut[s.NF * s.NFM + j] = u[base + j];
}

// reference wind on the vector Dubiner basis: uc[a*N + i] = sum_j Cb[a*N+i][j] ut[j]
__device__ void bdm_to_dubiner(const DevMesh& m, const double* ut, double* uc) {
  const int NW = m.s.NW;
  for (int b = 0; b < NW; ++b) {
    double acc = 0.0;
    const double* row = m.Cb + (long)b * NW;
    for (int j = 0; j < NW; ++j) acc += row[j] * ut[j];
    uc[b] = acc;
  }
}

template <typename T>
__global__ void wind_prep_kernel(DevMesh m, const double* __restrict__ u, T* __restrict__ Uw, T* __restrict__ Fw) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const Sizes& s = m.s;
  const int D = s.D, N = s.N;
  const long E = m.E;
  double ut[MAXW], uc[MAXW];
  gather_local(m, e, u, ut);
  bdm_to_dubiner(m, ut, uc);
  // affine: the diagonal mass |det J| folded in as 1/det J; curved: only the sign of
  // det J, the stage kernel applies the inverse mass block
  const bool curved = m.cid && m.cid[e] >= 0;
  const double inv = curved ? (m.detJ[e] > 0 ? 1.0 : -1.0) : 1.0 / m.detJ[e];
  for (int q = 0; q < s.QV; ++q)
    for (int a = 0; a < D; ++a) {
      double acc = 0.0;
      for (int i = 0; i < N; ++i) acc += m.Bv[q * N + i] * uc[a * N + i];
      Uw[m.hex ? ((long)e * s.QV + q) * D + a : (long)(q * D + a) * E + e] = (T)(inv * m.wv[q] * acc);
    }
  for (int f = 0; f < s.NF; ++f)
    for (int q = 0; q < s.QF; ++q) {
      double acc = 0.0;
      for (int a = 0; a < D; ++a) {
        const double g = ref_dir(m, f, a);
        if (g == 0.0) continue;
        double ua = 0.0;
        for (int i = 0; i < N; ++i) ua += m.Bf[(long)(f * s.QF + q) * N + i] * uc[a * N + i];
        acc += g * ua;
      }
      Fw[m.hex ? ((long)e * s.NF + f) * s.QF + q : (long)(f * s.QF + q) * E + e] = (T)(inv * m.wf[q] * acc);
    }
}

// wind on the vector Dubiner basis scaled by 1/det J, float, zero padded to nk
__global__ void wind_coeffs_kernel(DevMesh m, const double* __restrict__ u, float* __restrict__ wc, int nk) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const Sizes& s = m.s;
  double ut[MAXW], uc[MAXW];
  gather_local(m, e, u, ut);
  bdm_to_dubiner(m, ut, uc);
  const double inv = 1.0 / m.detJ[e];
  // tile-blocked [tile][a][i][128] (tile = 128 consecutive elements)
  float* wt = wc + (long)(e >> 7) * s.D * nk * 128 + (e & 127);
  for (int a = 0; a < s.D; ++a)
    for (int i = 0; i < nk; ++i) wt[(long)(a * nk + i) * 128] = i < s.N ? (float)(inv * uc[a * s.N + i]) : 0.f;
}

// tetrahedral tensor-core path, step 1: the wind on the vector Dubiner basis scaled
// by 1/det J, FP64, tile-blocked [tile][d][i][40] (tile of 40 elements), and the
// frozen reference flux at the facet points, (1/det J) w^f_q (u^ . -grad lambda_f),
// tile-blocked [tile][f][q][40]
__global__ void wind_tc3_kernel(DevMesh m, const double* __restrict__ u, double* __restrict__ uc3,
                                float* __restrict__ fw3) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const Sizes& s = m.s;
  const int N = s.N;
  double ut[MAXW], uc[MAXW];
  gather_local(m, e, u, ut);
  bdm_to_dubiner(m, ut, uc);
  const double inv = 1.0 / m.detJ[e];
  const int tile = e / 40, el = e % 40;
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < N; ++i) uc3[(((size_t)tile * 3 + c) * N + i) * 40 + el] = inv * uc[c * N + i];
  float* fb = fw3 + (size_t)tile * s.NF * s.QF * 40 + el;
  for (int f = 0; f < s.NF; ++f)
    for (int q = 0; q < s.QF; ++q) {
      double acc = 0.0;
      for (int a = 0; a < 3; ++a) {
        const double g = ref_dir(m, f, a);
        if (g == 0.0) continue;
        double ua = 0.0;
        for (int i = 0; i < N; ++i) ua += m.Bf[(long)(f * s.QF + q) * N + i] * uc[a * N + i];
        acc += g * ua;
      }
      fb[(size_t)(f * s.QF + q) * 40] = (float)(inv * m.wf[q] * acc);
    }
}

// step 2: the wind at the volume points, u_d(xi_q) = sum_i psi^_i(xi_q) uc3[d][i],
// in FP64, rounded once, in chunks of 16 points [tile][chunk][d][16][40]; padding
// points and elements past E are zero
__global__ void wind_pts_tc3_kernel(DevMesh m, const double* __restrict__ uc3, float* __restrict__ wq3,
                                    long total) {
  const long o = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= total) return;
  const Sizes& s = m.s;
  const int N = s.N, nch = (s.QV + 15) / 16;
  const int el = (int)(o % 40);
  const int qq = (int)((o / 40) % 16);
  const int d = (int)((o / 640) % 3);
  const long tj = o / 1920;
  const long tile = tj / nch;
  const int q = (int)(tj % nch) * 16 + qq;
  double acc = 0.0;
  if (q < s.QV && tile * 40 + el < m.E) {
    const double* uc = uc3 + ((size_t)tile * 3 + d) * N * 40 + el;
    const double* B = m.Bv + (size_t)q * N;
    for (int i = 0; i < N; ++i) acc += B[i] * uc[(size_t)i * 40];
  }
  wq3[o] = (float)acc;
}

// w_{c,i} = (1/det J) sum_a J[c][a] uc[a][i]   (= (1/|det J|) int_T u_c psi_i)
__global__ void transfer_kernel(DevMesh m, const double* __restrict__ u, double* __restrict__ w) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const Sizes& s = m.s;
  const int D = s.D, N = s.N;
  double ut[MAXW], uc[MAXW];
  gather_local(m, e, u, ut);
  bdm_to_dubiner(m, ut, uc);
  const double inv = 1.0 / m.detJ[e];
  const double* J = m.J + (long)e * D * D;
  double* we = w + (long)e * D * N;
  for (int c = 0; c < D; ++c)
    for (int i = 0; i < N; ++i) {
      double acc = 0.0;
      for (int a = 0; a < D; ++a) acc += J[c * D + a] * uc[a * N + i];
      we[c * N + i] = inv * acc;
    }
}

// transpose: y = (J/det J)^T f, z = Cb^T y; interior entries go straight to g,
// facet entries (with their signs) to zbuf[e][f][m] for the facet reduction.
__global__ void transfer_T_kernel(DevMesh m, const double* __restrict__ f, double* __restrict__ g,
                                  double* __restrict__ zbuf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const Sizes& s = m.s;
  const int D = s.D, N = s.N, NW = s.NW;
  double y[MAXW];
  const double inv = 1.0 / m.detJ[e];
  const double* J = m.J + (long)e * D * D;
  const double* fe = f + (long)e * D * N;
  for (int a = 0; a < D; ++a)
    for (int i = 0; i < N; ++i) {
      double acc = 0.0;
      for (int c = 0; c < D; ++c) acc += J[c * D + a] * fe[c * N + i];
      y[a * N + i] = inv * acc;
    }
  const double sg = m.detJ[e] > 0 ? 1.0 : -1.0;
  for (int j = 0; j < NW; ++j) {
    double z = 0.0;
    for (int b = 0; b < NW; ++b) z += m.Cb[(long)b * NW + j] * y[b];
    if (j < s.NF * s.NFM) {
      const int lf = j / s.NFM;
      int jg;
      const double sf = sg * (double)m.orient[(long)e * s.NF + lf] * facet_mode(m, e, lf, j % s.NFM, &jg);
      zbuf[(long)e * s.NF * s.NFM + lf * s.NFM + jg] = sf * z;
    } else {
      g[(long)m.nF * s.NFM + (long)e * s.NINT + (j - s.NF * s.NFM)] = z;
    }
  }
}

// deterministic facet sums: owner side first, then the other side
__global__ void facet_reduce_kernel(DevMesh m, const double* __restrict__ zbuf, double* __restrict__ g) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int NFM = m.s.NFM, NF = m.s.NF;
  if (t >= (long)m.nF * NFM) return;
  const long fg = t / NFM;
  const int j = (int)(t % NFM);
  const int sh = NF > 4 ? 3 : 2, mk = (1 << sh) - 1;     // (e << sh) | f
  int s0 = m.facet_sides[2 * fg], s1 = m.facet_sides[2 * fg + 1];
  if (!gather_ok(s0 >> sh, m.E, m.status)) s0 = -1;
  s1 = checked_code(s1, sh, m.E, m.status);
  if (s0 < 0) {   // only in the checked build, after a recorded violation
    g[t] = 0.0;
    return;
  }
  double v = zbuf[((long)(s0 >> sh) * NF + (s0 & mk)) * NFM + j];
  if (s1 >= 0) v += zbuf[((long)(s1 >> sh) * NF + (s1 & mk)) * NFM + j];
  g[t] = v;
}

__global__ void mass_kernel(DevMesh m, const double* __restrict__ v, double* out, bool inverse) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = (long)m.s.D * m.s.N;
  if (t >= (long)m.E * per) return;
  if (m.cid && m.cid[t / per] >= 0) return;   // curved elements: curved_mass_kernel
  const double a = fabs(m.detJ[t / per]);
  out[t] = inverse ? v[t] / a : v[t] * a;
}

// inverse of the row-major D x D matrix J (det given)
__device__ void invert_jacobian(int D, const double* J, double det, double* Jinv) {
  if (D == 2) {
    Jinv[0] = J[3] / det;
    Jinv[1] = -J[1] / det;
    Jinv[2] = -J[2] / det;
    Jinv[3] = J[0] / det;
  } else {
    Jinv[0] = (J[4] * J[8] - J[5] * J[7]) / det;
    Jinv[1] = (J[2] * J[7] - J[1] * J[8]) / det;
    Jinv[2] = (J[1] * J[5] - J[2] * J[4]) / det;
    Jinv[3] = (J[5] * J[6] - J[3] * J[8]) / det;
    Jinv[4] = (J[0] * J[8] - J[2] * J[6]) / det;
    Jinv[5] = (J[2] * J[3] - J[0] * J[5]) / det;
    Jinv[6] = (J[3] * J[7] - J[4] * J[6]) / det;
    Jinv[7] = (J[1] * J[6] - J[0] * J[7]) / det;
    Jinv[8] = (J[0] * J[4] - J[1] * J[3]) / det;
  }
}

// reference field u^ = det J J^{-1} curl(potential interpolant) at one point
__device__ void curl_ref(const DevMesh& m, const double* pot, const double* Lg, const double* Jinv, double det,
                         double* uh) {
  const int D = m.s.D, NL = m.s.NLAG;
  const int nc = D == 2 ? 1 : 3;
  double gr[3][3] = {{0}};
  for (int n = 0; n < NL; ++n)
    for (int c = 0; c < nc; ++c)
      for (int a = 0; a < D; ++a) gr[c][a] += pot[n * nc + c] * Lg[n * D + a];
  double gp[3][3] = {{0}};   // physical gradient J^{-T} grad^
  for (int c = 0; c < nc; ++c)
    for (int b = 0; b < D; ++b)
      for (int a = 0; a < D; ++a) gp[c][b] += Jinv[a * D + b] * gr[c][a];
  double u[3];
  if (D == 2) {
    u[0] = gp[0][1];
    u[1] = -gp[0][0];
  } else {
    u[0] = gp[2][1] - gp[1][2];
    u[1] = gp[0][2] - gp[2][0];
    u[2] = gp[1][0] - gp[0][1];
  }
  for (int a = 0; a < D; ++a) {
    double acc = 0.0;
    for (int b = 0; b < D; ++b) acc += Jinv[a * D + b] * u[b];
    uh[a] = det * acc;
  }
}

__global__ void wind_from_potential_kernel(DevMesh m, const double* __restrict__ pot_all, double* __restrict__ u) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const Sizes& s = m.s;
  const int D = s.D, NL = s.NLAG, nc = D == 2 ? 1 : 3;
  const double* J = m.J + (long)e * D * D;
  double det = m.detJ[e];
  double Jinv[9];
  invert_jacobian(D, J, det, Jinv);
  const double sg = det > 0 ? 1.0 : -1.0;
  if (m.cid && m.cid[e] >= 0) {
    // curved: det J J^{-1} curl(psi) = the reference curl of psi^ at every point, for any
    // map (2D), so the DOFs need no Jacobian: evaluate with J = Id
    for (int j = 0; j < 9; ++j) Jinv[j] = (j % (D + 1) == 0) ? 1.0 : 0.0;
    det = 1.0;
  }
  double pot[MAXL * 3];
  for (int j = 0; j < NL * nc; ++j) pot[j] = pot_all[(long)e * NL * nc + j];
  double uh[3];
  // facet moments, computed by the facet's owner (orient = +1)
  for (int f = 0; f < s.NF; ++f) {
    if (m.orient[(long)e * s.NF + f] < 0) continue;
    double acc[MAXF];
    for (int j = 0; j < s.NFM; ++j) acc[j] = 0.0;
    for (int q = 0; q < s.QFD; ++q) {
      curl_ref(m, pot, m.Lg_fac + (long)(f * s.QFD + q) * NL * D, Jinv, det, uh);
      double flux = 0.0;
      for (int a = 0; a < D; ++a) flux += ref_dir(m, f, a) * uh[a];
      for (int j = 0; j < s.NFM; ++j) acc[j] += m.wfd[q] * flux * m.Qfd[q * s.NFM + j];
    }
    const long g = m.facet_id[(long)e * s.NF + f];
    if (!gather_ok(g, m.nF, m.status)) continue;
    for (int j = 0; j < s.NFM; ++j) {
      int jg;
      const double fm = facet_mode(m, e, f, j, &jg);
      u[g * s.NFM + jg] = sg * fm * acc[j];
    }
  }
  if (s.NINT) {
    double acc[MAXI];
    for (int j = 0; j < s.NINT; ++j) acc[j] = 0.0;
    for (int q = 0; q < s.QD; ++q) {
      curl_ref(m, pot, m.Lg_int + (long)q * NL * D, Jinv, det, uh);
      for (int j = 0; j < s.NINT; ++j) {
        double t = 0.0;
        for (int a = 0; a < D; ++a) t += uh[a] * m.Tint[((long)q * s.NINT + j) * D + a];
        acc[j] += m.wd[q] * t;
      }
    }
    const long base = (long)m.nF * s.NFM + (long)e * s.NINT;
    for (int j = 0; j < s.NINT; ++j) u[base + j] = acc[j];
  }
}

// BDM DOFs of a physical field given at the DOF points of every element:
// vals[e][f*QFD + q][:] on local facet f, vals[e][NF*QFD + q][:] inside.
__global__ void hdiv_interpolate_kernel(DevMesh m, const double* __restrict__ vals, double* __restrict__ u) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const Sizes& s = m.s;
  const int D = s.D;
  const int P = s.NF * s.QFD + s.QD;
  const double* J = m.J + (long)e * D * D;
  const double det = m.detJ[e];
  double Jinv[9];
  invert_jacobian(D, J, det, Jinv);
  const double sg = det > 0 ? 1.0 : -1.0;
  const double* ve = vals + (long)e * P * D;
  double uh[3];
  auto to_ref = [&](const double* x) {   // u^ = det J J^{-1} u
    for (int a = 0; a < D; ++a) {
      double acc = 0.0;
      for (int b = 0; b < D; ++b) acc += Jinv[a * D + b] * x[b];
      uh[a] = det * acc;
    }
  };
  for (int f = 0; f < s.NF; ++f) {
    if (m.orient[(long)e * s.NF + f] < 0) continue;
    double acc[MAXF];
    for (int j = 0; j < s.NFM; ++j) acc[j] = 0.0;
    for (int q = 0; q < s.QFD; ++q) {
      to_ref(ve + (long)(f * s.QFD + q) * D);
      double flux = 0.0;
      for (int a = 0; a < D; ++a) flux += ref_dir(m, f, a) * uh[a];
      for (int j = 0; j < s.NFM; ++j) acc[j] += m.wfd[q] * flux * m.Qfd[q * s.NFM + j];
    }
    const long g = m.facet_id[(long)e * s.NF + f];
    if (!gather_ok(g, m.nF, m.status)) continue;
    for (int j = 0; j < s.NFM; ++j) {
      int jg;
      const double fm = facet_mode(m, e, f, j, &jg);
      u[g * s.NFM + jg] = sg * fm * acc[j];
    }
  }
  if (s.NINT) {
    double acc[MAXI];
    for (int j = 0; j < s.NINT; ++j) acc[j] = 0.0;
    for (int q = 0; q < s.QD; ++q) {
      to_ref(ve + (long)(s.NF * s.QFD + q) * D);
      for (int j = 0; j < s.NINT; ++j) {
        double t = 0.0;
        for (int a = 0; a < D; ++a) t += uh[a] * m.Tint[((long)q * s.NINT + j) * D + a];
        acc[j] += m.wd[q] * t;
      }
    }
    const long base = (long)m.nF * s.NFM + (long)e * s.NINT;
    for (int j = 0; j < s.NINT; ++j) u[base + j] = acc[j];
  }
}

__global__ void project_kernel(DevMesh m, const double* __restrict__ vals, double* __restrict__ w) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const Sizes& s = m.s;
  const int D = s.D, N = s.N;
  for (int c = 0; c < D; ++c)
    for (int i = 0; i < N; ++i) {
      double acc = 0.0;
      for (int q = 0; q < s.QD; ++q) acc += m.wd[q] * vals[((long)e * s.QD + q) * D + c] * m.Bd[q * N + i];
      w[((long)e * D + c) * N + i] = acc;
    }
}

__global__ void max_speed_kernel(DevMesh m, const double* __restrict__ u, unsigned long long* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  if (m.cid && m.cid[e] >= 0) return;         // curved elements: curved_max_speed_kernel
  const Sizes& s = m.s;
  const int D = s.D, N = s.N;
  double ut[MAXW], uc[MAXW];
  gather_local(m, e, u, ut);
  bdm_to_dubiner(m, ut, uc);
  const double* J = m.J + (long)e * D * D;
  const double inv = 1.0 / fabs(m.detJ[e]);
  double vmax = 0.0;
  for (int q = 0; q < s.QV; ++q) {
    double uh[3];
    for (int a = 0; a < D; ++a) {
      double acc = 0.0;
      for (int i = 0; i < N; ++i) acc += m.Bv[q * N + i] * uc[a * N + i];
      uh[a] = acc;
    }
    double n2 = 0.0;
    for (int r = 0; r < D; ++r) {
      double x = 0.0;
      for (int a = 0; a < D; ++a) x += J[r * D + a] * uh[a];
      n2 += x * x;
    }
    vmax = fmax(vmax, sqrt(n2) * inv);
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(vmax));
}

// ---- curved (quadratic) triangles: remark on curved elements, Sec. 2.4 ------------
// J(xi_q) = sum_j X_j (grad^ phi_j(xi_q))^T of curved element c; returns det J
__device__ double curved_jacobian(const DevMesh& m, int c, const double* p2g, double* J) {
  const double* X = m.cnodes + (long)c * 12;
  J[0] = J[1] = J[2] = J[3] = 0.0;
  for (int j = 0; j < 6; ++j)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) J[a * 2 + b] += X[j * 2 + a] * p2g[j * 2 + b];
  return J[0] * J[3] - J[1] * J[2];
}

// M_T = sum_q w_q |det J(xi_q)| psi_i psi_j on the interior rule (degree 2k+2, exact),
// Cholesky-factored and inverted column by column into Minv[(i*N + j)*Ec + c]
__global__ void curved_geometry_kernel(DevMesh m) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.Ec) return;
  const int N = m.s.N;
  double L[MAXN * (MAXN + 1) / 2];                    // packed lower triangle, (i, j <= i)
  for (int j = 0; j < N * (N + 1) / 2; ++j) L[j] = 0.0;
  for (int q = 0; q < m.s.QD; ++q) {
    double J[4];
    const double w = m.wd[q] * fabs(curved_jacobian(m, c, m.p2d + (long)q * 12, J));
    const double* B = m.Bd + (long)q * N;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j <= i; ++j) L[i * (i + 1) / 2 + j] += w * B[i] * B[j];
  }
  for (int j = 0; j < N; ++j) {
    double d = L[j * (j + 1) / 2 + j];
    for (int l = 0; l < j; ++l) d -= L[j * (j + 1) / 2 + l] * L[j * (j + 1) / 2 + l];
    const double ljj = sqrt(d);                         // d > 0: M_T is SPD on an unfolded element
    L[j * (j + 1) / 2 + j] = ljj;
    for (int i = j + 1; i < N; ++i) {
      double x = L[i * (i + 1) / 2 + j];
      for (int l = 0; l < j; ++l) x -= L[i * (i + 1) / 2 + l] * L[j * (j + 1) / 2 + l];
      L[i * (i + 1) / 2 + j] = x / ljj;
    }
  }
  for (int col = 0; col < N; ++col) {                 // M^{-1} e_col = L^{-T} L^{-1} e_col
    double y[MAXN];
    for (int i = 0; i < N; ++i) {
      double x = i == col ? 1.0 : 0.0;
      for (int l = 0; l < i; ++l) x -= L[i * (i + 1) / 2 + l] * y[l];
      y[i] = x / L[i * (i + 1) / 2 + i];
    }
    for (int i = N - 1; i >= 0; --i) {
      double x = y[i];
      for (int l = i + 1; l < N; ++l) x -= L[l * (l + 1) / 2 + i] * y[l];
      y[i] = x / L[i * (i + 1) / 2 + i];
    }
    for (int i = 0; i < N; ++i) {
      m.Minv64[(long)(i * N + col) * m.Ec + c] = y[i];
      m.Minv32[(long)(i * N + col) * m.Ec + c] = (float)y[i];
    }
  }
}

// I u on curved elements, the L2 projection: w = M^{-1} sum_q w_q psi(xi_q) sign(det J) J(xi_q) u^(xi_q)
__global__ void curved_transfer_kernel(DevMesh m, const double* __restrict__ u, double* __restrict__ w) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.Ec) return;
  const int e = m.celem[c], N = m.s.N;
  double ut[MAXW], uc[MAXW], b[2 * MAXN];
  gather_local(m, e, u, ut);
  bdm_to_dubiner(m, ut, uc);
  const double sg = m.detJ[e] > 0 ? 1.0 : -1.0;
  for (int j = 0; j < 2 * N; ++j) b[j] = 0.0;
  for (int q = 0; q < m.s.QD; ++q) {
    double J[4];
    curved_jacobian(m, c, m.p2d + (long)q * 12, J);
    const double* B = m.Bd + (long)q * N;
    double uh[2] = {0.0, 0.0};
    for (int i = 0; i < N; ++i) {
      uh[0] += B[i] * uc[i];
      uh[1] += B[i] * uc[N + i];
    }
    for (int cc = 0; cc < 2; ++cc) {
      const double v = m.wd[q] * sg * (J[cc * 2] * uh[0] + J[cc * 2 + 1] * uh[1]);
      for (int i = 0; i < N; ++i) b[cc * N + i] += v * B[i];
    }
  }
  double* we = w + (long)e * 2 * N;
  for (int cc = 0; cc < 2; ++cc)
    for (int i = 0; i < N; ++i) {
      double acc = 0.0;
      for (int j = 0; j < N; ++j) acc += m.Minv64[(long)(i * N + j) * m.Ec + c] * b[cc * N + j];
      we[cc * N + i] = acc;
    }
}

// the transpose on curved elements: y = M^{-1} f, the adjoint of the point evaluation and
// Piola factor, then Cb^T; facet entries (signed) to zbuf, interior entries to g
__global__ void curved_transfer_T_kernel(DevMesh m, const double* __restrict__ f, double* __restrict__ g,
                                         double* __restrict__ zbuf) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.Ec) return;
  const Sizes& s = m.s;
  const int e = m.celem[c], N = s.N, NW = s.NW;
  const double* fe = f + (long)e * 2 * N;
  double y[2 * MAXN], ua[MAXW];
  for (int cc = 0; cc < 2; ++cc)
    for (int i = 0; i < N; ++i) {
      double acc = 0.0;
      for (int j = 0; j < N; ++j) acc += m.Minv64[(long)(i * N + j) * m.Ec + c] * fe[cc * N + j];
      y[cc * N + i] = acc;
    }
  for (int j = 0; j < NW; ++j) ua[j] = 0.0;
  const double sg = m.detJ[e] > 0 ? 1.0 : -1.0;
  for (int q = 0; q < s.QD; ++q) {
    double J[4];
    curved_jacobian(m, c, m.p2d + (long)q * 12, J);
    const double* B = m.Bd + (long)q * N;
    double Y[2] = {0.0, 0.0};
    for (int i = 0; i < N; ++i) {
      Y[0] += B[i] * y[i];
      Y[1] += B[i] * y[N + i];
    }
    for (int a = 0; a < 2; ++a) {
      const double v = m.wd[q] * sg * (J[a] * Y[0] + J[2 + a] * Y[1]);   // (J^T Y)_a
      for (int i = 0; i < N; ++i) ua[a * N + i] += v * B[i];
    }
  }
  for (int j = 0; j < NW; ++j) {
    double z = 0.0;
    for (int b = 0; b < NW; ++b) z += m.Cb[(long)b * NW + j] * ua[b];
    if (j < s.NF * s.NFM) {
      const int lf = j / s.NFM;
      zbuf[(long)e * s.NF * s.NFM + j] = sg * (double)m.orient[(long)e * s.NF + lf] * z;
    } else {
      g[(long)m.nF * s.NFM + (long)e * s.NINT + (j - s.NF * s.NFM)] = z;
    }
  }
}

// M^V v or (M^V)^{-1} v on curved elements (M v by quadrature, M^{-1} from the blocks)
__global__ void curved_mass_kernel(DevMesh m, const double* __restrict__ v, double* out, bool inverse) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.Ec) return;
  const int e = m.celem[c], N = m.s.N;
  double x[2 * MAXN], r[2 * MAXN];
  for (int j = 0; j < 2 * N; ++j) {
    x[j] = v[(long)e * 2 * N + j];
    r[j] = 0.0;
  }
  if (inverse) {
    for (int cc = 0; cc < 2; ++cc)
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) r[cc * N + i] += m.Minv64[(long)(i * N + j) * m.Ec + c] * x[cc * N + j];
  } else {
    for (int q = 0; q < m.s.QD; ++q) {
      double J[4];
      const double w = m.wd[q] * fabs(curved_jacobian(m, c, m.p2d + (long)q * 12, J));
      const double* B = m.Bd + (long)q * N;
      for (int cc = 0; cc < 2; ++cc) {
        double val = 0.0;
        for (int i = 0; i < N; ++i) val += B[i] * x[cc * N + i];
        for (int i = 0; i < N; ++i) r[cc * N + i] += w * val * B[i];
      }
    }
  }
  for (int j = 0; j < 2 * N; ++j) out[(long)e * 2 * N + j] = r[j];
}

// max |u| = |J u^| / |det J| over the volume points of the curved elements
__global__ void curved_max_speed_kernel(DevMesh m, const double* __restrict__ u, unsigned long long* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.Ec) return;
  const int e = m.celem[c], N = m.s.N;
  double ut[MAXW], uc[MAXW];
  gather_local(m, e, u, ut);
  bdm_to_dubiner(m, ut, uc);
  double vmax = 0.0;
  for (int q = 0; q < m.s.QV; ++q) {
    double J[4];
    const double det = curved_jacobian(m, c, m.p2v + (long)q * 12, J);
    double uh[2] = {0.0, 0.0};
    for (int i = 0; i < N; ++i) {
      uh[0] += m.Bv[q * N + i] * uc[i];
      uh[1] += m.Bv[q * N + i] * uc[N + i];
    }
    const double x0 = J[0] * uh[0] + J[1] * uh[1], x1 = J[2] * uh[0] + J[3] * uh[1];
    vmax = fmax(vmax, sqrt(x0 * x0 + x1 * x1) / fabs(det));
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(vmax));
}

}  // namespace

cudaError_t launch_geometry(const DevMesh& m, cudaStream_t s) {
  if (m.E == 0) return cudaSuccess;
  geometry_kernel<<<grid_for(m.E), BLOCK, 0, s>>>(m);
  if (m.Ec > 0) curved_geometry_kernel<<<grid_for(m.Ec), BLOCK, 0, s>>>(m);
  return cudaGetLastError();
}

cudaError_t launch_wind_prep(const DevMesh& m, const double* u, void* Uw, void* Fw, bool fp32, cudaStream_t s) {
  if (m.E == 0) return cudaSuccess;
  if (fp32)
    wind_prep_kernel<float><<<grid_for(m.E), BLOCK, 0, s>>>(m, u, (float*)Uw, (float*)Fw);
  else
    wind_prep_kernel<double><<<grid_for(m.E), BLOCK, 0, s>>>(m, u, (double*)Uw, (double*)Fw);
  return cudaGetLastError();
}

cudaError_t launch_wind_tc3(const DevMesh& m, const double* u, double* uc3, float* wq3, float* fw3, cudaStream_t s) {
  if (m.E == 0) return cudaSuccess;
  wind_tc3_kernel<<<grid_for(m.E), BLOCK, 0, s>>>(m, u, uc3, fw3);
  const long total = wind_pts_tc3_len(m.s.QV, m.E);
  wind_pts_tc3_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(m, uc3, wq3, total);
  return cudaGetLastError();
}

cudaError_t launch_wind_coeffs(const DevMesh& m, const double* u, float* wc, int nk, cudaStream_t s) {
  if (m.E == 0) return cudaSuccess;
  wind_coeffs_kernel<<<grid_for(m.E), BLOCK, 0, s>>>(m, u, wc, nk);
  return cudaGetLastError();
}

cudaError_t launch_transfer(const DevMesh& m, const double* u, double* w, cudaStream_t s) {
  if (m.E == 0) return cudaSuccess;
  transfer_kernel<<<grid_for(m.E), BLOCK, 0, s>>>(m, u, w);
  if (m.Ec > 0) curved_transfer_kernel<<<grid_for(m.Ec), BLOCK, 0, s>>>(m, u, w);   // overwrites
  return cudaGetLastError();
}

cudaError_t launch_transfer_T(const DevMesh& m, const double* f, double* g, double* zbuf, cudaStream_t s) {
  if (m.E == 0) return cudaSuccess;
  transfer_T_kernel<<<grid_for(m.E), BLOCK, 0, s>>>(m, f, g, zbuf);
  if (m.Ec > 0) curved_transfer_T_kernel<<<grid_for(m.Ec), BLOCK, 0, s>>>(m, f, g, zbuf);   // overwrites
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  facet_reduce_kernel<<<grid_for((long)m.nF * m.s.NFM), BLOCK, 0, s>>>(m, zbuf, g);
  return cudaGetLastError();
}

// ---- diagnostics: mass per component and energy of a DG field, deterministic ----
namespace {

constexpr int DIAG_BLOCK = 256;

// sum of the DIAG_BLOCK values x[t] of a block in a fixed tree order (t = 0 gets it)
__device__ double block_tree_sum(double x, double* sh) {
  const int t = threadIdx.x;
  sh[t] = x;
  __syncthreads();
  for (int h = DIAG_BLOCK / 2; h > 0; h >>= 1) {
    if (t < h) sh[t] += sh[t + h];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// pass 1: per element, int_T w_c = c0 (M_T v_c)_0 (psi^_0 is the constant 1 / c0,
// c0^2 the reference measure) and int_T |w|^2 = sum_c v_c . (M_T v_c); one partial
// [D + 2] per block (mass per component, energy, non-finite coefficient count)
__global__ void diag_partial_kernel(DevMesh m, const double* __restrict__ v, const double* __restrict__ mv,
                                    double c0, double* __restrict__ partials) {
  __shared__ double sh[DIAG_BLOCK];
  const long e = (long)blockIdx.x * DIAG_BLOCK + threadIdx.x;
  const int D = m.s.D, N = m.s.N;
  double mass[3] = {0.0, 0.0, 0.0}, energy = 0.0, bad = 0.0;
  if (e < m.E) {
    for (int c = 0; c < D; ++c) {
      const double* x = v + (e * D + c) * N;
      const double* y = mv + (e * D + c) * N;
      mass[c] = c0 * y[0];
      for (int i = 0; i < N; ++i) {
        energy += x[i] * y[i];
        bad += isfinite(x[i]) ? 0.0 : 1.0;
      }
    }
  }
  double* out = partials + (long)blockIdx.x * (D + 2);
  for (int c = 0; c < D; ++c) {
    const double s = block_tree_sum(mass[c], sh);
    if (threadIdx.x == 0) out[c] = s;
  }
  const double se = block_tree_sum(energy, sh);
  const double sb = block_tree_sum(bad, sh);
  if (threadIdx.x == 0) {
    out[D] = se;
    out[D + 1] = sb;
  }
}

// pass 2: one block sums the partials in a fixed order; a non-finite coefficient
// sets bit 2 of the status word
__global__ void diag_final_kernel(const double* __restrict__ partials, int nblocks, int D, double* out,
                                  int* status) {
  __shared__ double sh[DIAG_BLOCK];
  for (int j = 0; j < D + 2; ++j) {
    double x = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += DIAG_BLOCK) x += partials[(long)b * (D + 2) + j];
    const double s = block_tree_sum(x, sh);
    if (threadIdx.x == 0) {
      out[j] = s;
      if (j == D + 1 && s > 0.0) atomicOr(status, 4);
    }
  }
}

}  // namespace

int diag_blocks(long E) { return (int)((E + DIAG_BLOCK - 1) / DIAG_BLOCK); }

cudaError_t launch_diagnostics(const DevMesh& m, const double* v, double* mv, double* partials, double* out,
                               int* status, cudaStream_t s) {
  cudaError_t err = launch_mass(m, v, mv, false, s);
  if (err != cudaSuccess) return err;
  const int nb = diag_blocks(m.E);
  // c0^2: the measure of the reference element (simplex 1/D!, square and cube 1)
  const double c0 = (m.quad || m.hex) ? 1.0 : std::sqrt(m.s.D == 2 ? 0.5 : 1.0 / 6.0);
  if (nb > 0) diag_partial_kernel<<<nb, DIAG_BLOCK, 0, s>>>(m, v, mv, c0, partials);
  diag_final_kernel<<<1, DIAG_BLOCK, 0, s>>>(partials, nb, m.s.D, out, status);
  return cudaGetLastError();
}

cudaError_t launch_mass(const DevMesh& m, const double* v, double* out, bool inverse, cudaStream_t s) {
  const long n = (long)m.E * m.s.D * m.s.N;
  if (n == 0) return cudaSuccess;
  mass_kernel<<<grid_for(n), BLOCK, 0, s>>>(m, v, out, inverse);
  if (m.Ec > 0) curved_mass_kernel<<<grid_for(m.Ec), BLOCK, 0, s>>>(m, v, out, inverse);
  return cudaGetLastError();
}

cudaError_t launch_wind_from_potential(const DevMesh& m, const double* pot, double* u, cudaStream_t s) {
  if (m.E == 0) return cudaSuccess;
  wind_from_potential_kernel<<<grid_for(m.E), BLOCK, 0, s>>>(m, pot, u);
  return cudaGetLastError();
}

cudaError_t launch_hdiv_interpolate(const DevMesh& m, const double* vals, double* u, cudaStream_t s) {
  if (m.E == 0) return cudaSuccess;
  hdiv_interpolate_kernel<<<grid_for(m.E), BLOCK, 0, s>>>(m, vals, u);
  return cudaGetLastError();
}

cudaError_t launch_project(const DevMesh& m, const double* vals, double* w, cudaStream_t s) {
  if (m.E == 0) return cudaSuccess;
  project_kernel<<<grid_for(m.E), BLOCK, 0, s>>>(m, vals, w);
  return cudaGetLastError();
}

cudaError_t launch_max_speed(const DevMesh& m, const double* u, unsigned long long* out, cudaStream_t s) {
  if (m.E == 0) return cudaSuccess;
  max_speed_kernel<<<grid_for(m.E), BLOCK, 0, s>>>(m, u, out);
  if (m.Ec > 0) curved_max_speed_kernel<<<grid_for(m.Ec), BLOCK, 0, s>>>(m, u, out);
  return cudaGetLastError();
}

}  // namespace dgc
