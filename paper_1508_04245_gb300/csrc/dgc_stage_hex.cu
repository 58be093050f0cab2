// Fused RK stage kernel for parallelepipeds with sum-factorised contractions:
// steps a3-a7 of the explicit upwind-DG convection step on [Q^k]^3, one warp per
// element (four elements per block, warp-level synchronisation only), the three
// velocity components one after the other.
//
// On the reference cube (contravariant Piola, as for simplices and
// parallelograms) the operator of Sec. 2.3 divided by the mass |det J| is
//
//   r_{abc} = - sum_{pqs} W(g_p, g_q, g_s) [ U0 l_a' l_b l_c + U1 l_a l_b' l_c + U2 l_a l_b l_c' ]
//             + sum_f sum_{face points} F_f w^ psi_{abc}
//
// with the frozen wind U_d = w_p w_q w_s u^_d / det J and F_f = w w (u^ . n^_f) / det J
// (element-major, prepared once per call).  Volume, one direction at a time in
// shared memory: three contractions to the m^3 points (t1 = sum_a l_a w,
// t2 = sum_b l_b t1, W = sum_c l_c t2), the three wind products, and three back
// (in the last direction l_c or l_c', in the middle l_b or l_b', in the first
// l_a or l_a').  Faces: the modal trace of the state (one contraction with l(0)
// or l(1) along the normal axis), the neighbour's trace on its own face carried
// into this face's parameter (through the face's global parameter: a transpose
// and sign flips (-1)^alpha, (-1)^beta per element face), the values at the m^2
// face points by two 1D contractions, the upwind flux, its projection back by two
// contractions and the outer product with l(0) or l(1) along the normal axis.
//
// Epilogue (a7): vout = alpha vn + beta vin - gamma r in FP64.
#include "dgc_kernels.h"
#include "dgc_stage.cuh"

namespace dgc {
namespace {

// normal axis and side of face f (zeta = 0, eta = 0, xi = 1, eta = 1, xi = 0, zeta = 1)
__device__ __forceinline__ int face_axis(int f) { return (f == 2 || f == 4) ? 0 : (f == 1 || f == 3) ? 1 : 2; }
__device__ __forceinline__ int face_side(int f) { return (f == 2 || f == 3 || f == 5) ? 1 : 0; }

constexpr int kHexWarps = 4;   // elements (warps) per block

template <int K, typename T>
struct HexScratch {                  // one element's working set in shared memory
  static constexpr int n = K + 1, N = n * n * n, m = (3 * K) / 2 + 1, QV = m * m * m, QF = m * m, NFM = n * n;
  T w[N], r[3 * N];
  T t1[m * n * n], t2[m * m * n], F[3][QV], G[3][m * m * n], H[2][m * n * n];
  T to[NFM], tn[NFM], vo[m * n], vn[m * n], P[QF], Qb[m * n];
};

template <int K, typename T>
__global__ void __launch_bounds__(32 * kHexWarps) stage_hex_kernel(StageArgs a, const signed char* __restrict__ fcode) {
  constexpr int n = K + 1, N = n * n * n, m = (3 * K) / 2 + 1, QV = m * m * m, QF = m * m, NFM = n * n;
  __shared__ T L[m * n], Dl[m * n], Eb[2 * n];
  __shared__ HexScratch<K, T> scr[kHexWarps];
  const T* gtab = static_cast<const T*>(a.tab);
  for (int j = threadIdx.x; j < 2 * m * n + 2 * n; j += blockDim.x) {
    const T v = gtab[j];
    if (j < m * n)
      L[j] = v;
    else if (j < 2 * m * n)
      Dl[j - m * n] = v;
    else
      Eb[j - 2 * m * n] = v;
  }
  __syncthreads();
  const int wid = threadIdx.x >> 5;
  const int e = blockIdx.x * kHexWarps + wid;
  if (e >= a.E) return;                                  // whole warps leave; no block barrier follows
  const long E = a.E;
  const int tid = threadIdx.x & 31, nt = 32;
  HexScratch<K, T>& S = scr[wid];
  T* w = S.w;
  T* r = S.r;
  T* t1 = S.t1;
  T* t2 = S.t2;
  T(*F)[QV] = S.F;
  T(*G)[m * m * n] = S.G;
  T(*H)[m * n * n] = S.H;
  T* to = S.to;
  T* tn = S.tn;
  T* vo = S.vo;
  T* vn = S.vn;
  T* P = S.P;
  T* Qb = S.Qb;
  const T* __restrict__ Uw = static_cast<const T*>(a.Uw) + (long)e * QV * 3;
  const T* __restrict__ Fw = static_cast<const T*>(a.Fw) + (long)e * 6 * QF;
  const double* __restrict__ vin_e = a.vin + (long)e * 3 * N;

  for (int c = 0; c < 3; ++c) {
    __syncwarp();
    for (int j = tid; j < N; j += nt) w[j] = (T)vin_e[c * N + j];
    __syncwarp();
    // ---- volume: to the points ------------------------------------------------------
    for (int o = tid; o < m * n * n; o += nt) {        // t1[p][b][cc] = sum_a l_a(g_p) w[a][b][cc]
      const int p = o / (n * n), bc = o % (n * n);
      T acc = (T)0;
      for (int aa = 0; aa < n; ++aa) acc += L[p * n + aa] * w[aa * n * n + bc];
      t1[o] = acc;
    }
    __syncwarp();
    for (int o = tid; o < m * m * n; o += nt) {        // t2[p][q][cc] = sum_b l_b(g_q) t1[p][b][cc]
      const int p = o / (m * n), q = (o / n) % m, cc = o % n;
      T acc = (T)0;
      for (int b = 0; b < n; ++b) acc += L[q * n + b] * t1[(p * n + b) * n + cc];
      t2[o] = acc;
    }
    __syncwarp();
    for (int o = tid; o < QV; o += nt) {               // W at (p, q, s), times the wind
      const int pq = o / m, s = o % m;
      T W = (T)0;
      for (int cc = 0; cc < n; ++cc) W += L[s * n + cc] * t2[pq * n + cc];
      for (int d = 0; d < 3; ++d) F[d][o] = Uw[(long)o * 3 + d] * W;
    }
    __syncwarp();
    // ---- volume: back to the modes ---------------------------------------------------
    for (int o = tid; o < m * m * n; o += nt) {        // last direction: l_c, l_c, l_c'
      const int pq = o / n, cc = o % n;
      T g0 = (T)0, g1 = (T)0, g2 = (T)0;
      for (int s = 0; s < m; ++s) {
        g0 += F[0][pq * m + s] * L[s * n + cc];
        g1 += F[1][pq * m + s] * L[s * n + cc];
        g2 += F[2][pq * m + s] * Dl[s * n + cc];
      }
      G[0][o] = g0;
      G[1][o] = g1;
      G[2][o] = g2;
    }
    __syncwarp();
    for (int o = tid; o < m * n * n; o += nt) {        // middle direction: l_b, l_b' (+) l_b
      const int p = o / (n * n), b = (o / n) % n, cc = o % n;
      T h0 = (T)0, h1 = (T)0;
      for (int q = 0; q < m; ++q) {
        const int gi = (p * m + q) * n + cc;
        h0 += G[0][gi] * L[q * n + b];
        h1 += G[1][gi] * Dl[q * n + b] + G[2][gi] * L[q * n + b];
      }
      H[0][o] = h0;
      H[1][o] = h1;
    }
    __syncwarp();
    for (int o = tid; o < N; o += nt) {                // first direction: l_a', l_a
      const int aa = o / (n * n), bc = o % (n * n);
      T acc = (T)0;
      for (int p = 0; p < m; ++p) acc += H[0][p * n * n + bc] * Dl[p * n + aa] + H[1][p * n * n + bc] * L[p * n + aa];
      r[c * N + o] = -acc;
    }
    // ---- faces -----------------------------------------------------------------------
    for (int f = 0; f < 6; ++f) {
      const int ax = face_axis(f);
      const int ta = ax == 0 ? 1 : 0, tb = ax == 2 ? 1 : 2;     // tangential axes, increasing
      const T* Es = Eb + face_side(f) * n;
      const int code = checked_code(a.nbr[(long)e * 6 + f], 3, a.E, a.status);
      __syncwarp();
      for (int j = tid; j < NFM; j += nt) {            // own modal trace, and the neighbour's
        const int al = j / n, be = j % n;
        int deg[3];
        deg[ta] = al;
        deg[tb] = be;
        T acc = (T)0;
        for (int g = 0; g < n; ++g) {
          deg[ax] = g;
          acc += w[(deg[0] * n + deg[1]) * n + deg[2]] * Es[g];
        }
        to[j] = acc;
        T nbv = (T)0;
        if (code >= 0) {
          const int ne = code >> 3, fn = code & 7;
          const int c0 = fcode[(long)e * 6 + f], c1 = fcode[(long)ne * 6 + fn];
          // this face's local mode (al, be) <- global mode <- the neighbour's local mode
          const int T0 = c0 & 1, o01 = (c0 >> 1) & 1, o02 = (c0 >> 2) & 1;
          const int ga = T0 ? be : al, gb = T0 ? al : be;      // global (a, b)
          const int s0 = T0 ? (be * o02 + al * o01) : (al * o01 + be * o02);
          const int T1 = c1 & 1, o11 = (c1 >> 1) & 1, o12 = (c1 >> 2) & 1;
          const int na = T1 ? gb : ga, nb = T1 ? ga : gb;      // the neighbour's local (alpha, beta)
          const int s1 = T1 ? (gb * o11 + ga * o12) : (ga * o11 + gb * o12);
          const int axn = face_axis(fn);
          const int tan = axn == 0 ? 1 : 0, tbn = axn == 2 ? 1 : 2;
          const T* En = Eb + face_side(fn) * n;
          const double* wn = a.vin + ((long)ne * 3 + c) * N;
          int dn[3];
          dn[tan] = na;
          dn[tbn] = nb;
          for (int g = 0; g < n; ++g) {
            dn[axn] = g;
            nbv += (T)wn[(dn[0] * n + dn[1]) * n + dn[2]] * En[g];
          }
          if ((s0 + s1) & 1) nbv = -nbv;
        }
        tn[j] = nbv;
      }
      __syncwarp();
      for (int o = tid; o < m * n; o += nt) {          // first face direction to the points
        const int pa = o / n, be = o % n;
        T x0 = (T)0, x1 = (T)0;
        for (int al = 0; al < n; ++al) {
          x0 += L[pa * n + al] * to[al * n + be];
          x1 += L[pa * n + al] * tn[al * n + be];
        }
        vo[o] = x0;
        vn[o] = x1;
      }
      __syncwarp();
      for (int o = tid; o < QF; o += nt) {             // values, upwind flux
        const int pa = o / m, pb = o % m;
        T x0 = (T)0, x1 = (T)0;
        for (int be = 0; be < n; ++be) {
          x0 += L[pb * n + be] * vo[pa * n + be];
          x1 += L[pb * n + be] * vn[pa * n + be];
        }
        const T fw = Fw[f * QF + o];
        P[o] = fw * (fw >= (T)0 ? x0 : (code >= 0 ? x1 : (T)0));
      }
      __syncwarp();
      for (int o = tid; o < m * n; o += nt) {          // back: second face direction
        const int pa = o / n, be = o % n;
        T acc = (T)0;
        for (int pb = 0; pb < m; ++pb) acc += P[pa * m + pb] * L[pb * n + be];
        Qb[o] = acc;
      }
      __syncwarp();
      for (int o = tid; o < NFM; o += nt) {            // first face direction, into r
        const int al = o / n, be = o % n;
        T acc = (T)0;
        for (int pa = 0; pa < m; ++pa) acc += Qb[pa * n + be] * L[pa * n + al];
        int deg[3];
        deg[ta] = al;
        deg[tb] = be;
        for (int g = 0; g < n; ++g) {
          deg[ax] = g;
          r[c * N + (deg[0] * n + deg[1]) * n + deg[2]] += acc * Es[g];
        }
      }
    }
  }
  __syncwarp();
  // ---- epilogue: RK stage combination in FP64 -----------------------------------------
  double* vout_e = a.vout + (long)e * 3 * N;
  const double* vn_e = a.vn ? a.vn + (long)e * 3 * N : nullptr;
  for (int o = tid; o < 3 * N; o += nt) {
    double x = a.beta * vin_e[o] - a.gamma * (double)r[o];
    if (vn_e) x += a.alpha * vn_e[o];
    vout_e[o] = x;
  }
  (void)E;
}

template <int K, typename T>
cudaError_t launch_hex_t(const StageArgs* ap, const signed char* fcode, cudaStream_t stream) {
  if (!ap) return cudaSuccess;
  if (ap->E == 0) return cudaSuccess;
  stage_hex_kernel<K, T><<<(ap->E + kHexWarps - 1) / kHexWarps, 32 * kHexWarps, 0, stream>>>(*ap, fcode);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stage_hex(int K, bool fp32, const StageArgs* a, const signed char* fcode, cudaStream_t s) {
  switch (K) {
#define DGC_CASE(k) \
  case k: return fp32 ? launch_hex_t<k, float>(a, fcode, s) : launch_hex_t<k, double>(a, fcode, s);
    DGC_CASE(1) DGC_CASE(2) DGC_CASE(3)
#undef DGC_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dgc
