// Fused RK stage kernel for parallelograms with sum-factorised (tensor-product)
// contractions: steps a3-a7 of the explicit upwind-DG convection step on
// [Q^k]^2, one thread per (element, velocity component).
//
// With psi_{ab}(xi, eta) = l_a(xi) l_b(eta) and Gauss points g_0..g_{m-1} per
// direction, the operator of Sec. 2.3 divided by the mass |det J| reads, on the
// reference square (contravariant Piola, as for simplices),
//
//   r_{ab} = - sum_{p,q} W(g_p, g_q) [ U0_{pq} l_a'(g_p) l_b(g_q) + U1_{pq} l_a(g_p) l_b'(g_q) ]
//            + sum_f sum_q F_{f,q} w^(x_fq) psi_{ab}(x_fq)
//
// with the frozen wind data U_{pq} = w_p w_q u^(g_p, g_q) / det J and
// F_{f,q} = w_q (u^ . n^_f)(x_fq) / det J (prepared once per call), W the
// state at the point and w^ its upwind value.  Every sum runs one direction
// at a time (sum factorisation):
//   * volume, for each row p: the row trace t_b = sum_a w_ab l_a(g_p), the
//     values W(g_p, g_q) = sum_b t_b l_b(g_q), the row projections
//     P_b = sum_q U0 W l_b(g_q) and P'_b = sum_q U1 W l_b'(g_q), and
//     r_ab -= l_a'(g_p) P_b + l_a(g_p) P'_b: O(m k^2 + m^2 k) per row instead
//     of O(m^2 k^2);
//   * facets: the modal trace of the state on the facet (a contraction with
//     l(0) or l(1) along the normal direction), the neighbour's the same way
//     on its own facet with (-1)^j when its facet parameter runs the other
//     way, the upwind values at the facet points, their projection on l_j and
//     its outer product with l(0) or l(1) back into r.
//
// The 1D tables live in constant memory (one slot per order).
// Epilogue (a7): vout = alpha vn + beta vin - gamma r in FP64.
#include "dgc_kernels.h"
#include "dgc_stage.cuh"

namespace dgc {
namespace {

// The 1D tables of every order, in constant memory: every thread reads the same
// entry at the same time, so the FMAs take them as constant-bank operands with no
// load instruction (filled by quad_tables_to_constant at mesh upload).
constexpr int kQuadTabMax = 2 * 10 * 7 + 2 * 7;   // m <= 10 points, n <= 7 modes (k <= 6)
__constant__ float kQuadTab32[7][kQuadTabMax];
__constant__ double kQuadTab64[7][kQuadTabMax];

template <int K, typename T>
__device__ __forceinline__ T qtab(int j) {
  if constexpr (sizeof(T) == 4)
    return kQuadTab32[K][j];
  else
    return kQuadTab64[K][j];
}

template <int K>
struct QuadDims {
  static constexpr int n = K + 1;             // 1D modes
  static constexpr int N = n * n;
  static constexpr int m = (3 * K) / 2 + 1;   // Gauss points per direction
  static constexpr int QV = m * m;
  // table blob: L [m][n] | Dl [m][n] | E [2][n]
  static constexpr int oL = 0, oD = m * n, oE = 2 * m * n, size = 2 * m * n + 2 * n;
};

template <int K, typename T>
__global__ void __launch_bounds__(128) stage_quad_kernel(StageArgs a) {
  using Q = QuadDims<K>;
  constexpr int n = Q::n, N = Q::N, m = Q::m, QV = Q::QV;
  auto L = [](int j) { return qtab<K, T>(Q::oL + j); };
  auto Dl = [](int j) { return qtab<K, T>(Q::oD + j); };
  auto E0 = [](int j) { return qtab<K, T>(Q::oE + j); };
  auto E1 = [](int j) { return qtab<K, T>(Q::oE + n + j); };

  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2L * a.E) return;
  const int e = (int)(t >> 1), c = (int)(t & 1);
  const long E = a.E;
  const double* __restrict__ vin_e = a.vin + ((long)e * 2 + c) * N;
  const T* __restrict__ Uw = static_cast<const T*>(a.Uw);
  const T* __restrict__ Fw = static_cast<const T*>(a.Fw);

  // FP32 inside an RK sequence: the FP32 copy of the stage input, so that neither
  // the own nor the neighbours' coefficients go through FP64 -> FP32 conversions
  // (they run on the FP64 pipe, 1/64 of the FP32 rate on this part)
  const float* __restrict__ v32 = sizeof(T) == 4 ? a.vin32 : nullptr;
  T w[N], r[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    w[i] = v32 ? (T)v32[((long)e * 2 + c) * N + i] : (T)vin_e[i];
    r[i] = (T)0;
  }

  // ---- volume ------------------------------------------------------------------
#pragma unroll 1
  for (int p = 0; p < m; ++p) {
    T tb[n], P0[n], P1[n];
#pragma unroll
    for (int b = 0; b < n; ++b) {
      T acc = (T)0;
#pragma unroll
      for (int aa = 0; aa < n; ++aa) acc += w[aa * n + b] * L(p * n + aa);
      tb[b] = acc;
      P0[b] = (T)0;
      P1[b] = (T)0;
    }
#pragma unroll
    for (int q = 0; q < m; ++q) {
      T W = (T)0;
#pragma unroll
      for (int b = 0; b < n; ++b) W += tb[b] * L(q * n + b);
      const int pq = p * m + q;
      const T f0 = Uw[(long)(pq * 2) * E + e] * W;
      const T f1 = Uw[(long)(pq * 2 + 1) * E + e] * W;
#pragma unroll
      for (int b = 0; b < n; ++b) {
        P0[b] += f0 * L(q * n + b);
        P1[b] += f1 * Dl(q * n + b);
      }
    }
#pragma unroll
    for (int aa = 0; aa < n; ++aa) {
      const T la = L(p * n + aa), da = Dl(p * n + aa);
#pragma unroll
      for (int b = 0; b < n; ++b) r[aa * n + b] -= da * P0[b] + la * P1[b];
    }
  }
  static_assert(QV == m * m, "tensor rule");

  // ---- facets -------------------------------------------------------------------
  // facet f: 0 eta = 0, 1 xi = 1, 2 eta = 1, 3 xi = 0; parameter xi (0, 2) or eta (1, 3)
  // (unrolled: the direction of every contraction is known at compile time)
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const bool along_xi = (f & 1) == 0;
    // the basis at the normal coordinate 0 (f = 0, 3) or 1 (f = 1, 2)
    auto Ef = [f](int j) { return (f == 0 || f == 3) ? qtab<K, T>(Q::oE + j) : qtab<K, T>(Q::oE + n + j); };
    T to[n], tn[n], ph[n];
#pragma unroll
    for (int j = 0; j < n; ++j) {
      T acc = (T)0;
#pragma unroll
      for (int l = 0; l < n; ++l) acc += (along_xi ? w[j * n + l] : w[l * n + j]) * Ef(l);
      to[j] = acc;
      tn[j] = (T)0;
      ph[j] = (T)0;
    }
    const int code = checked_code(a.nbr[(long)e * 4 + f], 3, a.E, a.status);
    if (code >= 0) {
      const int ne = code >> 3, fn = code & 3;
      const bool rev = (code & 4) != 0;
      const bool nxi = (fn & 1) == 0;
      const int oEn = Q::oE + ((fn == 0 || fn == 3) ? 0 : n);   // runtime facet of the neighbour
      const double* __restrict__ wn = a.vin + ((long)ne * 2 + c) * N;
#pragma unroll
      for (int j = 0; j < n; ++j) {
        T acc = (T)0;
#pragma unroll
        for (int l = 0; l < n; ++l) {
          const int i2 = nxi ? j * n + l : l * n + j;
          acc += (v32 ? (T)v32[((long)ne * 2 + c) * N + i2] : (T)wn[i2]) * qtab<K, T>(oEn + l);
        }
        tn[j] = (rev && (j & 1)) ? -acc : acc;
      }
    }
#pragma unroll
    for (int q = 0; q < m; ++q) {
      T o = (T)0, nb = (T)0;
#pragma unroll
      for (int j = 0; j < n; ++j) {
        o += to[j] * L(q * n + j);
        nb += tn[j] * L(q * n + j);
      }
      const T fw = Fw[(long)(f * m + q) * E + e];
      const T val = fw * (fw >= (T)0 ? o : nb);
#pragma unroll
      for (int j = 0; j < n; ++j) ph[j] += val * L(q * n + j);
    }
#pragma unroll
    for (int j = 0; j < n; ++j)
#pragma unroll
      for (int l = 0; l < n; ++l) {
        if (along_xi)
          r[j * n + l] += ph[j] * Ef(l);
        else
          r[l * n + j] += ph[j] * Ef(l);
      }
  }

  // ---- epilogue: RK stage combination in FP64 ------------------------------------
  double* vout_e = a.vout + ((long)e * 2 + c) * N;
  const double* vn_e = a.vn ? a.vn + ((long)e * 2 + c) * N : nullptr;
#pragma unroll
  float* out32 = a.vout32 ? a.vout32 + ((long)e * 2 + c) * N : nullptr;
  for (int i = 0; i < N; ++i) {
    double x = a.beta * vin_e[i] - a.gamma * (double)r[i];
    if (vn_e) x += a.alpha * vn_e[i];
    vout_e[i] = x;
    if (out32) out32[i] = (float)x;
  }
}

template <int K, typename T>
cudaError_t launch_quad_t(const StageArgs* ap, cudaStream_t stream) {
  if (!ap) return cudaSuccess;
  const StageArgs& a = *ap;
  constexpr int BLOCK = 128;
  const long work = 2L * a.E;
  const int grid = (int)((work + BLOCK - 1) / BLOCK);
  if (grid == 0) return cudaSuccess;
  stage_quad_kernel<K, T><<<grid, BLOCK, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t quad_tables_to_constant(int K, const std::vector<double>& tab) {
  if (K < 1 || K > 6 || (int)tab.size() > kQuadTabMax) return cudaErrorInvalidValue;
  std::vector<float> t32(tab.begin(), tab.end());
  cudaError_t err = cudaMemcpyToSymbol(kQuadTab64, tab.data(), tab.size() * sizeof(double),
                                       (size_t)K * kQuadTabMax * sizeof(double));
  if (err != cudaSuccess) return err;
  return cudaMemcpyToSymbol(kQuadTab32, t32.data(), t32.size() * sizeof(float), (size_t)K * kQuadTabMax * sizeof(float));
}

cudaError_t launch_stage_quad(int K, bool fp32, const StageArgs* a, cudaStream_t s) {
  switch (K) {
#define DGC_CASE(k) \
  case k: return fp32 ? launch_quad_t<k, float>(a, s) : launch_quad_t<k, double>(a, s);
    DGC_CASE(1) DGC_CASE(2) DGC_CASE(3) DGC_CASE(4) DGC_CASE(5) DGC_CASE(6)
#undef DGC_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dgc
