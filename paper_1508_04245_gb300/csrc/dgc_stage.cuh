// Fused RK stage kernel: steps a3-a7 of the explicit upwind-DG convection
// step for one element per thread (or one element-component group).
//
// For element T with reference wind u^ (contravariant Piola) the upwind DG
// operator of Sec. 2.3 divided by the diagonal mass |det J| (Sec. 2.3,
// orthonormal basis) reads, on the reference simplex,
//
//   r_{c,i} = (1/det J) [ - sum_q w_q w_c(xi_q) (u^ . grad^ psi^_i)(xi_q)
//                         + sum_f sum_q w^f_q (u^ . -grad lambda_f) w^_c psi^_i ]
//
// where w^_c is the upwind trace: the element's own trace where the flux
// leaves T (sign of (1/det J)(u^ . -grad lambda_f) >= 0), the neighbour's
// trace otherwise, zero on inflow boundary facets.  The frozen wind enters
// only through Uw = (1/det J) w_q u^(xi_q) and Fw = (1/det J) w^f_q
// (u^ . -grad lambda_f)(xi_fq), prepared once per call.
//
// Facet traces go through the facet polynomial basis: the trace of psi^_i
// on facet f equals sum_m Ef[f][m][i] q_m exactly, and because every
// element orders its vertices by global id, both elements of a facet see the
// same facet parametrisation, so the neighbour's trace at facet point q is
// sum_m Qt[q][m] (Ef[f'] w')_m with no permutation.
//
// Epilogue (step a7): vout = alpha vn + beta vin + gamma L(vin), L = -r,
// accumulated in FP64.
#pragma once

#include <cuda_runtime.h>

#include "dgc_internal.h"

namespace dgc {

struct StageArgs {
  const double* vin;   // stage input [E][D][N]
  const double* vn;    // substep start state (null when alpha == 0); may equal vout
  double* vout;        // stage output
  const void* Uw;      // [QV*D][E]
  const void* Fw;      // [NF*QF][E]
  const int* nbr;      // [E][NF]: (neighbour << 2) | neighbour's local facet, or -1
  const void* tab;     // stage table blob (StageTab layout)
  int E;
  double alpha, beta, gamma;
};

template <int D, int K>
struct StageTab {
  using Dm = Dims<D, K>;
  static constexpr int pad(int n) { return (n + 3) / 4 * 4; }
  static constexpr int oB = 0;                                        // [QV][N]
  static constexpr int oG = pad(Dm::QV * Dm::N);                      // [QV][N][D]
  static constexpr int oE = oG + pad(Dm::QV * Dm::N * D);             // [NF][NFM][N]
  static constexpr int oQ = oE + pad(Dm::NF * Dm::NFM * Dm::N);       // [QF][NFM]
  static constexpr int size = oQ + pad(Dm::QF * Dm::NFM);
};

template <typename T, int D, int K>
constexpr bool stage_tab_in_smem() {
  return StageTab<D, K>::size * (int)sizeof(T) <= 200 * 1024;
}

// components handled by one thread
template <typename T, int D, int K>
constexpr int stage_cpt() {
  return (D == 2 && sizeof(T) == 4) ? 2 : 1;
}

// Threads per block: a per-(dim, order, precision) choice made by the autotuner
// (dgc_autotune) among kStageBlocks, the default until it runs.  Every element
// is computed by one thread independently of the block shape, so the choice
// changes the speed only, never a result.
constexpr int kStageBlocks[4] = {64, 128, 192, 256};
template <typename T, int D, int K>
constexpr int stage_block_default() {
  return D == 2 ? 128 : 256;
}
int stage_block_get(int D, int K, bool fp32);   // tuned value or 0

template <int D, int K, typename T, int CPT, bool SMEM>
__global__ void __launch_bounds__(256) stage_kernel(StageArgs a) {
  using Dm = Dims<D, K>;
  using TB = StageTab<D, K>;
  constexpr int N = Dm::N, QV = Dm::QV, QF = Dm::QF, NFM = Dm::NFM, NF = Dm::NF;
  constexpr int G = D / CPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const T* __restrict__ gtab = static_cast<const T*>(a.tab);
  const T* tab = gtab;
  if (SMEM) {
    T* st = reinterpret_cast<T*>(smem_raw);
    for (int j = threadIdx.x; j < TB::size; j += blockDim.x) st[j] = gtab[j];
    __syncthreads();
    tab = st;
  }
  const T* Bv = tab + TB::oB;
  const T* Gv = tab + TB::oG;
  const T* Ef = tab + TB::oE;
  const T* Qt = tab + TB::oQ;

  const long wi = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (wi >= (long)a.E * G) return;
  const int e = (int)(wi / G);
  const int c0 = (int)(wi % G) * CPT;
  const long E = a.E;
  const double* __restrict__ vin_e = a.vin + ((long)e * D + c0) * N;
  const T* __restrict__ Uw = static_cast<const T*>(a.Uw);
  const T* __restrict__ Fw = static_cast<const T*>(a.Fw);

  T w[CPT][N], r[CPT][N];
#pragma unroll
  for (int c = 0; c < CPT; ++c)
#pragma unroll
    for (int i = 0; i < N; ++i) {
      w[c][i] = (T)vin_e[c * N + i];
      r[c][i] = (T)0;
    }

  // ---- volume term: r -= sum_q sum_a Uw[q][a] w(xi_q) d_a psi_i(xi_q) ------
#pragma unroll 1
  for (int q = 0; q < QV; ++q) {
    const T* Bq = Bv + q * N;
    T wq[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) wq[c] = (T)0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const T b = Bq[i];
#pragma unroll
      for (int c = 0; c < CPT; ++c) wq[c] += b * w[c][i];
    }
    T p[CPT][D];
#pragma unroll
    for (int aa = 0; aa < D; ++aa) {
      const T u = Uw[(long)(q * D + aa) * E + e];
#pragma unroll
      for (int c = 0; c < CPT; ++c) p[c][aa] = u * wq[c];
    }
    const T* Gq = Gv + q * N * D;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int aa = 0; aa < D; ++aa) {
        const T g = Gq[i * D + aa];
#pragma unroll
        for (int c = 0; c < CPT; ++c) r[c][i] -= p[c][aa] * g;
      }
  }

  // ---- facet terms ----------------------------------------------------------
#pragma unroll 1
  for (int f = 0; f < NF; ++f) {
    const int code = a.nbr[(long)e * NF + f];
    const T* Eo = Ef + f * NFM * N;
    T to[CPT][NFM], tn[CPT][NFM], phi[CPT][NFM];
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
      for (int m = 0; m < NFM; ++m) {
        T acc = (T)0;
#pragma unroll
        for (int i = 0; i < N; ++i) acc += Eo[m * N + i] * w[c][i];
        to[c][m] = acc;
        tn[c][m] = (T)0;
        phi[c][m] = (T)0;
      }
    if (code >= 0) {
      const int ne = code >> 2, fn = code & 3;
      const T* En = Ef + fn * NFM * N;
      const double* __restrict__ wn = a.vin + ((long)ne * D + c0) * N;
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const T x = (T)wn[c * N + i];
#pragma unroll
          for (int m = 0; m < NFM; ++m) tn[c][m] += En[m * N + i] * x;
        }
    }
#pragma unroll 1
    for (int q = 0; q < QF; ++q) {
      const T fw = Fw[(long)(f * QF + q) * E + e];
      const T* Qq = Qt + q * NFM;
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        T o = (T)0, n = (T)0;
#pragma unroll
        for (int m = 0; m < NFM; ++m) {
          o += Qq[m] * to[c][m];
          n += Qq[m] * tn[c][m];
        }
        const T val = fw * (fw >= (T)0 ? o : n);
#pragma unroll
        for (int m = 0; m < NFM; ++m) phi[c][m] += Qq[m] * val;
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        T acc = (T)0;
#pragma unroll
        for (int m = 0; m < NFM; ++m) acc += Eo[m * N + i] * phi[c][m];
        r[c][i] += acc;
      }
  }

  // ---- epilogue: RK stage combination in FP64 --------------------------------
  double* vout_e = a.vout + ((long)e * D + c0) * N;
  const double* vn_e = a.vn ? a.vn + ((long)e * D + c0) * N : nullptr;
#pragma unroll
  for (int c = 0; c < CPT; ++c)
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double x = a.beta * vin_e[c * N + i] - a.gamma * (double)r[c][i];
      if (vn_e) x += a.alpha * vn_e[c * N + i];
      vout_e[c * N + i] = x;
    }
}

// a == nullptr: only set the kernel's shared-memory attribute (done before
// any stream capture, as attribute changes are not stream work).
template <int D, int K, typename T>
cudaError_t launch_stage_t(const StageArgs* ap, cudaStream_t stream) {
  constexpr int CPT = stage_cpt<T, D, K>();
  constexpr bool SMEM = stage_tab_in_smem<T, D, K>();
  const int tuned = stage_block_get(D, K, sizeof(T) == 4);
  const int BLOCK = tuned > 0 ? tuned : stage_block_default<T, D, K>();
  const size_t smem = SMEM ? StageTab<D, K>::size * sizeof(T) : 0;
  auto kern = stage_kernel<D, K, T, CPT, SMEM>;
  if (!ap) {
    if (smem > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
  }
  const StageArgs& a = *ap;
  const long work = (long)a.E * (D / CPT);
  const int grid = (int)((work + BLOCK - 1) / BLOCK);
  if (grid == 0) return cudaSuccess;
  kern<<<grid, BLOCK, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace dgc
