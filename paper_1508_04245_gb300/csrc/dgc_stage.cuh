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
  int* status = nullptr;   // [2] device status words (gather checks of the checked build)
  const void* tab;     // stage table blob (StageTab layout)
  int E;
  double alpha, beta, gamma;
  // curved triangles (null cid: none): the residual of element e with cid[e] >= 0 is
  // multiplied by its inverse mass block Minv[(i*N + j)*Ec + cid[e]] (T-typed), the
  // frozen wind of such an element carrying sign(det J) instead of 1/det J
  const int* cid = nullptr;
  const void* Minv = nullptr;
  int Ec = 0;
  // FP32 contraction of parallelograms inside an RK sequence: an FP32 copy of vin
  // (read instead of converting vin and the neighbours' coefficients) and the FP32
  // copy of vout to write; null outside such a sequence
  const float* vin32 = nullptr;
  float* vout32 = nullptr;
};

// Rows padded to multiples of 4 values (zero filled) so the kernel reads them in
// 16-byte-aligned groups of four.
template <int D, int K>
struct StageTab {
  using Dm = Dims<D, K>;
  static constexpr int pad(int n) { return (n + 3) / 4 * 4; }
  static constexpr int NP4 = pad(Dm::N), NFM4 = pad(Dm::NFM);
  static constexpr int oB = 0;                                        // [QV][NP4]
  static constexpr int oG = oB + Dm::QV * NP4;                        // [QV][D][NP4]
  static constexpr int oE = oG + Dm::QV * D * NP4;                    // [NF][NFM][NP4]
  static constexpr int oQ = oE + Dm::NF * Dm::NFM * NP4;              // [QF][NFM4]
  static constexpr int size = oQ + Dm::QF * NFM4;
};

// four consecutive table values from a 16-byte-aligned address
__device__ __forceinline__ void load4(const float* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double* o) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = a.x;
  o[1] = a.y;
  o[2] = b.x;
  o[3] = b.y;
}

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

template <int D, int K, typename T, int CPT, bool SMEM, bool CURVED>
__global__ void __launch_bounds__(256, 1) stage_kernel(StageArgs a) {
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

  // FP32 inside an RK sequence: the FP32 copy of the stage input, so that neither the
  // own nor the neighbours' coefficients go through FP64 -> FP32 conversions (those
  // run on the FP64 pipe, 1/64 of the FP32 rate on this part)
  const float* __restrict__ v32 = sizeof(T) == 4 ? a.vin32 : nullptr;
  T w[CPT][N], r[CPT][N];
#pragma unroll
  for (int c = 0; c < CPT; ++c)
#pragma unroll
    for (int i = 0; i < N; ++i) {
      w[c][i] = v32 ? (T)v32[((long)e * D + c0 + c) * N + i] : (T)vin_e[c * N + i];
      r[c][i] = (T)0;
    }

  // ---- volume term: r -= sum_q sum_a Uw[q][a] w(xi_q) d_a psi_i(xi_q) ------
  // Table rows are read four values at a time, except for FP32 tetrahedra with
  // k >= 4, where the wider unrolled form no longer fits the register file and
  // the one-value form is kept.
  constexpr int NP4 = TB::NP4, NFM4 = TB::NFM4;
  constexpr bool VEC = !(D == 3 && K >= 4 && sizeof(T) == 4);
#pragma unroll 1
  for (int q = 0; q < QV; ++q) {
    const T* Bq = Bv + q * NP4;
    T wq[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) wq[c] = (T)0;
    if constexpr (!VEC) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const T b = Bq[i];
#pragma unroll
        for (int c = 0; c < CPT; ++c) wq[c] += b * w[c][i];
      }
    } else
#pragma unroll
    for (int i4 = 0; i4 < NP4; i4 += 4) {
      T b[4];
      load4(Bq + i4, b);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i4 + u < N ? i4 + u : N - 1;
        if (i4 + u < N)
#pragma unroll
          for (int c = 0; c < CPT; ++c) wq[c] += b[u] * w[c][i];
      }
    }
    T p[CPT][D];
#pragma unroll
    for (int aa = 0; aa < D; ++aa) {
      const T uu = Uw[(long)(q * D + aa) * E + e];
#pragma unroll
      for (int c = 0; c < CPT; ++c) p[c][aa] = uu * wq[c];
    }
    const T* Gq = Gv + q * D * NP4;
    if constexpr (!VEC) {
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int aa = 0; aa < D; ++aa) {
          const T g = Gq[aa * NP4 + i];
#pragma unroll
          for (int c = 0; c < CPT; ++c) r[c][i] -= p[c][aa] * g;
        }
    } else
#pragma unroll
    for (int aa = 0; aa < D; ++aa)
#pragma unroll
      for (int i4 = 0; i4 < NP4; i4 += 4) {
        T g[4];
        load4(Gq + aa * NP4 + i4, g);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i4 + u < N ? i4 + u : N - 1;
          if (i4 + u < N)
#pragma unroll
            for (int c = 0; c < CPT; ++c) r[c][i] -= p[c][aa] * g[u];
        }
      }
  }

  // ---- facet terms ----------------------------------------------------------
#pragma unroll 1
  for (int f = 0; f < NF; ++f) {
    const int code = checked_code(a.nbr[(long)e * NF + f], 2, a.E, a.status);
    const T* Eo = Ef + f * NFM * NP4;
    T to[CPT][NFM], tn[CPT][NFM], phi[CPT][NFM];
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
      for (int m = 0; m < NFM; ++m) {
        T acc = (T)0;
        if constexpr (!VEC) {
#pragma unroll
          for (int i = 0; i < N; ++i) acc += Eo[m * NP4 + i] * w[c][i];
        } else
#pragma unroll
        for (int i4 = 0; i4 < NP4; i4 += 4) {
          T ev[4];
          load4(Eo + m * NP4 + i4, ev);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (i4 + u < N) acc += ev[u] * w[c][i4 + u < N ? i4 + u : N - 1];
        }
        to[c][m] = acc;
        tn[c][m] = (T)0;
        phi[c][m] = (T)0;
      }
    if (code >= 0) {
      const int ne = code >> 2, fn = code & 3;
      const T* En = Ef + fn * NFM * NP4;
      const double* __restrict__ wn = a.vin + ((long)ne * D + c0) * N;
      const float* __restrict__ wn32 = v32 ? v32 + ((long)ne * D + c0) * N : nullptr;
      if constexpr (!VEC) {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            const T x = wn32 ? (T)wn32[c * N + i] : (T)wn[c * N + i];
#pragma unroll
            for (int m = 0; m < NFM; ++m) tn[c][m] += En[m * NP4 + i] * x;
          }
      } else
#pragma unroll
      for (int i4 = 0; i4 < NP4; i4 += 4) {
        T x[CPT][4];
#pragma unroll
        for (int c = 0; c < CPT; ++c)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = i4 + u < N ? i4 + u : 0;
            x[c][u] = i4 + u < N ? (wn32 ? (T)wn32[c * N + i] : (T)wn[c * N + i]) : (T)0;
          }
#pragma unroll
        for (int m = 0; m < NFM; ++m) {
          T ev[4];
          load4(En + m * NP4 + i4, ev);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (i4 + u < N)
#pragma unroll
              for (int c = 0; c < CPT; ++c) tn[c][m] += ev[u] * x[c][u];
        }
      }
    }
#pragma unroll 1
    for (int q = 0; q < QF; ++q) {
      const T fw = Fw[(long)(f * QF + q) * E + e];
      T qq[NFM4];
#pragma unroll
      for (int m4 = 0; m4 < NFM4; m4 += 4) load4(Qt + q * NFM4 + m4, qq + m4);
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        T o = (T)0, n = (T)0;
#pragma unroll
        for (int m = 0; m < NFM; ++m) {
          o += qq[m] * to[c][m];
          n += qq[m] * tn[c][m];
        }
        const T val = fw * (fw >= (T)0 ? o : n);
#pragma unroll
        for (int m = 0; m < NFM; ++m) phi[c][m] += qq[m] * val;
      }
    }
    if constexpr (!VEC) {
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          T acc = (T)0;
#pragma unroll
          for (int m = 0; m < NFM; ++m) acc += Eo[m * NP4 + i] * phi[c][m];
          r[c][i] += acc;
        }
    } else
#pragma unroll
    for (int i4 = 0; i4 < NP4; i4 += 4) {
      T acc[CPT][4];
#pragma unroll
      for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[c][u] = (T)0;
#pragma unroll
      for (int m = 0; m < NFM; ++m) {
        T ev[4];
        load4(Eo + m * NP4 + i4, ev);
#pragma unroll
        for (int c = 0; c < CPT; ++c)
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[c][u] += ev[u] * phi[c][m];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i4 + u < N)
#pragma unroll
          for (int c = 0; c < CPT; ++c) r[c][i4 + u < N ? i4 + u : N - 1] += acc[c][u];
    }
  }

  // ---- epilogue: RK stage combination in FP64 --------------------------------
  double* vout_e = a.vout + ((long)e * D + c0) * N;
  const double* vn_e = a.vn ? a.vn + ((long)e * D + c0) * N : nullptr;
  if constexpr (CURVED) {
    // curved element: the residual times its inverse mass block (remark on curved
    // elements, Sec. 2.4), one output row at a time
    const int ci = a.cid[e];
    if (ci >= 0) {
      const T* __restrict__ Mi = static_cast<const T*>(a.Minv) + ci;
#pragma unroll 1
      for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          T acc = (T)0;
#pragma unroll
          for (int j = 0; j < N; ++j) acc += Mi[(long)(i * N + j) * a.Ec] * r[c][j];
          double x = a.beta * vin_e[c * N + i] - a.gamma * (double)acc;
          if (vn_e) x += a.alpha * vn_e[c * N + i];
          vout_e[c * N + i] = x;
          if (a.vout32) a.vout32[((long)e * D + c0) * N + c * N + i] = (float)x;
        }
      }
      return;
    }
  }
#pragma unroll
  for (int c = 0; c < CPT; ++c)
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double x = a.beta * vin_e[c * N + i] - a.gamma * (double)r[c][i];
      if (vn_e) x += a.alpha * vn_e[c * N + i];
      vout_e[c * N + i] = x;
      if (a.vout32) a.vout32[((long)e * D + c0) * N + c * N + i] = (float)x;
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
  // the curved-element variant exists for triangles only
  auto kern_c = stage_kernel<D, K, T, CPT, SMEM, D == 2>;
  auto kern = stage_kernel<D, K, T, CPT, SMEM, false>;
  if (!ap) {
    if (smem > 48 * 1024) {
      cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err == cudaSuccess && D == 2)
        err = cudaFuncSetAttribute(kern_c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      return err;
    }
    return cudaSuccess;
  }
  const StageArgs& a = *ap;
  if (D == 2 && a.cid) kern = kern_c;
  const long work = (long)a.E * (D / CPT);
  const int grid = (int)((work + BLOCK - 1) / BLOCK);
  if (grid == 0) return cudaSuccess;
  kern<<<grid, BLOCK, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace dgc
