// Tensor-core RK stage kernel for triangles: steps a3-a7 with the two dense
// contractions of the upwind DG operator on tcgen05 (kind::tf32, three-pass
// head/tail split, FP32 accumulation in TMEM) and the FP64 stage combination.
//
// Per tile of 128 elements (one CTA, 128 threads, thread t = element t =
// GEMM row t = TMEM lane t):
//   1. bulk copies (TMA) bring the table blob and the tile's wind
//      coefficients into shared memory; every thread loads its element's FP64
//      state and writes the head/tail TF32 operands of the state fields;
//   2. GEMM A (one issuing thread): state and wind evaluated at the volume
//      points, the wind also at the facet points (weights and 1/det J folded
//      into the wind's table and coefficients);
//   3. CUDA cores, per element: own and neighbour facet traces on the facet
//      basis (the neighbour's from its FP64 state), upwind selection at the
//      facet points by the sign of (1/det J) w_q (u^ . -grad lambda_f),
//      projection back onto the facet basis (Sec. 2.3 upwind flux);
//   4. GEMM B in K-chunks of 8 through a 4-slot shared-memory ring: the
//      threads produce -Uw w_c(xi_q) products and the facet projections, one
//      thread issues the MMAs as chunks fill;
//   5. epilogue: r from TMEM, vout = alpha vn + beta vin - gamma r in FP64.
// The kernel is persistent (two CTAs per SM loop over tiles): the tables are
// loaded once per CTA, the next tile's wind block is bulk-copied as soon as
// the staging buffer is free, and the next tile's FP64 state blocks are
// prefetched into L2.  Every mbarrier wait is bounded; a timeout sets bit 1
// of the status word and the CTA stops (TMEM is still released).
#pragma once

#include <cuda_runtime.h>

#include "dgc_tc.cuh"
#include "dgc_tc_layout.h"

namespace dgc {

struct StageTcArgs {
  const double* vin;    // [E][2][N]
  const double* vn;     // substep start state or null (alpha == 0); may equal vout
  double* vout;
  const float* wcoef;   // [E][2][NK] wind on the Dubiner basis, scaled by 1/det J
  const int* nbr;       // [E][3]
  const float* blob;    // TcLayout2D<K> table blob
  int* status;          // device status word
  int E;
  double alpha, beta, gamma;
};

namespace tcimpl {

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// head/tail TF32 split of an FP32 value
__device__ __forceinline__ void split(float x, float& h, float& t) {
  h = tc::to_tf32(x);
  t = tc::to_tf32(x - h);
}

template <int NCOL>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float* v) {
  static_assert(NCOL % 8 == 0, "TMEM loads in groups of 8 columns");
#pragma unroll
  for (int c = 0; c < NCOL; c += 8) tc::tmem_ld8(taddr + c, v + c);
  tc::tmem_wait_ld();
}

}  // namespace tcimpl

template <int K>
__global__ void __launch_bounds__(128, 1) stage_tc_kernel(StageTcArgs a) {
  using L = TcLayout2D<K>;
  constexpr int N = L::N, QV = L::QV, QF = L::QF, NFM = L::NFM, NF = L::NF, NK = L::NK;
  constexpr int NP4 = L::NP4, NFM4 = L::NFM4;
  extern __shared__ __align__(1024) float sm[];
  float* blob = sm;
  float* wst = sm + L::oWst;
  float* op = sm + L::oOp;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::SMEM_FLOATS);
  uint64_t* bar_tab = bars + 0;
  uint64_t* bar_w = bars + 1;
  uint64_t* bar_A = bars + 2;
  uint64_t* bar_B = bars + 3;
  uint64_t* full = bars + 4;                 // NSLOT
  uint64_t* empty = bars + 4 + L::NSLOT;     // NSLOT
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4 + 2 * L::NSLOT);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int ntiles = (a.E + 127) / 128;
  const bool vin_al = (reinterpret_cast<uintptr_t>(a.vin) & 15) == 0;
  const bool vn_al = a.vn && (reinterpret_cast<uintptr_t>(a.vn) & 15) == 0;
  auto tile_valid = [&](int tile) { return min(128, a.E - tile * 128); };
  auto prefetch_state = [&](int tile) {   // next tile's FP64 state blocks into L2
    const uint32_t bytes = (uint32_t)tile_valid(tile) * 2 * N * 8;
    if (vin_al) tc::bulk_prefetch_l2(a.vin + (size_t)tile * 128 * 2 * N, bytes);
    if (vn_al) tc::bulk_prefetch_l2(a.vn + (size_t)tile * 128 * 2 * N, bytes);
  };
  auto load_wind = [&](int tile) {        // tile's wind coefficients into the staging buffer
    const uint32_t bytes = (uint32_t)tile_valid(tile) * 2 * NK * 4;
    tc::mbar_arrive_expect_tx(bar_w, bytes);
    tc::bulk_g2s(wst, a.wcoef + (size_t)tile * 128 * 2 * NK, bytes, bar_w);
  };

  if (t == 0) {
    tc::mbar_init(bar_tab, 1);
    tc::mbar_init(bar_w, 1);
    tc::mbar_init(bar_A, 1);
    tc::mbar_init(bar_B, 1);
    for (int s = 0; s < L::NSLOT; ++s) {
      tc::mbar_init(full + s, 128);
      tc::mbar_init(empty + s, 1);
    }
    *abort_flag = 0;
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (t == 0) {
    tc::mbar_arrive_expect_tx(bar_tab, L::BLOB * 4);
    tc::bulk_g2s(blob, a.blob, L::BLOB * 4, bar_tab);
    load_wind(blockIdx.x);
    prefetch_state(blockIdx.x);
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, L::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);
  if (!tc::mbar_wait(bar_tab, 0)) *abort_flag = 1;
  const float* Ef = blob + L::oEf;   // [NF][NFM][NP4]
  const float* Qt = blob + L::oQt;   // [QF][NFM4]
  const uint32_t op_s = tc::smem_u32(op);
  const uint32_t bl_s = tc::smem_u32(blob);
  const uint32_t tb_s = tc::smem_u32(blob + L::oTB);
  uint32_t chunk_ctr = 0;

  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int e = tile * 128 + t;
    const bool valid = e < a.E;
    const int next = tile + gridDim.x;
    if (t == 0 && next < ntiles) prefetch_state(next);

    // ---- own FP64 state -> registers, state operands (head / tail) ---------------
    float w[2][NP4];
    {
      const double* vin_e = a.vin + (size_t)e * 2 * N;
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int i = 0; i < NP4; ++i) w[c][i] = (valid && i < N) ? (float)vin_e[c * N + i] : 0.f;
    }
    // op layout: field f (0,1 state; 2,3 wind) x part (0 head, 1 tail) x [128 x NK]
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int k4 = 0; k4 < NK; k4 += 4) {
        float h[4], tl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float x = (k4 + u < NP4) ? w[c][(k4 + u < NP4) ? k4 + u : 0] : 0.f;
          tcimpl::split(x, h[u], tl[u]);
        }
        const uint32_t o = tc::kmajor_off32(t, k4, L::LBO, L::SBO_NK) / 4;
        tc::st_shared_v4(op + (c * 2 + 0) * L::szOpA + o, h[0], h[1], h[2], h[3]);
        tc::st_shared_v4(op + (c * 2 + 1) * L::szOpA + o, tl[0], tl[1], tl[2], tl[3]);
      }
    // ---- wind operands from the staged coefficients --------------------------------
    if (*abort_flag == 0 && !tc::mbar_wait(bar_w, it & 1)) *abort_flag = 1;
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
      for (int k4 = 0; k4 < NK; k4 += 4) {
        float h[4], tl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float x = valid ? wst[(t * 2 + d) * NK + k4 + u] : 0.f;
          tcimpl::split(x, h[u], tl[u]);
        }
        const uint32_t o = tc::kmajor_off32(t, k4, L::LBO, L::SBO_NK) / 4;
        tc::st_shared_v4(op + ((2 + d) * 2 + 0) * L::szOpA + o, h[0], h[1], h[2], h[3]);
        tc::st_shared_v4(op + ((2 + d) * 2 + 1) * L::szOpA + o, tl[0], tl[1], tl[2], tl[3]);
      }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool run = *abort_flag == 0;
    if (t == 0 && run) {
      if (next < ntiles) load_wind(next);   // the staging buffer is free again
      // ---- GEMM A ------------------------------------------------------------------
      for (int f = 0; f < 4; ++f) {
        const bool wind = f >= 2;
        const uint32_t idesc = tc::idesc_tf32(128, wind ? L::NAW : L::NAS);
        const uint32_t dcol = wind ? L::cW + (f - 2) * L::NAW : L::cS + f * L::NAS;
        const uint32_t tab = bl_s + 4u * (wind ? L::oTAw : L::oTAs);
        const uint32_t tsz = 4u * (wind ? L::szTAw : L::szTAs);
        uint32_t acc = 0;
        for (int pass = 0; pass < 3; ++pass) {
          const uint32_t a_op = op_s + 4u * ((f * 2 + (pass == 2 ? 1 : 0)) * L::szOpA);
          const uint32_t b_op = tab + (pass == 1 ? tsz : 0u);
          for (int ks = 0; ks < NK / 8; ++ks) {
            const uint64_t ad = tc::smem_desc(a_op + ks * 2 * L::LBO, L::LBO, L::SBO_NK);
            const uint64_t bd = tc::smem_desc(b_op + ks * 2 * L::LBO, L::LBO, L::SBO_NK);
            tc::mma_tf32(tbase + dcol, ad, bd, idesc, acc);
            acc = 1;
          }
        }
      }
      tc::mma_commit(bar_A);
    }

    // ---- facet traces on the facet basis (CUDA cores) -----------------------------
    float town[2][NF][NFM], tnb[2][NF][NFM];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int code = valid ? a.nbr[(size_t)e * NF + f] : -1;
      float wn[2][NP4];
      if (code >= 0) {
        const double* src = a.vin + (size_t)(code >> 2) * 2 * N;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int i = 0; i < NP4; ++i) wn[c][i] = i < N ? (float)src[c * N + (i < N ? i : 0)] : 0.f;
      } else {
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int i = 0; i < NP4; ++i) wn[c][i] = 0.f;
      }
      const int fn = code >= 0 ? (code & 3) : 0;
#pragma unroll
      for (int m = 0; m < NFM; ++m) {
        const float4* eo = reinterpret_cast<const float4*>(Ef + (f * NFM + m) * NP4);
        const float4* en = reinterpret_cast<const float4*>(Ef + (fn * NFM + m) * NP4);
        float ao[2] = {0.f, 0.f}, an[2] = {0.f, 0.f};
#pragma unroll
        for (int i4 = 0; i4 < NP4 / 4; ++i4) {
          const float4 x = eo[i4], y = en[i4];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            ao[c] += x.x * w[c][4 * i4] + x.y * w[c][4 * i4 + 1] + x.z * w[c][4 * i4 + 2] + x.w * w[c][4 * i4 + 3];
            an[c] += y.x * wn[c][4 * i4] + y.y * wn[c][4 * i4 + 1] + y.z * wn[c][4 * i4 + 2] +
                     y.w * wn[c][4 * i4 + 3];
          }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          town[c][f][m] = ao[c];
          tnb[c][f][m] = an[c];
        }
      }
    }

    // ---- wait for GEMM A -------------------------------------------------------------
    if (run && *abort_flag == 0 && !tc::mbar_wait(bar_A, it & 1)) *abort_flag = 1;
    tc::fence_after_sync();
    __syncthreads();
    const bool run2 = *abort_flag == 0;

    // ---- upwind facet fluxes projected on the facet basis ---------------------------
    float phi[2][NF * NFM];
#pragma unroll
    for (int j = 0; j < NF * NFM; ++j) phi[0][j] = phi[1][j] = 0.f;
    if (run2) {
      constexpr int NFP = NF * QF;                   // facet points
      constexpr int c0 = QV / 8 * 8, skip = QV - c0;
      constexpr int NL = (skip + NFP + 7) / 8 * 8;
      float uf[2][NL];
#pragma unroll
      for (int d = 0; d < 2; ++d) tcimpl::tmem_load<NL>(lane_base + L::cW + d * L::NAW + c0, uf[d]);
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int q = 0; q < QF; ++q) {
          // (1/det J) w_q (u^ . -grad lambda_f): -grad lambda_0 = (1,1), _1 = (-1,0), _2 = (0,-1)
          const float u0 = uf[0][skip + f * QF + q], u1 = uf[1][skip + f * QF + q];
          const float fw = f == 0 ? u0 + u1 : (f == 1 ? -u0 : -u1);
          float qq[NFM4];
#pragma unroll
          for (int m4 = 0; m4 < NFM4; m4 += 4) {
            const float4 x = *reinterpret_cast<const float4*>(Qt + q * NFM4 + m4);
            qq[m4] = x.x;
            qq[m4 + 1] = x.y;
            qq[m4 + 2] = x.z;
            qq[m4 + 3] = x.w;
          }
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            float o = 0.f, nb = 0.f;
#pragma unroll
            for (int m = 0; m < NFM; ++m) {
              o += qq[m] * town[c][f][m];
              nb += qq[m] * tnb[c][f][m];
            }
            const float val = fw * (fw >= 0.f ? o : nb);
#pragma unroll
            for (int m = 0; m < NFM; ++m) phi[c][f * NFM + m] += qq[m] * val;
          }
        }
    }

    // ---- GEMM B: produce K-chunks into the slot ring, thread 0 issues ----------------
    const uint32_t idescB = tc::idesc_tf32(128, L::NB);
    float wq[2][8], uq[2][8];
#pragma unroll
    for (int j = 0; j < L::NCH; ++j) {
      if (!run2) break;
      const uint32_t g = chunk_ctr + j;
      const int s = (int)(g % L::NSLOT);
      const uint32_t use = g / L::NSLOT;
      if (use > 0 && *abort_flag == 0 && !tc::mbar_wait(empty + s, (use - 1) & 1)) *abort_flag = 1;
      float vals[2][8];
      if (j < L::NCHF) {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int idx = j * 8 + kk;
#pragma unroll
          for (int c = 0; c < 2; ++c) vals[c][kk] = idx < NF * NFM ? phi[c][idx < NF * NFM ? idx : 0] : 0.f;
        }
      } else {
        // volume chunk: K index 2 q + dd for q = 4 jv .. 4 jv + 3
        const int jv = j - L::NCHF;
        if ((jv & 1) == 0) {
          const int q0 = jv * 4;
#pragma unroll
          for (int c = 0; c < 2; ++c) tcimpl::tmem_load<8>(lane_base + L::cS + c * L::NAS + q0, wq[c]);
#pragma unroll
          for (int d = 0; d < 2; ++d) tcimpl::tmem_load<8>(lane_base + L::cW + d * L::NAW + q0, uq[d]);
        }
        const int qo = (jv & 1) * 4;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int ql = qo + kk / 2, d = kk & 1;
          const int q = jv * 4 + kk / 2;
#pragma unroll
          for (int c = 0; c < 2; ++c) vals[c][kk] = (q < QV && valid) ? -uq[d][ql] * wq[c][ql] : 0.f;
        }
      }
      float* slot = op + s * (2 * 2 * L::szChunk);
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int k4 = 0; k4 < 8; k4 += 4) {
          float h[4], tl[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) tcimpl::split(vals[c][k4 + u], h[u], tl[u]);
          const uint32_t o = tc::kmajor_off32(t, k4, L::LBO, L::SBO_CH) / 4;
          tc::st_shared_v4(slot + (c * 2 + 0) * L::szChunk + o, h[0], h[1], h[2], h[3]);
          tc::st_shared_v4(slot + (c * 2 + 1) * L::szChunk + o, tl[0], tl[1], tl[2], tl[3]);
        }
      tc::fence_proxy_async_smem();
      tcimpl::mbar_arrive(full + s);
      if (t == 0 && *abort_flag == 0) {
        if (!tc::mbar_wait(full + s, use & 1)) {
          *abort_flag = 1;
        } else {
          tc::fence_after_sync();
          const uint32_t sl = op_s + 4u * (s * 2 * 2 * L::szChunk);
          for (int c = 0; c < 2; ++c)
            for (int pass = 0; pass < 3; ++pass) {
              const uint32_t a_op = sl + 4u * ((c * 2 + (pass == 2 ? 1 : 0)) * L::szChunk);
              const uint32_t b_op = tb_s + (pass == 1 ? 4u * L::szTB : 0u) + j * 2 * L::LBO;
              tc::mma_tf32(tbase + L::cB + c * L::NB, tc::smem_desc(a_op, L::LBO, L::SBO_CH),
                           tc::smem_desc(b_op, L::LBO, L::SBO_KB), idescB, (j > 0 || pass > 0) ? 1u : 0u);
            }
          tc::mma_commit(empty + s);
          if (j == L::NCH - 1) tc::mma_commit(bar_B);
        }
      }
    }
    chunk_ctr += L::NCH;

    // ---- epilogue: FP64 stage combination ---------------------------------------------
    const double* vin_e = a.vin + (size_t)e * 2 * N;
    const double* vn_e = a.vn ? a.vn + (size_t)e * 2 * N : nullptr;
    if (valid) {   // pull this element's lines into L1 while the last MMAs finish
#pragma unroll
      for (int b = 0; b < 2 * N * 8; b += 128) {
        asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<const char*>(vin_e) + b));
        if (vn_e) asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<const char*>(vn_e) + b));
      }
    }
    if (run2 && *abort_flag == 0 && !tc::mbar_wait(bar_B, it & 1)) *abort_flag = 1;
    tc::fence_after_sync();
    __syncthreads();
    const bool fin = run2 && *abort_flag == 0;   // uniform after the barrier
    if (fin) {
      float r[2][L::NB];
#pragma unroll
      for (int c = 0; c < 2; ++c) tcimpl::tmem_load<L::NB>(lane_base + L::cB + c * L::NB, r[c]);
      if (valid) {
        double* vout_e = a.vout + (size_t)e * 2 * N;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int i = 0; i < N; ++i) {
            double x = a.beta * vin_e[c * N + i] - a.gamma * (double)r[c][i];
            if (vn_e) x += a.alpha * vn_e[c * N + i];
            vout_e[c * N + i] = x;
          }
      }
    } else {
      if (t == 0) atomicOr(a.status, 2);   // a bounded wait gave up: this CTA stops
      break;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, L::TMEM_COLS);
}

}  // namespace dgc
