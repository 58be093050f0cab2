// Tensor-core RK stage kernel for tetrahedra (k = 1..4): steps a3-a7 of the
// upwind DG operator with both dense contractions on tcgen05 (split BF16x3
// operands, FP32 accumulation in TMEM) and the FP64 stage combination.
//
// On the reference simplex the stage residual of element T, component c, is
//   r_{c,i} = sum_q sum_d u_d(xi_q) w_c(xi_q) G[(d,q), i]
//           + sum_f sum_m Ef[f][m][i] phi_f[m],
//   G[(d,q), i] = -w_q d_d psi^_i(xi_q),  u = u^ / det J (contravariant Piola,
//   the diagonal mass |det J| folded in, Sec. 2.3), and the facet projection
//   phi_f[m] = sum_q Qt[q][m] Fw_f(q) w^_c(q) of the upwind flux, Fw the frozen
//   reference flux (1/det J) w^f_q (u^ . -grad lambda_f), w^ the own trace where
//   Fw >= 0 and the neighbour's otherwise (zero on inflow boundary facets).
//
// One persistent CTA per SM, 544 threads in three roles that work on
// different tiles at the same time:
//   volume warps 0-7 (two threads per GEMM row): write the tile's state and
//     wind operands into TMEM, then per chunk of 16 volume points read the
//     evaluated state and wind (GEMM A), exchange the wind components of an
//     element by warp shuffles, and write the products u_d w_c, split into
//     BF16 pieces, into TMEM as the A operand of GEMM B;
//   facet warps 8-15 (two threads per row, facets 2h, 2h + 1): the upwind
//     facet terms of a tile on CUDA cores from the facet traces of the stage
//     input (the own ones and the neighbour's, written by the previous stage)
//     while its volume part runs, then the epilogue once GEMM B has finished:
//     the increment, in the last stage of a substep the FP64 accumulation, and
//     the facet traces of the stage output;
//   warp 16: one thread issues every MMA and bulk copy (table chunks through
//     a ring of shared-memory slots, the tile's facet flux block).
// Two TMEM buffers each for the GEMM A results, the GEMM B operands and the
// GEMM B chunk partials (summed by the volume warps, round to nearest) let the
// volume warps run a tile ahead of the facet warps.  Every
// mbarrier wait is bounded; a timeout sets bit 1 of the status word, every
// role stops at its next check, in-flight copies and MMAs are drained and TMEM
// is released.
#pragma once

#include <cuda_runtime.h>

#include "dgc_stage_tc.cuh"
#include "dgc_tc.cuh"
#include "dgc_tc3_layout.h"

namespace dgc {

namespace tc3impl {

// named barrier of the 256 facet-warp threads
__device__ __forceinline__ void fw_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// the three BF16 pieces of NK values into TMEM columns col, col + NKC, col + 2 NKC
template <int NK, int NKC>
__device__ __forceinline__ void put3_tmem(uint32_t taddr, const float* x) {
#pragma unroll
  for (int k8 = 0; k8 < NK; k8 += 8) {
    uint32_t hw[4], mw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) tcimpl::split3_bf16x2(x[k8 + 2 * j], x[k8 + 2 * j + 1], hw[j], mw[j], lw[j]);
    tc::tmem_st4(taddr + k8 / 2, hw[0], hw[1], hw[2], hw[3]);
    tc::tmem_st4(taddr + NKC + k8 / 2, mw[0], mw[1], mw[2], mw[3]);
    tc::tmem_st4(taddr + 2 * NKC + k8 / 2, lw[0], lw[1], lw[2], lw[3]);
  }
}

}  // namespace tc3impl

template <int K>
__global__ void __launch_bounds__(544, 1) stage_tc3_kernel(StageTcArgs a) {
  using L = TcLayout3D<K>;
  constexpr int N = L::N, NFM = L::NFM, QF = L::QF, NK = L::NK, NKC = L::NKC, NR = L::NR, NCH = L::NCH;
  constexpr int NP4 = L::NP4, NFM4 = L::NFM4, EPT = L::EPT, SLOTS = L::SLOTS;
  extern __shared__ __align__(1024) unsigned char smb[];
  unsigned char* ring = smb + L::oRing;
  const float* fwt = reinterpret_cast<const float*>(smb + L::oFwt);
  float* fws = reinterpret_cast<float*>(smb + L::oFws);
  float* phis = reinterpret_cast<float*>(smb + L::oPhi);
  float* xs = reinterpret_cast<float*>(smb + L::oXs);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smb + L::oBar);
  uint64_t* bar_tab = bars + 0;       // [4] table chunk landed
  uint64_t* bar_tfree = bars + 4;     // [4] table slot free (GEMM B of its chunk done)
  uint64_t* bar_ops = bars + 8;       // operands of a tile written (8 volume warps)
  uint64_t* bar_afree = bars + 9;     // last GEMM A of a tile done: operands free
  uint64_t* bar_x = bars + 10;        // [2] GEMM A results ready
  uint64_t* bar_xfree = bars + 12;    // [2] GEMM A results read (8 volume warps)
  uint64_t* bar_p = bars + 14;        // [2] GEMM B operands written (8 volume warps)
  uint64_t* bar_pfree = bars + 16;    // [2] GEMM B done with its operands
  uint64_t* bar_r = bars + 18;        // the tile's residual summed into cRf (8 volume warps)
  uint64_t* bar_rfree = bars + 20;    // the residual read (8 facet warps)
  uint64_t* bar_ftab = bars + 22;     // facet tables landed
  uint64_t* bar_fws = bars + 23;      // [2] facet flux block of a tile landed
  uint64_t* bar_fwsfree = bars + 25;  // [2] facet flux block read (8 facet warps)
  uint64_t* bar_fin = bars + 27;      // every MMA of the CTA done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 28);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 29);
  volatile int* fw_stop = reinterpret_cast<volatile int*>(bars + 30);

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int ntiles = (a.E + EPT - 1) / EPT;
  const int nmy = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const float* vf_in = a.vf;
  const float* tr_in = a.trin;

  if (t == 0) {
    for (int i = 0; i < 4; ++i) {
      tc::mbar_init(bar_tab + i, 1);
      tc::mbar_init(bar_tfree + i, 1);
    }
    tc::mbar_init(bar_ops, 8);
    tc::mbar_init(bar_afree, 1);
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(bar_x + i, 1);
      tc::mbar_init(bar_xfree + i, 8);
      tc::mbar_init(bar_p + i, 8);
      tc::mbar_init(bar_pfree + i, 1);
      tc::mbar_init(bar_r + i, 8);
      tc::mbar_init(bar_rfree + i, 8);
      tc::mbar_init(bar_fws + i, 1);
      tc::mbar_init(bar_fwsfree + i, 8);
    }
    tc::mbar_init(bar_ftab, 1);
    tc::mbar_init(bar_fin, 1);
    *abort_flag = 0;
    *fw_stop = 0;
    tc::mbar_fence_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, L::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;

  if (warp == 16) {
    // ============================ issuer ======================================
    if (lane == 0) {
      const unsigned char* chunks = reinterpret_cast<const unsigned char*>(a.blob);
      const uint32_t ring_s = tc::smem_u32(ring);
      const int total = nmy * NCH;   // chunk uses of this CTA
      int ld = 0, lw = 0;            // table loads issued / waited (ring)
      int fws_ld[2] = {0, 0};        // flux block loads issued per buffer
      bool ok = true;
      auto fail = [&]() {
        ok = false;
        *abort_flag = 1;
      };
      auto load_chunk = [&](int Lx) {   // table chunk use Lx into its slot
        const int s = L::RESIDENT ? Lx : Lx % SLOTS;
        tc::mbar_arrive_expect_tx(bar_tab + s, L::CH_BYTES);
        tc::bulk_g2s(ring + (size_t)s * L::CH_BYTES, chunks + (size_t)(Lx % NCH) * L::CH_BYTES, L::CH_BYTES,
                     bar_tab + s);
      };
      auto load_fws = [&](int itl) {
        const int b = itl & 1;
        const int tile = blockIdx.x + itl * gridDim.x;
        tc::mbar_arrive_expect_tx(bar_fws + b, L::FWS * 4);
        tc::bulk_g2s(fws + b * L::FWS, a.fw3 + (size_t)tile * L::FWS, L::FWS * 4, bar_fws + b);
        ++fws_ld[b];
      };
      auto prefetch_tile = [&](int itl) {   // a tile's streamed inputs toward L2
        const int tile = blockIdx.x + itl * gridDim.x;
        const uint32_t blk = (uint32_t)N * 128 * 4;
        tc::bulk_prefetch_l2(vf_in + (size_t)tile * N * 128, blk);
        tc::bulk_prefetch_l2(a.wcoef + (size_t)tile * N * 128, blk);
        if (a.din) tc::bulk_prefetch_l2(a.din + (size_t)tile * N * 128, blk);
        tc::bulk_prefetch_l2(tr_in + (size_t)tile * L::NF * NFM * 128, (uint32_t)L::NF * NFM * 128 * 4);
        if (a.mode == 1) tc::bulk_prefetch_l2(a.v + (size_t)tile * N * 128, 2 * blk);
      };
      tc::mbar_arrive_expect_tx(bar_ftab, L::FWT * 4);
      tc::bulk_g2s(const_cast<float*>(fwt), a.ftab, L::FWT * 4, bar_ftab);
      if (nmy > 0) {
        if (L::RESIDENT) {
          for (int j = 0; j < NCH; ++j) load_chunk(j);
          ld = NCH;
        } else {
          for (; ld < 2 && ld < total; ++ld) load_chunk(ld);
        }
        load_fws(0);
        prefetch_tile(0);
        if (nmy > 1) load_fws(1);
      }
      const uint32_t idA = tc::idesc_bf16(128, 16);
      const uint32_t idB = tc::idesc_bf16(128, NR);
      // products of pieces (A piece, B piece), smallest first (see the triangle kernel)
      constexpr int PA[6] = {1, 2, 0, 1, 0, 0}, PB[6] = {1, 0, 2, 0, 1, 0};

      auto gemm_b = [&](int gg) {   // the volume test contraction of chunk use gg, a fresh partial
        const int jj = gg % NCH, b = gg & 1;
        if (!tc::mbar_wait(bar_p + b, (gg >> 1) & 1)) return fail();
        tc::fence_after_sync();
        const int s = L::RESIDENT ? jj : gg % SLOTS;
        const uint32_t sb = ring_s + (uint32_t)s * L::CH_BYTES + L::oBG;
#pragma unroll
        for (int pr = 0; pr < 6; ++pr)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const uint32_t at = tbase + L::cP + b * L::PCOLS + (d * 3 + PA[pr]) * 8;
            const uint64_t bd = tc::smem_desc(sb + (uint32_t)(d * 3 + PB[pr]) * L::szBG, 128, L::SBO_G);
            tc::mma_bf16_ts(tbase + L::cRp + b * NR, at, bd, idB, (pr | d) != 0);
          }
        tc::mma_commit(bar_pfree + b);
        if (!L::RESIDENT) tc::mma_commit(bar_tfree + s);
      };

      for (int it = 0; it < nmy && ok; ++it) {
        if (it >= 2) {   // the flux block of this tile into the buffer tile it - 2 used
          if (!tc::mbar_wait(bar_fwsfree + (it & 1), ((it >> 1) - 1) & 1)) {
            fail();
            break;
          }
          load_fws(it);
        }
        if (it + 1 < nmy) prefetch_tile(it + 1);
        if (!tc::mbar_wait(bar_ops, it & 1)) {
          fail();
          break;
        }
        tc::fence_after_sync();
        for (int j = 0; j < NCH && ok; ++j) {
          const int g = it * NCH + j, b = g & 1;
          const int s = L::RESIDENT ? j : g % SLOTS;
          if (L::RESIDENT) {
            if (it == 0 && !tc::mbar_wait(bar_tab + s, 0)) {
              fail();
              break;
            }
          } else {
            if (!tc::mbar_wait(bar_tab + s, (g / SLOTS) & 1)) {
              fail();
              break;
            }
            lw = g + 1;
          }
          if (g >= 2 && !tc::mbar_wait(bar_xfree + b, ((g >> 1) - 1) & 1)) {
            fail();
            break;
          }
          tc::fence_after_sync();
          // ---- GEMM A: state and wind at the chunk's 16 volume points ----------------
          const uint32_t sa = ring_s + (uint32_t)s * L::CH_BYTES + L::oBA;
#pragma unroll 1
          for (int fld = 0; fld < 2; ++fld) {
            const uint32_t dcol = tbase + L::cX + b * L::XCOLS + fld * 16;
            const uint32_t acol = tbase + (fld ? L::cAw : L::cAs);
            uint32_t acc = 0;
#pragma unroll
            for (int pr = 0; pr < 6; ++pr)
#pragma unroll
              for (int ks = 0; ks < NK / 16; ++ks) {
                const uint64_t bd = tc::smem_desc(sa + (uint32_t)PB[pr] * L::szBA + ks * 256, 128, L::SBO_A);
                tc::mma_bf16_ts(dcol, acol + PA[pr] * NKC + ks * 8, bd, idA, acc);
                acc = 1;
              }
          }
          tc::mma_commit(bar_x + b);
          if (j == NCH - 1) tc::mma_commit(bar_afree);
          if (j >= 1) {
            gemm_b(g - 1);
            if (!ok) break;
          }
          // ---- ring: the chunk two uses ahead into the slot GEMM B(g - 2) has freed ------
          if (!L::RESIDENT && ld < total && ld <= g + 2) {
            const int s2 = ld % SLOTS;
            if (ld >= SLOTS && !tc::mbar_wait(bar_tfree + s2, ((ld / SLOTS) - 1) & 1)) {
              fail();
              break;
            }
            load_chunk(ld);
            ++ld;
          }
        }
        if (ok) gemm_b(it * NCH + NCH - 1);
      }
      // ---- drain: every MMA, then every copy still in flight ------------------------
      tc::mma_commit(bar_fin);
      tc::mbar_wait(bar_fin, 0);
      if (L::RESIDENT) {
        if (nmy > 0)
          for (int j = 0; j < NCH; ++j) tc::mbar_wait(bar_tab + j, 0);
      } else {
        for (int Lx = lw; Lx < ld; ++Lx) tc::mbar_wait(bar_tab + Lx % SLOTS, (Lx / SLOTS) & 1);
      }
      for (int b = 0; b < 2; ++b)
        if (fws_ld[b]) tc::mbar_wait(bar_fws + b, (fws_ld[b] - 1) & 1);
      tc::mbar_wait(bar_ftab, 0);
      if (!ok) atomicOr(a.status, 2);
    }
  } else if (warp < 8) {
    // ============================ volume warps ===================================
    const int r = t & 127, h = t >> 7;
    const int rg = r >> 5, ln = r & 31, sl = ln / 3, c = ln % 3;
    const uint32_t lb = tbase + ((uint32_t)(rg * 32) << 16);
    constexpr int NRH = NR / 2;                 // residual columns this thread sums
    const uint32_t rcol = (uint32_t)(h * NRH);
    float racc[NRH];
    bool ok = true;
    auto wait_all = [&](uint64_t* bar, uint32_t parity) -> bool {   // warp-uniform bounded wait
      const bool w = *abort_flag == 0 && tc::mbar_wait(bar, parity);
      if (__all_sync(0xffffffffu, w)) return true;
      *abort_flag = 1;
      ok = false;
      return false;
    };
    auto collect = [&](int gg) {   // add the partial of chunk use gg (GEMM B(gg) has completed)
#pragma unroll
      for (int c8 = 0; c8 < NRH; c8 += 8) {
        float v8[8];
        tc::tmem_ld8(lb + L::cRp + (gg & 1) * NR + rcol + c8, v8);
        tc::tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 8; ++u) racc[c8 + u] += v8[u];
      }
    };
    auto finish = [&](int itp) {   // the last partials of tile itp, then its residual to the facet warps
      for (int jj = NCH >= 2 ? NCH - 2 : 0; jj < NCH; ++jj) {
        const int gg = itp * NCH + jj;
        if (!wait_all(bar_pfree + (gg & 1), (gg >> 1) & 1)) return;
        tc::fence_after_sync();
        collect(gg);
      }
      if (itp >= 1 && !wait_all(bar_rfree, (itp - 1) & 1)) return;
      tc::fence_after_sync();
#pragma unroll
      for (int c4 = 0; c4 < NRH; c4 += 4)
        tc::tmem_st4(lb + L::cRf + rcol + c4, __float_as_uint(racc[c4]), __float_as_uint(racc[c4 + 1]),
                     __float_as_uint(racc[c4 + 2]), __float_as_uint(racc[c4 + 3]));
      tc::tmem_wait_st();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tcimpl::mbar_arrive(bar_r);
    };
    for (int it = 0; it < nmy && ok; ++it) {
      const int tile = blockIdx.x + it * gridDim.x;
      const int e = tile * EPT + rg * 10 + sl;
      const bool valid = ln < 30 && e < a.E;
      if (it >= 1 && !wait_all(bar_afree, (it - 1) & 1)) break;
      tc::fence_after_sync();
      // ---- the tile's operands: h = 0 the state component c, h = 1 the wind's ------
      {
        float x[NK];
#pragma unroll
        for (int i = 0; i < NK; ++i) x[i] = 0.f;
        if (valid) {
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const size_t ix = tc3_index(tile, i, r, N);
            x[i] = h == 0 ? vf_in[ix] + (a.din ? a.din[ix] : 0.f) : a.wcoef[ix];
          }
        }
        tc3impl::put3_tmem<NK, NKC>(lb + (h ? L::cAw : L::cAs), x);
      }
      tc::tmem_wait_st();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tcimpl::mbar_arrive(bar_ops);
      if (it >= 1) {
        finish(it - 1);
        if (!ok) break;
      }
#pragma unroll
      for (int i = 0; i < NRH; ++i) racc[i] = 0.f;
      for (int j = 0; j < NCH; ++j) {
        const int g = it * NCH + j, b = g & 1;
        if (!wait_all(bar_x + b, (g >> 1) & 1)) break;
        tc::fence_after_sync();
        // this thread's 8 points of the chunk: w_c and u_c there
        float wq[8], uq[8];
        tc::tmem_ld8(lb + L::cX + b * L::XCOLS + 8 * h, wq);
        tc::tmem_ld8(lb + L::cX + b * L::XCOLS + 16 + 8 * h, uq);
        tc::tmem_wait_ld();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tcimpl::mbar_arrive(bar_xfree + b);
        // the element's three wind components from its three rows (same warp)
        float pv[3][8];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int q = 0; q < 8; ++q) pv[d][q] = __shfl_sync(0xffffffffu, uq[q], 3 * sl + d) * wq[q];
        if (g >= 2) {   // GEMM B(g - 2) is done with P[b] and its partial
          if (!wait_all(bar_pfree + b, ((g - 2) >> 1) & 1)) break;
          tc::fence_after_sync();
          if (j >= 2) collect(g - 2);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          uint32_t hw[4], mw[4], lw[4];
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
            tcimpl::split3_bf16x2(pv[d][2 * jj], pv[d][2 * jj + 1], hw[jj], mw[jj], lw[jj]);
          const uint32_t pc = lb + L::cP + b * L::PCOLS + d * 24 + 4 * h;
          tc::tmem_st4(pc, hw[0], hw[1], hw[2], hw[3]);
          tc::tmem_st4(pc + 8, mw[0], mw[1], mw[2], mw[3]);
          tc::tmem_st4(pc + 16, lw[0], lw[1], lw[2], lw[3]);
        }
        tc::tmem_wait_st();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tcimpl::mbar_arrive(bar_p + b);
      }
    }
    if (ok && nmy > 0) finish(nmy - 1);
  } else {
    // ============================ facet warps ====================================
    const int ft = t - 256;
    const int r = ft & 127, h = ft >> 7;
    const int rg = r >> 5, ln = r & 31, sl = ln / 3, c = ln % 3;
    const int el = rg * 10 + sl;
    const uint32_t lb = tbase + ((uint32_t)(rg * 32) << 16);
    const float* Ef = fwt + L::oEf;   // [NF][NFM][NP4]
    const float* Qt = fwt + L::oQt;   // [QF][NFM4]
    constexpr int NH = (N + 1) / 2;   // coefficients per thread in the epilogue
    const int i0 = h * NH;
    bool ok = tc::mbar_wait(bar_ftab, 0);
    if (!ok) *abort_flag = 1;
    for (int it = 0; it < nmy; ++it) {
      if (ft == 0) *fw_stop = *abort_flag;
      tc3impl::fw_sync();
      if (*fw_stop) break;   // uniform over the facet warps
      const int tile = blockIdx.x + it * gridDim.x;
      const int e = tile * EPT + el;
      const bool valid = ln < 30 && e < a.E;
      const int b = it & 1;
      bool w = *abort_flag == 0 && tc::mbar_wait(bar_fws + b, (it >> 1) & 1);
      if (!w) *abort_flag = 1;
      const float* fwb = fws + b * L::FWS;
      // ---- upwind facet terms of facets 2h, 2h + 1 (CUDA cores, FP32) ----------------
      float phi[2][NFM];
#pragma unroll
      for (int ff = 0; ff < 2; ++ff) {
        const int f = 2 * h + ff;
        float to[NFM], tn[NFM];
        const int code = valid ? a.nbr[(size_t)e * 4 + f] : -1;
        const int ne = code >> 2, fn = code & 3;
        const int nrow = code >= 0 ? tc3_row(ne % EPT, c) : 0;
#pragma unroll
        for (int m = 0; m < NFM; ++m) {
          to[m] = valid ? tr_in[tc3_tr_index(tile, f, m, r, NFM)] : 0.f;
          tn[m] = code >= 0 ? tr_in[tc3_tr_index(ne / EPT, fn, m, nrow, NFM)] : 0.f;
          phi[ff][m] = 0.f;
        }
#pragma unroll 1
        for (int q = 0; q < QF; ++q) {
          const float fw = valid ? fwb[(f * QF + q) * EPT + el] : 0.f;
          float qq[NFM4];
#pragma unroll
          for (int m4 = 0; m4 < NFM4; m4 += 4) {
            const float4 y = *reinterpret_cast<const float4*>(Qt + q * NFM4 + m4);
            qq[m4] = y.x;
            qq[m4 + 1] = y.y;
            qq[m4 + 2] = y.z;
            qq[m4 + 3] = y.w;
          }
          float o0 = 0.f, o1 = 0.f, n0 = 0.f, n1 = 0.f;
#pragma unroll
          for (int m = 0; m < NFM; m += 2) {
            o0 += qq[m] * to[m];
            n0 += qq[m] * tn[m];
            if (m + 1 < NFM) {
              o1 += qq[m + 1] * to[m + 1];
              n1 += qq[m + 1] * tn[m + 1];
            }
          }
          const float val = fw * (fw >= 0.f ? o0 + o1 : n0 + n1);
#pragma unroll
          for (int m = 0; m < NFM; ++m) phi[ff][m] += qq[m] * val;
        }
      }
      __syncwarp();
      if (lane == 0) tcimpl::mbar_arrive(bar_fwsfree + b);
      // the projections into shared memory (free since the last barrier of the previous tile)
#pragma unroll
      for (int ff = 0; ff < 2; ++ff)
#pragma unroll
        for (int m = 0; m < NFM; ++m) phis[((2 * h + ff) * NFM + m) * 128 + r] = phi[ff][m];
      // ---- the tile's residual from GEMM B -------------------------------------------
      w = *abort_flag == 0 && tc::mbar_wait(bar_r, it & 1);
      if (!w) *abort_flag = 1;
      tc::fence_after_sync();
      constexpr int NG = (NH + 7) / 8 + 1;   // 8-column groups covering [i0, i0 + NH)
      float rr[NG * 8];
      const int g0 = i0 / 8;
#pragma unroll
      for (int gq = 0; gq < NG; ++gq)
        if ((g0 + gq) * 8 < NR) tc::tmem_ld8(lb + L::cRf + (g0 + gq) * 8, rr + 8 * gq);
      tc::tmem_wait_ld();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tcimpl::mbar_arrive(bar_rfree);
      tc3impl::fw_sync();
      // ---- epilogue on coefficients i0 .. i0 + NH - 1 -------------------------------
      float ri[NH];
#pragma unroll
      for (int ii = 0; ii < NH; ++ii) ri[ii] = rr[i0 - 8 * g0 + ii];
#pragma unroll 1
      for (int fm = 0; fm < L::NF * NFM; ++fm) {
        const float p = phis[fm * 128 + r];
        const float* Er = Ef + fm * NP4 + i0;
#pragma unroll
        for (int ii = 0; ii < NH; ++ii)
          if (i0 + ii < N) ri[ii] += Er[ii] * p;
      }
#pragma unroll
      for (int ii = 0; ii < NH; ++ii) {
        const int i = i0 + ii;
        if (i >= N) break;
        float x = 0.f;
        if (valid) {
          const size_t ix = tc3_index(tile, i, r, N);
          const float ed = a.din ? a.din[ix] : 0.f;
          const float inc = fmaf(a.p_hi, ed, fmaf(a.p_lo, ed, -fmaf(a.q_hi, ri[ii], a.q_lo * ri[ii])));
          if (a.mode == 0) {
            a.dout[ix] = inc;
            x = vf_in[ix] + inc;
          } else if (a.mode == 1) {
            const double xv = a.v[ix] + tc::f32_to_f64(inc);   // FP64 state accumulation
            a.v[ix] = xv;
            x = tc::f64_to_f32_rn(xv);
            a.vf_out[ix] = x;
          } else {
            a.v[ix] = tc::f32_to_f64(inc);
          }
        }
        xs[i * 128 + r] = x;
      }
      tc3impl::fw_sync();
      // ---- facet traces of the stage output, facets 2h, 2h + 1 -----------------------
      if (valid && a.mode != 2) {
        float xo[NP4];
#pragma unroll
        for (int i = 0; i < NP4; ++i) xo[i] = i < N ? xs[i * 128 + r] : 0.f;
#pragma unroll
        for (int ff = 0; ff < 2; ++ff) {
          const int f = 2 * h + ff;
#pragma unroll 1
          for (int m = 0; m < NFM; ++m) {
            const float* Er = Ef + (f * NFM + m) * NP4;
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int i4 = 0; i4 < NP4; i4 += 4) {
              const float4 y = *reinterpret_cast<const float4*>(Er + i4);
              s0 += y.x * xo[i4] + y.y * xo[i4 + 1];
              s1 += y.z * xo[i4 + 2] + y.w * xo[i4 + 3];
            }
            a.trout[tc3_tr_index(tile, f, m, r, NFM)] = s0 + s1;
          }
        }
      }
      tc3impl::fw_sync();   // phis and xs are reused by the next tile
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, L::TMEM_COLS);
}

// ABI layout [E][3][N] -> the tile-blocked rows (FP64 and FP32 copy) and the facet
// traces of the FP32 copy; padding rows and elements past E are written as zero
template <int K>
__global__ void __launch_bounds__(128) tc3_in_kernel(const double* __restrict__ v, double* __restrict__ vt,
                                                     float* __restrict__ vft, float* __restrict__ tr,
                                                     const float* __restrict__ ftab, int E) {
  using L = TcLayout3D<K>;
  constexpr int N = L::N, NFM = L::NFM, NP4 = L::NP4;
  const int tile = blockIdx.x, r = threadIdx.x;
  const int ln = r & 31, c = ln % 3;
  const int e = tile * L::EPT + (r >> 5) * 10 + ln / 3;
  const bool valid = ln < 30 && e < E;
  float x[NP4];
#pragma unroll
  for (int i = 0; i < NP4; ++i) x[i] = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double d = valid ? v[((size_t)e * 3 + c) * N + i] : 0.0;
    vt[tc3_index(tile, i, r, N)] = d;
    x[i] = tc::f64_to_f32_rn(d);
    vft[tc3_index(tile, i, r, N)] = x[i];
  }
  const float* Ef = ftab + L::oEf;
#pragma unroll 1
  for (int fm = 0; fm < L::NF * NFM; ++fm) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) s += Ef[fm * NP4 + i] * x[i];
    tr[tc3_tr_index(tile, fm / NFM, fm % NFM, r, NFM)] = s;
  }
}

// tile-blocked rows (FP64) -> ABI layout [E][3][N]
template <int K>
__global__ void __launch_bounds__(256) tc3_out_kernel(const double* __restrict__ vt, double* __restrict__ v, int E) {
  using L = TcLayout3D<K>;
  constexpr int N = L::N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)E * 3 * N) return;
  const int i = (int)(gid % N);
  const int c = (int)((gid / N) % 3);
  const int e = (int)(gid / (3 * N));
  v[gid] = vt[tc3_index(e / L::EPT, i, tc3_row(e % L::EPT, c), N)];
}

}  // namespace dgc
