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
// One persistent CTA per SM, 640 threads in four roles that work on
// different tiles at the same time:
//   volume warps 0-7 (two threads per GEMM row): write the tile's state
//     operand into TMEM, then per chunk of 16 volume points read the evaluated
//     state (GEMM A) and the wind there (a shared-memory ring), and write the
//     products u_d w_c, split into BF16 pieces on the row's grid for the chunk
//     (both threads of a row form all 48 products and take the same largest
//     magnitude), into TMEM as the A operand of GEMM B;
//   facet warps 8-15 (two threads per row, facets 2h, 2h + 1): the upwind
//     facet terms of a tile on CUDA cores from the facet traces of the stage
//     input (the own ones and the neighbour's, written by the previous stage)
//     while its volume part runs, then the epilogue once GEMM B has finished:
//     the increment, in the last stage of a substep the FP64 accumulation, and
//     the facet traces of the stage output;
//   warp 16: the bulk copies (table chunks and the chunks' wind blocks through
//     rings of shared-memory slots, the tiles' facet flux blocks, L2 prefetch
//     of the next tile), issued as their slots free up;
//   warps 17-19: one thread each issues the MMAs of GEMM A (even, odd chunks)
//     and of GEMM B -- a single issuing thread sustains only about one
//     tcgen05.mma per 50 cycles, so independent chains come from separate warps.
// Two TMEM buffers each for the GEMM A results, the GEMM B operands and the
// GEMM B head partials (summed by the volume warps, round to nearest) let the
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

// the grid 2^(e - 8) of a group of values whose largest magnitude is mx = f 2^e
// (f in [0.5, 1)): heads rint(x / g) g are then integers of at most 256 grid
// units, exact in BF16 (g = 1 for an all-zero group)
__device__ __forceinline__ void grid_of(float mx, float& g, float& gi) {
  int ex = 0;
  frexpf(mx, &ex);
  ex = ex < -100 ? -100 : ex;
  g = mx > 0.f ? ldexpf(1.f, ex - 8) : 1.f;
  gi = mx > 0.f ? ldexpf(1.f, 8 - ex) : 1.f;
}

// two values split exactly into BF16 pieces: the head on the grid g, the remainder
// (exact in FP32) rounded into a middle and a low piece; lower value in the low half
__device__ __forceinline__ void split_grid(float a, float b, float g, float gi, uint32_t& hw, uint32_t& mw,
                                           uint32_t& lw) {
  const float ha = rintf(a * gi) * g, hb = rintf(b * gi) * g;
  hw = tcimpl::bf16x2_rn(ha, hb);   // exact
  const float ra = a - ha, rb = b - hb;   // exact
  mw = tcimpl::bf16x2_rn(ra, rb);
  lw = tcimpl::bf16x2_rn(ra - __uint_as_float(mw << 16), rb - __uint_as_float(mw & 0xFFFF0000u));
}

// the three BF16 pieces of NK values into TMEM columns col, col + NKC, col + 2 NKC,
// heads on the grid of the largest |x|; of the groups of 8 values the caller
// writes those of parity part (the two threads of a row share the work)
template <int NK, int NKC>
__device__ __forceinline__ void put3_tmem(uint32_t taddr, const float* x, int part) {
  float mx = 0.f;
#pragma unroll
  for (int k = 0; k < NK; ++k) mx = fmaxf(mx, fabsf(x[k]));
  float g, gi;
  grid_of(mx, g, gi);
#pragma unroll
  for (int k8 = 0; k8 < NK; k8 += 8) {
    if (((k8 >> 3) & 1) != part) continue;
    uint32_t hw[4], mw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) split_grid(x[k8 + 2 * j], x[k8 + 2 * j + 1], g, gi, hw[j], mw[j], lw[j]);
    tc::tmem_st4(taddr + k8 / 2, hw[0], hw[1], hw[2], hw[3]);
    tc::tmem_st4(taddr + NKC + k8 / 2, mw[0], mw[1], mw[2], mw[3]);
    tc::tmem_st4(taddr + 2 * NKC + k8 / 2, lw[0], lw[1], lw[2], lw[3]);
  }
}

}  // namespace tc3impl

template <int K>
__global__ void __launch_bounds__(640, 1) stage_tc3_kernel(StageTcArgs a) {
  using L = TcLayout3D<K>;
  constexpr int N = L::N, NFM = L::NFM, QF = L::QF, NK = L::NK, NKC = L::NKC, NR = L::NR, NCH = L::NCH;
  constexpr int NP4 = L::NP4, NFM4 = L::NFM4, EPT = L::EPT, SLOTS = L::SLOTS;
  extern __shared__ __align__(1024) unsigned char smb[];
  unsigned char* ring = smb + L::oRing;
  const float* fwt = reinterpret_cast<const float*>(smb + L::oFwt);
  float* fws = reinterpret_cast<float*>(smb + L::oFws);
  float* phis = reinterpret_cast<float*>(smb + L::oPhi);
  float* xs = reinterpret_cast<float*>(smb + L::oXs);
  float* wnd = reinterpret_cast<float*>(smb + L::oWnd);
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
  uint64_t* bar_wnd = bars + 31;      // [4] wind block of a chunk landed
  uint64_t* bar_wfree = bars + 35;    // [4] wind slot consumed (8 volume warps)
  const uint32_t poll = a.poll ? a.poll : tc::kWaitPolls;   // polls per bounded wait

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int ntiles = (a.E + EPT - 1) / EPT;
  const int nmy = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const float* vf_in = a.vf;
  const float* tr_in = a.trin;

  if (t == 0) {
    for (int i = 0; i < 4; ++i) {
      tc::mbar_init(bar_tab + i, 1);
      tc::mbar_init(bar_tfree + i, 2);   // GEMM A and GEMM B of the slot's chunk
    }
    tc::mbar_init(bar_ops, 8);
    tc::mbar_init(bar_afree, NCH >= 2 ? 2 : 1);   // both GEMM A issuers, when both have chunks in a tile
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
    for (int i = 0; i < L::WSLOTS; ++i) {
      tc::mbar_init(bar_wnd + i, 1);
      tc::mbar_init(bar_wfree + i, 8);
    }
    tc::mbar_init(bar_ftab, 1);
    tc::mbar_init(bar_fin, 3);   // the three MMA-issuing threads
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

  if (warp >= 16) {
    // ============ warp 16: bulk copies; 17, 18: GEMM A; 19: GEMM B ===============
    // (one tcgen05.mma issuing thread sustains one MMA per ~50 cycles, so the GEMM A
    // MMAs of even and odd chunks, which use separate TMEM buffers, come from two
    // warps; GEMM B has half as many MMAs)
    if (lane == 0) {
      const int role = warp - 16;
      const unsigned char* chunks = reinterpret_cast<const unsigned char*>(a.blob);
      const uint32_t ring_s = tc::smem_u32(ring);
      const int total = nmy * NCH;   // chunk uses of this CTA
      bool ok = true;
      auto fail = [&]() {
        ok = false;
        *abort_flag = 1;
      };
      auto slot = [&](int g) { return L::RESIDENT ? g % NCH : g % SLOTS; };
      auto tab_ready = [&](int g) {   // the table chunk of use g has landed
        return tc::mbar_wait(bar_tab + slot(g), L::RESIDENT ? 0u : (uint32_t)((g / SLOTS) & 1), poll);
      };
      // products of pieces (A piece, B piece), smallest first (see the triangle kernel)
      constexpr int PA[6] = {1, 2, 0, 1, 0, 0}, PB[6] = {1, 0, 2, 0, 1, 0};
      if (role == 0) {
        // ---- producer: table chunks and wind blocks through their rings, the tiles'
        //      facet flux blocks, L2 prefetch of a tile's streamed inputs; each copy is
        //      issued as soon as its slot is free (polled, so that no full ring holds
        //      up the others) --------------------------------------------------------
        int ld = 0;      // table loads issued
        int wl = 0;      // wind loads issued
        int fl = 0;      // flux block loads issued (tiles)
        auto load_chunk = [&](int Lx) {
          const int s2 = slot(Lx);
          tc::mbar_arrive_expect_tx(bar_tab + s2, L::CH_BYTES);
          tc::bulk_g2s(ring + (size_t)s2 * L::CH_BYTES, chunks + (size_t)(Lx % NCH) * L::CH_BYTES, L::CH_BYTES,
                       bar_tab + s2);
        };
        auto load_wind = [&](int g) {
          const int s2 = g % L::WSLOTS;
          const int tile = blockIdx.x + (g / NCH) * gridDim.x;
          tc::mbar_arrive_expect_tx(bar_wnd + s2, L::WCH * 4);
          tc::bulk_g2s(wnd + (size_t)s2 * L::WCH, a.wq3 + ((size_t)tile * NCH + g % NCH) * L::WCH, L::WCH * 4,
                       bar_wnd + s2);
        };
        auto load_fws = [&](int itl) {
          const int b = itl & 1;
          const int tile = blockIdx.x + itl * gridDim.x;
          tc::mbar_arrive_expect_tx(bar_fws + b, L::FWS * 4);
          tc::bulk_g2s(fws + b * L::FWS, a.fw3 + (size_t)tile * L::FWS, L::FWS * 4, bar_fws + b);
        };
        auto prefetch_tile = [&](int itl) {
          const int tile = blockIdx.x + itl * gridDim.x;
          const uint32_t blk = (uint32_t)N * 128 * 4;
          tc::bulk_prefetch_l2(vf_in + (size_t)tile * N * 128, blk);
          if (a.din) tc::bulk_prefetch_l2(a.din + (size_t)tile * N * 128, blk);
          tc::bulk_prefetch_l2(tr_in + (size_t)tile * L::NF * 128 * NFM4, (uint32_t)L::NF * 128 * NFM4 * 4);
          if (a.mode == 1) tc::bulk_prefetch_l2(a.v + (size_t)tile * N * 128, 2 * blk);
        };
        const int nmy_ld = a.stall ? 0 : nmy;   // the stall hook issues no copy at all
        if (!a.stall) {
          tc::mbar_arrive_expect_tx(bar_ftab, L::FWT * 4);
          tc::bulk_g2s(const_cast<float*>(fwt), a.ftab, L::FWT * 4, bar_ftab);
        }
        if (nmy_ld > 0) {
          const int first = L::RESIDENT ? NCH : (total < SLOTS ? total : SLOTS);
          for (; ld < first; ++ld) load_chunk(ld);
        }
        const int total_ld = nmy_ld * NCH;
        const int ldn = L::RESIDENT ? ld : total_ld;   // table loads in all
        uint32_t idle = 0;
        while (ok && (fl < nmy_ld || wl < total_ld || ld < ldn)) {
          bool moved = false;
          // the flux block of tile fl into the buffer tile fl - 2 has released
          if (fl < nmy_ld && (fl < 2 || tc::mbar_try_wait(bar_fwsfree + (fl & 1), ((fl >> 1) - 1) & 1))) {
            load_fws(fl);
            prefetch_tile(fl);
            ++fl;
            moved = true;
          }
          // the wind block of chunk use wl into the slot use wl - WSLOTS has released
          if (wl < total_ld &&
              (wl < L::WSLOTS || tc::mbar_try_wait(bar_wfree + wl % L::WSLOTS, ((wl / L::WSLOTS) - 1) & 1))) {
            load_wind(wl);
            ++wl;
            moved = true;
          }
          // the table chunk of use ld into the slot use ld - SLOTS has released
          if (ld < ldn && tc::mbar_try_wait(bar_tfree + ld % SLOTS, ((ld / SLOTS) - 1) & 1)) {
            load_chunk(ld);
            ++ld;
            moved = true;
          }
          if (moved) {
            idle = 0;
          } else if (++idle > poll || *abort_flag) {
            fail();
          } else {
            __nanosleep(200);   // nothing to issue yet: leave the issue slots to the compute warps
          }
        }
        // drain: the copies still in flight land before the CTA exits
        if (L::RESIDENT) {
          if (nmy_ld > 0)
            for (int j = 0; j < NCH; ++j) tc::mbar_wait(bar_tab + j, 0, poll);
        } else {
          for (int Lx = ld - SLOTS > 0 ? ld - SLOTS : 0; Lx < ld; ++Lx)
            tc::mbar_wait(bar_tab + Lx % SLOTS, (Lx / SLOTS) & 1, poll);
        }
        for (int g = wl - L::WSLOTS > 0 ? wl - L::WSLOTS : 0; g < wl; ++g)
          tc::mbar_wait(bar_wnd + g % L::WSLOTS, (g / L::WSLOTS) & 1, poll);
        for (int itl = fl - 2 > 0 ? fl - 2 : 0; itl < fl; ++itl) tc::mbar_wait(bar_fws + (itl & 1), (itl >> 1) & 1, poll);
        if (!a.stall) tc::mbar_wait(bar_ftab, 0, poll);
        if (a.stall) fail();
      } else if (role <= 2) {
        // ---- GEMM A of the chunk uses of parity p: the state at 16 volume points --------
        const int p = role - 1;
        const uint32_t idA = tc::idesc_bf16(128, 16);
        int cur = -1;   // the tile whose operands this issuer has seen written
        for (int g = p; g < total && ok; g += 2) {
          const int it = g / NCH;
          if (it != cur) {
            if (!tc::mbar_wait(bar_ops, it & 1, poll)) {
              fail();
              break;
            }
            cur = it;
          }
          if (!tab_ready(g) || (g >= 2 && !tc::mbar_wait(bar_xfree + p, ((g >> 1) - 1) & 1, poll))) {
            fail();
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = ring_s + (uint32_t)slot(g) * L::CH_BYTES + L::oBA;
          {
            // [hh | corr]: the grid-aligned head x head sum (exact), then the five correction
            // products smallest first
            const uint32_t dcol = tbase + L::cX + p * L::XCOLS;
            const uint32_t acol = tbase + L::cAs;
            const uint64_t bd0 = tc::smem_desc(sa, 128, L::SBO_A);
#pragma unroll
            for (int ks = 0; ks < NK / 16; ++ks)   // the address field of a descriptor is address / 16
              tc::mma_bf16_ts(dcol, acol + ks * 8, bd0 + (uint64_t)((ks * 256) >> 4), idA, ks != 0);
#pragma unroll
            for (int pr = 0; pr < 5; ++pr)
#pragma unroll
              for (int ks = 0; ks < NK / 16; ++ks)
                tc::mma_bf16_ts(dcol + 16, acol + PA[pr] * NKC + ks * 8,
                                bd0 + (uint64_t)((PB[pr] * L::szBA + ks * 256) >> 4), idA, (pr | ks) != 0);
          }
          tc::mma_commit(bar_x + p);
          if (!L::RESIDENT) tc::mma_commit(bar_tfree + slot(g));
          if (g + 2 >= (it + 1) * NCH) tc::mma_commit(bar_afree);   // this issuer's last chunk of the tile
        }
        tc::mma_commit(bar_fin);
        tc::mbar_wait(bar_fin, 0, poll);
      } else {
        // ---- GEMM B of every chunk use: the head x head sum (exact) into a fresh partial,
        //      the correction products into the tile's correction accumulator ---------
        const uint32_t idB = tc::idesc_bf16(128, NR);
        for (int g = 0; g < total && ok; ++g) {
          const int p = g & 1;
          if (!tab_ready(g) || !tc::mbar_wait(bar_p + p, (g >> 1) & 1, poll)) {
            fail();
            break;
          }
          tc::fence_after_sync();
          const uint64_t bd0 = tc::smem_desc(ring_s + (uint32_t)slot(g) * L::CH_BYTES + L::oBG, 128, L::SBO_G);
          const uint32_t pa = tbase + L::cP + p * L::PCOLS;
#pragma unroll
          for (int d = 0; d < 3; ++d)
            tc::mma_bf16_ts(tbase + L::cRh + p * NR, pa + d * 24, bd0 + (uint64_t)((d * 3 * L::szBG) >> 4), idB,
                            d != 0);
          const bool first = g % NCH == 0;   // the tile's first chunk starts the correction sum
#pragma unroll
          for (int pr = 0; pr < 5; ++pr)
#pragma unroll
            for (int d = 0; d < 3; ++d)
              tc::mma_bf16_ts(tbase + L::cRc, pa + (d * 3 + PA[pr]) * 8,
                              bd0 + (uint64_t)(((d * 3 + PB[pr]) * L::szBG) >> 4), idB, !first || (pr | d) != 0);
          tc::mma_commit(bar_pfree + p);
          if (!L::RESIDENT) tc::mma_commit(bar_tfree + slot(g));
        }
        tc::mma_commit(bar_fin);
        tc::mbar_wait(bar_fin, 0, poll);
      }
      if (!ok) atomicOr(a.status, 2);
    }
  } else if (warp < 8) {
    // ============================ volume warps ===================================
    const int r = t & 127, h = t >> 7;
    const int rg = r >> 5, ln = r & 31;
    const int elw = rg * 10 + (ln < 30 ? ln / 3 : 0);   // element whose wind the row reads
    const uint32_t lb = tbase + ((uint32_t)(rg * 32) << 16);
    constexpr int NRH = NR / 2;                 // residual columns this thread sums
    const uint32_t rcol = (uint32_t)(h * NRH);
    float racc[NRH];
    bool ok = true;
    auto wait_all = [&](uint64_t* bar, uint32_t parity) -> bool {   // warp-uniform bounded wait
      const bool w = *abort_flag == 0 && tc::mbar_wait(bar, parity, poll);
      if (__all_sync(0xffffffffu, w)) return true;
      *abort_flag = 1;
      ok = false;
      return false;
    };
    auto add_cols = [&](uint32_t col) {   // racc += TMEM columns col + rcol .. + NRH - 1 of the row
#pragma unroll
      for (int c8 = 0; c8 < NRH; c8 += 8) {
        float v8[8];
        tc::tmem_ld8(lb + col + rcol + c8, v8);
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
        add_cols(L::cRh + (gg & 1) * NR);
      }
      add_cols(L::cRc);   // the tile's correction sum (complete with its last chunk)
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
      const int e = tile * EPT + rg * 10 + ln / 3;
      const bool valid = ln < 30 && e < a.E;
      if (it >= 1 && !wait_all(bar_afree, (it - 1) & 1)) break;
      tc::fence_after_sync();
      // ---- the tile's state operand (both threads of a row write half of its columns) ---
      {
        float x[NK];
#pragma unroll
        for (int i = 0; i < NK; ++i) x[i] = 0.f;
        if (valid) {
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const size_t ix = tc3_index(tile, i, r, N);
            x[i] = vf_in[ix] + (a.din ? a.din[ix] : 0.f);
          }
        }
        tc3impl::put3_tmem<NK, NKC>(lb + L::cAs, x, h);
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
        const int g = it * NCH + j, b = g & 1, ws = g % L::WSLOTS;
        if (!wait_all(bar_x + b, (g >> 1) & 1)) break;
        tc::fence_after_sync();
        // the state at the chunk's 16 points: this thread's 8 (wo) and the partner's (wx)
        float wo[8], wx[8];
        {
          float ho[8], co[8], hx[8], cx[8];
          const uint32_t xb = lb + L::cX + b * L::XCOLS;
          tc::tmem_ld8(xb + 8 * h, ho);
          tc::tmem_ld8(xb + 16 + 8 * h, co);
          tc::tmem_ld8(xb + 8 * (1 - h), hx);
          tc::tmem_ld8(xb + 16 + 8 * (1 - h), cx);
          tc::tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            wo[q] = ho[q] + co[q];
            wx[q] = hx[q] + cx[q];
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tcimpl::mbar_arrive(bar_xfree + b);
        if (!wait_all(bar_wnd + ws, (g / L::WSLOTS) & 1)) break;
        // the products u_d w_c at this thread's points, and the largest |u_d w_c| of the
        // row over all 48 of the chunk (both threads of the row form the same products)
        float pv[3][8];
        float mx = 0.f;
        {
          const float* wb = wnd + ws * L::WCH + elw;
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              pv[d][q] = wb[(d * 16 + 8 * h + q) * EPT] * wo[q];
              const float px = wb[(d * 16 + 8 * (1 - h) + q) * EPT] * wx[q];
              mx = fmaxf(mx, fmaxf(fabsf(pv[d][q]), fabsf(px)));
            }
        }
        if (g >= 2) {   // GEMM B(g - 2) is done with P[b] and its partial
          if (!wait_all(bar_pfree + b, ((g - 2) >> 1) & 1)) break;
          tc::fence_after_sync();
          if (j >= 2) add_cols(L::cRh + b * NR);
        }
        float gs, gi;
        tc3impl::grid_of(mx, gs, gi);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          uint32_t hw[4], mw[4], lw[4];
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
            tc3impl::split_grid(pv[d][2 * jj], pv[d][2 * jj + 1], gs, gi, hw[jj], mw[jj], lw[jj]);
          const uint32_t pc = lb + L::cP + b * L::PCOLS + d * 24 + 4 * h;
          tc::tmem_st4(pc, hw[0], hw[1], hw[2], hw[3]);
          tc::tmem_st4(pc + 8, mw[0], mw[1], mw[2], mw[3]);
          tc::tmem_st4(pc + 16, lw[0], lw[1], lw[2], lw[3]);
        }
        tc::tmem_wait_st();
        tc::fence_before_sync();
        __syncwarp();
        // every value read from the wind slot has been consumed into TMEM by now, so the
        // next bulk copy into the slot cannot overtake a read still in flight
        if (lane == 0) {
          tcimpl::mbar_arrive(bar_p + b);
          tcimpl::mbar_arrive(bar_wfree + ws);
        }
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
    // coefficients of this thread in the epilogue: a 4-aligned half, [i0, i0 + NH)
    constexpr int NH = ((N + 1) / 2 + 3) / 4 * 4;
    const int i0 = h * NH;
    bool ok = tc::mbar_wait(bar_ftab, 0, poll);
    if (!ok) *abort_flag = 1;
    for (int it = 0; it < nmy; ++it) {
      if (ft == 0) *fw_stop = *abort_flag;
      tc3impl::fw_sync();
      if (*fw_stop) break;   // uniform over the facet warps
      const int tile = blockIdx.x + it * gridDim.x;
      const int e = tile * EPT + el;
      const bool valid = ln < 30 && e < a.E;
      const int b = it & 1;
      bool w = *abort_flag == 0 && tc::mbar_wait(bar_fws + b, (it >> 1) & 1, poll);
      if (!w) *abort_flag = 1;
      const float* fwb = fws + b * L::FWS;
      // ---- upwind facet terms of facets 2h, 2h + 1 (CUDA cores, FP32, packed pairs) ------
      // own and neighbour traces of a facet as pairs of modes (NFM4 / 2 pairs each)
      constexpr int NP2 = NFM4 / 2;
#pragma unroll
      for (int ff = 0; ff < 2; ++ff) {
        const int f = 2 * h + ff;
        unsigned long long to2[NP2], tn2[NP2];
        {
          const int code = valid ? checked_code(a.nbr[(size_t)e * 4 + f], 2, a.E, a.status) : -1;
          const ulonglong2* po = reinterpret_cast<const ulonglong2*>(tr_in + tc3_tr_index(tile, f, 0, r, NFM4));
          const ulonglong2* pn = reinterpret_cast<const ulonglong2*>(
              tr_in + tc3_tr_index(code >= 0 ? (code >> 2) / EPT : 0, code & 3, 0,
                                   code >= 0 ? tc3_row((code >> 2) % EPT, c) : 0, NFM4));
#pragma unroll
          for (int j = 0; j < NP2 / 2; ++j) {
            const ulonglong2 x = valid ? po[j] : make_ulonglong2(0ull, 0ull);
            const ulonglong2 y = code >= 0 ? pn[j] : make_ulonglong2(0ull, 0ull);
            to2[2 * j] = x.x;
            to2[2 * j + 1] = x.y;
            tn2[2 * j] = y.x;
            tn2[2 * j + 1] = y.y;
          }
        }
        unsigned long long ph2[NP2];
#pragma unroll
        for (int j = 0; j < NP2; ++j) ph2[j] = 0ull;
#pragma unroll 4
        for (int q = 0; q < QF; ++q) {
          const float fw = valid ? fwb[(f * QF + q) * EPT + el] : 0.f;
          const ulonglong2* Qr = reinterpret_cast<const ulonglong2*>(Qt + q * NFM4);
          unsigned long long qq2[NP2];
#pragma unroll
          for (int j = 0; j < NP2 / 2; ++j) {
            const ulonglong2 y = Qr[j];
            qq2[2 * j] = y.x;
            qq2[2 * j + 1] = y.y;
          }
          // two partial sums per trace: dependency chains of NP2 / 2 packed FMAs
          unsigned long long oa = 0ull, ob = 0ull, na = 0ull, nb = 0ull;
#pragma unroll
          for (int j = 0; j < NP2; j += 2) {
            oa = tc::f2_fma(qq2[j], to2[j], oa);
            na = tc::f2_fma(qq2[j], tn2[j], na);
            if (j + 1 < NP2) {
              ob = tc::f2_fma(qq2[j + 1], to2[j + 1], ob);
              nb = tc::f2_fma(qq2[j + 1], tn2[j + 1], nb);
            }
          }
          float oal, oah, obl, obh, nal, nah, nbl, nbh;
          tc::f2_unpack(oa, oal, oah);
          tc::f2_unpack(ob, obl, obh);
          tc::f2_unpack(na, nal, nah);
          tc::f2_unpack(nb, nbl, nbh);
          const float val = fw * (fw >= 0.f ? (oal + obl) + (oah + obh) : (nal + nbl) + (nah + nbh));
          const unsigned long long vv = tc::f2_pack(val, val);
#pragma unroll
          for (int j = 0; j < NP2; ++j) ph2[j] = tc::f2_fma(qq2[j], vv, ph2[j]);
        }
        // the projection into shared memory (free since the last barrier of the previous tile)
#pragma unroll
        for (int j = 0; j < NP2; ++j) {
          float lo, hi;
          tc::f2_unpack(ph2[j], lo, hi);
          if (2 * j < NFM) phis[(f * NFM + 2 * j) * 128 + r] = lo;
          if (2 * j + 1 < NFM) phis[(f * NFM + 2 * j + 1) * 128 + r] = hi;
        }
      }
      __syncwarp();
      if (lane == 0) tcimpl::mbar_arrive(bar_fwsfree + b);
      // ---- the tile's residual, this thread's coefficients --------------------------
      w = *abort_flag == 0 && tc::mbar_wait(bar_r, it & 1, poll);
      if (!w) *abort_flag = 1;
      tc::fence_after_sync();
      float ri[NH];
#pragma unroll
      for (int c4 = 0; c4 < NH; c4 += 4)
        if (i0 + c4 < NR) tc::tmem_ld4(lb + L::cRf + i0 + c4, ri + c4);
      tc::tmem_wait_ld();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tcimpl::mbar_arrive(bar_rfree);
      tc3impl::fw_sync();
      // ---- epilogue on coefficients i0 .. i0 + NH - 1 -------------------------------
      {
        unsigned long long r2[NH / 2];
#pragma unroll
        for (int j = 0; j < NH / 2; ++j) r2[j] = tc::f2_pack(ri[2 * j], ri[2 * j + 1]);
#pragma unroll 4   // loads of later iterations overlap the FMAs of earlier ones
        for (int fm = 0; fm < L::NF * NFM; ++fm) {
          const float pv = phis[fm * 128 + r];
          const unsigned long long pp = tc::f2_pack(pv, pv);
          const ulonglong2* Er = reinterpret_cast<const ulonglong2*>(Ef + fm * NP4 + i0);
#pragma unroll
          for (int j4 = 0; j4 < NH / 4; ++j4) {
            if (i0 + 4 * j4 >= NP4) break;
            const ulonglong2 y = Er[j4];
            r2[2 * j4] = tc::f2_fma(y.x, pp, r2[2 * j4]);
            r2[2 * j4 + 1] = tc::f2_fma(y.y, pp, r2[2 * j4 + 1]);
          }
        }
#pragma unroll
        for (int j = 0; j < NH / 2; ++j) tc::f2_unpack(r2[j], ri[2 * j], ri[2 * j + 1]);
      }
      // in two halves: every global load of a half is issued before its stores, so
      // the loads do not wait one after another behind possibly aliasing stores
      constexpr int NQ = NH / 2;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        float ed[NQ], xb[NQ];
        double xd[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int i = i0 + hh * NQ + q;
          ed[q] = 0.f;
          xb[q] = 0.f;
          xd[q] = 0.0;
          if (valid && i < N) {
            const size_t ix = tc3_index(tile, i, r, N);
            if (a.din) ed[q] = a.din[ix];
            if (a.mode == 0) xb[q] = vf_in[ix];
            if (a.mode == 1) xd[q] = a.v[ix];
          }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int ii = hh * NQ + q, i = i0 + ii;
          if (i >= N) break;
          float x = 0.f;
          if (valid) {
            const size_t ix = tc3_index(tile, i, r, N);
            const float inc = fmaf(a.p_hi, ed[q], fmaf(a.p_lo, ed[q], -fmaf(a.q_hi, ri[ii], a.q_lo * ri[ii])));
            if (a.mode == 0) {
              a.dout[ix] = inc;
              x = xb[q] + inc;
            } else if (a.mode == 1) {
              const double xv = xd[q] + tc::f32_to_f64(inc);   // FP64 state accumulation
              a.v[ix] = xv;
              x = tc::f64_to_f32_rn(xv);
              a.vf_out[ix] = x;
            } else {
              a.v[ix] = tc::f32_to_f64(inc);
            }
          }
          xs[i * 128 + r] = x;
        }
      }
      tc3impl::fw_sync();
      // ---- facet traces of the stage output, facets 2h, 2h + 1 -----------------------
      if (valid && a.mode != 2) {
        unsigned long long x2[NP4 / 2];
#pragma unroll
        for (int j = 0; j < NP4 / 2; ++j)
          x2[j] = tc::f2_pack(2 * j < N ? xs[2 * j * 128 + r] : 0.f, 2 * j + 1 < N ? xs[(2 * j + 1) * 128 + r] : 0.f);
#pragma unroll
        for (int ff = 0; ff < 2; ++ff) {
          const int f = 2 * h + ff;
          float tv[NFM4];
#pragma unroll
          for (int m = 0; m < NFM4; ++m) {
            unsigned long long s2 = 0ull;
            if (m < NFM) {
              const ulonglong2* Er = reinterpret_cast<const ulonglong2*>(Ef + (f * NFM + m) * NP4);
#pragma unroll
              for (int j4 = 0; j4 < NP4 / 4; ++j4) {
                const ulonglong2 y = Er[j4];
                s2 = tc::f2_fma(y.x, x2[2 * j4], s2);
                s2 = tc::f2_fma(y.y, x2[2 * j4 + 1], s2);
              }
            }
            float lo, hi;
            tc::f2_unpack(s2, lo, hi);
            tv[m] = lo + hi;
          }
          float4* dst = reinterpret_cast<float4*>(a.trout + tc3_tr_index(tile, f, 0, r, NFM4));
#pragma unroll
          for (int m4 = 0; m4 < NFM4 / 4; ++m4)
            dst[m4] = make_float4(tv[4 * m4], tv[4 * m4 + 1], tv[4 * m4 + 2], tv[4 * m4 + 3]);
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
  constexpr int NFM4 = L::NFM4;
#pragma unroll 1
  for (int f = 0; f < L::NF; ++f) {
    float tv[NFM4];
#pragma unroll
    for (int m = 0; m < NFM4; ++m) {
      float s = 0.f;
      if (m < NFM)
#pragma unroll
        for (int i = 0; i < N; ++i) s += Ef[(f * NFM + m) * NP4 + i] * x[i];
      tv[m] = s;
    }
    float4* dst = reinterpret_cast<float4*>(tr + tc3_tr_index(tile, f, 0, r, NFM4));
#pragma unroll
    for (int m4 = 0; m4 < NFM4 / 4; ++m4) dst[m4] = make_float4(tv[4 * m4], tv[4 * m4 + 1], tv[4 * m4 + 2], tv[4 * m4 + 3]);
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
