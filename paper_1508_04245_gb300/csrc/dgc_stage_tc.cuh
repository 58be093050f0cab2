// Tensor-core RK stage kernel for triangles: steps a3-a7 of the upwind DG
// operator with its dense contraction on tcgen05 (kind::tf32, three-pass
// head/tail split, FP32 accumulation in TMEM) and the FP64 stage combination.
//
// Per tile of 128 elements (one CTA, 256 threads: thread (r, c) handles
// velocity component c of element r; element r = GEMM row r = TMEM lane r):
//   1. the tile's FP32 state and stage-input increment and its wind
//      coefficients arrive in shared memory by bulk copies (TMA) issued one
//      tile ahead; every thread writes the head/tail TF32 operands of its
//      state component and of one wind component;
//   2. GEMM A (one issuing thread): state and wind evaluated at the volume
//      points, the wind also at the facet points (weights and 1/det J folded
//      into the wind's table and coefficients);
//   3. CUDA cores, per element and component, in FP32: own and neighbour
//      facet traces on the facet basis (from the trace buffer), upwind
//      selection at the facet points by the sign of (1/det J) w_q (u^ .
//      -grad lambda_f), projection back onto the facet basis and restriction
//      to the element basis (Sec. 2.3 upwind flux); then the volume term,
//      products -(1/det J) w_q u^_d w_c(xi_q) against the basis gradients;
//   4. epilogue: the stage increment, in the last stage of a substep the FP64
//      state accumulation, and the facet traces of the stage output.
// The kernel is persistent (two CTAs per SM loop over tiles): the tables are
// loaded once per CTA.  State vectors use a tile-blocked SoA layout (TSOA) so
// every warp access is coalesced, and each stage writes the facet traces of
// its output (TR) for the next stage, which reads its own and its neighbours'
// traces instead of recomputing them from the coefficients.  Every mbarrier
// wait is bounded; a timeout sets bit 1 of the status word and the CTA stops
// (its bulk copies are drained and TMEM is still released).
#pragma once

#include <cuda_runtime.h>

#include "dgc_tc.cuh"
#include "dgc_tc_layout.h"

namespace dgc {

// Internal layouts of the tensor-core path (tile = 128 consecutive elements,
// r = element % 128): state "TSOA" [tile][c][i][128] FP64 and facet traces
// "TR" [tile][c][f][m][128] FP32, so a warp touches 32 consecutive elements.
__host__ __device__ __forceinline__ size_t tsoa_index(int e, int c, int i, int N) {
  return ((size_t)(e >> 7) * 2 * N + (size_t)c * N + i) * 128 + (e & 127);
}
__host__ __device__ __forceinline__ size_t tr_index(int e, int c, int f, int m, int NFM) {
  return ((size_t)(e >> 7) * 2 * 3 * NFM + ((size_t)c * 3 + f) * NFM + m) * 128 + (e & 127);
}

// One SSP-RK stage in increment form: the stage input is v^n + din, the
// kernel forms inc = p din + q L(v^n + din) with L = -(M^V)^{-1} C^V, and
//   mode 0: writes inc (FP32) and the facet traces of v^n + inc;
//   mode 1: v <- v + inc in FP64 (the substep's state accumulation), writes
//           the FP32 copy of the new v and its facet traces;
//   mode 2: v <- inc in FP64 (the operator itself, for conv_apply);
//   mode 3: one pseudo-time (Richardson) iteration of Sec. 3.3.2 with the
//           buffer sets selected by the parity of the iteration count i =
//           ctrl[1]: from v_i (FP64 v2[i&1], its FP32 copy vf2[i&1] and
//           traces tr2[i&1]) it forms r = (M^V)^{-1} C^V v_i, the residual
//           rho = g - v_i - tau r and v_i + ds rho in FP64, writes the latter
//           (FP64, FP32 copy, traces) into the other set, and per tile the
//           sum over its elements of |det J| rho^2 into partials[tile].
struct StageTcArgs {
  const float* vf;      // TSOA FP32 copy of v^n
  const float* din;     // TSOA FP32 increment of the stage input, null = none
  const float* trin;    // TR facet traces of the stage input
  float* dout;          // mode 0: TSOA FP32 increment out
  double* v;            // modes 1, 2: TSOA FP64 state
  float* vf_out;        // mode 1: FP32 copy of the new state (may equal vf)
  float* trout;         // modes 0, 1: facet traces of the stage output
  const float* wcoef;   // [tile][2][NK][128] wind on the Dubiner basis, scaled by 1/det J
  const int* nbr;       // [E][3]
  const float* blob;    // TcLayout2D<K> table blob
  int* status;          // device status word
  int E;
  int mode;
  // the coefficients p, q of the increment as FP32 pairs (hi + lo = the FP64 value
  // to 2^-48): a single FP32 rounding of q = c ds would scale every substep's
  // time step by the same (1 + eps), an error that grows linearly in time
  float p_hi, p_lo, q_hi, q_lo;
  // mode 3
  const double* ctrl;   // [1] = iteration count (as a double)
  const float* vf2[2];
  float* tr2[2];
  double* v2[2];
  const double* g;      // TSOA FP64 right-hand side
  const double* detJ;   // [E]
  double tau, ds;
  double* partials;     // [tiles]
  // tetrahedra (stage_tc3_kernel): the frozen facet flux in tile blocks
  // [tile][f][q][40], the FP32 facet tables (Ef, Qt) and the wind at the volume
  // points; blob then holds the BF16 table chunks, wcoef is unused and every
  // state vector has the row layout of TcLayout3D
  const float* fw3;
  const float* ftab;
  const float* wq3;     // the wind at the volume points, [tile][chunk][d][16][40]
  // bounded waits: polls of an mbarrier before a wait gives up (0 = tc::kWaitPolls); stall != 0
  // (a test hook) issues no bulk copy at all, so every wait runs out with nothing in
  // flight and the kernel reports the timeout in bit 1 of the status word
  uint32_t poll;
  int stall;
  // batched launch (triangles): one kernel over the tiles of several meshes of the same
  // order and stage kind.  list[j] holds mesh j's arguments (their own list null),
  // tile_off[j] the launch's number of mesh j's first tile (nondecreasing, tile_off[0] = 0),
  // batch_tiles the launch's tile count (= tile_off[n_list]); in this struct mode, din's
  // nullness, blob, poll and stall hold for every mesh, and the per-mesh fields are unused.
  // null list: one mesh, described by this struct.
  const StageTcArgs* list;
  const int* tile_off;
  int n_list;
  int batch_tiles;
};

// the mesh of tile `tile` in a batched launch: the last j with tile_off[j] <= tile
__device__ __forceinline__ int batch_instance(const int* tile_off, int n, int tile) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_off[mid] <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

namespace tcimpl {

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// head/tail TF32 split of an FP32 value
__device__ __forceinline__ void split(float x, float& h, float& t) {
  h = tc::to_tf32(x);
  t = tc::to_tf32(x - h);
}

// two FP32 values to a packed BF16 pair (round to nearest even), lo in the low half
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
// exact three-piece BF16 split of two FP32 values: a = h + m + l (each residual
// is exact in FP32 and the last has at most 8 significant bits)
__device__ __forceinline__ void split3_bf16x2(float a, float b, uint32_t& h, uint32_t& m, uint32_t& l) {
  h = bf16x2_rn(a, b);
  const float ra = a - __uint_as_float(h << 16), rb = b - __uint_as_float(h & 0xFFFF0000u);
  m = bf16x2_rn(ra, rb);
  l = bf16x2_rn(ra - __uint_as_float(m << 16), rb - __uint_as_float(m & 0xFFFF0000u));
}

// The pieces of NK values x of this thread's operand row r into the pieces of one
// field (base = first piece, pieces szOpA words apart), K-major core-matrix layout.
template <int K, int P>
__device__ __forceinline__ void put_operand(float* base, int r, const float* x) {
  using L = TcLayout2D<K, P>;
  const uint32_t row = (uint32_t)((r & 7) * 16 + (r >> 3) * L::SBO_NK);
  if constexpr (P == kTf32x3) {
#pragma unroll
    for (int k4 = 0; k4 < L::NK; k4 += 4) {
      float h[4], tl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) split(x[k4 + u], h[u], tl[u]);
      const uint32_t o = (row + (k4 / 4) * L::LBO) / 4;
      tc::st_shared_v4(base + o, h[0], h[1], h[2], h[3]);
      tc::st_shared_v4(base + L::szOpA + o, tl[0], tl[1], tl[2], tl[3]);
    }
  } else {
#pragma unroll
    for (int k8 = 0; k8 < L::NK; k8 += 8) {
      uint32_t hw[4], mw[4], lw[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) split3_bf16x2(x[k8 + 2 * j], x[k8 + 2 * j + 1], hw[j], mw[j], lw[j]);
      const uint32_t o = (row + (k8 / 8) * L::LBO) / 4;
      tc::st_shared_v4u(base + o, hw[0], hw[1], hw[2], hw[3]);
      tc::st_shared_v4u(base + L::szOpA + o, mw[0], mw[1], mw[2], mw[3]);
      tc::st_shared_v4u(base + 2 * L::szOpA + o, lw[0], lw[1], lw[2], lw[3]);
    }
  }
}

template <int NCOL>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float* v) {
  static_assert(NCOL % 8 == 0, "TMEM loads in groups of 8 columns");
#pragma unroll
  for (int c = 0; c < NCOL; c += 8) tc::tmem_ld8(taddr + c, v + c);
  tc::tmem_wait_ld();
}

}  // namespace tcimpl

// own facet traces of one component on the facet bases: tr[f][m] = sum_i Ef[f][m][i] x[i]
template <int N, int NF, int NFM, int NP4>
__device__ __forceinline__ void facet_traces(const float* Ef, const float* x, float (*tr)[NFM]) {
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int m = 0; m < NFM; ++m) {
      float a0 = 0.f, a1 = 0.f;
#pragma unroll
      for (int i4 = 0; i4 < NP4 / 4; ++i4) {
        const float4 y = *reinterpret_cast<const float4*>(Ef + (f * NFM + m) * NP4 + 4 * i4);
        a0 += y.x * x[4 * i4] + y.y * x[4 * i4 + 1];
        a1 += y.z * x[4 * i4 + 2] + y.w * x[4 * i4 + 3];
      }
      tr[f][m] = a0 + a1;
    }
}

// RICH: the variant for mode 3 (pseudo-time iteration); modes 0-2 compile without it
// resident CTAs per SM: two for k <= 4, one for k = 5, 6 (their shared memory and
// TMEM exceed half of the SM's); the register budget follows
__host__ __device__ constexpr int tc_ctas_per_sm(int K) { return K <= 4 ? 2 : 1; }

// BATCH: the tiles of the meshes in a.list (a batched launch); per tile, the mesh's own
// buffers, size, neighbours, status word and stage coefficients
template <int K, int P, bool RICH, bool BATCH = false>
__global__ void __launch_bounds__(288, tc_ctas_per_sm(K)) stage_tc_kernel(StageTcArgs a) {
  static_assert(!(RICH && BATCH), "the pseudo-time iteration runs on one mesh");
  using L = TcLayout2D<K, P>;
  constexpr int N = L::N, QV = L::QV, QF = L::QF, NFM = L::NFM, NF = L::NF, NK = L::NK;
  constexpr int NP4 = L::NP4, NFM4 = L::NFM4;
  constexpr bool EARLY_TRACES = tc_ctas_per_sm(K) == 1;
  extern __shared__ __align__(1024) float sm[];
  float* blob = sm;
  float* wst = sm + L::oWst;
  float* op = sm + L::oOp;
  float* stg = sm + L::oStg;                 // next tile's [vf | din] (wind half of op)
  float* epi = sm + L::oEpi;                 // this tile's [vf | din] (state half of op)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::SMEM_FLOATS);
  uint64_t* bar_tab = bars + 0;
  uint64_t* bar_w = bars + 1;
  uint64_t* bar_A = bars + 2;
  uint64_t* bar_st = bars + 3;
  uint64_t* bar_ep = bars + 4;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const uint32_t poll = a.poll ? a.poll : tc::kWaitPolls;   // polls per bounded wait
  double* red = reinterpret_cast<double*>(bars + 6);   // per-warp sums of mode 3 (8)

  // threads 0..255: (element row r of the tile, velocity component c); warps
  // 0-3 and 4-7 read the same TMEM lanes (a warp sees lanes 32 (warp % 4) ..
  // + 31).  Warp 8 only issues the MMAs and bulk copies (thread 256).
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const bool producer = t < 256;
  const int r = t & 127;
  const int c = (t >> 7) & 1;
  const int issuer_t = 256;
  const int ntiles = BATCH ? a.batch_tiles : (a.E + 127) / 128;
  // input and output buffers (mode 3 picks its pair by the parity of the iteration count)
  const float* vf_in = a.vf;
  const float* tr_in = a.trin;
  double* v_state = a.v;
  double* v_out = a.v;
  float* vf_out = a.vf_out;
  float* tr_out = a.trout;
  if constexpr (RICH) {
    const int par = ((int)a.ctrl[1]) & 1;
    vf_in = a.vf2[par];
    tr_in = a.tr2[par];
    v_state = a.v2[par];
    v_out = a.v2[par ^ 1];
    vf_out = const_cast<float*>(a.vf2[par ^ 1]);
    tr_out = a.tr2[par ^ 1];
  }
  // the epilogue reads the stage-input increment (modes 0, 1) and v^n (mode 0)
  const bool epi_din = a.din != nullptr;
  const bool epi_vf = a.mode == 0;
  // issuer-side counts of bulk copies into the staging buffers (drained at exit)
  uint32_t w_issued = 0, st_issued = 0, ep_issued = 0;
  // the next tile's contiguous TR block into L2 ahead of use
  // the sources of a tile's bulk copies: its mesh's buffers and its number within that mesh
  struct TileSrc {
    int lt;
    const float *wcoef, *vf, *din, *tr;
  };
  auto tile_src = [&](int tile) {
    TileSrc s{tile, a.wcoef, vf_in, a.din, tr_in};
    if constexpr (BATCH) {
      const int j = batch_instance(a.tile_off, a.n_list, tile);
      const StageTcArgs& b = a.list[j];
      s = TileSrc{tile - a.tile_off[j], b.wcoef, b.vf, b.din, b.trin};
    }
    return s;
  };
  auto prefetch_tile = [&](const TileSrc& s) {
    const uint32_t ntr = 128u * 2 * NF * NFM;  // values per tile in TR
    tc::bulk_prefetch_l2(s.tr + (size_t)s.lt * ntr, ntr * 4);
  };
  auto load_wind = [&](const TileSrc& s) {        // a tile's wind coefficients into the staging buffer
    const uint32_t bytes = (uint32_t)L::WSTAGE * 4;   // whole tile block ([c][k][128])
    tc::mbar_arrive_expect_tx(bar_w, bytes);
    tc::bulk_g2s(wst, s.wcoef + (size_t)s.lt * L::WSTAGE, bytes, bar_w);
    ++w_issued;
  };
  // a tile's blocks of v^n (FP32 copy) and of the stage-input increment into dst
  // (TSOA vectors are allocated in whole tiles: complete, 16-byte aligned blocks)
  const uint32_t blk = (uint32_t)L::TSOA_TILE * 4;
  auto load_state = [&](float* dst, uint64_t* bar, const TileSrc& s, bool vf, bool din) {
    tc::mbar_arrive_expect_tx(bar, (vf ? blk : 0u) + (din ? blk : 0u));
    if (vf) tc::bulk_g2s(dst, s.vf + (size_t)s.lt * L::TSOA_TILE, blk, bar);
    if (din) tc::bulk_g2s(dst + L::TSOA_TILE, s.din + (size_t)s.lt * L::TSOA_TILE, blk, bar);
  };

  if (t == 0) {
    tc::mbar_init(bar_tab, 1);
    tc::mbar_init(bar_w, 1);
    tc::mbar_init(bar_A, 1);
    tc::mbar_init(bar_st, 1);
    tc::mbar_init(bar_ep, 1);
    *abort_flag = 0;
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (t == issuer_t && !a.stall) {
    tc::mbar_arrive_expect_tx(bar_tab, L::SBLOB * 4);
    tc::bulk_g2s(blob, a.blob, L::SBLOB * 4, bar_tab);
    const TileSrc s0 = tile_src(blockIdx.x);
    load_wind(s0);
    load_state(stg, bar_st, s0, true, epi_din);
    ++st_issued;
    prefetch_tile(s0);
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, L::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t lane_base = tbase + ((uint32_t)((warp & 3) * 32) << 16);
  if (!tc::mbar_wait(bar_tab, 0, poll)) *abort_flag = 1;
  const float* G = (L::G_GLOBAL ? a.blob : blob) + L::oG;     // [QV][2][NP4]
  const float* Ef = blob + L::oEf;   // [NF][NFM][NP4]
  const float* Qt = blob + L::oQt;   // [QF][NFM4]
  const uint32_t op_s = tc::smem_u32(op);
  const uint32_t bl_s = tc::smem_u32(blob);

  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    // the tile's mesh (batched launches) and the tile's number lt within it
    int lt = tile;
    const StageTcArgs* ia = nullptr;
    if constexpr (BATCH) {
      const int j = batch_instance(a.tile_off, a.n_list, tile);
      ia = a.list + j;
      lt = tile - a.tile_off[j];
    }
    const int E = BATCH ? ia->E : a.E;
    const int* nbr = BATCH ? ia->nbr : a.nbr;
    int* status = BATCH ? ia->status : a.status;
    const float* tr_t = BATCH ? ia->trin : tr_in;
    const int e = lt * 128 + r;
    const bool valid = e < E;
    const int next = tile + gridDim.x;

    // ---- stage input v^n + din (staged by bulk copy) -> state operand of component c
    if (producer) {
    if (*abort_flag == 0 && !tc::mbar_wait(bar_st, it & 1, poll)) *abort_flag = 1;
    float w[NK];
#pragma unroll
    for (int i = 0; i < NK; ++i) {
      const int si = (c * N + (i < N ? i : 0)) * 128 + r;
      w[i] = (valid && i < N) ? stg[si] + (epi_din ? stg[L::TSOA_TILE + si] : 0.f) : 0.f;
    }
    tcimpl::put_operand<K, P>(op + c * L::PIECES * L::szOpA, r, w);
    }   // producer
    __syncthreads();   // the staged state has been read: its space takes the wind operands
    if (producer) {
    // ---- wind operand of dimension d = c from the staged coefficients --------------
    if (*abort_flag == 0 && !tc::mbar_wait(bar_w, it & 1, poll)) *abort_flag = 1;
    float x[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) x[k] = valid ? wst[(c * NK + k) * 128 + r] : 0.f;   // conflict-free
    tcimpl::put_operand<K, P>(op + (2 + c) * L::PIECES * L::szOpA, r, x);
    }   // producer
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool run = *abort_flag == 0;
    if (t == issuer_t && run) {
      // ---- GEMM A ------------------------------------------------------------------
      // products of pieces (A piece, B piece), smallest first: the tensor-core FP32
      // accumulation rounds partly toward zero, so the small correction products
      // are summed while the accumulator is still small and the dominant head x
      // head product comes last.  TF32: th, ht, hh; BF16: mm, lh, hl, mh, hm, hh
      constexpr int PA3[3] = {1, 0, 0}, PB3[3] = {0, 1, 0};
      constexpr int PA6[6] = {1, 2, 0, 1, 0, 0}, PB6[6] = {1, 0, 2, 0, 1, 0};
      const int* PA = P == kBf16x3 ? PA6 : PA3;
      const int* PB = P == kBf16x3 ? PB6 : PB3;
      for (int f = 0; f < 4; ++f) {
        const bool wind = f >= 2;
        const int NA = wind ? L::NAW : L::NAS;
        const uint32_t idesc = P == kBf16x3 ? tc::idesc_bf16(128, NA) : tc::idesc_tf32(128, NA);
        const uint32_t dcol = wind ? L::cW + (f - 2) * L::NAW : L::cS + f * L::NAS;
        const uint32_t tab = bl_s + 4u * (wind ? L::oTAw : L::oTAs);
        const uint32_t tsz = 4u * (wind ? L::szTAw : L::szTAs);
        uint32_t acc = 0;
        for (int pr = 0; pr < L::NPROD; ++pr) {
          const uint32_t a_op = op_s + 4u * ((f * L::PIECES + PA[pr]) * L::szOpA);
          const uint32_t b_op = tab + PB[pr] * tsz;
          for (int ks = 0; ks < NK / L::KSTEP; ++ks) {
            const uint64_t ad = tc::smem_desc(a_op + ks * 2 * L::LBO, L::LBO, L::SBO_NK);
            const uint64_t bd = tc::smem_desc(b_op + ks * 2 * L::LBO, L::LBO, L::SBO_NK);
            if constexpr (P == kBf16x3) tc::mma_bf16(tbase + dcol, ad, bd, idesc, acc);
            else tc::mma_tf32(tbase + dcol, ad, bd, idesc, acc);
            acc = 1;
          }
        }
      }
      tc::mma_commit(bar_A);
    }
    // ---- own and neighbour facet traces from the trace buffer: with one CTA per SM
    //      (k = 5, 6; registers to spare) loaded while GEMM A runs, with two (k <= 4) after
    //      the volume part, from L2 (the tile's block is prefetched with its state) ----
    float to[NF][NFM], tn[NF][NFM];
    auto load_traces = [&]() {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int code = (producer && valid) ? checked_code(nbr[(size_t)e * NF + f], 2, E, status) : -1;
        const int ne = code >> 2, fn = code & 3;
#pragma unroll
        for (int m = 0; m < NFM; ++m) {
          to[f][m] = (producer && valid) ? tr_t[tr_index(e, c, f, m, NFM)] : 0.f;
          tn[f][m] = code >= 0 ? tr_t[tr_index(ne, c, fn, m, NFM)] : 0.f;
        }
      }
    };
    if constexpr (EARLY_TRACES) load_traces();
    if (producer && run && *abort_flag == 0 && !tc::mbar_wait(bar_A, it & 1, poll)) *abort_flag = 1;
    tc::fence_after_sync();
    __syncthreads();
    const bool run2 = *abort_flag == 0;
    // ---- issuer: GEMM A has read both operand halves: this tile's state for the
    //      epilogue into the state half, the next tile's into the wind half ---------
    if (t == issuer_t && run2) {
      tc::fence_proxy_async_smem();
      // the FP64 state the epilogue accumulates into (mode 1), toward L2
      if (RICH || a.mode == 1)
        tc::bulk_prefetch_l2((BATCH ? ia->v : v_state) + (size_t)lt * L::TSOA_TILE, (uint32_t)L::TSOA_TILE * 8);
      if constexpr (RICH) tc::bulk_prefetch_l2(a.g + (size_t)tile * L::TSOA_TILE, (uint32_t)L::TSOA_TILE * 8);
      if (epi_vf || epi_din) {
        load_state(epi, bar_ep, TileSrc{lt, nullptr, BATCH ? ia->vf : vf_in, BATCH ? ia->din : a.din, nullptr},
                   epi_vf, epi_din);
        ++ep_issued;
      }
      if (next < ntiles) {
        const TileSrc sn = tile_src(next);
        load_state(stg, bar_st, sn, true, epi_din);
        ++st_issued;
        prefetch_tile(sn);
      }
    }

    // ---- test contractions on CUDA cores (FP32): r_i = volume part + facet part ------
    // r is held as packed pairs (i = 2j, 2j + 1); the tables' padding rows are zero.
    // Volume part, split by output halves: thread (r, c) accumulates the outputs i of
    // half c (i in [c NH, c NH + NH)) of BOTH components, so each value of G it loads
    // serves two products; the other component's half goes to thread (r, 1 - c) through
    // the wind staging buffer (free from the wind operand until the next tile's wind is
    // loaded after the epilogue wait).
    constexpr int NP2 = NP4 / 2;
    constexpr int NH = NP4 / 2, NH2 = NH / 2;    // outputs per half, as packed pairs
    static_assert(NH * 256 <= L::WSTAGE, "the exchange fits the wind staging buffer");
    unsigned long long va[NH2], vb[NH2];         // half c of component c (va) and 1 - c (vb)
#pragma unroll
    for (int j = 0; j < NH2; ++j) va[j] = vb[j] = 0ull;
    if (run2 && producer) {
      // volume: r_i -= sum_q sum_d (Uw[q][d] w_c(xi_q)) G[q][d][i], 4 points per TMEM load
      // (the state columns are padded to a multiple of 16, so a group never runs past them)
#pragma unroll 1
      for (int q0 = 0; q0 < QV; q0 += 4) {
        float wa[4], wb[4], uq0[4], uq1[4];
        tc::tmem_ld4(lane_base + L::cS + c * L::NAS + q0, wa);
        tc::tmem_ld4(lane_base + L::cS + (1 - c) * L::NAS + q0, wb);
        tc::tmem_ld4(lane_base + L::cW + q0, uq0);
        tc::tmem_ld4(lane_base + L::cW + L::NAW + q0, uq1);
        tc::tmem_wait_ld();
#pragma unroll
        for (int ql = 0; ql < 4; ++ql) {
          if (q0 + ql >= QV) break;
          const float a0 = valid ? -uq0[ql] * wa[ql] : 0.f, a1 = valid ? -uq1[ql] * wa[ql] : 0.f;
          const float b0 = valid ? -uq0[ql] * wb[ql] : 0.f, b1 = valid ? -uq1[ql] * wb[ql] : 0.f;
          const unsigned long long pa0 = tc::f2_pack(a0, a0), pa1 = tc::f2_pack(a1, a1);
          const unsigned long long pb0 = tc::f2_pack(b0, b0), pb1 = tc::f2_pack(b1, b1);
          const float* Gq = G + (q0 + ql) * 2 * NP4 + c * NH;   // G[q][0][half c], then G[q][1][half c]
          if constexpr (NH % 4 == 0) {
            const ulonglong2* g0p = reinterpret_cast<const ulonglong2*>(Gq);
            const ulonglong2* g1p = reinterpret_cast<const ulonglong2*>(Gq + NP4);
#pragma unroll
            for (int j4 = 0; j4 < NH / 4; ++j4) {
              ulonglong2 g0, g1;
              if constexpr (L::G_GLOBAL) {
                g0 = tc::ld_keep_u64x2(g0p + j4);
                g1 = tc::ld_keep_u64x2(g1p + j4);
              } else {
                g0 = g0p[j4];
                g1 = g1p[j4];
              }
              va[2 * j4] = tc::f2_fma(pa1, g1.x, tc::f2_fma(pa0, g0.x, va[2 * j4]));
              va[2 * j4 + 1] = tc::f2_fma(pa1, g1.y, tc::f2_fma(pa0, g0.y, va[2 * j4 + 1]));
              vb[2 * j4] = tc::f2_fma(pb1, g1.x, tc::f2_fma(pb0, g0.x, vb[2 * j4]));
              vb[2 * j4 + 1] = tc::f2_fma(pb1, g1.y, tc::f2_fma(pb0, g0.y, vb[2 * j4 + 1]));
            }
          } else {
            const unsigned long long* g0p = reinterpret_cast<const unsigned long long*>(Gq);
            const unsigned long long* g1p = reinterpret_cast<const unsigned long long*>(Gq + NP4);
#pragma unroll
            for (int j = 0; j < NH2; ++j) {
              const unsigned long long g0 = L::G_GLOBAL ? tc::ld_keep_u64(g0p + j) : g0p[j];
              const unsigned long long g1 = L::G_GLOBAL ? tc::ld_keep_u64(g1p + j) : g1p[j];
              va[j] = tc::f2_fma(pa1, g1, tc::f2_fma(pa0, g0, va[j]));
              vb[j] = tc::f2_fma(pb1, g1, tc::f2_fma(pb0, g0, vb[j]));
            }
          }
        }
      }
      // component 1 - c of half c to thread (r, 1 - c): [i within the half][thread]
#pragma unroll
      for (int j = 0; j < NH2; ++j) {
        float lo, hi;
        tc::f2_unpack(vb[j], lo, hi);
        wst[(2 * j) * 256 + t] = lo;
        wst[(2 * j + 1) * 256 + t] = hi;
      }
    }
    __syncthreads();
    unsigned long long r2[NP2];   // component c, every output
#pragma unroll
    for (int j = 0; j < NH2; ++j) {
      // half 1 - c of component c, from thread (r, 1 - c)
      const unsigned long long o = (run2 && producer)
                                       ? tc::f2_pack(wst[(2 * j) * 256 + (t ^ 128)], wst[(2 * j + 1) * 256 + (t ^ 128)])
                                       : 0ull;
      r2[j] = c == 0 ? va[j] : o;
      r2[NH2 + j] = c == 0 ? o : va[j];
    }
    if constexpr (!EARLY_TRACES) load_traces();
    if (run2 && producer) {
      // facets: upwind flux at the facet points, projected onto the facet basis, then
      // r_i += sum_{f,m} Ef[f][m][i] phi[f][m]
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        // wind at this facet's points: (1/det J) w_q u^_dd, columns QV + f QF + q
        float u0[QF], u1[QF];
#pragma unroll
        for (int q = 0; q < QF; ++q) {
          uint32_t x0, x1;
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                       : "=r"(x0)
                       : "r"(lane_base + L::cW + QV + f * QF + q));
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                       : "=r"(x1)
                       : "r"(lane_base + L::cW + L::NAW + QV + f * QF + q));
          u0[q] = __uint_as_float(x0);
          u1[q] = __uint_as_float(x1);
        }
        tc::tmem_wait_ld();
        float phi[NFM];
#pragma unroll
        for (int m = 0; m < NFM; ++m) phi[m] = 0.f;
#pragma unroll
        for (int q = 0; q < QF; ++q) {
          // -grad lambda_0 = (1,1), -grad lambda_1 = (-1,0), -grad lambda_2 = (0,-1)
          const float fw = f == 0 ? u0[q] + u1[q] : (f == 1 ? -u0[q] : -u1[q]);
          float qq[NFM4];
#pragma unroll
          for (int m4 = 0; m4 < NFM4; m4 += 4) {
            const float4 x = *reinterpret_cast<const float4*>(Qt + q * NFM4 + m4);
            qq[m4] = x.x;
            qq[m4 + 1] = x.y;
            qq[m4 + 2] = x.z;
            qq[m4 + 3] = x.w;
          }
          float o = 0.f, nb = 0.f;
#pragma unroll
          for (int m = 0; m < NFM; ++m) {
            o += qq[m] * to[f][m];
            nb += qq[m] * tn[f][m];
          }
          const float val = valid ? fw * (fw >= 0.f ? o : nb) : 0.f;
#pragma unroll
          for (int m = 0; m < NFM; ++m) phi[m] += qq[m] * val;
        }
#pragma unroll
        for (int m = 0; m < NFM; ++m) {
          const ulonglong2* Er = reinterpret_cast<const ulonglong2*>(Ef + (f * NFM + m) * NP4);
          const unsigned long long pp = tc::f2_pack(phi[m], phi[m]);
#pragma unroll
          for (int j4 = 0; j4 < NP4 / 4; ++j4) {
            const ulonglong2 y = Er[j4];
            r2[2 * j4] = tc::f2_fma(y.x, pp, r2[2 * j4]);
            r2[2 * j4 + 1] = tc::f2_fma(y.y, pp, r2[2 * j4 + 1]);
          }
        }
      }
    }

    float rr[NP4];
#pragma unroll
    for (int j = 0; j < NP2; ++j) tc::f2_unpack(r2[j], rr[2 * j], rr[2 * j + 1]);
    // ---- epilogue: increment, FP64 accumulation (mode 1), output traces --------------
    double ex[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
      ex[i] = (producer && valid && a.mode == 1) ? (BATCH ? ia->v : v_state)[tsoa_index(e, c, i, N)] : 0.0;
    if (producer && run2 && (epi_vf || epi_din) && *abort_flag == 0 && !tc::mbar_wait(bar_ep, it & 1, poll))
      *abort_flag = 1;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool fin = run2 && *abort_flag == 0;   // uniform after the barrier
    if (fin && t == issuer_t && next < ntiles) {
      tc::fence_proxy_async_smem();   // the exchange's reads of the staging buffer come first
      load_wind(tile_src(next));
    }
    if (!fin) {
      // a bounded wait gave up: this CTA stops (in a batched launch its later tiles may
      // belong to any of the meshes: each is told)
      if (t == 0) {
        if constexpr (BATCH) {
          for (int j = 0; j < a.n_list; ++j) atomicOr(a.list[j].status, 2);
        } else {
          atomicOr(a.status, 2);
        }
      }
      break;
    }
    double racc = 0.0;   // mode 3: sum of rho^2 over this thread's coefficients
    if (producer && valid) {
      double* vs_t = BATCH ? ia->v : v_state;
      double* vo_t = BATCH ? ia->v : v_out;
      float* vfo_t = BATCH ? ia->vf_out : vf_out;
      float* tro_t = BATCH ? ia->trout : tr_out;
      float* dout_t = BATCH ? ia->dout : a.dout;
      const float p_hi = BATCH ? ia->p_hi : a.p_hi, p_lo = BATCH ? ia->p_lo : a.p_lo;
      const float q_hi = BATCH ? ia->q_hi : a.q_hi, q_lo = BATCH ? ia->q_lo : a.q_lo;
      // inc = p din + q L, L = -r (r carries FP32 accuracy)
      float xo[NP4];
#pragma unroll
      for (int i = 0; i < NP4; ++i) xo[i] = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const size_t ix = tsoa_index(e, c, i, N);
        const int si = (c * N + i) * 128 + r;
        const float ed = epi_din ? epi[L::TSOA_TILE + si] : 0.f;
        const float inc = fmaf(p_hi, ed, fmaf(p_lo, ed, -fmaf(q_hi, rr[i], q_lo * rr[i])));
        if (RICH) {
          // rho = g - v - tau r and the next iterate, in FP64
          const double vx = vs_t[ix];
          const double rho = (a.g[ix] - vx) - a.tau * tc::f32_to_f64(rr[i]);
          const double vn = vx + a.ds * rho;
          vo_t[ix] = vn;
          xo[i] = tc::f64_to_f32_rn(vn);
          vfo_t[ix] = xo[i];
          racc += rho * rho;
        } else if (a.mode == 0) {
          dout_t[ix] = inc;
          xo[i] = epi[si] + inc;
        } else if (a.mode == 1) {
          const double x = ex[i] + tc::f32_to_f64(inc);   // FP64 state accumulation
          vo_t[ix] = x;
          xo[i] = tc::f64_to_f32_rn(x);
          vfo_t[ix] = xo[i];
        } else {
          vo_t[ix] = tc::f32_to_f64(inc);
        }
      }
      if (a.mode != 2) {
        float tr[NF][NFM];
        facet_traces<N, NF, NFM, NP4>(Ef, xo, tr);
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
          for (int m = 0; m < NFM; ++m) tro_t[tr_index(e, c, f, m, NFM)] = tr[f][m];
      }
      if constexpr (RICH) racc *= fabs(a.detJ[e]);
    }
    if (RICH && producer) {   // per-warp sum in a fixed order
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) racc += __shfl_xor_sync(0xffffffffu, racc, o);
      if ((t & 31) == 0) red[warp] = racc;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (RICH && t == 0) {
      double sum = 0.0;
#pragma unroll
      for (int w8 = 0; w8 < 8; ++w8) sum += red[w8];
      a.partials[tile] = sum;
    }
  }
  // bulk copies still in flight (only after a timeout) land before the CTA exits
  if (t == issuer_t) {
    if (st_issued) tc::mbar_wait(bar_st, (st_issued - 1) & 1, poll);
    if (ep_issued) tc::mbar_wait(bar_ep, (ep_issued - 1) & 1, poll);
    if (w_issued) tc::mbar_wait(bar_w, (w_issued - 1) & 1, poll);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, L::TMEM_COLS);
}

// ABI layout [E][2][N] -> TSOA (FP64 and its FP32 copy), plus the facet traces (TR)
template <int K>
__global__ void __launch_bounds__(256) tsoa_in_kernel(const double* __restrict__ v, double* __restrict__ vt,
                                                      float* __restrict__ vft, float* __restrict__ tr,
                                                      const float* __restrict__ blob, int E) {
  using L = TcLayout2D<K>;
  constexpr int N = L::N, NF = L::NF, NFM = L::NFM, NP4 = L::NP4;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int e = (int)(gid >> 1), c = (int)(gid & 1);
  if (e >= E) return;
  float x[NP4];
#pragma unroll
  for (int i = 0; i < NP4; ++i) x[i] = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double d = v[((size_t)e * 2 + c) * N + i];
    vt[tsoa_index(e, c, i, N)] = d;
    x[i] = tc::f64_to_f32_rn(d);
    vft[tsoa_index(e, c, i, N)] = x[i];
  }
  float t[NF][NFM];
  facet_traces<N, NF, NFM, NP4>(blob + L::oEf, x, t);
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int m = 0; m < NFM; ++m) tr[tr_index(e, c, f, m, NFM)] = t[f][m];
}

// ABI layout [E][2][N] -> TSOA, FP64 only
template <int K>
__global__ void __launch_bounds__(256) tsoa_in64_kernel(const double* __restrict__ v, double* __restrict__ vt,
                                                        int E) {
  constexpr int N = TcLayout2D<K>::N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)E * 2 * N) return;
  const int i = (int)(gid % N);
  const int c = (int)((gid / N) % 2);
  const int e = (int)(gid / (2 * N));
  vt[tsoa_index(e, c, i, N)] = v[gid];
}

// TSOA -> ABI layout from the buffer of a pair selected by the parity of ctrl[1]
template <int K>
__global__ void __launch_bounds__(256) tsoa_out_sel_kernel(const double* __restrict__ vt0,
                                                           const double* __restrict__ vt1,
                                                           const double* __restrict__ ctrl, double* __restrict__ v,
                                                           int E) {
  constexpr int N = TcLayout2D<K>::N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)E * 2 * N) return;
  const int i = (int)(gid % N);
  const int c = (int)((gid / N) % 2);
  const int e = (int)(gid / (2 * N));
  const double* vt = (((int)ctrl[1]) & 1) ? vt1 : vt0;
  v[gid] = vt[tsoa_index(e, c, i, N)];
}

// TSOA -> ABI layout
template <int K>
__global__ void __launch_bounds__(256) tsoa_out_kernel(const double* __restrict__ vt, double* __restrict__ v, int E) {
  constexpr int N = TcLayout2D<K>::N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)E * 2 * N) return;
  const int i = (int)(gid % N);
  const int c = (int)((gid / N) % 2);
  const int e = (int)(gid / (2 * N));
  v[gid] = vt[tsoa_index(e, c, i, N)];
}

}  // namespace dgc
