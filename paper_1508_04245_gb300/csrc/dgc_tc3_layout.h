// Compile-time layout of the tensor-core stage kernel for tetrahedra (dim 3).
//
// GEMM rows are (element, velocity component) pairs: a tile holds 40
// elements, rows 32 g + 3 s + c for element 10 g + s (g = 0..3, s = 0..9) and
// component c; rows 32 g + 30 and 32 g + 31 are padding.  Each row carries one
// field of the state (its component):
//
//   GEMM A (per chunk of 16 volume points, A from TMEM, B = basis table):
//     X[r, q] = sum_j A_s[r, j] Bv[q, j]          state component c at xi_q
//   GEMM B (the volume test contraction, A = products from TMEM), per chunk:
//     R_j[r, i] = sum_{d, q in chunk j} P[r, (d, q)] G[(d, q), i],  R = sum_j R_j,
//     P[r, (d, q)] = u_d(xi_q) w_c(xi_q),  G[(d, q), i] = -w_q d_d psi^_i(xi_q)
//
// The wind is frozen over a call, so its values at the volume points,
// u_d(xi_q) = (1/det J) sum_i uc[d][i] psi^_i(xi_q), are evaluated once per
// call in FP64 (rounded to FP32) and streamed per chunk, [tile][chunk][d][16][40].
//
// Every operand is split exactly into three BF16 pieces (kind::f16, six
// products, FP32 accumulation), with the head pieces on a grid: the head of
// an operand row is a multiple of 2^(e - 7), e the exponent of the largest
// value the row contributes to one accumulation (the state coefficients of
// the row; the 48 products P of the row in the chunk), and the head of a table
// column a multiple of 2^(f - 7) likewise (a point of the GEMM A table; a
// basis function i over the chunk in G).  Every head x head product is then an
// integer multiple of 2^(e + f - 14) of at most 2^16 units and their sum over
// K <= 48 stays below 2^22 units: exact in FP32.  That sum accumulates on its
// own, the five correction products (about 2^-8 of it) on theirs, and the two
// are added on CUDA cores, so the truncating accumulation of the tensor cores
// biases neither the evaluated state nor the residual.  The tables of a chunk
// (Bv and the three G blocks, all pieces) are one contiguous blob bulk-copied
// into a ring of shared-memory slots; the facet terms run on CUDA cores in FP32
// from the facet traces of the stage input and the frozen facet flux.
#pragma once

namespace dgc {

template <int K>
struct TcLayout3D {
  static constexpr int pad(int n, int m) { return (n + m - 1) / m * m; }
  static constexpr int D = 3;
  static constexpr int NF = 4;
  static constexpr int N = (K + 1) * (K + 2) * (K + 3) / 6;
  static constexpr int NFM = (K + 1) * (K + 2) / 2;
  static constexpr int NQ1V = (3 * K - 1) / 2 + 1;
  static constexpr int QV = NQ1V * NQ1V * NQ1V;
  static constexpr int NQ1F = (3 * K) / 2 + 1;
  static constexpr int QF = NQ1F * NQ1F;
  static constexpr int EPT = 40;                       // elements per tile
  static constexpr int NK = pad(N, 16);                // K of GEMM A
  static constexpr int NR = pad(N, 16);                // N of GEMM B
  static constexpr int QC = 16;                        // volume points per chunk
  static constexpr int NCH = (QV + QC - 1) / QC;       // chunks per tile

  // TMEM columns (32-bit); a BF16 piece of a K = NK operand row takes NK / 2
  static constexpr int NKC = NK / 2;
  static constexpr int cAs = 0;                        // state operand, pieces h, m, l
  // GEMM A results, two buffers of [hh | corr] (16 columns each): the head-piece
  // products accumulate apart from the five correction products
  static constexpr int cX = pad(3 * NKC, 16);
  static constexpr int XCOLS = 32;
  static constexpr int cP = cX + 2 * XCOLS;            // GEMM B operands, two buffers: [d][piece][8 columns]
  static constexpr int PCOLS = 72;
  // GEMM B: the head sums of a chunk into a fresh partial (two buffers), the
  // correction products of all chunks of a tile into one accumulator, both added
  // on CUDA cores; then the tile's summed residual handed to the facet warps
  static constexpr int cRh = cP + 2 * PCOLS;
  static constexpr int cRc = cRh + 2 * NR;
  static constexpr int cRf = cRc + NR;
  static constexpr int TMEM_USED = cRf + NR;
  static constexpr int TMEM_COLS = 512;
  static_assert(TMEM_USED <= TMEM_COLS, "tensor memory");

  // chunk blob (bytes): [Bv pieces: 3 x (16 x NK)] [G: d x piece x (NR x 16)], BF16
  static constexpr int szBA = 16 * NK * 2;             // one piece of the GEMM A table chunk
  static constexpr int szBG = NR * 16 * 2;             // one piece of one G block
  static constexpr int oBA = 0;
  static constexpr int oBG = 3 * szBA;
  static constexpr int CH_BYTES = oBG + 9 * szBG;
  static constexpr unsigned SBO_A = (NK / 8) * 128;    // 8-row groups of the GEMM A table
  static constexpr unsigned SBO_G = 256;               // 8-row groups of a G block (K = 16)
  static constexpr bool RESIDENT = NCH <= 4;           // every chunk kept, else a ring
  static constexpr int SLOTS = RESIDENT ? NCH : 4;

  // FP32 tables of the facet terms: Ef [NF][NFM][NP4], Qt [QF][NFM4]
  static constexpr int NP4 = pad(N, 4);
  static constexpr int NFM4 = pad(NFM, 4);
  static constexpr int oEf = 0;
  static constexpr int oQt = NF * NFM * NP4;
  static constexpr int FWT = pad(oQt + QF * NFM4, 4);  // floats

  // frozen facet flux of a tile: [f][q][EPT] floats
  static constexpr int FWS = NF * QF * EPT;
  // the wind at the 16 points of a chunk: [d][q][EPT] floats, through a ring
  static constexpr int WCH = 3 * QC * EPT;
  static constexpr int WSLOTS = 4;

  // shared memory (bytes)
  static constexpr int oRing = 0;
  static constexpr int oFwt = oRing + SLOTS * CH_BYTES;
  static constexpr int oFws = oFwt + FWT * 4;          // two tile buffers
  static constexpr int oPhi = oFws + 2 * FWS * 4;      // [f][m][128] facet projections
  static constexpr int oXs = oPhi + NF * NFM * 128 * 4;  // [i][128] stage output (for its traces)
  static constexpr int oWnd = oXs + N * 128 * 4;       // wind ring, WSLOTS x WCH floats
  static constexpr int oBar = oWnd + WSLOTS * WCH * 4;
  static constexpr int NBAR = 40;
  static constexpr int SMEM_BYTES = oBar + NBAR * 8 + 64;
  static_assert(SMEM_BYTES <= 232448, "shared memory per block");
};

// tile-blocked row layouts of the tetrahedral tensor-core path
__host__ __device__ __forceinline__ int tc3_row(int el, int c) { return (el / 10) * 32 + (el % 10) * 3 + c; }
__host__ __device__ __forceinline__ size_t tc3_index(int tile, int i, int r, int N) {
  return ((size_t)tile * N + i) * 128 + r;
}
// facet traces [tile][f][row][NFM4]: the modes of one (row, facet) contiguous, so a
// neighbour's trace is one short aligned run (two sectors at k = 4) read by vector loads
__host__ __device__ __forceinline__ size_t tc3_tr_index(int tile, int f, int m, int r, int NFM4) {
  return (((size_t)tile * 4 + f) * 128 + r) * NFM4 + m;
}

}  // namespace dgc
