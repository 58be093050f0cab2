// Compile-time layout of the tensor-core stage kernel for triangles (dim 2).
//
// One CTA handles a tile of 128 elements; element t of the tile is GEMM row t
// and TMEM lane t.  The dense contraction of the stage, the evaluation of the
// state and of the wind at the quadrature points, runs on tcgen05 with FP32
// accumulation in TMEM, every operand split into low-precision pieces:
//   TF32X3 (kind::tf32): two TF32 pieces (head, tail), three products
//          (hh + ht + th), about 22 significand bits per operand;
//   BF16X3 (kind::f16, both operands BF16): three BF16 pieces, which hold an
//          FP32 value exactly, six products (hh + hm + mh + hl + lh + mm).
//
//   GEMM A   X_f[128 x NA] = C_f[128 x NK] * TA[NA x NK]^T   for the fields
//            f = state components w_0, w_1 (TA = TAs: basis at the volume
//            points) and wind components u^_0/det J, u^_1/det J (TA = TAw:
//            weighted basis at the volume points and at the facet points).
//
// The test contractions (against the basis gradients at the volume points and
// against the facet restriction Ef) are narrow (N = dim P^k outputs per
// element and component) and run on CUDA cores in FP32 from the FP32 tables G
// and Ef.
//
// Operands are K-major without swizzle (see dgc_tc.cuh): a core matrix is 8
// rows x 16 bytes (4 TF32 or 8 BF16 values), LBO = 128 bytes between core
// matrices along K, SBO = (K / values per core row) * 128 bytes between 8-row
// groups.
#pragma once

namespace dgc {

enum TcPrec { kTf32x3 = 0, kBf16x3 = 1 };

template <int K, int P = kTf32x3>
struct TcLayout2D {
  static constexpr int pad(int n, int m) { return (n + m - 1) / m * m; }
  static constexpr int ESZ = P == kBf16x3 ? 2 : 4;     // operand element bytes
  static constexpr int PIECES = P == kBf16x3 ? 3 : 2;
  static constexpr int NPROD = P == kBf16x3 ? 6 : 3;   // products per field
  static constexpr int KSTEP = 32 / ESZ;               // K of one MMA (32 bytes)
  static constexpr int CORE_K = 16 / ESZ;              // K of one core matrix (16 bytes)
  static constexpr int D = 2;
  static constexpr int N = (K + 1) * (K + 2) / 2;
  static constexpr int NF = 3;
  static constexpr int NFM = K + 1;
  static constexpr int NQ1V = (3 * K - 1) / 2 + 1;
  static constexpr int QV = NQ1V * NQ1V;
  static constexpr int QF = (3 * K) / 2 + 1;
  static constexpr int NK = pad(N, 16);                // K of GEMM A (and of the wind layout)
  static constexpr int NAS = pad(QV, 16);              // N of the state GEMM A
  static constexpr int NAW = pad(QV + NF * QF, 16);    // N of the wind GEMM A

  // TMEM columns (FP32 accumulators)
  static constexpr int cS = 0;                         // state fields, NAS each
  static constexpr int cW = 2 * NAS;                   // wind fields, NAW each
  static constexpr int TMEM_USED = cW + 2 * NAW;
  static constexpr int TMEM_COLS = TMEM_USED <= 32 ? 32 : TMEM_USED <= 64 ? 64 : TMEM_USED <= 128 ? 128
                                 : TMEM_USED <= 256 ? 256 : 512;

  // table blob (32-bit words), sections each a multiple of 4 words
  static constexpr int szTAs = NAS * NK * ESZ / 4, szTAw = NAW * NK * ESZ / 4;   // one piece, in words
  static constexpr int NP4 = pad(N, 4);                // rows padded for 16-byte loads
  static constexpr int NFM4 = pad(NFM, 4);
  static constexpr int szG = QV * D * NP4;             // G[q][d][i] = d_d psi^_i (xi_q)
  static constexpr int szEf = NF * NFM * NP4, szQt = QF * NFM4;
  static constexpr int oTAs = 0;
  static constexpr int oTAw = oTAs + PIECES * szTAs;
  static constexpr int oEf = oTAw + PIECES * szTAw;
  static constexpr int oQt = oEf + szEf;
  static constexpr int oG = oQt + szQt;
  static constexpr int BLOB = oG + szG;
  // the blob part copied into shared memory: all of it, except G for k >= 6, which
  // the kernel then reads from global memory (through L1) to fit one CTA per SM
  static constexpr bool G_GLOBAL = K >= 6;
  static constexpr int SBLOB = G_GLOBAL ? oG : BLOB;

  // shared memory (floats): blob | wind staging | operand region
  static constexpr int WSTAGE = 128 * D * NK;          // wind coefficients of the tile
  static constexpr int szOpA = 128 * NK * ESZ / 4;     // one GEMM A operand piece, words
  static constexpr int OPREG = 2 * D * PIECES * szOpA; // 4 fields x pieces
  static constexpr int HALF_A = 2 * PIECES * szOpA;    // the state half (then the wind half)
  static constexpr int TSOA_TILE = D * N * 128;        // one tile block of a TSOA vector
  static constexpr int STG = 2 * TSOA_TILE;            // a tile's v^n (FP32) and stage increment
  // The next tile's staged state lives in the wind half when it fits there: it is
  // read before the wind operands are written and refilled once GEMM A has
  // completed; otherwise it has its own region.  Once GEMM A has completed, the
  // start of the operand region takes this tile's state again for the epilogue.
  static constexpr bool STG_ALIAS = STG <= HALF_A;
  static_assert(STG <= OPREG, "the epilogue's state must fit in the GEMM A operands");
  static constexpr int oWst = SBLOB;
  static constexpr int oOp = pad(oWst + WSTAGE, 32);   // 128-byte aligned
  static constexpr int oStg = STG_ALIAS ? oOp + HALF_A : oOp + OPREG;   // next tile's [vf | din]
  static constexpr int oEpi = oOp;                     // this tile's [vf | din] for the epilogue
  static constexpr int SMEM_FLOATS = STG_ALIAS ? oOp + OPREG : oStg + STG;
  static constexpr int SMEM_BYTES = SMEM_FLOATS * 4 + 256;   // + barriers

  static constexpr unsigned LBO = 128;                 // next core matrix along K
  static constexpr unsigned SBO_NK = (NK / CORE_K) * 128;   // next 8-row group
};

}  // namespace dgc
