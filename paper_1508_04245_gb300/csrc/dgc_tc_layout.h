// Compile-time layout of the tensor-core stage kernel for triangles (dim 2).
//
// One CTA handles a tile of 128 elements; element t of the tile is GEMM row t
// and TMEM lane t.  Two GEMMs per stage, both on tcgen05 (kind::tf32) with
// FP32 accumulation, each operand split into a TF32 head and a TF32 tail and
// multiplied in three passes (head*head + head*tail + tail*head):
//
//   GEMM A   X_f[128 x NA] = C_f[128 x NK] * TA[NA x NK]^T   for the fields
//            f = state components w_0, w_1 (TA = TAs: basis at the volume
//            points) and wind components u^_0/det J, u^_1/det J (TA = TAw:
//            weighted basis at the volume points and at the facet points).
//   GEMM B   R_c[128 x NB] = P_c[128 x KB] * TB[NB x KB]^T, where P_c holds
//            the upwind facet projections (K columns [0, KF)) and
//            -Uw[q][dd] w_c(xi_q) (K columns [KF, KF + 2 QV)); TB holds the
//            facet restriction Ef and the basis gradients G.
//
// Operands are K-major without swizzle (see dgc_tc.cuh): LBO = 128 bytes,
// SBO = (K / 4) * 128 bytes.
#pragma once

namespace dgc {

template <int K>
struct TcLayout2D {
  static constexpr int pad(int n, int m) { return (n + m - 1) / m * m; }
  static constexpr int D = 2;
  static constexpr int N = (K + 1) * (K + 2) / 2;
  static constexpr int NF = 3;
  static constexpr int NFM = K + 1;
  static constexpr int NQ1V = (3 * K - 1) / 2 + 1;
  static constexpr int QV = NQ1V * NQ1V;
  static constexpr int QF = (3 * K) / 2 + 1;
  static constexpr int NK = pad(N, 8);                 // K of GEMM A
  static constexpr int NAS = pad(QV, 16);              // N of the state GEMM A
  static constexpr int NAW = pad(QV + NF * QF, 16);    // N of the wind GEMM A
  static constexpr int NB = pad(N, 16);                // N of GEMM B
  static constexpr int KF = pad(NF * NFM, 8);          // facet part of GEMM B's K
  static constexpr int KV = pad(2 * QV, 8);            // volume part of GEMM B's K
  static constexpr int KB = KF + KV;
  static constexpr int NCH = KB / 8;                   // GEMM B K-chunks of 8
  static constexpr int NCHF = KF / 8;                  // of which facet chunks
  static constexpr int NSLOT = 2;                      // GEMM B chunk buffers

  // TMEM columns (FP32 accumulators)
  static constexpr int cS = 0;                         // state fields, NAS each
  static constexpr int cW = 2 * NAS;                   // wind fields, NAW each
  static constexpr int cB = 2 * NAS + 2 * NAW;         // GEMM B, NB each
  static constexpr int TMEM_USED = cB + 2 * NB;
  static constexpr int TMEM_COLS = TMEM_USED <= 32 ? 32 : TMEM_USED <= 64 ? 64 : TMEM_USED <= 128 ? 128
                                 : TMEM_USED <= 256 ? 256 : 512;

  // table blob (floats), sections in operand layout, each a multiple of 4 floats
  static constexpr int szTAs = NAS * NK, szTAw = NAW * NK, szTB = NB * KB;
  static constexpr int NP4 = pad(N, 4);                // Ef rows padded for 16-byte loads
  static constexpr int NFM4 = pad(NFM, 4);             // Qt rows padded for 16-byte loads
  static constexpr int szEf = NF * NFM * NP4, szQt = QF * NFM4;
  static constexpr int oTAs = 0;                       // head, tail
  static constexpr int oTAw = oTAs + 2 * szTAs;
  static constexpr int oTB = oTAw + 2 * szTAw;
  static constexpr int oEf = oTB + 2 * szTB;
  static constexpr int oQt = oEf + szEf;
  static constexpr int BLOB = oQt + szQt;

  // shared memory (floats): blob | wind staging | operand region (| state staging)
  static constexpr int WSTAGE = 128 * D * NK;          // wind coefficients of the tile
  static constexpr int TSOA_TILE = D * N * 128;        // one tile block of a TSOA vector
  static constexpr int STG = 2 * TSOA_TILE;            // the tile's v^n (FP32) and stage increment
  static constexpr int szOpA = 128 * NK;               // one GEMM A operand part
  static constexpr int szChunk = 128 * 8;              // one GEMM B chunk operand part
  static constexpr int OPREG_A = 2 * D * 2 * szOpA;    // 4 fields x head/tail
  static constexpr int OPREG_B = NSLOT * 2 * 2 * szChunk;   // slots x comps x head/tail
  static constexpr int OPREG = OPREG_A > OPREG_B ? OPREG_A : OPREG_B;
  static constexpr int oWst = BLOB;
  static constexpr int oOp = pad(oWst + WSTAGE, 32);   // 128-byte aligned
  // The tile's staged state lives in the wind-operand half of the GEMM A operands
  // when the GEMM B ring fits in the state half: it is read before the wind
  // operands are written and refilled for the next tile once GEMM A has completed.
  static constexpr int HALF_A = 2 * 2 * szOpA;
  static constexpr bool STG_ALIAS = OPREG_B <= HALF_A && STG <= HALF_A;
  static constexpr int oStg = STG_ALIAS ? oOp + HALF_A : pad(oOp + OPREG, 32);
  static constexpr int SMEM_FLOATS = STG_ALIAS ? oOp + OPREG : oStg + STG;
  static constexpr int SMEM_BYTES = SMEM_FLOATS * 4 + 256;   // + barriers

  static constexpr unsigned LBO = 128;
  static constexpr unsigned SBO_NK = (NK / 4) * 128;
  static constexpr unsigned SBO_KB = (KB / 4) * 128;
  static constexpr unsigned SBO_CH = (8 / 4) * 128;
};

}  // namespace dgc
