// Tensor-core stage kernel for tetrahedra: host tables (the BF16 table chunks
// of both GEMMs, split exactly into three pieces from the FP64 reference
// tables; the FP32 facet tables), launchers and the row-layout transposes.
#include <cstring>
#include <vector>

#include "dgc_kernels.h"
#include "dgc_stage_tc3.cuh"

namespace dgc {
namespace {

template <int K>
std::vector<unsigned char> chunks_t(const Tables& t) {
  using L = TcLayout3D<K>;
  constexpr int N = L::N, QV = L::QV;
  std::vector<unsigned char> b((size_t)L::NCH * L::CH_BYTES, 0);
  // head pieces on the grid of a table column, 2^(f - 8) for the largest magnitude
  // 2^f x [0.5, 1) in the column (integers of at most 256 units, exact in BF16),
  // the remainder (exact in FP64) in two BF16 pieces, so head x head products with
  // the grid-aligned operand rows sum exactly in FP32
  auto grid_of = [](double mx) {
    int ex = 0;
    std::frexp(mx, &ex);
    return mx > 0.0 ? std::ldexp(1.0, ex - 8) : 1.0;
  };
  auto put_grid = [&](size_t piece0, size_t piece_bytes, size_t off, double x, double g) {
    const double hd = std::nearbyint(x / g) * g;
    uint16_t ph[3], pr[3];
    bf16x3_pieces(hd, ph);
    bf16x3_pieces(x - hd, pr);
    const uint16_t pc[3] = {ph[0], pr[0], pr[1]};
    for (int k = 0; k < 3; ++k) std::memcpy(b.data() + piece0 + k * piece_bytes + off, &pc[k], 2);
  };
  for (int j = 0; j < L::NCH; ++j) {
    const size_t base = (size_t)j * L::CH_BYTES;
    for (int n = 0; n < L::QC; ++n) {
      const int q = j * L::QC + n;
      if (q >= QV) break;   // padding points: zero rows and columns
      // GEMM A table: row n (point), K index k (basis function), K-major core matrices;
      // its column of the product is the point, the grid the point's
      double mx = 0.0;
      for (int k = 0; k < N; ++k) mx = std::max(mx, std::fabs(t.Bv[(size_t)q * N + k]));
      const double g = grid_of(mx);
      for (int k = 0; k < N; ++k)
        put_grid(base + L::oBA, L::szBA, (size_t)((n & 7) * 16 + (n >> 3) * L::SBO_A + (k & 7) * 2 + (k >> 3) * 128),
                 t.Bv[(size_t)q * N + k], g);
    }
    // GEMM B tables, one per direction d: row i (basis function), K index n (point);
    // the column of the product is the basis function, its grid taken over the chunk's
    // 3 x 16 entries
    auto G = [&](int n, int i, int d) {
      const int q = j * L::QC + n;
      return q < QV ? -t.wv[q] * t.Gv[((size_t)q * N + i) * 3 + d] : 0.0;
    };
    for (int i = 0; i < N; ++i) {
      double mx = 0.0;
      for (int d = 0; d < 3; ++d)
        for (int n = 0; n < L::QC; ++n) mx = std::max(mx, std::fabs(G(n, i, d)));
      const double g = grid_of(mx);
      for (int d = 0; d < 3; ++d)
        for (int n = 0; n < L::QC; ++n)
          put_grid(base + L::oBG + (size_t)d * 3 * L::szBG, L::szBG,
                   (size_t)((i & 7) * 16 + (i >> 3) * L::SBO_G + (n & 7) * 2 + (n >> 3) * 128), G(n, i, d), g);
    }
  }
  return b;
}

template <int K>
std::vector<float> ftab_t(const Tables& t) {
  using L = TcLayout3D<K>;
  std::vector<float> f(L::FWT, 0.f);
  for (int fm = 0; fm < L::NF * L::NFM; ++fm)
    for (int i = 0; i < L::N; ++i) f[L::oEf + fm * L::NP4 + i] = (float)t.Ef[(size_t)fm * L::N + i];
  for (int q = 0; q < L::QF; ++q)
    for (int m = 0; m < L::NFM; ++m) f[L::oQt + q * L::NFM4 + m] = (float)t.Qt[(size_t)q * L::NFM + m];
  return f;
}

template <int K>
cudaError_t launch_t(const StageTcArgs* a, cudaStream_t s) {
  using L = TcLayout3D<K>;
  if (!a) return cudaFuncSetAttribute(stage_tc3_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM_BYTES);
  const int tiles = (a->E + L::EPT - 1) / L::EPT;
  if (tiles == 0) return cudaSuccess;
  // persistent: one CTA per SM (all of its tensor memory)
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int grid = tiles < sms ? tiles : sms;
  stage_tc3_kernel<K><<<grid, 640, L::SMEM_BYTES, s>>>(*a);
  return cudaGetLastError();
}

template <int K>
cudaError_t in_t(const double* v, double* vt, float* vft, float* tr, const float* ftab, int E, cudaStream_t s) {
  const int tiles = (E + TcLayout3D<K>::EPT - 1) / TcLayout3D<K>::EPT;
  if (tiles == 0) return cudaSuccess;
  tc3_in_kernel<K><<<tiles, 128, 0, s>>>(v, vt, vft, tr, ftab, E);
  return cudaGetLastError();
}

template <int K>
cudaError_t out_t(const double* vt, double* v, int E, cudaStream_t s) {
  const long n = 3L * E * TcLayout3D<K>::N;
  if (n == 0) return cudaSuccess;
  tc3_out_kernel<K><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(vt, v, E);
  return cudaGetLastError();
}

template <template <int> class F, typename... Args>
auto by_order(int K, Args... args) {
  switch (K) {
    case 1: return F<1>::run(args...);
    case 2: return F<2>::run(args...);
    case 3: return F<3>::run(args...);
    default: return F<4>::run(args...);
  }
}

template <int K>
struct Lens {
  static size_t run(int which, int E) {
    using L = TcLayout3D<K>;
    const size_t tiles = ((size_t)E + L::EPT - 1) / L::EPT;
    if (which == 0) return tiles * L::N * 128;
    if (which == 1) return tiles * L::NF * 128 * L::NFM4;
    return tiles * L::FWS;
  }
};

}  // namespace

std::vector<unsigned char> tc3_chunks(int K, const Tables& t) {
  switch (K) {
    case 1: return chunks_t<1>(t);
    case 2: return chunks_t<2>(t);
    case 3: return chunks_t<3>(t);
    case 4: return chunks_t<4>(t);
    default: return {};
  }
}

std::vector<float> tc3_ftab(int K, const Tables& t) {
  switch (K) {
    case 1: return ftab_t<1>(t);
    case 2: return ftab_t<2>(t);
    case 3: return ftab_t<3>(t);
    case 4: return ftab_t<4>(t);
    default: return {};
  }
}

cudaError_t launch_stage_tc3(int K, const StageTcArgs* a, cudaStream_t s) {
  switch (K) {
    case 1: return launch_t<1>(a, s);
    case 2: return launch_t<2>(a, s);
    case 3: return launch_t<3>(a, s);
    case 4: return launch_t<4>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

size_t tc3_rows_len(int K, int E) { return K >= 1 && K <= 4 ? by_order<Lens>(K, 0, E) : 0; }
size_t tc3_tr_len(int K, int E) { return K >= 1 && K <= 4 ? by_order<Lens>(K, 1, E) : 0; }
size_t tc3_fw_len(int K, int E) { return K >= 1 && K <= 4 ? by_order<Lens>(K, 2, E) : 0; }

cudaError_t launch_tc3_in(int K, const double* v, double* vt, float* vft, float* tr, const float* ftab, int E,
                          cudaStream_t s) {
  switch (K) {
    case 1: return in_t<1>(v, vt, vft, tr, ftab, E, s);
    case 2: return in_t<2>(v, vt, vft, tr, ftab, E, s);
    case 3: return in_t<3>(v, vt, vft, tr, ftab, E, s);
    case 4: return in_t<4>(v, vt, vft, tr, ftab, E, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tc3_out(int K, const double* vt, double* v, int E, cudaStream_t s) {
  switch (K) {
    case 1: return out_t<1>(vt, v, E, s);
    case 2: return out_t<2>(vt, v, E, s);
    case 3: return out_t<3>(vt, v, E, s);
    case 4: return out_t<4>(vt, v, E, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dgc
