// Tensor-core stage kernel: host table blob (GEMM A operands with the head/tail
// TF32 split of the FP64 reference tables, FP32 test tables) and launcher,
// triangles k = 1..4.
#include <cstring>
#include <vector>

#include "dgc_kernels.h"
#include "dgc_stage_tc.cuh"

namespace dgc {
namespace {

// round to TF32, nearest with ties away from zero (as cvt.rna.tf32.f32)
float tf32_rna(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x1000u;
  u &= 0xFFFFE000u;
  std::memcpy(&x, &u, 4);
  return x;
}

// BF16 bits of a value, round to nearest even (from its FP32 rounding)
uint16_t bf16_rn(double x) {
  const float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// byte offset of element (row, k) in a K-major operand of esz-byte elements (LBO 128 B)
size_t kbyte(int row, int k, unsigned sbo, int esz) {
  const int ck = 16 / esz;
  return (size_t)((row & 7) * 16 + (row >> 3) * sbo + (k % ck) * esz + (k / ck) * 128);
}

// value x of operand element (row, k) split into the pieces of the scheme; pieces
// start at word `base` of the blob and lie `size` words apart
template <int P>
void put_split(std::vector<float>& b, size_t base, size_t size, int row, int k, unsigned sbo, double x) {
  unsigned char* bytes = reinterpret_cast<unsigned char*>(b.data());
  if (P == kTf32x3) {
    const float h = tf32_rna((float)x);
    const float t = tf32_rna((float)(x - (double)h));
    const size_t o = kbyte(row, k, sbo, 4);
    std::memcpy(bytes + 4 * base + o, &h, 4);
    std::memcpy(bytes + 4 * (base + size) + o, &t, 4);
  } else {
    const uint16_t h = bf16_rn(x);
    const double r = x - bf16_value(h);
    const uint16_t m = bf16_rn(r);
    const uint16_t l = bf16_rn(r - bf16_value(m));
    const size_t o = kbyte(row, k, sbo, 2);
    std::memcpy(bytes + 4 * base + o, &h, 2);
    std::memcpy(bytes + 4 * (base + size) + o, &m, 2);
    std::memcpy(bytes + 4 * (base + 2 * size) + o, &l, 2);
  }
}

template <int K, int P>
std::vector<float> blob_t(const Tables& t) {
  using L = TcLayout2D<K, P>;
  const int N = L::N, QV = L::QV, QF = L::QF, NFM = L::NFM;
  std::vector<float> b(L::BLOB, 0.f);
  for (int n = 0; n < QV; ++n)
    for (int k = 0; k < N; ++k) {
      put_split<P>(b, L::oTAs, L::szTAs, n, k, L::SBO_NK, t.Bv[n * N + k]);
      put_split<P>(b, L::oTAw, L::szTAw, n, k, L::SBO_NK, t.wv[n] * t.Bv[n * N + k]);
    }
  for (int f = 0; f < L::NF; ++f)
    for (int q = 0; q < QF; ++q)
      for (int k = 0; k < N; ++k)
        put_split<P>(b, L::oTAw, L::szTAw, QV + f * QF + q, k, L::SBO_NK, t.wf[q] * t.Bf[(f * QF + q) * N + k]);
  for (int q = 0; q < QV; ++q)
    for (int dd = 0; dd < 2; ++dd)
      for (int i = 0; i < N; ++i) b[L::oG + (q * 2 + dd) * L::NP4 + i] = (float)t.Gv[(q * N + i) * 2 + dd];
  for (int fm = 0; fm < L::NF * NFM; ++fm)
    for (int i = 0; i < N; ++i) b[L::oEf + fm * L::NP4 + i] = (float)t.Ef[fm * N + i];
  for (int q = 0; q < QF; ++q)
    for (int m = 0; m < NFM; ++m) b[L::oQt + q * L::NFM4 + m] = (float)t.Qt[q * NFM + m];
  return b;
}

template <int K, int P>
cudaError_t launch_t(const StageTcArgs* a, cudaStream_t s) {
  using L = TcLayout2D<K, P>;
  static_assert(L::SMEM_BYTES <= 232448, "shared memory per block");
  static_assert(L::TMEM_COLS * tc_ctas_per_sm(K) <= 512, "tensor memory per SM");
  if (!a) {
    cudaError_t e0 = cudaFuncSetAttribute(stage_tc_kernel<K, P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          L::SMEM_BYTES);
    if (e0 == cudaSuccess)
      e0 = cudaFuncSetAttribute(stage_tc_kernel<K, P, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                L::SMEM_BYTES);
    if (e0 != cudaSuccess) return e0;
    return cudaFuncSetAttribute(stage_tc_kernel<K, P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                L::SMEM_BYTES);
  }
  const bool batch = a->list != nullptr;
  if (batch && a->mode == 3) return cudaErrorInvalidValue;
  auto kern = a->mode == 3 ? stage_tc_kernel<K, P, true>
                           : (batch ? stage_tc_kernel<K, P, false, true> : stage_tc_kernel<K, P, false>);
  const int tiles = batch ? a->batch_tiles : (a->E + 127) / 128;
  if (tiles == 0) return cudaSuccess;
  // persistent: two resident CTAs per SM for k <= 4 (shared memory and TMEM allow
  // two), one for k = 5, 6 (more than half of either)
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int per_sm = tc_ctas_per_sm(K);
  const int grid = tiles < per_sm * sms ? tiles : per_sm * sms;
  kern<<<grid, 288, L::SMEM_BYTES, s>>>(*a);
  return cudaGetLastError();
}

template <int K>
cudaError_t tsoa_in_t(const double* v, double* vt, float* vft, float* tr, const float* blob, int E,
                      cudaStream_t s) {
  const long n = 2L * E;
  if (n == 0) return cudaSuccess;
  tsoa_in_kernel<K><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, vt, vft, tr, blob, E);
  return cudaGetLastError();
}

template <int K>
cudaError_t tsoa_out_t(const double* vt, double* v, int E, cudaStream_t s) {
  const long n = 2L * E * TcLayout2D<K>::N;
  if (n == 0) return cudaSuccess;
  tsoa_out_kernel<K><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(vt, v, E);
  return cudaGetLastError();
}

template <int K>
cudaError_t tsoa_in64_t(const double* v, double* vt, int E, cudaStream_t s) {
  const long n = 2L * E * TcLayout2D<K>::N;
  if (n == 0) return cudaSuccess;
  tsoa_in64_kernel<K><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, vt, E);
  return cudaGetLastError();
}

template <int K>
cudaError_t tsoa_out_sel_t(const double* vt0, const double* vt1, const double* ctrl, double* v, int E,
                           cudaStream_t s) {
  const long n = 2L * E * TcLayout2D<K>::N;
  if (n == 0) return cudaSuccess;
  tsoa_out_sel_kernel<K><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(vt0, vt1, ctrl, v, E);
  return cudaGetLastError();
}

}  // namespace

void bf16x3_pieces(double x, uint16_t* p) {
  p[0] = bf16_rn(x);
  const double r = x - bf16_value(p[0]);
  p[1] = bf16_rn(r);
  p[2] = bf16_rn(r - bf16_value(p[1]));
}

cudaError_t launch_tsoa_in64(int D, int K, const double* v, double* vt, int E, cudaStream_t s) {
  if (D != 2) return cudaErrorInvalidValue;
  switch (K) {
    case 1: return tsoa_in64_t<1>(v, vt, E, s);
    case 2: return tsoa_in64_t<2>(v, vt, E, s);
    case 3: return tsoa_in64_t<3>(v, vt, E, s);
    case 4: return tsoa_in64_t<4>(v, vt, E, s);
    case 5: return tsoa_in64_t<5>(v, vt, E, s);
    case 6: return tsoa_in64_t<6>(v, vt, E, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tsoa_out_sel(int D, int K, const double* vt0, const double* vt1, const double* ctrl, double* v,
                                int E, cudaStream_t s) {
  if (D != 2) return cudaErrorInvalidValue;
  switch (K) {
    case 1: return tsoa_out_sel_t<1>(vt0, vt1, ctrl, v, E, s);
    case 2: return tsoa_out_sel_t<2>(vt0, vt1, ctrl, v, E, s);
    case 3: return tsoa_out_sel_t<3>(vt0, vt1, ctrl, v, E, s);
    case 4: return tsoa_out_sel_t<4>(vt0, vt1, ctrl, v, E, s);
    case 5: return tsoa_out_sel_t<5>(vt0, vt1, ctrl, v, E, s);
    case 6: return tsoa_out_sel_t<6>(vt0, vt1, ctrl, v, E, s);
    default: return cudaErrorInvalidValue;
  }
}

size_t tc_tsoa_len(int D, int K, int E) {
  const size_t tiles = ((size_t)E + 127) / 128;
  return tiles * 128 * D * ((size_t)(K + 1) * (K + 2) / 2);
}
size_t tc_tr_len(int D, int K, int E) {
  const size_t tiles = ((size_t)E + 127) / 128;
  return tiles * 128 * D * (D + 1) * (size_t)(K + 1);
}

cudaError_t launch_tsoa_in(int D, int K, const double* v, double* vt, float* vft, float* tr, const float* blob,
                           int E, cudaStream_t s) {
  if (D != 2) return cudaErrorInvalidValue;
  switch (K) {
    case 1: return tsoa_in_t<1>(v, vt, vft, tr, blob, E, s);
    case 2: return tsoa_in_t<2>(v, vt, vft, tr, blob, E, s);
    case 3: return tsoa_in_t<3>(v, vt, vft, tr, blob, E, s);
    case 4: return tsoa_in_t<4>(v, vt, vft, tr, blob, E, s);
    case 5: return tsoa_in_t<5>(v, vt, vft, tr, blob, E, s);
    case 6: return tsoa_in_t<6>(v, vt, vft, tr, blob, E, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tsoa_out(int D, int K, const double* vt, double* v, int E, cudaStream_t s) {
  if (D != 2) return cudaErrorInvalidValue;
  switch (K) {
    case 1: return tsoa_out_t<1>(vt, v, E, s);
    case 2: return tsoa_out_t<2>(vt, v, E, s);
    case 3: return tsoa_out_t<3>(vt, v, E, s);
    case 4: return tsoa_out_t<4>(vt, v, E, s);
    case 5: return tsoa_out_t<5>(vt, v, E, s);
    case 6: return tsoa_out_t<6>(vt, v, E, s);
    default: return cudaErrorInvalidValue;
  }
}

bool tc_supported(int D, int K) { return K >= 1 && (D == 2 ? K <= 6 : (D == 3 && K <= 4)); }

int tc_nk(int D, int K) {
  if (D != 2) return 0;
  switch (K) {
    case 1: return TcLayout2D<1>::NK;
    case 2: return TcLayout2D<2>::NK;
    case 3: return TcLayout2D<3>::NK;
    case 4: return TcLayout2D<4>::NK;
    case 5: return TcLayout2D<5>::NK;
    case 6: return TcLayout2D<6>::NK;
    default: return 0;
  }
}

std::vector<float> tc_blob(int D, int K, int P, const Tables& t) {
  if (D != 2) return {};
  switch (K * 2 + (P == kBf16x3 ? 1 : 0)) {
    case 2: return blob_t<1, kTf32x3>(t);
    case 3: return blob_t<1, kBf16x3>(t);
    case 4: return blob_t<2, kTf32x3>(t);
    case 5: return blob_t<2, kBf16x3>(t);
    case 6: return blob_t<3, kTf32x3>(t);
    case 7: return blob_t<3, kBf16x3>(t);
    case 8: return blob_t<4, kTf32x3>(t);
    case 9: return blob_t<4, kBf16x3>(t);
    case 10: return blob_t<5, kTf32x3>(t);
    case 11: return blob_t<5, kBf16x3>(t);
    case 12: return blob_t<6, kTf32x3>(t);
    case 13: return blob_t<6, kBf16x3>(t);
    default: return {};
  }
}

cudaError_t launch_stage_tc(int D, int K, int P, const StageTcArgs* a, cudaStream_t s) {
  if (D != 2) return cudaErrorInvalidValue;
  switch (K * 2 + (P == kBf16x3 ? 1 : 0)) {
    case 2: return launch_t<1, kTf32x3>(a, s);
    case 3: return launch_t<1, kBf16x3>(a, s);
    case 4: return launch_t<2, kTf32x3>(a, s);
    case 5: return launch_t<2, kBf16x3>(a, s);
    case 6: return launch_t<3, kTf32x3>(a, s);
    case 7: return launch_t<3, kBf16x3>(a, s);
    case 8: return launch_t<4, kTf32x3>(a, s);
    case 9: return launch_t<4, kBf16x3>(a, s);
    case 10: return launch_t<5, kTf32x3>(a, s);
    case 11: return launch_t<5, kBf16x3>(a, s);
    case 12: return launch_t<6, kTf32x3>(a, s);
    case 13: return launch_t<6, kBf16x3>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dgc
