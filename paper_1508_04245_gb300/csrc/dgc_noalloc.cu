// dgc_transfer_T_noalloc: the transpose transfer I^T without any device
// allocation at call time.
//
// dgc_transfer_T keeps its facet scratch (one value per element, local facet
// and facet moment) in a buffer the library allocates on the mesh handle at
// the first call.  Callers that may not allocate device memory when they
// call -- an application that reserves its device memory at start-up, or a
// host loop that must not block on the device-wide synchronisation of
// cudaMalloc / cudaFree -- use this variant instead: its scratch is a
// file-scope device array of fixed size, present on every GPU that loads the
// library until the process ends.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/dgconv.h"
#include "dgc_kernels.h"

namespace {

// 16 MiB of FP64 scratch: E * (facets per element) * n_fm doubles must fit.
constexpr long long kNoallocScratchDoubles = DGC_NOALLOC_SCRATCH_DOUBLES;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device; in host code the array's name is only a host-side stand-in).
cudaError_t scratch_address(double** out) {
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return err;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

namespace dgc {
// defined in dgc_api.cu: the device view of a handle and the error setter
bool mesh_view(const dgc_mesh* mesh, DevMesh* out);
dgc_status set_error(dgc_status code, const char* msg);
}  // namespace dgc

extern "C" dgc_status dgc_transfer_T_noalloc(dgc_mesh* mesh, const double* f_dg, double* g_hdiv, void* stream) {
  dgc::DevMesh m;
  if (!dgc::mesh_view(mesh, &m)) return dgc::set_error(DGC_ERR_ARG, "mesh handle is NULL");
  if (!f_dg || !g_hdiv) return dgc::set_error(DGC_ERR_ARG, "NULL vector");
  const long long need = (long long)m.E * m.s.NF * m.s.NFM;
  if (need > kNoallocScratchDoubles) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "dgc_transfer_T_noalloc: mesh needs %lld scratch doubles (elements x facets x facet moments), "
             "the fixed maximum is %lld; use dgc_transfer_T",
             need, kNoallocScratchDoubles);
    return dgc::set_error(DGC_ERR_ARG, buf);
  }
  double* scratch = nullptr;
  cudaError_t err = scratch_address(&scratch);
  if (err != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof(buf), "dgc_transfer_T_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(err));
    return dgc::set_error(DGC_ERR_CUDA, buf);
  }
  // every scratch entry the facet reduction reads is written first by this call
  err = dgc::launch_transfer_T(m, f_dg, g_hdiv, scratch, reinterpret_cast<cudaStream_t>(stream));
  if (err != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof(buf), "dgc_transfer_T_noalloc: launch failed: %s", cudaGetErrorString(err));
    return dgc::set_error(DGC_ERR_CUDA, buf);
  }
  return DGC_OK;
}
