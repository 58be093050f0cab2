// C-ABI of the dgconv library: argument checking, the mesh handle (host
// connectivity, device geometry, reference tables, scratch) and the launch
// sequences of the entry points declared in include/dgconv.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dgconv.h"
#include "dgc_kernels.h"
#include "dgc_stage.cuh"
#include "dgc_stage_tc.cuh"

using dgc::DevMesh;
using dgc::Sizes;

namespace {

thread_local std::string g_last_error;

// Host-side fault injection for tests of error propagation (no GPU is ever made
// to fault): DGC_FAULT=alloc makes device allocations fail, =capture makes graph
// captures fail to start, =launch makes kernel launches fail, each before the
// CUDA call is made; =stall launches the tensor-core stage kernels with no bulk
// copy issued and a short poll budget, so their bounded waits run out with
// nothing in flight and the timeout reaches the status word (dgc_check).
bool injected(const char* what) {
  const char* f = std::getenv("DGC_FAULT");
  return f && std::strcmp(f, what) == 0;
}

// NVTX range over one entry point (a no-op unless a profiler is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
#define DGC_RANGE() NvtxRange dgc_range_(__func__)

dgc_status fail(dgc_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define DGC_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t err_ = (call);                                                              \
    if (err_ != cudaSuccess)                                                                \
      return fail(DGC_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(err_),   \
                  __FILE__, __LINE__);                                                      \
  } while (0)

template <typename T>
struct DevBuf {
  T* ptr = nullptr;
  size_t n = 0;
  cudaError_t alloc(size_t count) {
    if (count <= n && ptr) return cudaSuccess;
    if (injected("alloc")) return cudaErrorMemoryAllocation;
    release();
    n = count;
    return cudaMalloc(&ptr, std::max<size_t>(count, 1) * sizeof(T));
  }
  cudaError_t upload(const std::vector<T>& v) {
    cudaError_t e = alloc(v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    n = 0;
  }
};

struct GraphKey {
  const double* wind;
  double* v;
  double ds;
  int nsteps, scheme, prec;
  bool stall;   // captured under DGC_FAULT=stall
  bool operator==(const GraphKey& o) const {
    return wind == o.wind && v == o.v && ds == o.ds && nsteps == o.nsteps && scheme == o.scheme &&
           prec == o.prec && stall == o.stall;
  }
};

}  // namespace

struct dgc_mesh;

namespace {
// cached graphs of dgc_batch_rk_substeps: key = every argument of the call
struct BatchGraph {
  std::vector<uint64_t> key;
  std::vector<dgc_mesh*> meshes;
  cudaGraphExec_t exec = nullptr;
  void* lists = nullptr;   // device stage argument lists and tile offsets of the merged groups
};
std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch_cache;
constexpr int kBatchBranches = 8;
cudaStream_t g_batch_streams[kBatchBranches + 1] = {nullptr};
}  // namespace

struct dgc_mesh {
  Sizes s;
  int E = 0, nF = 0, nV = 0;
  int quad = 0;                    // 1: parallelograms (dgc_mesh_upload_quad)
  int hex = 0;                     // 1: parallelepipeds (dgc_mesh_upload_hex)
  DevBuf<signed char> fcode;       // [E][6] face codes of a parallelepiped mesh
  DevBuf<float> q32[3];            // FP32 copies of v, v1, v2 in an FP32 RK sequence
  DevBuf<signed char> flip;        // [E][4] facet-parameter flips of a parallelogram mesh
  DevBuf<int> qnbr;                // [E][4] neighbour codes of the parallelogram stage kernel
  // curved (quadratic) triangles, dgc_mesh_upload_curved
  int Ec = 0;
  std::vector<int> h_cid;          // [E] curved index or -1
  std::vector<double> h_cnodes;    // [Ec][6][2]
  DevBuf<int> celem, cid;
  DevBuf<double> cnodes, p2d, p2v, Minv64;
  DevBuf<float> Minv32;
  std::vector<double> h_verts;     // [nV][D]
  std::vector<int> h_elems;        // [E][NF] sorted
  double h_min = 0.0;
  DevBuf<double> verts, J, detJ;
  DevBuf<int> elems, nbr, facet_id, facet_sides;
  DevBuf<signed char> orient;
  // FP64 tables
  DevBuf<double> Bv, wv, wf, Bf, Cb, Lg_int, Lg_fac, Tint, wd, wfd, Qfd, Bd;
  // stage-table blobs
  DevBuf<double> tab64;
  DevBuf<float> tab32, tcblob, tcblob16, wcoef, trA, trB;   // tensor-core blobs: TF32x3, BF16x3
  // tetrahedral tensor-core path: BF16 table chunks (the FP32 facet tables in tcblob),
  // the tile-blocked frozen facet flux and wind at the volume points, and the wind's
  // FP64 coefficients they are evaluated from
  DevBuf<unsigned char> tc3chunks;
  DevBuf<float> fw3, wq3;
  DevBuf<double> uc3;
  DevBuf<double> ts0;              // tile-blocked FP64 state of the tensor-core path
  DevBuf<float> tsf, d1, d2;       // its FP32 copy and the FP32 stage increments
  DevBuf<double> ts1, tsg;         // pseudo-time solve on that path: second state, right-hand side
  DevBuf<double> diag_mv, diag_part;   // dgc_diagnostics: M v and the per-block partial sums
  DevBuf<float> tsf1;              // and the second state's FP32 copy
  DevBuf<int> status;
  // scratch
  DevBuf<double> Uw64, Fw64, stage1, stage2, zbuf;
  DevBuf<float> Uw32, Fw32;
  DevBuf<unsigned long long> reduce;
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  GraphKey graph_key{};
  // H(div)-side compositions: DG state, its mass image, the mixed wind, the OIFS graph
  DevBuf<double> ov, omv, wmix;
  cudaGraphExec_t oifs_graph = nullptr;
  std::vector<uint64_t> oifs_key;
  // pseudo-time solve: residual, operator output, norm partials, [norm0, i], its graph
  DevBuf<double> rho, rop, partials, rstate;
  cudaStream_t body_stream = nullptr;
  cudaGraphExec_t rich_graph = nullptr;
  std::vector<uint64_t> rich_key;

  DevMesh view() const {
    DevMesh m;
    m.s = s;
    m.E = E;
    m.nF = nF;
    m.nV = nV;
    m.verts = verts.ptr;
    m.elems = elems.ptr;
    m.J = J.ptr;
    m.detJ = detJ.ptr;
    m.nbr = nbr.ptr;
    m.facet_id = facet_id.ptr;
    m.status = status.ptr;
#if DGC_CHECKED
    m.inject_bad_facet = injected("gather") ? 1 : 0;
#endif
    m.orient = orient.ptr;
    m.facet_sides = facet_sides.ptr;
    m.Bv = Bv.ptr;
    m.wv = wv.ptr;
    m.wf = wf.ptr;
    m.Bf = Bf.ptr;
    m.Cb = Cb.ptr;
    m.Lg_int = Lg_int.ptr;
    m.Lg_fac = Lg_fac.ptr;
    m.Tint = Tint.ptr;
    m.wd = wd.ptr;
    m.wfd = wfd.ptr;
    m.Qfd = Qfd.ptr;
    m.Bd = Bd.ptr;
    m.quad = quad;
    m.flip = flip.ptr;
    m.hex = hex;
    m.fcode = fcode.ptr;
    m.Ec = Ec;
    m.celem = celem.ptr;
    m.cid = Ec ? cid.ptr : nullptr;
    m.cnodes = cnodes.ptr;
    m.p2d = p2d.ptr;
    m.p2v = p2v.ptr;
    m.Minv64 = Minv64.ptr;
    m.Minv32 = Minv32.ptr;
    return m;
  }

  void release_all() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    if (rich_graph) cudaGraphExecDestroy(rich_graph);
    rich_graph = nullptr;
    if (oifs_graph) cudaGraphExecDestroy(oifs_graph);
    oifs_graph = nullptr;
    for (auto* b : {&ov, &omv, &wmix}) b->release();
    if (capture_stream) cudaStreamDestroy(capture_stream);
    capture_stream = nullptr;
    if (body_stream) cudaStreamDestroy(body_stream);
    body_stream = nullptr;
    for (auto* b : {&rho, &rop, &partials, &rstate}) b->release();
    for (auto* b : {&verts, &J, &detJ, &Bv, &wv, &wf, &Bf, &Cb, &Lg_int, &Lg_fac, &Tint, &wd, &wfd, &Qfd,
                    &Bd, &tab64, &Uw64, &Fw64, &stage1, &stage2, &zbuf})
      b->release();
    for (auto* b : {&elems, &nbr, &facet_id, &facet_sides}) b->release();
    orient.release();
    flip.release();
    fcode.release();
    for (auto& b : q32) b.release();
    qnbr.release();
    for (auto* b : {&celem, &cid}) b->release();
    for (auto* b : {&cnodes, &p2d, &p2v, &Minv64}) b->release();
    Minv32.release();
    tab32.release();
    tcblob.release();
    tcblob16.release();
    tc3chunks.release();
    fw3.release();
    wq3.release();
    diag_mv.release();
    diag_part.release();
    uc3.release();
    wcoef.release();
    trA.release();
    trB.release();
    ts0.release();
    tsf.release();
    ts1.release();
    tsg.release();
    tsf1.release();
    d1.release();
    d2.release();
    status.release();
    Uw32.release();
    Fw32.release();
    reduce.release();
  }
};

namespace {

// stage-table blob in the layout of dgc::StageTab (rows padded to 4 values)
template <typename T>
std::vector<T> stage_blob(const dgc::Tables& t) {
  const Sizes& s = t.s;
  const int D = s.D, N = s.N, NFM = s.NFM, NF = s.NF;
  const int NP4 = (N + 3) / 4 * 4, NFM4 = (NFM + 3) / 4 * 4;
  const size_t oG = (size_t)s.QV * NP4, oE = oG + (size_t)s.QV * D * NP4, oQ = oE + (size_t)NF * NFM * NP4;
  std::vector<T> out(oQ + (size_t)s.QF * NFM4, (T)0);
  for (int q = 0; q < s.QV; ++q)
    for (int i = 0; i < N; ++i) {
      out[(size_t)q * NP4 + i] = (T)t.Bv[(size_t)q * N + i];
      for (int d = 0; d < D; ++d) out[oG + ((size_t)q * D + d) * NP4 + i] = (T)t.Gv[((size_t)q * N + i) * D + d];
    }
  for (int fm = 0; fm < NF * NFM; ++fm)
    for (int i = 0; i < N; ++i) out[oE + (size_t)fm * NP4 + i] = (T)t.Ef[(size_t)fm * N + i];
  for (int q = 0; q < s.QF; ++q)
    for (int m = 0; m < NFM; ++m) out[oQ + (size_t)q * NFM4 + m] = (T)t.Qt[(size_t)q * NFM + m];
  return out;
}

// the 1D tables of the parallelogram stage kernel: l at the Gauss points | l' there | l(0), l(1)
template <typename T>
std::vector<T> quad_stage_blob(const dgc::Tables& t) {
  std::vector<T> out;
  for (const std::vector<double>* v : {&t.q1L, &t.q1D, &t.q1E})
    for (double x : *v) out.push_back((T)x);
  return out;
}

dgc_status check_mesh(const dgc_mesh* m) {
  if (!m) return fail(DGC_ERR_ARG, "mesh handle is NULL");
  return DGC_OK;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

dgc_status ensure_wind_scratch(dgc_mesh* m, bool fp32) {
  cudaError_t perr = m->hex        ? dgc::launch_stage_hex(m->s.K, fp32, nullptr, nullptr, nullptr)
                     : m->quad     ? dgc::launch_stage_quad(m->s.K, fp32, nullptr, nullptr)
                     : m->s.D == 2 ? dgc::launch_stage_2d(m->s.K, fp32, nullptr, nullptr)
                                   : dgc::launch_stage_3d(m->s.K, fp32, nullptr, nullptr);
  if (perr != cudaSuccess) return fail(DGC_ERR_CUDA, "stage kernel setup failed: %s", cudaGetErrorString(perr));
  const size_t nu = (size_t)m->s.QV * m->s.D * m->E, nf = (size_t)m->s.NF * m->s.QF * m->E;
  if (fp32) {
    DGC_CUDA(m->Uw32.alloc(nu));
    DGC_CUDA(m->Fw32.alloc(nf));
  } else {
    DGC_CUDA(m->Uw64.alloc(nu));
    DGC_CUDA(m->Fw64.alloc(nf));
  }
  return DGC_OK;
}

dgc_status launch_stage(dgc_mesh* m, bool fp32, const double* vin, const double* vn, double* vout,
                        double alpha, double beta, double gamma, cudaStream_t st, const float* vin32 = nullptr,
                        float* vout32 = nullptr) {
  if (injected("launch")) return fail(DGC_ERR_CUDA, "stage kernel launch failed (injected)");
  dgc::StageArgs a;
  a.vin = vin;
  a.vn = vn;
  a.vout = vout;
  a.Uw = fp32 ? (const void*)m->Uw32.ptr : (const void*)m->Uw64.ptr;
  a.Fw = fp32 ? (const void*)m->Fw32.ptr : (const void*)m->Fw64.ptr;
  a.nbr = (m->quad || m->hex) ? m->qnbr.ptr : m->nbr.ptr;
  a.tab = fp32 ? (const void*)m->tab32.ptr : (const void*)m->tab64.ptr;
  a.E = m->E;
  a.status = m->status.ptr;
  a.alpha = alpha;
  a.beta = beta;
  a.gamma = gamma;
  a.vin32 = vin32;
  a.vout32 = vout32;
  if (m->Ec > 0) {
    a.cid = m->cid.ptr;
    a.Minv = fp32 ? (const void*)m->Minv32.ptr : (const void*)m->Minv64.ptr;
    a.Ec = m->Ec;
  }
  cudaError_t err = m->hex        ? dgc::launch_stage_hex(m->s.K, fp32, &a, m->fcode.ptr, st)
                    : m->quad     ? dgc::launch_stage_quad(m->s.K, fp32, &a, st)
                    : m->s.D == 2 ? dgc::launch_stage_2d(m->s.K, fp32, &a, st)
                                  : dgc::launch_stage_3d(m->s.K, fp32, &a, st);
  if (err != cudaSuccess) return fail(DGC_ERR_CUDA, "stage kernel launch failed: %s", cudaGetErrorString(err));
  return DGC_OK;
}

// the tensor-core precisions (split operands on tcgen05)
bool is_tc(dgc_prec prec) { return prec == DGC_TF32X3 || prec == DGC_BF16X3; }

// the tensor-core stage kernels cover triangles with k <= 6 and tetrahedra with k <= 4
bool mesh_tc(const dgc_mesh* m) {
  return !m->quad && !m->hex && m->Ec == 0 && dgc::tc_supported(m->s.D, m->s.K);
}

dgc_status check_prec(const dgc_mesh* m, dgc_prec prec) {
  if (prec == DGC_FP64 || prec == DGC_FP32) return DGC_OK;
  if (is_tc(prec)) {
    if (mesh_tc(m) && m->s.D == 3 && prec == DGC_TF32X3)
      return fail(DGC_ERR_UNSUPPORTED, "DGC_TF32X3 is available for triangles; tetrahedra take DGC_BF16X3");
    if (mesh_tc(m)) return DGC_OK;
    return fail(DGC_ERR_UNSUPPORTED, "%s is available for affine triangles with k <= 6 and tetrahedra with k <= 4 (dim %d, k %d%s)",
                prec == DGC_TF32X3 ? "DGC_TF32X3" : "DGC_BF16X3", m->s.D, m->s.K,
                m->quad ? ", parallelograms" : (m->hex ? ", parallelepipeds" : (m->Ec ? ", curved elements" : "")));
  }
  return fail(DGC_ERR_ARG, "unknown precision %d", (int)prec);
}

dgc_status ensure_tc_scratch(dgc_mesh* m) {
  if (m->s.D == 3) {
    cudaError_t perr = dgc::launch_stage_tc3(m->s.K, nullptr, nullptr);
    if (perr != cudaSuccess)
      return fail(DGC_ERR_CUDA, "tensor-core stage setup failed: %s", cudaGetErrorString(perr));
    const size_t nt = dgc::tc3_rows_len(m->s.K, m->E), nr = dgc::tc3_tr_len(m->s.K, m->E);
    const size_t nw = dgc::tc3_fw_len(m->s.K, m->E);
    // the wind at the points is written in full (zero at padding points and elements)
    DGC_CUDA(m->wq3.alloc((size_t)dgc::wind_pts_tc3_len(m->s.QV, m->E)));
    DGC_CUDA(m->uc3.alloc(((size_t)m->E + 39) / 40 * 3 * m->s.N * 40));
    // facet flux entries the kernel never writes (elements past E) must read as zero
    if (m->fw3.n < nw) {
      DGC_CUDA(m->fw3.alloc(nw));
      DGC_CUDA(cudaMemset(m->fw3.ptr, 0, nw * sizeof(float)));
    }
    DGC_CUDA(m->ts0.alloc(nt));
    DGC_CUDA(m->tsf.alloc(nt));
    DGC_CUDA(m->d1.alloc(nt));
    DGC_CUDA(m->d2.alloc(nt));
    DGC_CUDA(m->trA.alloc(nr));
    DGC_CUDA(m->trB.alloc(nr));
    return DGC_OK;
  }
  for (int P = 0; P < 2; ++P) {
    cudaError_t perr = dgc::launch_stage_tc(m->s.D, m->s.K, P, nullptr, nullptr);
    if (perr != cudaSuccess)
      return fail(DGC_ERR_CUDA, "tensor-core stage setup failed: %s", cudaGetErrorString(perr));
  }
  DGC_CUDA(m->wcoef.alloc(((size_t)m->E + 127) / 128 * 128 * m->s.D * dgc::tc_nk(m->s.D, m->s.K)));
  const size_t nt = dgc::tc_tsoa_len(m->s.D, m->s.K, m->E), nr = dgc::tc_tr_len(m->s.D, m->s.K, m->E);
  DGC_CUDA(m->ts0.alloc(nt));
  DGC_CUDA(m->tsf.alloc(nt));
  DGC_CUDA(m->d1.alloc(nt));
  DGC_CUDA(m->d2.alloc(nt));
  DGC_CUDA(m->trA.alloc(nr));
  DGC_CUDA(m->trB.alloc(nr));
  return DGC_OK;
}

// the arguments of one tensor-core stage in increment form (see dgc::StageTcArgs)
dgc::StageTcArgs tc_args(dgc_mesh* m, dgc_prec prec, int mode, const float* din, const float* trin, float* dout,
                         float* trout, double p, double q, double* v) {
  const int P = prec == DGC_BF16X3 ? 1 : 0;
  dgc::StageTcArgs a{};   // every pointer a mode does not use is null
  a.vf = m->tsf.ptr;
  a.din = din;
  a.trin = trin;
  a.dout = dout;
  a.v = v;
  a.vf_out = m->tsf.ptr;
  a.trout = trout;
  a.wcoef = m->wcoef.ptr;
  a.nbr = m->nbr.ptr;
  a.blob = P ? m->tcblob16.ptr : m->tcblob.ptr;
  a.status = m->status.ptr;
  a.E = m->E;
  a.mode = mode;
  a.p_hi = (float)p;
  a.p_lo = (float)(p - (double)a.p_hi);
  a.q_hi = (float)q;
  a.q_lo = (float)(q - (double)a.q_hi);
  if (injected("stall")) {
    a.stall = 1;
    a.poll = 1u << 12;
  }
  if (m->s.D == 3) {
    a.blob = reinterpret_cast<const float*>(m->tc3chunks.ptr);
    a.ftab = m->tcblob.ptr;
    a.fw3 = m->fw3.ptr;
    a.wq3 = m->wq3.ptr;
  }
  return a;
}

// stage j of an SSP-RK substep in increment form on the tensor-core path:
//   RK3: d1 = ds L(v),  d2 = d1/4 + ds/4 L(v + d1),  v += 2/3 d2 + 2/3 ds L(v + d2)
//   RK2: d1 = ds L(v),  v += d1/2 + ds/2 L(v + d1)
// (identical to the Shu-Osher / Heun forms).  Each stage reads the facet traces of its
// input from one buffer and writes those of its output to the other; RK3 has an odd
// number of stages, so `parity` (the substep's number mod 2) says which buffer holds v's.
dgc::StageTcArgs tc_rk_stage(dgc_mesh* m, dgc_prec prec, int scheme, int parity, int j, double ds) {
  float* cur = parity ? m->trB.ptr : m->trA.ptr;
  float* oth = parity ? m->trA.ptr : m->trB.ptr;
  if (scheme == DGC_SSPRK2) {
    if (j == 0) return tc_args(m, prec, 0, nullptr, cur, m->d1.ptr, oth, 0.0, ds, nullptr);
    return tc_args(m, prec, 1, m->d1.ptr, oth, nullptr, cur, 0.5, 0.5 * ds, m->ts0.ptr);
  }
  if (j == 0) return tc_args(m, prec, 0, nullptr, cur, m->d1.ptr, oth, 0.0, ds, nullptr);
  if (j == 1) return tc_args(m, prec, 0, m->d1.ptr, oth, m->d2.ptr, cur, 0.25, 0.25 * ds, nullptr);
  return tc_args(m, prec, 1, m->d2.ptr, cur, nullptr, oth, 2.0 / 3.0, 2.0 / 3.0 * ds, m->ts0.ptr);
}

// launch one tensor-core stage (or, with a.list set, a batched stage over the triangle
// meshes of one order, dim and precision given by d, k, prec)
dgc_status launch_tc(int d, int k, dgc_prec prec, const dgc::StageTcArgs& a, cudaStream_t st) {
  if (injected("launch")) return fail(DGC_ERR_CUDA, "tensor-core stage launch failed (injected)");
  cudaError_t err = d == 3 ? dgc::launch_stage_tc3(k, &a, st)
                           : dgc::launch_stage_tc(d, k, prec == DGC_BF16X3 ? 1 : 0, &a, st);
  if (err != cudaSuccess) return fail(DGC_ERR_CUDA, "tensor-core stage launch failed: %s", cudaGetErrorString(err));
  return DGC_OK;
}

// one tensor-core stage in increment form (see dgc::StageTcArgs)
dgc_status launch_stage_tc(dgc_mesh* m, dgc_prec prec, int mode, const float* din, const float* trin, float* dout,
                           float* trout, double p, double q, double* v, cudaStream_t st) {
  return launch_tc(m->s.D, m->s.K, prec, tc_args(m, prec, mode, din, trin, dout, trout, p, q, v), st);
}

// one fused pseudo-time iteration on the tensor-core path (mode 3 of dgc::StageTcArgs)
dgc_status launch_rich_tc(dgc_mesh* m, dgc_prec prec, double tau, double ds, cudaStream_t st) {
  const int P = prec == DGC_BF16X3 ? 1 : 0;
  if (injected("launch")) return fail(DGC_ERR_CUDA, "tensor-core stage launch failed (injected)");
  dgc::StageTcArgs a{};
  a.din = nullptr;
  a.wcoef = m->wcoef.ptr;
  a.nbr = m->nbr.ptr;
  a.blob = P ? m->tcblob16.ptr : m->tcblob.ptr;
  a.status = m->status.ptr;
  a.E = m->E;
  a.mode = 3;
  a.ctrl = m->rstate.ptr;
  a.vf2[0] = m->tsf.ptr;
  a.vf2[1] = m->tsf1.ptr;
  a.tr2[0] = m->trA.ptr;
  a.tr2[1] = m->trB.ptr;
  a.v2[0] = m->ts0.ptr;
  a.v2[1] = m->ts1.ptr;
  a.g = m->tsg.ptr;
  a.detJ = m->detJ.ptr;
  a.tau = tau;
  a.ds = ds;
  a.partials = m->partials.ptr;
  cudaError_t err = dgc::launch_stage_tc(m->s.D, m->s.K, P, &a, st);
  if (err != cudaSuccess) return fail(DGC_ERR_CUDA, "tensor-core stage launch failed: %s", cudaGetErrorString(err));
  return DGC_OK;
}

dgc_status tc_transpose_in(dgc_mesh* m, const double* v, float* tr, cudaStream_t st) {
  cudaError_t err = m->s.D == 3
                        ? dgc::launch_tc3_in(m->s.K, v, m->ts0.ptr, m->tsf.ptr, tr, m->tcblob.ptr, m->E, st)
                        : dgc::launch_tsoa_in(m->s.D, m->s.K, v, m->ts0.ptr, m->tsf.ptr, tr, m->tcblob.ptr, m->E, st);
  if (err != cudaSuccess) return fail(DGC_ERR_CUDA, "layout transpose failed: %s", cudaGetErrorString(err));
  return DGC_OK;
}

dgc_status tc_transpose_out(dgc_mesh* m, const double* vt, double* v, cudaStream_t st) {
  cudaError_t err = m->s.D == 3 ? dgc::launch_tc3_out(m->s.K, vt, v, m->E, st)
                                : dgc::launch_tsoa_out(m->s.D, m->s.K, vt, v, m->E, st);
  if (err != cudaSuccess) return fail(DGC_ERR_CUDA, "layout transpose failed: %s", cudaGetErrorString(err));
  return DGC_OK;
}

// The wind of the propagation: frozen (prev == nullptr, prepared once before the
// substeps) or extrapolated linearly from (now, prev) to the midpoint of each
// substep, theta_j = (j + 1/2) ds / dt_prev, wind_j = (1 + theta_j) now - theta_j prev.
struct WindPlan {
  const double* now = nullptr;
  const double* prev = nullptr;
  double dt_prev = 0.0;
};

dgc_status prepare_wind(dgc_mesh* m, dgc_prec prec, const double* wind, cudaStream_t st);

dgc_status substep_wind(dgc_mesh* m, dgc_prec prec, const WindPlan& w, double ds, int j, cudaStream_t st) {
  if (!w.prev) return DGC_OK;
  const double theta = (j + 0.5) * ds / w.dt_prev;
  dgc::CombineArgs a{};
  a.x[0] = w.now;
  a.x[1] = w.prev;
  a.c[0] = 1.0 + theta;
  a.c[1] = -theta;
  a.nterms = 2;
  const long n = (long)m->nF * m->s.NFM + (long)m->E * m->s.NINT;
  DGC_CUDA(dgc::launch_combine(m->wmix.ptr, a, n, st));
  return prepare_wind(m, prec, m->wmix.ptr, st);
}

// SSP-RK substeps on the tensor-core path, increment form (tc_rk_stage): v^(i) = v^n + d_i;
// the state v is accumulated in FP64 once per substep, the increments are FP32.
// ABI -> TSOA once, back at the end.
dgc_status rk_sequence_tc(dgc_mesh* m, dgc_prec prec, double* v, double ds, int nsteps, int scheme,
                          const WindPlan& wp, cudaStream_t st) {
  if (dgc_status rc = tc_transpose_in(m, v, m->trA.ptr, st)) return rc;
  const int stages = scheme == DGC_SSPRK2 ? 2 : 3;
  for (int n = 0; n < nsteps; ++n) {
    if (dgc_status rc = substep_wind(m, prec, wp, ds, n, st)) return rc;
    const int parity = scheme == DGC_SSPRK2 ? 0 : (n & 1);
    for (int j = 0; j < stages; ++j)
      if (dgc_status rc = launch_tc(m->s.D, m->s.K, prec, tc_rk_stage(m, prec, scheme, parity, j, ds), st)) return rc;
  }
  return tc_transpose_out(m, m->ts0.ptr, v, st);
}

// one stage vout = alpha vn + beta vin + gamma L(vin), any precision
dgc_status stage(dgc_mesh* m, dgc_prec prec, const double* vin, const double* vn, double* vout, double alpha,
                 double beta, double gamma, cudaStream_t st, const float* vin32 = nullptr, float* vout32 = nullptr) {
  return launch_stage(m, prec == DGC_FP32, vin, vn, vout, alpha, beta, gamma, st, vin32, vout32);
}

// frozen-wind data for the chosen precision
dgc_status prepare_wind(dgc_mesh* m, dgc_prec prec, const double* wind, cudaStream_t st) {
  cudaError_t err;
  if (is_tc(prec) && m->s.D == 3) {
    err = dgc::launch_wind_tc3(m->view(), wind, m->uc3.ptr, m->wq3.ptr, m->fw3.ptr, st);
  } else if (is_tc(prec)) {
    err = dgc::launch_wind_coeffs(m->view(), wind, m->wcoef.ptr, dgc::tc_nk(m->s.D, m->s.K), st);
  } else {
    const bool fp32 = prec == DGC_FP32;
    err = dgc::launch_wind_prep(m->view(), wind, fp32 ? (void*)m->Uw32.ptr : (void*)m->Uw64.ptr,
                                fp32 ? (void*)m->Fw32.ptr : (void*)m->Fw64.ptr, fp32, st);
  }
  if (err != cudaSuccess) return fail(DGC_ERR_CUDA, "wind preparation failed: %s", cudaGetErrorString(err));
  return DGC_OK;
}

dgc_status ensure_prec_scratch(dgc_mesh* m, dgc_prec prec) {
  if (is_tc(prec)) return ensure_tc_scratch(m);
  if (prec == DGC_FP32 && !m->hex)
    for (auto& b : m->q32) DGC_CUDA(b.alloc((size_t)m->E * m->s.D * m->s.N));
  return ensure_wind_scratch(m, prec == DGC_FP32);
}

// The launch sequence of dgc_rk_substeps (also what gets captured); with
// wind_prev the wind is extrapolated per substep (see WindPlan).
dgc_status rk_sequence(dgc_mesh* m, const double* wind, double* v, double ds, int nsteps, int scheme, dgc_prec prec,
                       cudaStream_t st, const double* wind_prev = nullptr, double dt_prev = 0.0) {
  WindPlan wp;
  wp.now = wind;
  wp.prev = wind_prev;
  wp.dt_prev = dt_prev;
  if (!wind_prev)
    if (dgc_status rc = prepare_wind(m, prec, wind, st)) return rc;
  if (is_tc(prec)) return rk_sequence_tc(m, prec, v, ds, nsteps, scheme, wp, st);
  double* v1 = m->stage1.ptr;
  double* v2 = m->stage2.ptr;
  // FP32 contractions (simplices, curved triangles, parallelograms) carry FP32 copies
  // of v, v1, v2 from stage to stage
  const bool mirror = prec == DGC_FP32 && !m->hex && nsteps > 0;
  float* f0 = mirror ? m->q32[0].ptr : nullptr;
  float* f1 = mirror ? m->q32[1].ptr : nullptr;
  float* f2 = mirror ? m->q32[2].ptr : nullptr;
  if (mirror) DGC_CUDA(dgc::launch_to_float(v, f0, (long)m->E * m->s.D * m->s.N, st));
  for (int n = 0; n < nsteps; ++n) {
    dgc_status rc;
    if ((rc = substep_wind(m, prec, wp, ds, n, st))) return rc;
    if (scheme == DGC_SSPRK2) {
      // v1 = v + ds L(v);  v = 1/2 v + 1/2 (v1 + ds L(v1))
      if ((rc = stage(m, prec, v, nullptr, v1, 0.0, 1.0, ds, st, f0, f1))) return rc;
      if ((rc = stage(m, prec, v1, v, v, 0.5, 0.5, 0.5 * ds, st, f1, f0))) return rc;
    } else {
      // Shu-Osher SSP-RK3
      if ((rc = stage(m, prec, v, nullptr, v1, 0.0, 1.0, ds, st, f0, f1))) return rc;
      if ((rc = stage(m, prec, v1, v, v2, 0.75, 0.25, 0.25 * ds, st, f1, f2))) return rc;
      if ((rc = stage(m, prec, v2, v, v, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0 * ds, st, f2, f0))) return rc;
    }
  }
  return DGC_OK;
}

// begin a stream capture (fails before any CUDA call under DGC_FAULT=capture)
cudaError_t begin_capture(cudaStream_t st) {
  if (injected("capture")) return cudaErrorStreamCaptureUnsupported;
  return cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
}

// forget the cached batch graphs that contain this mesh
void drop_batch_graphs(const dgc_mesh* mesh) {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  for (size_t j = 0; j < g_batch_cache.size();) {
    BatchGraph& b = g_batch_cache[j];
    if (std::find(b.meshes.begin(), b.meshes.end(), mesh) != b.meshes.end()) {
      if (b.exec) cudaGraphExecDestroy(b.exec);
      if (b.lists) cudaFree(b.lists);
      g_batch_cache.erase(g_batch_cache.begin() + j);
    } else {
      ++j;
    }
  }
}

// out = (M^V)^-1 C^V w = -L(w) with the wind prepared for prec
dgc_status apply_operator(dgc_mesh* m, dgc_prec prec, const double* w, double* out, cudaStream_t st) {
  if (is_tc(prec)) {
    if (dgc_status rc = tc_transpose_in(m, w, m->trA.ptr, st)) return rc;
    // mode 2 with q = -1: v <- -L(w)
    if (dgc_status rc =
            launch_stage_tc(m, prec, 2, nullptr, m->trA.ptr, nullptr, nullptr, 0.0, -1.0, m->ts0.ptr, st))
      return rc;
    return tc_transpose_out(m, m->ts0.ptr, out, st);
  }
  return stage(m, prec, w, nullptr, out, 0.0, 0.0, -1.0, st);
}

// rho = g - v - tau A v with the norm partials, then the control kernel
dgc_status rich_step(dgc_mesh* m, dgc_prec prec, const double* g, const double* v, double tau, double reduction,
                     int max_iter, bool first, cudaGraphConditionalHandle h, int32_t* iters, double* res,
                     cudaStream_t st) {
  const long n = (long)m->E * m->s.D * m->s.N;
  const int nb = dgc::rich_blocks(n);
  if (dgc_status rc = apply_operator(m, prec, v, m->rop.ptr, st)) return rc;
  DGC_CUDA(dgc::launch_rich_resid(g, v, m->rop.ptr, tau, m->rho.ptr, m->detJ.ptr, m->s.D * m->s.N, n,
                                  m->partials.ptr, nb, st));
  DGC_CUDA(dgc::launch_rich_control(m->partials.ptr, nb, m->rstate.ptr, iters, res, reduction, max_iter, first, h,
                                    m->status.ptr, st));
  return DGC_OK;
}

// Graph of the whole solve: wind, first residual and decision, then
// WHILE(continue) { v += ds rho; residual; decision }.
dgc_status rich_build(dgc_mesh* m, const double* wind, const double* g, double* v, double tau, double ds,
                      double reduction, int max_iter, dgc_prec prec, int32_t* iters, double* res,
                      cudaGraphExec_t* out) {
  if (!m->capture_stream) DGC_CUDA(cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking));
  if (!m->body_stream) DGC_CUDA(cudaStreamCreateWithFlags(&m->body_stream, cudaStreamNonBlocking));
  cudaStream_t cs = m->capture_stream, bs = m->body_stream;
  const long n = (long)m->E * m->s.D * m->s.N;
  // tensor-core precisions on triangles: the iteration stays in the tile-blocked layout, fused into
  // the stage kernel (tetrahedra take the separate kernels around the tensor-core operator)
  const bool tc = is_tc(prec) && m->s.D == 2;
  const int ntiles = (m->E + 127) / 128;
  DGC_CUDA(begin_capture(cs));
  cudaGraph_t graph = nullptr;
  dgc_status rc = DGC_OK;
  cudaError_t err = cudaSuccess;
  cudaGraphConditionalHandle h = 0;
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t cond;
  do {
    if ((err = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, nullptr, nullptr, nullptr)) != cudaSuccess) break;
    if ((err = cudaGraphConditionalHandleCreate(&h, graph, 0, 0)) != cudaSuccess) break;
    if ((rc = prepare_wind(m, prec, wind, cs))) break;
    if (tc) {
      // tile-blocked state (set 0) and right-hand side; iteration count 0 selects set 0
      if ((err = cudaMemsetAsync(m->rstate.ptr, 0, 2 * sizeof(double), cs)) != cudaSuccess) break;
      if ((rc = tc_transpose_in(m, v, m->trA.ptr, cs))) break;
      if ((err = dgc::launch_tsoa_in64(m->s.D, m->s.K, g, m->tsg.ptr, m->E, cs)) != cudaSuccess) break;
      if ((rc = launch_rich_tc(m, prec, tau, ds, cs))) break;
      if ((err = dgc::launch_rich_control(m->partials.ptr, ntiles, m->rstate.ptr, iters, res, reduction, max_iter,
                                          true, h, m->status.ptr, cs)) != cudaSuccess)
        break;
    } else if ((rc = rich_step(m, prec, g, v, tau, reduction, max_iter, true, h, iters, res, cs))) {
      break;
    }
    if ((err = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, &deps, nullptr, &ndeps)) != cudaSuccess) break;
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if ((err = cudaGraphAddNode(&cond, graph, deps, nullptr, ndeps, &cp)) != cudaSuccess) break;
    if ((err = cudaStreamUpdateCaptureDependencies(cs, &cond, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
      break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((err = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      break;
    cudaError_t e1 = cudaSuccess;
    dgc_status rc1 = DGC_OK;
    if (tc) {
      // one fused iteration: operator, residual, next iterate (other buffer set), partials
      rc1 = launch_rich_tc(m, prec, tau, ds, bs);
      if (rc1 == DGC_OK)
        e1 = dgc::launch_rich_control(m->partials.ptr, ntiles, m->rstate.ptr, iters, res, reduction, max_iter,
                                      false, h, m->status.ptr, bs);
    } else {
      e1 = dgc::launch_rich_update(v, m->rho.ptr, ds, n, bs);
      if (e1 == cudaSuccess) rc1 = rich_step(m, prec, g, v, tau, reduction, max_iter, false, h, iters, res, bs);
    }
    cudaError_t e2 = cudaStreamEndCapture(bs, &body);
    if (rc1) rc = rc1;
    else if (e1 != cudaSuccess) err = e1;
    else if (e2 != cudaSuccess) err = e2;
    if (rc != DGC_OK || err != cudaSuccess) break;
    // after the loop: the accepted iterate back to the caller's layout
    if (tc && (err = dgc::launch_tsoa_out_sel(m->s.D, m->s.K, m->ts0.ptr, m->ts1.ptr, m->rstate.ptr, v, m->E, cs)) !=
                  cudaSuccess)
      break;
  } while (false);
  cudaGraph_t done = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(cs, &done);
  if (rc != DGC_OK || err != cudaSuccess || e3 != cudaSuccess) {
    if (done) cudaGraphDestroy(done);
    if (rc != DGC_OK) return rc;
    return fail(DGC_ERR_CUDA, "pseudo-time graph construction failed: %s",
                cudaGetErrorString(err != cudaSuccess ? err : e3));
  }
  err = cudaGraphInstantiate(out, done, 0);
  cudaGraphDestroy(done);
  if (err != cudaSuccess) {
    *out = nullptr;
    return fail(DGC_ERR_CUDA, "pseudo-time graph instantiation failed: %s", cudaGetErrorString(err));
  }
  return DGC_OK;
}

}  // namespace

namespace dgc {
// autotuned threads per block of the CUDA-core stage kernel, [dim - 2][k][fp32]; 0 = default
std::atomic<int> g_stage_block[2][7][2];
int stage_block_get(int D, int K, bool fp32) {
  if (D < 2 || D > 3 || K < 1 || K > 6) return 0;
  return g_stage_block[D - 2][K][fp32 ? 1 : 0].load(std::memory_order_relaxed);
}
// helpers for entry points defined in other translation units
bool mesh_view(const dgc_mesh* mesh, DevMesh* out) {
  if (!mesh) return false;
  *out = mesh->view();
  return true;
}
dgc_status set_error(dgc_status code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace dgc

extern "C" {

dgc_status dgc_last_error(char* buf, int len) {
  if (!buf || len <= 0) return DGC_ERR_ARG;
  snprintf(buf, (size_t)len, "%s", g_last_error.c_str());
  return DGC_OK;
}

dgc_status dgc_mesh_upload(int dim, int k, int n_vert, const double* verts, int n_elem, const int32_t* elems,
                           void* stream, dgc_mesh** out) {
  DGC_RANGE();
  if (!out) return fail(DGC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (dim != 2 && dim != 3) return fail(DGC_ERR_UNSUPPORTED, "dim must be 2 or 3 (got %d)", dim);
  if (!dgc::supported(dim, k)) return fail(DGC_ERR_UNSUPPORTED, "order k=%d not supported for dim %d", k, dim);
  if (n_vert <= 0 || n_elem <= 0 || !verts || !elems)
    return fail(DGC_ERR_ARG, "empty mesh or NULL arrays (n_vert=%d, n_elem=%d)", n_vert, n_elem);
  const int NF = dim + 1;
  dgc_mesh* m = new dgc_mesh();
  m->s = dgc::make_sizes(dim, k);
  m->E = n_elem;
  m->nV = n_vert;
  m->h_verts.assign(verts, verts + (size_t)n_vert * dim);
  m->h_elems.assign(elems, elems + (size_t)n_elem * NF);
  // ---- connectivity (sorts each element's vertices) ---------------------------
  dgc::Connectivity con;
  std::string why = dgc::build_connectivity(dim, n_vert, n_elem, m->h_elems, con);
  if (!why.empty()) {
    delete m;
    return fail(DGC_ERR_ARG, "%s", why.c_str());
  }
  m->nF = con.n_facets;
  // ---- validate geometry, shortest edge ---------------------------------------
  double hmin = INFINITY;
  for (int e = 0; e < n_elem; ++e) {
    const int* v = &m->h_elems[(size_t)e * NF];
    double Jm[9];
    for (int c = 0; c < dim; ++c)
      for (int r = 0; r < dim; ++r) Jm[r * dim + c] = verts[(size_t)v[c + 1] * dim + r] - verts[(size_t)v[0] * dim + r];
    double det = dim == 2 ? Jm[0] * Jm[3] - Jm[1] * Jm[2]
                          : Jm[0] * (Jm[4] * Jm[8] - Jm[5] * Jm[7]) - Jm[1] * (Jm[3] * Jm[8] - Jm[5] * Jm[6]) +
                                Jm[2] * (Jm[3] * Jm[7] - Jm[4] * Jm[6]);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) {
      delete m;
      return fail(DGC_ERR_ARG, "element %d is degenerate (det J = %g)", e, det);
    }
    for (int a = 0; a < NF; ++a)
      for (int b = a + 1; b < NF; ++b) {
        double l2 = 0.0;
        for (int r = 0; r < dim; ++r) {
          double d = verts[(size_t)v[a] * dim + r] - verts[(size_t)v[b] * dim + r];
          l2 += d * d;
        }
        hmin = std::min(hmin, std::sqrt(l2));
      }
  }
  m->h_min = hmin;
  // ---- device data ------------------------------------------------------------
  cudaStream_t st = as_stream(stream);
  const dgc::Tables* tp;
  try {
    tp = &dgc::tables(dim, k);
  } catch (const std::exception& ex) {
    delete m;
    return fail(DGC_ERR_ARG, "reference table build failed: %s", ex.what());
  }
  const dgc::Tables& t = *tp;
  auto up = [&](cudaError_t err) -> bool { return err == cudaSuccess; };
  bool ok = up(m->verts.upload(m->h_verts)) && up(m->elems.upload(m->h_elems)) && up(m->nbr.upload(con.nbr)) &&
            up(m->facet_id.upload(con.facet_id)) && up(m->orient.upload(con.orient)) &&
            up(m->facet_sides.upload(con.sides)) &&
            up(m->J.alloc((size_t)n_elem * dim * dim)) && up(m->detJ.alloc(n_elem)) && up(m->Bv.upload(t.Bv)) &&
            up(m->wv.upload(t.wv)) && up(m->wf.upload(t.wf)) && up(m->Bf.upload(t.Bf)) && up(m->Cb.upload(t.Cb)) &&
            up(m->Lg_int.upload(t.Lg_int)) && up(m->Lg_fac.upload(t.Lg_fac)) && up(m->Tint.upload(t.Tint)) &&
            up(m->wd.upload(t.wd)) && up(m->wfd.upload(t.wfd)) && up(m->Qfd.upload(t.Qfd)) &&
            up(m->Bd.upload(t.Bd)) && up(m->tab64.upload(stage_blob<double>(t))) &&
            up(m->tab32.upload(stage_blob<float>(t))) && up(m->status.alloc(2)) &&
            up(cudaMemset(m->status.ptr, 0, 2 * sizeof(int))) &&
            (!dgc::tc_supported(dim, k) ||
             (dim == 2 ? (up(m->tcblob.upload(dgc::tc_blob(dim, k, 0, t))) &&
                          up(m->tcblob16.upload(dgc::tc_blob(dim, k, 1, t))))
                       : (up(m->tcblob.upload(dgc::tc3_ftab(k, t))) &&
                          up(m->tc3chunks.upload(dgc::tc3_chunks(k, t))))));
  if (!ok) {
    cudaError_t err = cudaGetLastError();
    m->release_all();
    delete m;
    return fail(DGC_ERR_ALLOC, "device upload failed: %s", cudaGetErrorString(err));
  }
  cudaError_t err = dgc::launch_geometry(m->view(), st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) {
    m->release_all();
    delete m;
    return fail(DGC_ERR_CUDA, "geometry kernel failed: %s", cudaGetErrorString(err));
  }
  *out = m;
  return DGC_OK;
}

dgc_status dgc_mesh_upload_quad(int k, int n_vert, const double* verts, int n_elem, const int32_t* elems,
                                void* stream, dgc_mesh** out) {
  DGC_RANGE();
  if (!out) return fail(DGC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!dgc::quad_supported(k)) return fail(DGC_ERR_UNSUPPORTED, "order k=%d not supported for parallelograms", k);
  if (n_vert <= 0 || n_elem <= 0 || !verts || !elems)
    return fail(DGC_ERR_ARG, "empty mesh or NULL arrays (n_vert=%d, n_elem=%d)", n_vert, n_elem);
  if (n_elem >= (1 << 28)) return fail(DGC_ERR_ARG, "at most 2^28 - 1 parallelograms (got %d)", n_elem);
  dgc_mesh* m = new dgc_mesh();
  m->quad = 1;
  m->s = dgc::make_quad_sizes(k);
  m->E = n_elem;
  m->nV = n_vert;
  m->h_verts.assign(verts, verts + (size_t)n_vert * 2);
  m->h_elems.assign(elems, elems + (size_t)n_elem * 4);
  dgc::Connectivity con;
  std::vector<signed char> flip;
  std::vector<int> qnbr;
  std::string why = dgc::build_quad_connectivity(n_vert, n_elem, m->h_elems, con, flip, qnbr);
  if (!why.empty()) {
    delete m;
    return fail(DGC_ERR_ARG, "%s", why.c_str());
  }
  m->nF = con.n_facets;
  // ---- validate: parallelogram (X_0 + X_2 = X_1 + X_3), non-degenerate; shortest edge
  double hmin = INFINITY;
  for (int e = 0; e < n_elem; ++e) {
    const int* v = &m->h_elems[(size_t)e * 4];
    const double* X[4];
    for (int a = 0; a < 4; ++a) X[a] = verts + (size_t)v[a] * 2;
    double scale = 0.0, gap = 0.0;
    for (int r = 0; r < 2; ++r) {
      scale = std::max(scale, std::fabs(X[1][r] - X[0][r]) + std::fabs(X[3][r] - X[0][r]));
      const double d = X[0][r] + X[2][r] - X[1][r] - X[3][r];
      gap += d * d;
    }
    if (!(std::sqrt(gap) <= 1e-12 * scale)) {
      delete m;
      return fail(DGC_ERR_ARG, "element %d is not a parallelogram (|X0 + X2 - X1 - X3| = %g)", e, std::sqrt(gap));
    }
    const double det = (X[1][0] - X[0][0]) * (X[3][1] - X[0][1]) - (X[3][0] - X[0][0]) * (X[1][1] - X[0][1]);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) {
      delete m;
      return fail(DGC_ERR_ARG, "element %d is degenerate (det J = %g)", e, det);
    }
    for (int f = 0; f < 4; ++f) {
      const double* A = X[dgc::kQuadFacet[f][0]];
      const double* B = X[dgc::kQuadFacet[f][1]];
      hmin = std::min(hmin, std::hypot(B[0] - A[0], B[1] - A[1]));
    }
  }
  m->h_min = hmin;
  cudaStream_t st = as_stream(stream);
  const dgc::Tables* tp;
  try {
    tp = &dgc::quad_tables(k);
  } catch (const std::exception& ex) {
    delete m;
    return fail(DGC_ERR_ARG, "reference table build failed: %s", ex.what());
  }
  const dgc::Tables& t = *tp;
  auto up = [&](cudaError_t err) -> bool { return err == cudaSuccess; };
  bool ok = up(m->verts.upload(m->h_verts)) && up(m->elems.upload(m->h_elems)) && up(m->nbr.upload(con.nbr)) &&
            up(m->facet_id.upload(con.facet_id)) && up(m->orient.upload(con.orient)) &&
            up(m->facet_sides.upload(con.sides)) && up(m->flip.upload(flip)) && up(m->qnbr.upload(qnbr)) &&
            up(m->J.alloc((size_t)n_elem * 4)) && up(m->detJ.alloc(n_elem)) && up(m->Bv.upload(t.Bv)) &&
            up(m->wv.upload(t.wv)) && up(m->wf.upload(t.wf)) && up(m->Bf.upload(t.Bf)) && up(m->Cb.upload(t.Cb)) &&
            up(m->Lg_int.upload(t.Lg_int)) && up(m->Lg_fac.upload(t.Lg_fac)) && up(m->Tint.upload(t.Tint)) &&
            up(m->wd.upload(t.wd)) && up(m->wfd.upload(t.wfd)) && up(m->Qfd.upload(t.Qfd)) &&
            up(m->Bd.upload(t.Bd)) && up(m->tab64.upload(quad_stage_blob<double>(t))) &&
            up(m->tab32.upload(quad_stage_blob<float>(t))) && up(m->status.alloc(2)) &&
            up(cudaMemset(m->status.ptr, 0, 2 * sizeof(int))) &&
            up(dgc::quad_tables_to_constant(k, quad_stage_blob<double>(t)));
  if (!ok) {
    cudaError_t err = cudaGetLastError();
    m->release_all();
    delete m;
    return fail(DGC_ERR_ALLOC, "device upload failed: %s", cudaGetErrorString(err));
  }
  cudaError_t err = dgc::launch_geometry(m->view(), st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) {
    m->release_all();
    delete m;
    return fail(DGC_ERR_CUDA, "geometry kernel failed: %s", cudaGetErrorString(err));
  }
  *out = m;
  return DGC_OK;
}

dgc_status dgc_mesh_upload_hex(int k, int n_vert, const double* verts, int n_elem, const int32_t* elems,
                               void* stream, dgc_mesh** out) {
  DGC_RANGE();
  if (!out) return fail(DGC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!dgc::hex_supported(k)) return fail(DGC_ERR_UNSUPPORTED, "order k=%d not supported for parallelepipeds", k);
  if (n_vert <= 0 || n_elem <= 0 || !verts || !elems)
    return fail(DGC_ERR_ARG, "empty mesh or NULL arrays (n_vert=%d, n_elem=%d)", n_vert, n_elem);
  if (n_elem >= (1 << 28)) return fail(DGC_ERR_ARG, "at most 2^28 - 1 parallelepipeds (got %d)", n_elem);
  dgc_mesh* m = new dgc_mesh();
  m->hex = 1;
  m->s = dgc::make_hex_sizes(k);
  m->E = n_elem;
  m->nV = n_vert;
  m->h_verts.assign(verts, verts + (size_t)n_vert * 3);
  m->h_elems.assign(elems, elems + (size_t)n_elem * 8);
  dgc::Connectivity con;
  std::vector<signed char> fcode;
  std::vector<int> qnbr;
  std::string why = dgc::build_hex_connectivity(n_vert, n_elem, m->h_elems, con, fcode, qnbr);
  if (!why.empty()) {
    delete m;
    return fail(DGC_ERR_ARG, "%s", why.c_str());
  }
  m->nF = con.n_facets;
  // ---- validate: every vertex at X_0 + J c for its reference corner c; shortest edge
  const int corner[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
  double hmin = INFINITY;
  for (int e = 0; e < n_elem; ++e) {
    const int* v = &m->h_elems[(size_t)e * 8];
    const double* X0 = verts + (size_t)v[0] * 3;
    double J[3][3], scale = 0.0;
    const int cols[3] = {1, 3, 4};
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < 3; ++r) {
        J[r][c] = verts[(size_t)v[cols[c]] * 3 + r] - X0[r];
        scale += std::fabs(J[r][c]);
      }
    double gap = 0.0;
    for (int a = 0; a < 8; ++a)
      for (int r = 0; r < 3; ++r) {
        double x = X0[r];
        for (int c = 0; c < 3; ++c) x += J[r][c] * corner[a][c];
        gap = std::max(gap, std::fabs(x - verts[(size_t)v[a] * 3 + r]));
      }
    if (!(gap <= 1e-12 * scale)) {
      delete m;
      return fail(DGC_ERR_ARG, "element %d is not a parallelepiped (vertex off by %g)", e, gap);
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) {
      delete m;
      return fail(DGC_ERR_ARG, "element %d is degenerate (det J = %g)", e, det);
    }
    for (int c = 0; c < 3; ++c) hmin = std::min(hmin, std::sqrt(J[0][c] * J[0][c] + J[1][c] * J[1][c] + J[2][c] * J[2][c]));
  }
  m->h_min = hmin;
  cudaStream_t st = as_stream(stream);
  const dgc::Tables* tp;
  try {
    tp = &dgc::hex_tables(k);
  } catch (const std::exception& ex) {
    delete m;
    return fail(DGC_ERR_ARG, "reference table build failed: %s", ex.what());
  }
  const dgc::Tables& t = *tp;
  auto up = [&](cudaError_t err) -> bool { return err == cudaSuccess; };
  bool ok = up(m->verts.upload(m->h_verts)) && up(m->elems.upload(m->h_elems)) && up(m->nbr.upload(con.nbr)) &&
            up(m->facet_id.upload(con.facet_id)) && up(m->orient.upload(con.orient)) &&
            up(m->facet_sides.upload(con.sides)) && up(m->fcode.upload(fcode)) && up(m->qnbr.upload(qnbr)) &&
            up(m->J.alloc((size_t)n_elem * 9)) && up(m->detJ.alloc(n_elem)) && up(m->Bv.upload(t.Bv)) &&
            up(m->wv.upload(t.wv)) && up(m->wf.upload(t.wf)) && up(m->Bf.upload(t.Bf)) && up(m->Cb.upload(t.Cb)) &&
            up(m->Lg_int.upload(t.Lg_int)) && up(m->Lg_fac.upload(t.Lg_fac)) && up(m->Tint.upload(t.Tint)) &&
            up(m->wd.upload(t.wd)) && up(m->wfd.upload(t.wfd)) && up(m->Qfd.upload(t.Qfd)) &&
            up(m->Bd.upload(t.Bd)) && up(m->tab64.upload(quad_stage_blob<double>(t))) &&
            up(m->tab32.upload(quad_stage_blob<float>(t))) && up(m->status.alloc(2)) &&
            up(cudaMemset(m->status.ptr, 0, 2 * sizeof(int)));
  if (!ok) {
    cudaError_t err = cudaGetLastError();
    m->release_all();
    delete m;
    return fail(DGC_ERR_ALLOC, "device upload failed: %s", cudaGetErrorString(err));
  }
  cudaError_t err = dgc::launch_geometry(m->view(), st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) {
    m->release_all();
    delete m;
    return fail(DGC_ERR_CUDA, "geometry kernel failed: %s", cudaGetErrorString(err));
  }
  *out = m;
  return DGC_OK;
}

dgc_status dgc_mesh_upload_curved(int k, int n_vert, const double* verts, int n_elem, const int32_t* elems,
                                  const double* edge_nodes, void* stream, dgc_mesh** out) {
  DGC_RANGE();
  if (!out) return fail(DGC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!edge_nodes) return fail(DGC_ERR_ARG, "edge_nodes is NULL");
  dgc_mesh* m = nullptr;
  if (dgc_status rc = dgc_mesh_upload(2, k, n_vert, verts, n_elem, elems, stream, &m)) return rc;
  // facet ids of the sorted elements (the same connectivity the upload built)
  std::vector<int> el = m->h_elems;
  dgc::Connectivity con;
  dgc::build_connectivity(2, n_vert, n_elem, el, con);
  const dgc::Tables& t = dgc::tables(2, k);
  // six nodes per element: sorted vertices, then the edge nodes m_01, m_02, m_12
  // (facets 2, 1, 0: local facet f is opposite local vertex f)
  const int node_of_facet[3] = {5, 4, 3};
  const int ends[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  std::vector<double> nodes((size_t)n_elem * 12);
  m->h_cid.assign(n_elem, -1);
  std::vector<int> celem;
  for (int e = 0; e < n_elem; ++e) {
    double* X = &nodes[(size_t)e * 12];
    const int* v = &m->h_elems[(size_t)e * 3];
    for (int a = 0; a < 3; ++a)
      for (int r = 0; r < 2; ++r) X[a * 2 + r] = verts[(size_t)v[a] * 2 + r];
    for (int f = 0; f < 3; ++f) {
      const int g = con.facet_id[(size_t)e * 3 + f];
      for (int r = 0; r < 2; ++r) X[node_of_facet[f] * 2 + r] = edge_nodes[(size_t)g * 2 + r];
    }
    double dev = 0.0, hmin = INFINITY;
    for (int j = 3; j < 6; ++j) {
      const double* A = X + ends[j][0] * 2;
      const double* B = X + ends[j][1] * 2;
      hmin = std::min(hmin, std::hypot(B[0] - A[0], B[1] - A[1]));
      for (int r = 0; r < 2; ++r) dev = std::max(dev, std::fabs(X[j * 2 + r] - 0.5 * (A[r] + B[r])));
    }
    if (dev > 1e-14 * hmin) {
      m->h_cid[e] = (int)celem.size();
      celem.push_back(e);
    }
  }
  // P2 reference gradients at a point
  auto p2grad = [](double x1, double x2, double* g) {
    const double x0 = 1.0 - x1 - x2;
    const double gg[12] = {-(4 * x0 - 1), -(4 * x0 - 1), 4 * x1 - 1, 0.0, 0.0, 4 * x2 - 1,
                           4 * (x0 - x1), -4 * x1, -4 * x2, 4 * (x0 - x2), 4 * x2, 4 * x1};
    for (int j = 0; j < 12; ++j) g[j] = gg[j];
  };
  auto table_at = [&](const std::vector<double>& pts) {
    std::vector<double> out(pts.size() / 2 * 12);
    for (size_t q = 0; q < pts.size() / 2; ++q) p2grad(pts[2 * q], pts[2 * q + 1], &out[q * 12]);
    return out;
  };
  const std::vector<double> p2d = table_at(t.xd), p2v = table_at(t.xv);
  // the map must not fold: det J keeps the sign of the vertices' affine map at the
  // nodes and at both rules
  std::vector<double> checkpts = t.xd;
  checkpts.insert(checkpts.end(), t.xv.begin(), t.xv.end());
  const double refnodes[12] = {0, 0, 1, 0, 0, 1, 0.5, 0, 0, 0.5, 0.5, 0.5};
  checkpts.insert(checkpts.end(), refnodes, refnodes + 12);
  const std::vector<double> p2c = table_at(checkpts);
  m->h_cnodes.clear();
  for (int c = 0; c < (int)celem.size(); ++c) {
    const int e = celem[c];
    const double* X = &nodes[(size_t)e * 12];
    const double* v0 = X;
    const double sa = (X[2] - v0[0]) * (X[5] - v0[1]) - (X[4] - v0[0]) * (X[3] - v0[1]);
    for (size_t q = 0; q < checkpts.size() / 2; ++q) {
      double J[4] = {0, 0, 0, 0};
      for (int j = 0; j < 6; ++j)
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) J[a * 2 + b] += X[j * 2 + a] * p2c[q * 12 + j * 2 + b];
      const double det = J[0] * J[3] - J[1] * J[2];
      if (!(det * sa > 0.0)) {
        dgc_mesh_free(m);
        return fail(DGC_ERR_ARG, "curved element %d folds over (det J changes sign)", e);
      }
    }
    m->h_cnodes.insert(m->h_cnodes.end(), X, X + 12);
  }
  m->Ec = (int)celem.size();
  if (m->Ec > 0) {
    const size_t nn = (size_t)m->s.N * m->s.N * m->Ec;
    cudaError_t err = cudaSuccess;
    for (cudaError_t e2 : {m->celem.upload(celem), m->cid.upload(m->h_cid), m->cnodes.upload(m->h_cnodes),
                           m->p2d.upload(p2d), m->p2v.upload(p2v), m->Minv64.alloc(nn), m->Minv32.alloc(nn)})
      if (e2 != cudaSuccess) err = e2;
    if (err == cudaSuccess) err = dgc::launch_geometry(m->view(), as_stream(stream));
    if (err == cudaSuccess) err = cudaStreamSynchronize(as_stream(stream));
    if (err != cudaSuccess) {
      dgc_mesh_free(m);
      return fail(DGC_ERR_CUDA, "curved geometry failed: %s", cudaGetErrorString(err));
    }
  }
  *out = m;
  return DGC_OK;
}

dgc_status dgc_mesh_free(dgc_mesh* mesh) {
  if (!mesh) return DGC_OK;
  drop_batch_graphs(mesh);
  mesh->release_all();
  delete mesh;
  return DGC_OK;
}

dgc_status dgc_sizes(const dgc_mesh* mesh, int64_t* n_dg, int64_t* n_hdiv) {
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (n_dg) *n_dg = (int64_t)mesh->E * mesh->s.D * mesh->s.N;
  if (n_hdiv) *n_hdiv = (int64_t)mesh->nF * mesh->s.NFM + (int64_t)mesh->E * mesh->s.NINT;
  return DGC_OK;
}

dgc_status dgc_mesh_info(const dgc_mesh* mesh, int64_t* info) {
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (!info) return fail(DGC_ERR_ARG, "info is NULL");
  const Sizes& s = mesh->s;
  const int64_t shape = mesh->quad ? 1 : mesh->hex ? 3 : (mesh->h_cid.empty() ? 0 : 2);
  int64_t v[13] = {s.D, s.K, mesh->E, mesh->nF, s.N, s.NW, s.NFM, s.NINT, s.NLAG, s.QD, s.NF * s.QFD + s.QD,
                   shape, mesh->Ec};
  std::memcpy(info, v, sizeof(v));
  return DGC_OK;
}

dgc_status dgc_geometry(dgc_mesh* mesh, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  DGC_CUDA(dgc::launch_geometry(mesh->view(), as_stream(stream)));
  return DGC_OK;
}

dgc_status dgc_transfer(dgc_mesh* mesh, const double* u_hdiv, double* w_dg, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (!u_hdiv || !w_dg) return fail(DGC_ERR_ARG, "NULL vector");
  DGC_CUDA(dgc::launch_transfer(mesh->view(), u_hdiv, w_dg, as_stream(stream)));
  return DGC_OK;
}

dgc_status dgc_transfer_T(dgc_mesh* mesh, const double* f_dg, double* g_hdiv, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (!f_dg || !g_hdiv) return fail(DGC_ERR_ARG, "NULL vector");
  DGC_CUDA(mesh->zbuf.alloc((size_t)mesh->E * mesh->s.NF * mesh->s.NFM));
  DGC_CUDA(dgc::launch_transfer_T(mesh->view(), f_dg, g_hdiv, mesh->zbuf.ptr, as_stream(stream)));
  return DGC_OK;
}

dgc_status dgc_mass_apply(dgc_mesh* mesh, const double* v_dg, double* out_dg, int inverse, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (!v_dg || !out_dg) return fail(DGC_ERR_ARG, "NULL vector");
  DGC_CUDA(dgc::launch_mass(mesh->view(), v_dg, out_dg, inverse != 0, as_stream(stream)));
  return DGC_OK;
}

dgc_status dgc_diagnostics(dgc_mesh* mesh, const double* v_dg, double* out, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (!v_dg || !out) return fail(DGC_ERR_ARG, "NULL vector");
  DGC_CUDA(mesh->diag_mv.alloc((size_t)mesh->E * mesh->s.D * mesh->s.N));
  DGC_CUDA(mesh->diag_part.alloc((size_t)std::max(dgc::diag_blocks(mesh->E), 1) * (mesh->s.D + 2)));
  DGC_CUDA(dgc::launch_diagnostics(mesh->view(), v_dg, mesh->diag_mv.ptr, mesh->diag_part.ptr, out,
                                   mesh->status.ptr, as_stream(stream)));
  return DGC_OK;
}

dgc_status dgc_conv_apply(dgc_mesh* mesh, const double* wind_hdiv, const double* w_dg, double* out_dg,
                          dgc_prec prec, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (dgc_status rc = check_prec(mesh, prec)) return rc;
  if (!wind_hdiv || !w_dg || !out_dg) return fail(DGC_ERR_ARG, "NULL vector");
  const size_t n = (size_t)mesh->E * mesh->s.D * mesh->s.N;
  if (out_dg < w_dg + n && w_dg < out_dg + n) return fail(DGC_ERR_ARG, "out_dg overlaps w_dg");
  if (dgc_status rc = ensure_prec_scratch(mesh, prec)) return rc;
  cudaStream_t st = as_stream(stream);
  if (dgc_status rc = prepare_wind(mesh, prec, wind_hdiv, st)) return rc;
  return apply_operator(mesh, prec, w_dg, out_dg, st);
}

dgc_status dgc_rk_substeps(dgc_mesh* mesh, const double* wind_hdiv, double* v_dg, double ds, int nsteps,
                           dgc_scheme scheme, dgc_prec prec, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (dgc_status rc = check_prec(mesh, prec)) return rc;
  if (!wind_hdiv || !v_dg) return fail(DGC_ERR_ARG, "NULL vector");
  if (scheme != DGC_SSPRK2 && scheme != DGC_SSPRK3) return fail(DGC_ERR_ARG, "unknown scheme %d", (int)scheme);
  if (nsteps < 0) return fail(DGC_ERR_ARG, "nsteps must be >= 0 (got %d)", nsteps);
  if (!(ds > 0.0) || !std::isfinite(ds)) return fail(DGC_ERR_ARG, "ds must be positive and finite (got %g)", ds);
  if (nsteps == 0) return DGC_OK;
  const size_t n = (size_t)mesh->E * mesh->s.D * mesh->s.N;
  if (dgc_status rc = ensure_prec_scratch(mesh, prec)) return rc;
  DGC_CUDA(mesh->stage1.alloc(n));
  DGC_CUDA(mesh->stage2.alloc(n));
  cudaStream_t st = as_stream(stream);
  GraphKey key{wind_hdiv, v_dg, ds, nsteps, (int)scheme, (int)prec, injected("stall")};
  if (!(mesh->graph && mesh->graph_key == key)) {
    if (mesh->graph) cudaGraphExecDestroy(mesh->graph);
    mesh->graph = nullptr;
    if (!mesh->capture_stream) DGC_CUDA(cudaStreamCreateWithFlags(&mesh->capture_stream, cudaStreamNonBlocking));
    DGC_CUDA(begin_capture(mesh->capture_stream));
    dgc_status rc = rk_sequence(mesh, wind_hdiv, v_dg, ds, nsteps, (int)scheme, prec, mesh->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t err = cudaStreamEndCapture(mesh->capture_stream, &g);
    if (rc != DGC_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (err != cudaSuccess) return fail(DGC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(err));
    err = cudaGraphInstantiate(&mesh->graph, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) {
      mesh->graph = nullptr;
      return fail(DGC_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(err));
    }
    mesh->graph_key = key;
  }
  DGC_CUDA(cudaGraphLaunch(mesh->graph, st));
  return DGC_OK;
}

dgc_status dgc_richardson(dgc_mesh* mesh, const double* wind_hdiv, const double* g_dg, double* v_dg, double tau,
                          double ds, double reduction, int max_iter, dgc_prec prec, int32_t* iters_dev,
                          double* res_dev, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (mesh->Ec) return fail(DGC_ERR_UNSUPPORTED, "the pseudo-time solve takes affine meshes (its norm uses |det J|)");
  if (dgc_status rc = check_prec(mesh, prec)) return rc;
  if (!wind_hdiv || !g_dg || !v_dg || !iters_dev) return fail(DGC_ERR_ARG, "NULL argument");
  if (!(tau > 0.0) || !std::isfinite(tau)) return fail(DGC_ERR_ARG, "tau must be positive and finite (got %g)", tau);
  if (!(ds > 0.0 && ds < 2.0)) return fail(DGC_ERR_ARG, "ds must lie in (0, 2) (got %g)", ds);
  if (!(reduction >= 0.0) || !std::isfinite(reduction))
    return fail(DGC_ERR_ARG, "reduction must be finite and >= 0 (got %g)", reduction);
  if (max_iter < 0) return fail(DGC_ERR_ARG, "max_iter must be >= 0 (got %d)", max_iter);
  const size_t n = (size_t)mesh->E * mesh->s.D * mesh->s.N;
  if (g_dg < v_dg + n && v_dg < g_dg + n) return fail(DGC_ERR_ARG, "v_dg overlaps g_dg");
  if (dgc_status rc = ensure_prec_scratch(mesh, prec)) return rc;
  DGC_CUDA(mesh->rho.alloc(n));
  DGC_CUDA(mesh->rop.alloc(n));
  DGC_CUDA(mesh->partials.alloc(std::max<size_t>((size_t)dgc::rich_blocks((long)n), ((size_t)mesh->E + 127) / 128)));
  DGC_CUDA(mesh->rstate.alloc(2));
  if (is_tc(prec) && mesh->s.D == 2) {
    const size_t nt = dgc::tc_tsoa_len(mesh->s.D, mesh->s.K, mesh->E);
    DGC_CUDA(mesh->ts1.alloc(nt));
    DGC_CUDA(mesh->tsg.alloc(nt));
    DGC_CUDA(mesh->tsf1.alloc(nt));
  }
  std::vector<uint64_t> key = {(uint64_t)(uintptr_t)wind_hdiv, (uint64_t)(uintptr_t)g_dg, (uint64_t)(uintptr_t)v_dg,
                               (uint64_t)(uintptr_t)iters_dev, (uint64_t)(uintptr_t)res_dev, (uint64_t)max_iter,
                               (uint64_t)prec};
  for (double x : {tau, ds, reduction}) {
    uint64_t b;
    std::memcpy(&b, &x, 8);
    key.push_back(b);
  }
  if (!(mesh->rich_graph && mesh->rich_key == key)) {
    if (mesh->rich_graph) cudaGraphExecDestroy(mesh->rich_graph);
    mesh->rich_graph = nullptr;
    if (dgc_status rc = rich_build(mesh, wind_hdiv, g_dg, v_dg, tau, ds, reduction, max_iter, prec, iters_dev,
                                   res_dev, &mesh->rich_graph))
      return rc;
    mesh->rich_key = key;
  }
  DGC_CUDA(cudaGraphLaunch(mesh->rich_graph, as_stream(stream)));
  return DGC_OK;
}

dgc_status dgc_autotune(dgc_mesh* mesh, const double* wind_hdiv, dgc_prec prec, int reps, int* block_out,
                        void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (dgc_status rc = check_prec(mesh, prec)) return rc;
  if (!wind_hdiv) return fail(DGC_ERR_ARG, "wind_hdiv is NULL");
  if (reps < 1 || reps > 1000) return fail(DGC_ERR_ARG, "reps must lie in 1..1000 (got %d)", reps);
  if (block_out) *block_out = 0;
  if (is_tc(prec)) return DGC_OK;   // the tensor-core kernels have one tile shape each
  if (mesh->quad || mesh->hex) return DGC_OK;   // the tensor-product kernels have one block shape (128)
  const bool fp32 = prec == DGC_FP32;
  const size_t n = (size_t)mesh->E * mesh->s.D * mesh->s.N;
  if (dgc_status rc = ensure_prec_scratch(mesh, prec)) return rc;
  DGC_CUDA(mesh->stage1.alloc(n));
  DGC_CUDA(mesh->stage2.alloc(n));
  cudaStream_t st = as_stream(stream);
  DGC_CUDA(cudaMemsetAsync(mesh->stage1.ptr, 0, n * sizeof(double), st));
  if (dgc_status rc = prepare_wind(mesh, prec, wind_hdiv, st)) return rc;
  cudaEvent_t e0, e1;
  DGC_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(DGC_ERR_CUDA, "event creation failed");
  }
  std::atomic<int>& slot = dgc::g_stage_block[mesh->s.D - 2][mesh->s.K][fp32 ? 1 : 0];
  const int before = slot.load();
  int best = 0;
  float best_ms = 0.f;
  dgc_status rc = DGC_OK;
  for (int b : dgc::kStageBlocks) {
    slot.store(b);
    // one untimed launch, then reps timed launches of one stage (stage1 -> stage2)
    for (int r = 0; r <= reps && rc == DGC_OK; ++r) {
      if (r == 1 && cudaEventRecord(e0, st) != cudaSuccess) rc = fail(DGC_ERR_CUDA, "event record failed");
      if (rc == DGC_OK) rc = stage(mesh, prec, mesh->stage1.ptr, nullptr, mesh->stage2.ptr, 0.0, 1.0, 1e-3, st);
    }
    float ms = 0.f;
    if (rc == DGC_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = fail(DGC_ERR_CUDA, "timing the stage kernel failed");
    if (rc != DGC_OK) break;
    if (best == 0 || ms < best_ms) {
      best = b;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != DGC_OK) {
    slot.store(before);
    return rc;
  }
  slot.store(best);
  // graphs captured before the choice keep their old launch shape: drop them
  if (mesh->graph) cudaGraphExecDestroy(mesh->graph);
  mesh->graph = nullptr;
  if (mesh->rich_graph) cudaGraphExecDestroy(mesh->rich_graph);
  mesh->rich_graph = nullptr;
  if (mesh->oifs_graph) cudaGraphExecDestroy(mesh->oifs_graph);
  mesh->oifs_graph = nullptr;
  drop_batch_graphs(mesh);
  if (block_out) *block_out = best;
  return DGC_OK;
}

dgc_status dgc_wind_extrapolate(dgc_mesh* mesh, int n_terms, const double* const* fields, const double* coefs,
                                double* out_hdiv, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (n_terms < 1 || n_terms > dgc::kMaxTerms)
    return fail(DGC_ERR_ARG, "n_terms must lie in 1..%d (got %d)", dgc::kMaxTerms, n_terms);
  if (!fields || !coefs || !out_hdiv) return fail(DGC_ERR_ARG, "NULL argument");
  dgc::CombineArgs a{};
  for (int t = 0; t < n_terms; ++t) {
    if (!fields[t]) return fail(DGC_ERR_ARG, "fields[%d] is NULL", t);
    if (!std::isfinite(coefs[t])) return fail(DGC_ERR_ARG, "coefs[%d] is not finite", t);
    a.x[t] = fields[t];
    a.c[t] = coefs[t];
  }
  a.nterms = n_terms;
  const long n = (long)mesh->nF * mesh->s.NFM + (long)mesh->E * mesh->s.NINT;
  DGC_CUDA(dgc::launch_combine(out_hdiv, a, n, as_stream(stream)));
  return DGC_OK;
}

dgc_status dgc_conv_apply_hdiv(dgc_mesh* mesh, const double* wind_hdiv, const double* u_hdiv, double* out_hdiv,
                               dgc_prec prec, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (dgc_status rc = check_prec(mesh, prec)) return rc;
  if (!wind_hdiv || !u_hdiv || !out_hdiv) return fail(DGC_ERR_ARG, "NULL vector");
  const size_t n = (size_t)mesh->E * mesh->s.D * mesh->s.N;
  const size_t nh = (size_t)mesh->nF * mesh->s.NFM + (size_t)mesh->E * mesh->s.NINT;
  if (out_hdiv < u_hdiv + nh && u_hdiv < out_hdiv + nh) return fail(DGC_ERR_ARG, "out_hdiv overlaps u_hdiv");
  if (dgc_status rc = ensure_prec_scratch(mesh, prec)) return rc;
  DGC_CUDA(mesh->ov.alloc(n));
  DGC_CUDA(mesh->omv.alloc(n));
  DGC_CUDA(mesh->rop.alloc(n));
  DGC_CUDA(mesh->zbuf.alloc((size_t)mesh->E * mesh->s.NF * mesh->s.NFM));
  cudaStream_t st = as_stream(stream);
  // out = I^T M^V ((M^V)^-1 C^V) I u
  DGC_CUDA(dgc::launch_transfer(mesh->view(), u_hdiv, mesh->ov.ptr, st));
  if (dgc_status rc = prepare_wind(mesh, prec, wind_hdiv, st)) return rc;
  if (dgc_status rc = apply_operator(mesh, prec, mesh->ov.ptr, mesh->rop.ptr, st)) return rc;
  DGC_CUDA(dgc::launch_mass(mesh->view(), mesh->rop.ptr, mesh->omv.ptr, false, st));
  DGC_CUDA(dgc::launch_transfer_T(mesh->view(), mesh->omv.ptr, out_hdiv, mesh->zbuf.ptr, st));
  return DGC_OK;
}

dgc_status dgc_oifs_rhs(dgc_mesh* mesh, const double* u_hdiv, const double* wind_hdiv, const double* wind_prev_hdiv,
                        double dt_prev, double* out_hdiv, double ds, int nsteps, dgc_scheme scheme, dgc_prec prec,
                        void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (dgc_status rc = check_prec(mesh, prec)) return rc;
  if (!u_hdiv || !wind_hdiv || !out_hdiv) return fail(DGC_ERR_ARG, "NULL vector");
  if (scheme != DGC_SSPRK2 && scheme != DGC_SSPRK3) return fail(DGC_ERR_ARG, "unknown scheme %d", (int)scheme);
  if (nsteps < 0) return fail(DGC_ERR_ARG, "nsteps must be >= 0 (got %d)", nsteps);
  if (!(ds > 0.0) || !std::isfinite(ds)) return fail(DGC_ERR_ARG, "ds must be positive and finite (got %g)", ds);
  if (wind_prev_hdiv && (!(dt_prev > 0.0) || !std::isfinite(dt_prev)))
    return fail(DGC_ERR_ARG, "dt_prev must be positive and finite with wind_prev (got %g)", dt_prev);
  const size_t n = (size_t)mesh->E * mesh->s.D * mesh->s.N;
  const size_t nh = (size_t)mesh->nF * mesh->s.NFM + (size_t)mesh->E * mesh->s.NINT;
  if (out_hdiv < u_hdiv + nh && u_hdiv < out_hdiv + nh) return fail(DGC_ERR_ARG, "out_hdiv overlaps u_hdiv");
  if (dgc_status rc = ensure_prec_scratch(mesh, prec)) return rc;
  DGC_CUDA(mesh->stage1.alloc(n));
  DGC_CUDA(mesh->stage2.alloc(n));
  DGC_CUDA(mesh->ov.alloc(n));
  DGC_CUDA(mesh->omv.alloc(n));
  DGC_CUDA(mesh->wmix.alloc(nh));
  DGC_CUDA(mesh->zbuf.alloc((size_t)mesh->E * mesh->s.NF * mesh->s.NFM));
  uint64_t b_ds, b_dt;
  std::memcpy(&b_ds, &ds, 8);
  std::memcpy(&b_dt, &dt_prev, 8);
  std::vector<uint64_t> key = {(uint64_t)(uintptr_t)u_hdiv, (uint64_t)(uintptr_t)wind_hdiv,
                               (uint64_t)(uintptr_t)wind_prev_hdiv, (uint64_t)(uintptr_t)out_hdiv, b_ds,
                               wind_prev_hdiv ? b_dt : 0u, (uint64_t)nsteps, (uint64_t)scheme, (uint64_t)prec,
                               (uint64_t)injected("stall")};
  if (!(mesh->oifs_graph && mesh->oifs_key == key)) {
    if (mesh->oifs_graph) cudaGraphExecDestroy(mesh->oifs_graph);
    mesh->oifs_graph = nullptr;
    if (!mesh->capture_stream) DGC_CUDA(cudaStreamCreateWithFlags(&mesh->capture_stream, cudaStreamNonBlocking));
    cudaStream_t cs = mesh->capture_stream;
    DGC_CUDA(begin_capture(cs));
    // a2: v = I u;  Q: nsteps substeps;  out = I^T M^V v
    dgc_status rc = DGC_OK;
    cudaError_t err = dgc::launch_transfer(mesh->view(), u_hdiv, mesh->ov.ptr, cs);
    if (err == cudaSuccess && nsteps > 0)
      rc = rk_sequence(mesh, wind_hdiv, mesh->ov.ptr, ds, nsteps, (int)scheme, prec, cs, wind_prev_hdiv, dt_prev);
    if (err == cudaSuccess && rc == DGC_OK) err = dgc::launch_mass(mesh->view(), mesh->ov.ptr, mesh->omv.ptr, false, cs);
    if (err == cudaSuccess && rc == DGC_OK)
      err = dgc::launch_transfer_T(mesh->view(), mesh->omv.ptr, out_hdiv, mesh->zbuf.ptr, cs);
    cudaGraph_t g = nullptr;
    cudaError_t err2 = cudaStreamEndCapture(cs, &g);
    if (rc != DGC_OK || err != cudaSuccess || err2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (rc != DGC_OK) return rc;
      return fail(DGC_ERR_CUDA, "OIFS graph capture failed: %s", cudaGetErrorString(err != cudaSuccess ? err : err2));
    }
    err = cudaGraphInstantiate(&mesh->oifs_graph, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) {
      mesh->oifs_graph = nullptr;
      return fail(DGC_ERR_CUDA, "OIFS graph instantiation failed: %s", cudaGetErrorString(err));
    }
    mesh->oifs_key = key;
  }
  DGC_CUDA(cudaGraphLaunch(mesh->oifs_graph, as_stream(stream)));
  return DGC_OK;
}

namespace {
// The triangle instances of one order on the tensor-core path advance together: each
// stage is one launch of the persistent kernel over the tiles of all of them
// (dgc::StageTcArgs::list), so small meshes share the SMs instead of each leaving most
// of them idle, and a substep takes one launch per stage instead of one per instance.
struct MergedGroup {
  int K = 0;
  std::vector<int> inst;                  // instance numbers, nsteps descending
  std::vector<dgc::StageTcArgs> lists;    // [parity][stage][instance], host copy
  std::vector<int> off;                   // first tile of each instance, then the total
  dgc::StageTcArgs* dlists = nullptr;     // device copies
  int* doff = nullptr;
};

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// the stage argument lists and tile offsets of a group (host side)
void merged_plan(MergedGroup& g, dgc_mesh* const* meshes, const double* ds, int scheme, dgc_prec prec) {
  const int n = (int)g.inst.size();
  const int stages = scheme == DGC_SSPRK2 ? 2 : 3, parities = scheme == DGC_SSPRK2 ? 1 : 2;
  g.lists.assign((size_t)parities * stages * n, dgc::StageTcArgs{});
  g.off.assign(n + 1, 0);
  for (int u = 0; u < n; ++u) {
    dgc_mesh* m = meshes[g.inst[u]];
    g.off[u + 1] = g.off[u] + (m->E + 127) / 128;
    for (int par = 0; par < parities; ++par)
      for (int j = 0; j < stages; ++j)
        g.lists[((size_t)par * stages + j) * n + u] = tc_rk_stage(m, prec, scheme, par, j, ds[g.inst[u]]);
  }
}

size_t merged_bytes(const MergedGroup& g) {
  return round256(g.lists.size() * sizeof(dgc::StageTcArgs)) + round256(g.off.size() * sizeof(int));
}

// the launches of a group on one stream (captured): per instance the wind data and the
// layout transpose in, the substeps, the transpose out
dgc_status rk_sequence_merged(const MergedGroup& g, dgc_mesh* const* meshes, const double* const* winds,
                              double* const* states, const int* nsteps, int scheme, dgc_prec prec, cudaStream_t st) {
  const int n = (int)g.inst.size();
  const int stages = scheme == DGC_SSPRK2 ? 2 : 3;
  for (int i : g.inst) {
    if (dgc_status rc = prepare_wind(meshes[i], prec, winds[i], st)) return rc;
    if (dgc_status rc = tc_transpose_in(meshes[i], states[i], meshes[i]->trA.ptr, st)) return rc;
  }
  int active = n;
  for (int step = 0; step < nsteps[g.inst[0]]; ++step) {
    while (active > 0 && nsteps[g.inst[active - 1]] <= step) --active;   // the instances still stepping
    const int parity = scheme == DGC_SSPRK2 ? 0 : (step & 1);
    for (int j = 0; j < stages; ++j) {
      const size_t l = ((size_t)parity * stages + j) * n;
      dgc::StageTcArgs a = g.lists[l];   // mode, stage kind, tables and wait budget of every instance
      a.list = g.dlists + l;
      a.tile_off = g.doff;
      a.n_list = active;
      a.batch_tiles = g.off[active];
      if (dgc_status rc = launch_tc(2, g.K, prec, a, st)) return rc;
    }
  }
  for (int i : g.inst)
    if (dgc_status rc = tc_transpose_out(meshes[i], meshes[i]->ts0.ptr, states[i], st)) return rc;
  return DGC_OK;
}
}  // namespace

dgc_status dgc_batch_rk_substeps(int n_inst, dgc_mesh* const* meshes, const double* const* winds,
                                 double* const* states, const double* ds, const int* nsteps, dgc_scheme scheme,
                                 dgc_prec prec, void* stream) {
  DGC_RANGE();
  if (n_inst < 0) return fail(DGC_ERR_ARG, "n_inst must be >= 0");
  if (n_inst == 0) return DGC_OK;
  if (!meshes || !winds || !states || !ds || !nsteps) return fail(DGC_ERR_ARG, "NULL argument array");
  if (scheme != DGC_SSPRK2 && scheme != DGC_SSPRK3) return fail(DGC_ERR_ARG, "unknown scheme %d", (int)scheme);
  if (prec != DGC_FP64 && prec != DGC_FP32 && !is_tc(prec))
    return fail(DGC_ERR_ARG, "precision %d not available", (int)prec);
  std::vector<dgc_prec> pr(n_inst);
  std::vector<uint64_t> key = {(uint64_t)n_inst, (uint64_t)scheme, (uint64_t)prec};
  for (int i = 0; i < n_inst; ++i) {
    dgc_mesh* m = meshes[i];
    if (!m || !winds[i] || !states[i]) return fail(DGC_ERR_ARG, "instance %d: NULL mesh or vector", i);
    if (!(ds[i] > 0.0) || !std::isfinite(ds[i])) return fail(DGC_ERR_ARG, "instance %d: ds must be positive", i);
    if (nsteps[i] < 0) return fail(DGC_ERR_ARG, "instance %d: nsteps must be >= 0", i);
    for (int j = 0; j < i; ++j)
      if (meshes[j] == m) return fail(DGC_ERR_ARG, "instances %d and %d share a mesh handle (scratch)", j, i);
    // the tensor-core path covers affine triangles k <= 6 and tetrahedra k <= 4 (BF16x3 only);
    // other instances run their stages in FP32
    pr[i] = (is_tc(prec) && (!mesh_tc(m) || (m->s.D == 3 && prec == DGC_TF32X3))) ? DGC_FP32 : prec;
    if (dgc_status rc = ensure_prec_scratch(m, pr[i])) return rc;
    const size_t n = (size_t)m->E * m->s.D * m->s.N;
    DGC_CUDA(m->stage1.alloc(n));
    DGC_CUDA(m->stage2.alloc(n));
    uint64_t dsbits;
    std::memcpy(&dsbits, &ds[i], 8);
    key.insert(key.end(), {(uint64_t)(uintptr_t)m, (uint64_t)(uintptr_t)winds[i], (uint64_t)(uintptr_t)states[i],
                           dsbits, (uint64_t)nsteps[i]});
  }
  key.push_back((uint64_t)injected("stall"));
  std::lock_guard<std::mutex> lock(g_batch_mu);
  BatchGraph* hit = nullptr;
  for (BatchGraph& b : g_batch_cache)
    if (b.key == key) hit = &b;
  if (!hit) {
    for (auto& st : g_batch_streams)
      if (!st) DGC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaStream_t main_st = g_batch_streams[0];
    // triangle instances on the tensor-core path: one merged group per order
    std::vector<MergedGroup> groups;
    std::vector<char> merged(n_inst, 0);
    for (int i = 0; i < n_inst; ++i) {
      dgc_mesh* m = meshes[i];
      if (!is_tc(pr[i]) || m->s.D != 2 || nsteps[i] == 0 || m->E == 0) continue;
      MergedGroup* g = nullptr;
      for (MergedGroup& h : groups)
        if (h.K == m->s.K) g = &h;
      if (!g) {
        groups.emplace_back();
        g = &groups.back();
        g->K = m->s.K;
      }
      g->inst.push_back(i);
      merged[i] = 1;
    }
    size_t lbytes = 0;
    for (MergedGroup& g : groups) {
      std::stable_sort(g.inst.begin(), g.inst.end(), [&](int x, int y) { return nsteps[x] > nsteps[y]; });
      merged_plan(g, meshes, ds, (int)scheme, prec);
      lbytes += merged_bytes(g);
    }
    void* lists = nullptr;
    if (lbytes) {
      DGC_CUDA(cudaMalloc(&lists, lbytes));
      char* p = static_cast<char*>(lists);
      cudaError_t cerr = cudaSuccess;
      for (MergedGroup& g : groups) {
        g.dlists = reinterpret_cast<dgc::StageTcArgs*>(p);
        g.doff = reinterpret_cast<int*>(p + round256(g.lists.size() * sizeof(dgc::StageTcArgs)));
        if (cerr == cudaSuccess)
          cerr = cudaMemcpy(g.dlists, g.lists.data(), g.lists.size() * sizeof(dgc::StageTcArgs), cudaMemcpyHostToDevice);
        if (cerr == cudaSuccess)
          cerr = cudaMemcpy(g.doff, g.off.data(), g.off.size() * sizeof(int), cudaMemcpyHostToDevice);
        p += merged_bytes(g);
      }
      if (cerr != cudaSuccess) {
        cudaFree(lists);
        return fail(DGC_ERR_CUDA, "batch argument upload failed: %s", cudaGetErrorString(cerr));
      }
    }
    std::vector<cudaEvent_t> evs;
    auto new_event = [&](cudaEvent_t* e) {
      cudaError_t err = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
      if (err == cudaSuccess) evs.push_back(*e);
      return err;
    };
    auto cleanup = [&]() {
      for (cudaEvent_t e : evs) cudaEventDestroy(e);
    };
    // Two phases: first the work whose CTAs leave room for a second one on an SM (the
    // triangle kernel for k <= 4, the CUDA-core kernels), then the work whose CTAs take a
    // whole SM (triangles k = 5, 6, the tetrahedral kernel).  Within a phase the merged
    // groups and the other instances run round robin on the branches (independent graph
    // paths).  Mixed in one phase, the two kinds of CTA leave SMs half used: a CTA that
    // needs a whole SM waits for an SM that a smaller one still half occupies.
    auto whole_sm = [&](int i) { return is_tc(pr[i]) && (meshes[i]->s.D == 3 || meshes[i]->s.K >= 5); };
    std::vector<std::vector<int>> phase(2);   // items: group g as g, instance i as -(i + 1)
    for (size_t g = 0; g < groups.size(); ++g) phase[groups[g].K >= 5].push_back((int)g);
    for (int i = 0; i < n_inst; ++i)
      if (nsteps[i] > 0 && !merged[i]) phase[whole_sm(i)].push_back(-(i + 1));
    if (phase[0].empty() && phase[1].empty()) return DGC_OK;   // no instance takes a substep
    DGC_CUDA(begin_capture(main_st));
    cudaError_t err = cudaSuccess;
    dgc_status rc = DGC_OK;
    for (const std::vector<int>& items : phase) {
      if (items.empty() || err != cudaSuccess || rc != DGC_OK) continue;
      const int branches = std::min((int)items.size(), kBatchBranches);
      cudaEvent_t fork;
      err = new_event(&fork);
      if (err == cudaSuccess) err = cudaEventRecord(fork, main_st);
      for (int b = 0; b < branches && err == cudaSuccess; ++b)
        err = cudaStreamWaitEvent(g_batch_streams[1 + b], fork, 0);
      for (size_t u = 0; u < items.size() && err == cudaSuccess && rc == DGC_OK; ++u) {
        cudaStream_t bs = g_batch_streams[1 + u % branches];
        const int it = items[u];
        if (it >= 0) {
          rc = rk_sequence_merged(groups[it], meshes, winds, states, nsteps, (int)scheme, prec, bs);
        } else {
          const int i = -it - 1;
          rc = rk_sequence(meshes[i], winds[i], states[i], ds[i], nsteps[i], (int)scheme, pr[i], bs);
        }
      }
      for (int b = 0; b < branches && err == cudaSuccess; ++b) {
        cudaEvent_t join;
        err = new_event(&join);
        if (err == cudaSuccess) err = cudaEventRecord(join, g_batch_streams[1 + b]);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(main_st, join, 0);
      }
    }
    cudaGraph_t g = nullptr;
    cudaError_t err2 = cudaStreamEndCapture(main_st, &g);
    cleanup();
    if (rc != DGC_OK || err != cudaSuccess || err2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (lists) cudaFree(lists);
      if (rc != DGC_OK) return rc;
      return fail(DGC_ERR_CUDA, "batch graph capture failed: %s",
                  cudaGetErrorString(err != cudaSuccess ? err : err2));
    }
    BatchGraph bg;
    bg.key = key;
    bg.meshes.assign(meshes, meshes + n_inst);
    bg.lists = lists;
    err = cudaGraphInstantiate(&bg.exec, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) {
      if (lists) cudaFree(lists);
      return fail(DGC_ERR_CUDA, "batch graph instantiation failed: %s", cudaGetErrorString(err));
    }
    g_batch_cache.push_back(bg);
    hit = &g_batch_cache.back();
  }
  DGC_CUDA(cudaGraphLaunch(hit->exec, as_stream(stream)));
  return DGC_OK;
}

dgc_status dgc_point_coords(const dgc_mesh* mesh, int kind, double* xyz, int64_t* count) {
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (kind < 0 || kind > 2) return fail(DGC_ERR_ARG, "kind must be 0, 1 or 2");
  const dgc::Tables& t = mesh->quad  ? dgc::quad_tables(mesh->s.K)
                         : mesh->hex ? dgc::hex_tables(mesh->s.K)
                                     : dgc::tables(mesh->s.D, mesh->s.K);
  const int D = mesh->s.D, NF = mesh->s.NF;
  std::vector<double> dofpts;
  if (kind == 2) {   // facet DOF points of every local facet, then the interior points
    dofpts = t.xfd;
    dofpts.insert(dofpts.end(), t.xd.begin(), t.xd.end());
  }
  const std::vector<double>& ref = kind == 0 ? t.lag_nodes : (kind == 1 ? t.xd : dofpts);
  const int P = (int)ref.size() / D;
  if (count) *count = (int64_t)mesh->E * P;
  if (!xyz) return DGC_OK;
  for (int e = 0; e < mesh->E; ++e) {
    const int* v = &mesh->h_elems[(size_t)e * (mesh->hex ? 8 : NF)];   // vertices per element
    const double* X0 = &mesh->h_verts[(size_t)v[0] * D];
    if (mesh->Ec && mesh->h_cid[e] >= 0) {   // curved: the quadratic map through the six nodes
      const double* X = &mesh->h_cnodes[(size_t)mesh->h_cid[e] * 12];
      for (int p = 0; p < P; ++p) {
        const double x1 = ref[p * 2], x2 = ref[p * 2 + 1], x0 = 1.0 - x1 - x2;
        const double phi[6] = {x0 * (2 * x0 - 1), x1 * (2 * x1 - 1), x2 * (2 * x2 - 1), 4 * x0 * x1, 4 * x0 * x2,
                               4 * x1 * x2};
        for (int r = 0; r < 2; ++r) {
          double x = 0.0;
          for (int j = 0; j < 6; ++j) x += phi[j] * X[j * 2 + r];
          xyz[((size_t)e * P + p) * 2 + r] = x;
        }
      }
      continue;
    }
    for (int p = 0; p < P; ++p)
      for (int r = 0; r < D; ++r) {
        double x = X0[r];
        for (int c = 0; c < D; ++c) {
          // simplex: X_{c+1}; parallelogram: X_1, X_3; parallelepiped: X_1, X_3, X_4
          const int vc = v[c == 0 ? 1 : (mesh->quad || mesh->hex) ? (c == 1 ? 3 : 4) : c + 1];
          x += (mesh->h_verts[(size_t)vc * D + r] - X0[r]) * ref[p * D + c];
        }
        xyz[((size_t)e * P + p) * D + r] = x;
      }
  }
  return DGC_OK;
}

dgc_status dgc_wind_from_potential(dgc_mesh* mesh, const double* pot, double* u_hdiv, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (!pot || !u_hdiv) return fail(DGC_ERR_ARG, "NULL vector");
  DGC_CUDA(dgc::launch_wind_from_potential(mesh->view(), pot, u_hdiv, as_stream(stream)));
  return DGC_OK;
}

dgc_status dgc_hdiv_interpolate(dgc_mesh* mesh, const double* vals, double* u_hdiv, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (mesh->Ec) return fail(DGC_ERR_UNSUPPORTED, "point-value input on curved elements is not available");
  if (!vals || !u_hdiv) return fail(DGC_ERR_ARG, "NULL vector");
  DGC_CUDA(dgc::launch_hdiv_interpolate(mesh->view(), vals, u_hdiv, as_stream(stream)));
  return DGC_OK;
}

dgc_status dgc_project(dgc_mesh* mesh, const double* vals, double* w_dg, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (mesh->Ec) return fail(DGC_ERR_UNSUPPORTED, "point-value input on curved elements is not available");
  if (!vals || !w_dg) return fail(DGC_ERR_ARG, "NULL vector");
  DGC_CUDA(dgc::launch_project(mesh->view(), vals, w_dg, as_stream(stream)));
  return DGC_OK;
}

dgc_status dgc_max_wind_speed(dgc_mesh* mesh, const double* wind_hdiv, double* out, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (!wind_hdiv || !out) return fail(DGC_ERR_ARG, "NULL argument");
  cudaStream_t st = as_stream(stream);
  DGC_CUDA(mesh->reduce.alloc(1));
  DGC_CUDA(cudaMemsetAsync(mesh->reduce.ptr, 0, sizeof(unsigned long long), st));
  DGC_CUDA(dgc::launch_max_speed(mesh->view(), wind_hdiv, mesh->reduce.ptr, st));
  unsigned long long bits = 0;
  DGC_CUDA(cudaMemcpyAsync(&bits, mesh->reduce.ptr, sizeof(bits), cudaMemcpyDeviceToHost, st));
  DGC_CUDA(cudaStreamSynchronize(st));
  double v;
  std::memcpy(&v, &bits, sizeof(v));
  *out = v;
  return DGC_OK;
}

dgc_status dgc_table(int dim, int k, const char* name, double* out, int64_t* count) {
  if (!name || !count) return fail(DGC_ERR_ARG, "NULL argument");
  if (!dgc::supported(dim, k)) return fail(DGC_ERR_UNSUPPORTED, "order k=%d not supported for dim %d", k, dim);
  const dgc::Tables* tp;
  try {
    tp = &dgc::tables(dim, k);
  } catch (const std::exception& ex) {
    return fail(DGC_ERR_ARG, "reference table build failed: %s", ex.what());
  }
  const dgc::Tables& t = *tp;
  const std::vector<double>* v = nullptr;
  const std::string n(name);
  if (n == "Bv") v = &t.Bv;
  else if (n == "Gv") v = &t.Gv;
  else if (n == "wv") v = &t.wv;
  else if (n == "xv") v = &t.xv;
  else if (n == "wf") v = &t.wf;
  else if (n == "sf") v = &t.sf;
  else if (n == "Ef") v = &t.Ef;
  else if (n == "Qt") v = &t.Qt;
  else if (n == "Cb") v = &t.Cb;
  else return fail(DGC_ERR_ARG, "unknown table '%s'", name);
  *count = (int64_t)v->size();
  if (out) std::memcpy(out, v->data(), v->size() * sizeof(double));
  return DGC_OK;
}

dgc_status dgc_quad_table(int k, const char* name, double* out, int64_t* count) {
  if (!name || !count) return fail(DGC_ERR_ARG, "NULL argument");
  if (!dgc::quad_supported(k)) return fail(DGC_ERR_UNSUPPORTED, "order k=%d not supported for parallelograms", k);
  const dgc::Tables* tp;
  try {
    tp = &dgc::quad_tables(k);
  } catch (const std::exception& ex) {
    return fail(DGC_ERR_ARG, "reference table build failed: %s", ex.what());
  }
  const dgc::Tables& t = *tp;
  const std::vector<double>* v = nullptr;
  const std::string n(name);
  if (n == "Bv") v = &t.Bv;
  else if (n == "Gv") v = &t.Gv;
  else if (n == "wv") v = &t.wv;
  else if (n == "xv") v = &t.xv;
  else if (n == "wf") v = &t.wf;
  else if (n == "sf") v = &t.sf;
  else if (n == "Bf") v = &t.Bf;
  else if (n == "Cb") v = &t.Cb;
  else if (n == "q1L") v = &t.q1L;
  else if (n == "q1D") v = &t.q1D;
  else if (n == "q1E") v = &t.q1E;
  else return fail(DGC_ERR_ARG, "unknown table '%s'", name);
  *count = (int64_t)v->size();
  if (out) std::memcpy(out, v->data(), v->size() * sizeof(double));
  return DGC_OK;
}

dgc_status dgc_quad_connectivity(int n_vert, int n_elem, const int32_t* elems, int32_t* facet_id, int32_t* nbr,
                                 int8_t* orient, int8_t* flip, int32_t* n_facets) {
  if (n_elem <= 0 || n_vert <= 0 || !elems) return fail(DGC_ERR_ARG, "empty mesh");
  std::vector<int> el(elems, elems + (size_t)n_elem * 4);
  dgc::Connectivity con;
  std::vector<signed char> fl;
  std::vector<int> qn;
  std::string why = dgc::build_quad_connectivity(n_vert, n_elem, el, con, fl, qn);
  if (!why.empty()) return fail(DGC_ERR_ARG, "%s", why.c_str());
  const size_t n = (size_t)n_elem * 4;
  for (size_t j = 0; j < n; ++j) {
    if (facet_id) facet_id[j] = con.facet_id[j];
    if (nbr) nbr[j] = qn[j];
    if (orient) orient[j] = con.orient[j];
    if (flip) flip[j] = fl[j];
  }
  if (n_facets) *n_facets = con.n_facets;
  return DGC_OK;
}

dgc_status dgc_hex_table(int k, const char* name, double* out, int64_t* count) {
  if (!name || !count) return fail(DGC_ERR_ARG, "NULL argument");
  if (!dgc::hex_supported(k)) return fail(DGC_ERR_UNSUPPORTED, "order k=%d not supported for parallelepipeds", k);
  const dgc::Tables* tp;
  try {
    tp = &dgc::hex_tables(k);
  } catch (const std::exception& ex) {
    return fail(DGC_ERR_ARG, "reference table build failed: %s", ex.what());
  }
  const dgc::Tables& t = *tp;
  const std::vector<double>* v = nullptr;
  const std::string n(name);
  if (n == "Bv") v = &t.Bv;
  else if (n == "wv") v = &t.wv;
  else if (n == "xv") v = &t.xv;
  else if (n == "wf") v = &t.wf;
  else if (n == "Bf") v = &t.Bf;
  else if (n == "Cb") v = &t.Cb;
  else if (n == "q1L") v = &t.q1L;
  else if (n == "q1D") v = &t.q1D;
  else if (n == "q1E") v = &t.q1E;
  else return fail(DGC_ERR_ARG, "unknown table '%s'", name);
  *count = (int64_t)v->size();
  if (out) std::memcpy(out, v->data(), v->size() * sizeof(double));
  return DGC_OK;
}

dgc_status dgc_hex_connectivity(int n_vert, int n_elem, const int32_t* elems, int32_t* facet_id, int32_t* nbr,
                                int8_t* orient, int8_t* fcode, int32_t* n_facets) {
  if (n_elem <= 0 || n_vert <= 0 || !elems) return fail(DGC_ERR_ARG, "empty mesh");
  std::vector<int> el(elems, elems + (size_t)n_elem * 8);
  dgc::Connectivity con;
  std::vector<signed char> fc;
  std::vector<int> qn;
  std::string why = dgc::build_hex_connectivity(n_vert, n_elem, el, con, fc, qn);
  if (!why.empty()) return fail(DGC_ERR_ARG, "%s", why.c_str());
  const size_t n = (size_t)n_elem * 6;
  for (size_t j = 0; j < n; ++j) {
    if (facet_id) facet_id[j] = con.facet_id[j];
    if (nbr) nbr[j] = qn[j];
    if (orient) orient[j] = con.orient[j];
    if (fcode) fcode[j] = fc[j];
  }
  if (n_facets) *n_facets = con.n_facets;
  return DGC_OK;
}

dgc_status dgc_connectivity(int dim, int n_vert, int n_elem, const int32_t* elems, int32_t* facet_id, int32_t* nbr,
                            int8_t* orient, int32_t* n_facets) {
  if (dim != 2 && dim != 3) return fail(DGC_ERR_UNSUPPORTED, "dim must be 2 or 3");
  if (n_elem <= 0 || n_vert <= 0 || !elems) return fail(DGC_ERR_ARG, "empty mesh");
  std::vector<int> el(elems, elems + (size_t)n_elem * (dim + 1));
  dgc::Connectivity con;
  std::string why = dgc::build_connectivity(dim, n_vert, n_elem, el, con);
  if (!why.empty()) return fail(DGC_ERR_ARG, "%s", why.c_str());
  const size_t n = (size_t)n_elem * (dim + 1);
  for (size_t j = 0; j < n; ++j) {
    if (facet_id) facet_id[j] = con.facet_id[j];
    if (nbr) nbr[j] = con.nbr[j];
    if (orient) orient[j] = con.orient[j];
  }
  if (n_facets) *n_facets = con.n_facets;
  return DGC_OK;
}

// ---- checkpoint / resume ----------------------------------------------------------
namespace {
struct StateHeader {
  char magic[4];          // "DGCS"
  uint32_t version;       // 1
  int32_t dim, k;
  int64_t n_elem, n_dg;
  double t;
  int64_t step;
  uint64_t checksum;      // FNV-1a 64 of the payload bytes
};
uint64_t fnv1a64(const unsigned char* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t j = 0; j < n; ++j) {
    h ^= p[j];
    h *= 1099511628211ull;
  }
  return h;
}
}  // namespace

dgc_status dgc_state_save(const dgc_mesh* mesh, const double* v_dg, double t, int64_t step, void* blob,
                          int64_t* size, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (!v_dg || !size) return fail(DGC_ERR_ARG, "NULL argument");
  const size_t n = (size_t)mesh->E * mesh->s.D * mesh->s.N;
  const size_t bytes = sizeof(StateHeader) + n * sizeof(double);
  if (!blob) {
    *size = (int64_t)bytes;
    return DGC_OK;
  }
  if (*size < (int64_t)bytes) return fail(DGC_ERR_ARG, "blob holds %lld bytes, %zu needed", (long long)*size, bytes);
  unsigned char* out = static_cast<unsigned char*>(blob);
  cudaStream_t st = as_stream(stream);
  DGC_CUDA(cudaMemcpyAsync(out + sizeof(StateHeader), v_dg, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  DGC_CUDA(cudaStreamSynchronize(st));
  StateHeader h;
  std::memcpy(h.magic, "DGCS", 4);
  h.version = 1;
  h.dim = mesh->s.D;
  h.k = mesh->s.K;
  h.n_elem = mesh->E;
  h.n_dg = (int64_t)n;
  h.t = t;
  h.step = step;
  h.checksum = fnv1a64(out + sizeof(StateHeader), n * sizeof(double));
  std::memcpy(out, &h, sizeof(h));
  *size = (int64_t)bytes;
  return DGC_OK;
}

dgc_status dgc_state_load(const dgc_mesh* mesh, const void* blob, int64_t size, double* v_dg, double* t,
                          int64_t* step, void* stream) {
  DGC_RANGE();
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (!blob || !v_dg) return fail(DGC_ERR_ARG, "NULL argument");
  if (size < (int64_t)sizeof(StateHeader)) return fail(DGC_ERR_ARG, "blob too short for a header");
  StateHeader h;
  std::memcpy(&h, blob, sizeof(h));
  const size_t n = (size_t)mesh->E * mesh->s.D * mesh->s.N;
  if (std::memcmp(h.magic, "DGCS", 4) != 0 || h.version != 1) return fail(DGC_ERR_ARG, "not a dgconv state blob");
  if (h.dim != mesh->s.D || h.k != mesh->s.K || h.n_elem != mesh->E || h.n_dg != (int64_t)n)
    return fail(DGC_ERR_ARG, "blob is for dim %d, k %d, %lld elements; mesh has dim %d, k %d, %d elements", h.dim, h.k,
                (long long)h.n_elem, mesh->s.D, mesh->s.K, mesh->E);
  if (size < (int64_t)(sizeof(StateHeader) + n * sizeof(double))) return fail(DGC_ERR_ARG, "blob truncated");
  const unsigned char* payload = static_cast<const unsigned char*>(blob) + sizeof(StateHeader);
  if (fnv1a64(payload, n * sizeof(double)) != h.checksum) return fail(DGC_ERR_ARG, "blob checksum mismatch");
  cudaStream_t st = as_stream(stream);
  DGC_CUDA(cudaMemcpyAsync(v_dg, payload, n * sizeof(double), cudaMemcpyHostToDevice, st));
  DGC_CUDA(cudaStreamSynchronize(st));
  if (t) *t = h.t;
  if (step) *step = h.step;
  return DGC_OK;
}

dgc_status dgc_check(dgc_mesh* mesh, void* stream) {
  if (dgc_status rc = check_mesh(mesh)) return rc;
  cudaStream_t st = as_stream(stream);
  int word[2] = {0, 0};
  DGC_CUDA(cudaMemcpyAsync(word, mesh->status.ptr, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  DGC_CUDA(cudaStreamSynchronize(st));
  if (word[0]) {
    DGC_CUDA(cudaMemsetAsync(mesh->status.ptr, 0, 2 * sizeof(int), st));
    DGC_CUDA(cudaStreamSynchronize(st));
    if (word[0] & 8)
      return fail(DGC_ERR_BOUNDS, "a gather index was out of range (checked build; first index %d, status word 0x%x)",
                  word[1], word[0]);
    if (word[0] & 2) return fail(DGC_ERR_TIMEOUT, "a bounded device-side wait gave up (status word 0x%x)", word[0]);
    if (word[0] & 4)
      return fail(DGC_ERR_NONFINITE, "dgc_diagnostics met a non-finite coefficient (status word 0x%x)", word[0]);
    return fail(DGC_ERR_NONFINITE, "non-finite residual norm in the pseudo-time iteration (status word 0x%x)",
                word[0]);
  }
  return DGC_OK;
}

dgc_status dgc_min_edge(const dgc_mesh* mesh, double* out) {
  if (dgc_status rc = check_mesh(mesh)) return rc;
  if (!out) return fail(DGC_ERR_ARG, "out is NULL");
  *out = mesh->h_min;
  return DGC_OK;
}

}  // extern "C"
