// Launch wrappers of the dgconv kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "dgc_checked.h"
#include "dgc_internal.h"

namespace dgc {

struct StageArgs;
struct StageTcArgs;

// Device view of a mesh and of its FP64 reference tables.
struct DevMesh {
  Sizes s;
  int E, nF, nV;
  const double* verts;        // [nV][D]
  const int* elems;           // [E][NF], sorted vertex ids
  double* J;                  // [E][D][D]
  double* detJ;               // [E]
  const int* nbr;             // [E][NF]  (e' << 2) | f', or -1
  const int* facet_id;        // [E][NF]
  int* status;                // [2] device status words (gather checks of the checked build)
  int inject_bad_facet = 0;   // checked build only: DGC_FAULT=gather offsets element 0's facet ids
  const signed char* orient;  // [E][NF]  +1 owner / boundary, -1 otherwise
  const int* facet_sides;     // [nF][2]  (e << 2) | f, second entry -1 on the boundary
  // FP64 tables
  const double* Bv;
  const double* wv;
  const double* wf;
  const double* Bf;
  const double* Cb;
  const double* Lg_int;
  const double* Lg_fac;
  const double* Tint;
  const double* wd;
  const double* wfd;
  const double* Qfd;
  const double* Bd;
  // parallelograms: element type and the facet-parameter flips [E][4]
  int quad = 0;
  const signed char* flip = nullptr;
  // parallelepipeds: element type and the face codes [E][6] (T | o1 << 1 | o2 << 2)
  int hex = 0;
  const signed char* fcode = nullptr;
  // curved (quadratic) triangles: Ec of them, celem [Ec] their element ids, cid [E]
  // the curved index of an element or -1, cnodes [Ec][6][2] their P2 nodes, the P2
  // reference gradients at the interior rule (p2d [QD][6][2]) and at the volume rule
  // (p2v [QV][6][2]), and their inverse mass blocks [N*N][Ec] (FP64 and FP32)
  int Ec = 0;
  const int* celem = nullptr;
  const int* cid = nullptr;
  const double* cnodes = nullptr;
  const double* p2d = nullptr;
  const double* p2v = nullptr;
  double* Minv64 = nullptr;
  float* Minv32 = nullptr;
};

// a == nullptr prepares the kernel (shared-memory attribute) without launching
cudaError_t launch_stage_2d(int K, bool fp32, const StageArgs* a, cudaStream_t s);
cudaError_t launch_stage_3d(int K, bool fp32, const StageArgs* a, cudaStream_t s);
// parallelograms, sum-factorised; a->nbr holds the (e' << 3) | (rev << 2) | f' codes
// and a->tab the 1D tables [l at the Gauss points | l' there | l(0), l(1)]
cudaError_t launch_stage_quad(int K, bool fp32, const StageArgs* a, cudaStream_t s);
// parallelepipeds, one block per element; a->nbr holds (e' << 3) | f', the frozen wind
// is element-major (Uw [E][QV][3], Fw [E][6][QF]), fcode the face codes [E][6]
cudaError_t launch_stage_hex(int K, bool fp32, const StageArgs* a, const signed char* fcode, cudaStream_t s);
// copy the order-K 1D tables [l at the Gauss points | l' there | l(0), l(1)] into the
// kernel's constant-memory slot (synchronous; call before any stream capture)
cudaError_t quad_tables_to_constant(int K, const std::vector<double>& tab);

// tensor-core stage kernels (triangles and tetrahedra, k <= 4); a == nullptr prepares the kernel
bool tc_supported(int D, int K);
// the three BF16 pieces (round to nearest even) of x: x = p0 + p1 + p2 to about 2^-24 |x|
void bf16x3_pieces(double x, uint16_t* p);
// tetrahedra: the BF16 table chunks (GEMM A basis, GEMM B gradients) as bytes,
// the FP32 facet tables, the launch and the row-layout transposes
std::vector<unsigned char> tc3_chunks(int K, const Tables& t);
std::vector<float> tc3_ftab(int K, const Tables& t);
cudaError_t launch_stage_tc3(int K, const StageTcArgs* a, cudaStream_t s);
size_t tc3_rows_len(int K, int E);    // one state vector in the row layout
size_t tc3_tr_len(int K, int E);      // its facet traces
size_t tc3_fw_len(int K, int E);      // the tile-blocked facet flux
cudaError_t launch_tc3_in(int K, const double* v, double* vt, float* vft, float* tr, const float* ftab, int E,
                          cudaStream_t s);
cudaError_t launch_tc3_out(int K, const double* vt, double* v, int E, cudaStream_t s);
// wind rows [tile][i][128] (component c of element e in row tc3_row, scaled by
// 1/det J) and the facet flux [tile][f][q][40] of the frozen wind
// tetrahedral tensor-core path: the wind coefficients (FP64 scratch uc3, tiles x 3 x N x 40),
// the wind at the volume points (wq3, wind_pts_tc3_len floats) and the facet flux (fw3)
cudaError_t launch_wind_tc3(const DevMesh& m, const double* u_hdiv, double* uc3, float* wq3, float* fw3, cudaStream_t s);
inline long wind_pts_tc3_len(int QV, long E) { return (E + 39) / 40 * ((QV + 15) / 16) * 1920L; }
int tc_nk(int D, int K);
// P: 0 = TF32 head/tail (3 products), 1 = BF16 three pieces (6 products)
std::vector<float> tc_blob(int D, int K, int P, const Tables& t);
cudaError_t launch_stage_tc(int D, int K, int P, const StageTcArgs* a, cudaStream_t s);
// tile-blocked layouts of the tensor-core path: lengths, and the ABI <-> TSOA transposes
// (the inward one also writes the facet traces of the state)
size_t tc_tsoa_len(int D, int K, int E);
size_t tc_tr_len(int D, int K, int E);
cudaError_t launch_tsoa_in(int D, int K, const double* v, double* vt, float* vft, float* tr, const float* blob,
                           int E, cudaStream_t s);
cudaError_t launch_tsoa_out(int D, int K, const double* vt, double* v, int E, cudaStream_t s);
// FP64-only ABI -> TSOA, and TSOA -> ABI from the buffer of a pair picked by the parity of ctrl[1]
cudaError_t launch_tsoa_in64(int D, int K, const double* v, double* vt, int E, cudaStream_t s);
cudaError_t launch_tsoa_out_sel(int D, int K, const double* vt0, const double* vt1, const double* ctrl, double* v,
                                int E, cudaStream_t s);
// wind on the Dubiner basis scaled by 1/det J, float, tile-blocked [tile][D][nk][128]
// (zero padded in i; entries of elements past E in the last tile are not written)
cudaError_t launch_wind_coeffs(const DevMesh& m, const double* u_hdiv, float* wc, int nk, cudaStream_t s);

cudaError_t launch_geometry(const DevMesh& m, cudaStream_t s);
// frozen-wind data of the stage kernels: Uw [QV*D][E], Fw [NF*QF][E] in float or double
cudaError_t launch_wind_prep(const DevMesh& m, const double* u_hdiv, void* Uw, void* Fw, bool fp32,
                             cudaStream_t s);
cudaError_t launch_transfer(const DevMesh& m, const double* u_hdiv, double* w_dg, cudaStream_t s);
cudaError_t launch_transfer_T(const DevMesh& m, const double* f_dg, double* g_hdiv, double* zbuf,
                              cudaStream_t s);
cudaError_t launch_mass(const DevMesh& m, const double* v, double* out, bool inverse, cudaStream_t s);
// mass per component and energy of a DG field (out [D + 2]: masses, energy, count of
// non-finite coefficients), deterministic two-pass reduction; mv [E D N] and
// partials [diag_blocks(E) (D + 2)] are scratch
int diag_blocks(long E);
cudaError_t launch_diagnostics(const DevMesh& m, const double* v, double* mv, double* partials, double* out,
                               int* status, cudaStream_t s);
cudaError_t launch_wind_from_potential(const DevMesh& m, const double* pot, double* u_hdiv, cudaStream_t s);
// BDM DOFs of a physical field given at the DOF points: vals [E][NF*QFD + QD][D]
cudaError_t launch_hdiv_interpolate(const DevMesh& m, const double* vals, double* u_hdiv, cudaStream_t s);
cudaError_t launch_project(const DevMesh& m, const double* vals, double* w_dg, cudaStream_t s);
cudaError_t launch_max_speed(const DevMesh& m, const double* u_hdiv, unsigned long long* out_bits,
                             cudaStream_t s);

// out = sum_t c[t] x[t] over n doubles
constexpr int kMaxTerms = 8;
struct CombineArgs {
  const double* x[kMaxTerms];
  double c[kMaxTerms];
  int nterms;
};
cudaError_t launch_combine(double* out, const CombineArgs& a, long n, cudaStream_t s);
// y = (float) x over n values
cudaError_t launch_to_float(const double* x, float* y, long n, cudaStream_t s);

// pseudo-time (Richardson) solve: residual + deterministic norm partials, update, control
int rich_blocks(long n);
cudaError_t launch_rich_resid(const double* g, const double* v, const double* r, double tau, double* rho,
                              const double* detJ, int DN, long n, double* partials, int nblocks, cudaStream_t s);
cudaError_t launch_rich_update(double* v, const double* rho, double ds, long n, cudaStream_t s);
cudaError_t launch_rich_control(const double* partials, int np, double* state, int* iters, double* res,
                                double reduction, int max_iter, bool first, cudaGraphConditionalHandle h,
                                int* status, cudaStream_t s);

}  // namespace dgc
