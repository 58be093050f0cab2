/*
 * dgconv -- the explicit upwind-DG convection step of Lehrenfeld & Schoeberl,
 * "High order exactly divergence-free Hybrid Discontinuous Galerkin Methods
 * for unsteady incompressible flows" (arXiv:1508.04245), on one GB300 GPU.
 *
 * The library evaluates, for affine triangles (dim = 2) and tetrahedra
 * (dim = 3) of polynomial order k, and for parallelograms, parallelepipeds and
 * quadratic (curved) triangles (dgc_mesh_upload_quad / _hex / _curved):
 *
 *   I        the transfer from the H(div)-conforming velocity space W_h
 *            (BDM_k) to the DG space V_h = [P^k]^dim            (Sec. 2.4)
 *   I^T      its transpose, from functionals on V_h to functionals on W_h
 *   M^-1 C   the upwind DG convection operator of Sec. 2.3 with the diagonal
 *            mass matrix of an L2-orthonormal basis
 *   Q        explicit SSP Runge-Kutta substeps of the propagation problem
 *            dv/ds + (M^V)^-1 C^V(u) v = 0 with a frozen wind u   (Sec. 3.2.2)
 *   (Id + tau M^-1 C)^-1   the implicit convection step, by pseudo-time
 *            (Richardson) iteration                              (Sec. 3.3.2)
 *   I^T M^V Q I, I^T C^V I   the OIFS right-hand side and the convection
 *            operator on W_h, each as one call        (Sec. 3.2, Sec. 2.4)
 *
 * Conventions shared by every call
 * --------------------------------
 * - Diagnostics: every compute entry point opens an NVTX range named after it
 *   (visible under a profiler, free otherwise).  For tests of error handling,
 *   the environment variable DGC_FAULT=alloc|capture|launch makes device
 *   allocations, graph captures or kernel launches fail on the host before the
 *   CUDA call is made; the call returns its DGC_ERR_* code and the handle stays
 *   usable.  In the checked build (libdgconv_checked.so, compiled with
 *   DGC_CHECKED=1: every neighbour code, facet DOF id and facet side is
 *   bounds-checked on the device), DGC_FAULT=gather offsets the facet DOF ids
 *   of element 0 out of range, which the checks catch (DGC_ERR_BOUNDS from
 *   dgc_check); the regular build ignores it.  DGC_FAULT=stall launches the tensor-core stage kernels with no
 *   bulk copy issued and a short poll budget: their bounded waits run out with
 *   nothing in flight, the results of that call are undefined, and dgc_check
 *   then returns DGC_ERR_TIMEOUT; the handle stays usable.
 * - Status: 0 (DGC_OK) on success, a negative DGC_ERR_* code otherwise; the
 *   message is available from dgc_last_error().  Argument errors are detected
 *   on the host before anything is launched.
 * - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is enqueued asynchronously; no call synchronizes unless its
 *   comment says so.
 * - Memory: every array argument marked "device" is caller-owned device memory
 *   of the stated length in doubles; "host" arrays are caller-owned host memory.
 *   The library owns only the dgc_mesh handle, its geometry, its scratch
 *   buffers and its cached CUDA graphs, all released by dgc_mesh_free().
 * - DG layout ("dg vector", n_dg = E * dim * N doubles): element-major
 *   [E][dim][N], coefficients of each velocity component on the orthonormal
 *   Dubiner basis of the element (N = dim P^k), so M^V_T = |det J_T| Id.
 * - H(div) layout ("hdiv vector", n_hdiv doubles): [n_facets][n_fm] facet
 *   normal moments int_F u.n_F q_m dS (n_F = outward normal of the facet's
 *   lower-index element, q_m the facet Dubiner basis in the facet's
 *   sorted-vertex parametrisation, n_fm = dim P^k(F)), then [E][n_int]
 *   interior moments against the unit-normalised Nedelec space N_{k-1}.
 *   Global facets are numbered by their sorted vertex tuples in lexicographic
 *   order.  The tangential facet unknowns of the HDG space have no part in
 *   convection (Sec. 2.4) and are not represented.
 * - Orders supported: dim 2, k = 1..6; dim 3, k = 1..5 (DGC_ERR_UNSUPPORTED
 *   otherwise).
 * - Parallelograms (handles from dgc_mesh_upload_quad, the uncurved
 *   quadrilaterals of Sec. 2 "Preliminaries"): V_h = [Q^k]^2 on the basis
 *   psi_{ab} = l_a(xi) l_b(eta), i = a (k+1) + b, l_a the orthonormal shifted
 *   Legendre polynomial on [0,1] (N = (k+1)^2, M^V_T = |det J_T| Id); W_h the
 *   H(div)-conforming subspace of the Piola images of [Q^k]^2, so W_h lies in
 *   V_h and I is an embedding (Sec. 2.4).  H(div) layout: [n_facets][k+1]
 *   facet moments int_F u.n_F l_m(s) dS, s running from the facet's lower to
 *   its higher global vertex id, then [E][2(k+1)(k-1)] interior moments of the
 *   reference field against (l_a l_b, 0), a <= k-2, b <= k, then
 *   (0, l_a l_b), a <= k, b <= k-2.  dgc_geometry, dgc_transfer,
 *   dgc_transfer_T(_noalloc), dgc_mass_apply, dgc_conv_apply, dgc_rk_substeps,
 *   dgc_batch_rk_substeps, dgc_richardson, dgc_oifs_rhs, dgc_conv_apply_hdiv,
 *   dgc_wind_extrapolate, dgc_wind_from_potential, dgc_hdiv_interpolate,
 *   dgc_project, dgc_point_coords, dgc_max_wind_speed, dgc_min_edge,
 *   dgc_state_save / _load and dgc_check accept them with DGC_FP64 and
 *   DGC_FP32 (the stage kernel contracts one direction at a time); the
 *   tensor-core precisions return DGC_ERR_UNSUPPORTED.  dgc_wind_from_potential
 *   takes the stream function at the (k+1)^2 nodes (a/k, b/k), index
 *   a (k+1) + b, of every element (dgc_point_coords kind 0).
 */
#ifndef DGCONV_H
#define DGCONV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgc_mesh dgc_mesh;
typedef int dgc_status;

#define DGC_OK 0
#define DGC_ERR_ARG (-1)          /* invalid argument (null pointer, bad size, degenerate mesh) */
#define DGC_ERR_CUDA (-2)         /* a CUDA runtime call or kernel launch failed */
#define DGC_ERR_UNSUPPORTED (-3)  /* dimension / order / precision not available */
#define DGC_ERR_TIMEOUT (-4)      /* a bounded device-side wait gave up */
#define DGC_ERR_NONFINITE (-5)    /* a NaN or Inf was produced */
#define DGC_ERR_ALLOC (-6)        /* device or host allocation failed */
#define DGC_ERR_BOUNDS (-7)       /* a gather index was out of range (checked build only) */

/* Contraction precision of the convection stages; the state is FP64 in every
 * mode.
 *   DGC_FP64    FP64 on CUDA cores
 *   DGC_FP32    FP32 on CUDA cores
 *   DGC_BF16X3  triangles, k <= 6: the evaluation at the quadrature points on
 *               tcgen05 tensor cores, kind::f16, each operand split exactly into
 *               three BF16 pieces, six products, FP32 accumulation; the test
 *               contractions in FP32 on CUDA cores; FP32 stage increments,
 *               FP64 accumulation once per substep
 *               tetrahedra, k <= 4: both contractions of the volume term on
 *               tcgen05 (the evaluation at the quadrature points and the test
 *               contraction against the basis gradients), the same split with
 *               the head pieces on grids that make every head x head sum exact,
 *               each chunk of 16 quadrature points accumulated separately and the
 *               chunks added in FP32 on CUDA cores; the facet terms in FP32 on
 *               CUDA cores; FP32 increments, FP64 accumulation once per substep
 *   DGC_TF32X3  triangles, k <= 6: as DGC_BF16X3 with kind::tf32 and a
 *               two-piece TF32 split (about 22 significand bits per operand),
 *               three products
 * Other orders, other element shapes and DGC_TF32X3 on tetrahedra return
 * DGC_ERR_UNSUPPORTED for the tensor-core precisions. */
typedef enum { DGC_FP64 = 0, DGC_FP32 = 1, DGC_BF16X3 = 2, DGC_TF32X3 = 3 } dgc_prec;
typedef enum { DGC_SSPRK2 = 2, DGC_SSPRK3 = 3 } dgc_scheme;

/* Build a mesh handle: connectivity on the host, then geometry on the device
 * (step a1).  verts: host [n_vert][dim]; elems: host [n_elem][dim+1] vertex
 * ids of affine simplices (any local order; the library sorts each element's
 * vertices by global id, which orients every facet consistently).  The mesh
 * must be conforming (a facet is shared by at most two elements) and no
 * element may be degenerate.  Synchronizes `stream` once at the end.
 * Sec. 2 "Preliminaries" (affine simplicial partition, facets). */
dgc_status dgc_mesh_upload(int dim, int k, int n_vert, const double* verts, int n_elem,
                           const int32_t* elems, void* stream, dgc_mesh** out);

/* Build a handle for a conforming mesh of parallelograms of order k = 1..6.
 * verts: host [n_vert][2]; elems: host [n_elem][4] vertex ids in cyclic order
 * (either sense of rotation, any starting corner; the order is kept:
 * x = X_0 + J xi with J[:, 0] = X_1 - X_0, J[:, 1] = X_3 - X_0 on [0,1]^2).
 * Every element must satisfy |X_0 + X_2 - X_1 - X_3| <= 1e-12 times its size
 * (a parallelogram: an uncurved quadrilateral, Sec. 2 "Preliminaries") and be
 * non-degenerate; n_elem < 2^28.  Local facets: eta = 0 (X_0 -> X_1),
 * xi = 1 (X_1 -> X_2), eta = 1 (X_3 -> X_2), xi = 0 (X_0 -> X_3).  Facets are
 * numbered by their sorted vertex pairs in lexicographic order, each owned by
 * its lower-index element.  Synchronizes `stream` once at the end.  Errors:
 * DGC_ERR_ARG (bad arrays, non-conforming, not a parallelogram, degenerate),
 * DGC_ERR_UNSUPPORTED (k), DGC_ERR_ALLOC, DGC_ERR_CUDA. */
dgc_status dgc_mesh_upload_quad(int k, int n_vert, const double* verts, int n_elem,
                                const int32_t* elems, void* stream, dgc_mesh** out);

/* Build a handle for a conforming mesh of parallelepipeds (uncurved hexahedra)
 * of order k = 1..3.  verts: host [n_vert][3]; elems: host [n_elem][8] vertex
 * ids in the local order (0,0,0), (1,0,0), (1,1,0), (0,1,0), (0,0,1), (1,0,1),
 * (1,1,1), (0,1,1) of the reference cube (kept: x = X_0 + J xi with
 * J = [X_1 - X_0, X_3 - X_0, X_4 - X_0]); every vertex must sit at X_0 + J c within
 * 1e-12 of the element's size.  V_h = [Q^k]^3 on psi_{abc} = l_a l_b l_c,
 * i = (a (k+1) + b)(k+1) + c; W_h the H(div) subspace of the Piola images of
 * [Q^k]^3.  H(div) layout: [n_faces][(k+1)^2] face moments
 * int_F u.n_F l_a(s1) l_b(s2) dS, mode a (k+1) + b, in the face's global parameter
 * (origin at its lowest vertex id, s1 towards the lower-id of the origin's two
 * face neighbours, s2 towards the other; n_F the lower-index element's outward
 * normal), then [E][3(k+1)^2(k-1)] interior moments of the reference field
 * against l_a l_b l_c in component d with the d-th degree <= k-2 (d outer, then
 * a, b, c).  Faces are numbered by their sorted vertex quadruples.  The same
 * entry points as for parallelograms accept such handles (DGC_FP64, DGC_FP32);
 * dgc_wind_from_potential takes the vector potential at the (k+1)^3 nodes
 * (a/k, b/k, c/k), [E][(k+1)^3][3].  Synchronizes `stream`. */
dgc_status dgc_mesh_upload_hex(int k, int n_vert, const double* verts, int n_elem, const int32_t* elems,
                               void* stream, dgc_mesh** out);

/* Build a handle for quadratic (curved) triangles of order k = 1..6 (remark on
 * curved elements, Sec. 2.4).  verts, elems as for dgc_mesh_upload with dim = 2;
 * edge_nodes: host [n_facets][2], the mid-node of every facet in the global facet
 * order (sorted vertex pairs, lexicographic; dgc_connectivity gives it).  Each
 * element is the image of the reference triangle under the P2 map through its
 * three (sorted) vertices and three edge nodes; an element whose edge nodes are
 * the chord midpoints (within 1e-14 of its shortest edge) is affine and keeps
 * the affine path.  On curved elements V_h holds the mapped Dubiner
 * polynomials, the mass matrix is a dense block (stored inverted, N*N doubles
 * and floats per curved element), I is the L2 projection, I^T its transpose;
 * the H(div) layout and DOFs are those of the affine case (Piola-mapped BDM_k).
 * Accepted on such handles: every entry point accepted on affine triangles with
 * DGC_FP64 / DGC_FP32, except dgc_richardson, dgc_hdiv_interpolate and
 * dgc_project (DGC_ERR_UNSUPPORTED); the tensor-core precisions return
 * DGC_ERR_UNSUPPORTED.  dgc_point_coords maps through the quadratic map.
 * Errors: those of dgc_mesh_upload; DGC_ERR_ARG when det J changes sign inside
 * an element (checked at the nodes and quadrature points).  Synchronizes
 * `stream`. */
dgc_status dgc_mesh_upload_curved(int k, int n_vert, const double* verts, int n_elem, const int32_t* elems,
                                  const double* edge_nodes, void* stream, dgc_mesh** out);

/* Release the handle and everything the library allocated for it. */
dgc_status dgc_mesh_free(dgc_mesh* mesh);

/* Lengths of the dg and hdiv vectors of this mesh. */
dgc_status dgc_sizes(const dgc_mesh* mesh, int64_t* n_dg, int64_t* n_hdiv);

/* info[0..12] = dim, k, n_elem, n_facets, N, N_W (=dim*N), n_fm, n_int,
 * n_lagrange (nodes of the potential interpolation per element), n_proj
 * (points of the projection rule), n_dofpts (points per element of the H(div)
 * interpolation), shape (0 simplices, 1 parallelograms, 2 quadratic triangles,
 * 3 parallelepipeds),
 * n_curved (curved elements; 0 unless shape 2).  info holds 13 entries. */
dgc_status dgc_mesh_info(const dgc_mesh* mesh, int64_t* info);

/* Step a1: recompute J (columns x_{i+1}-x_0 of the sorted vertices) and
 * det J of every element on the device.  Affine elements, Sec. 2. */
dgc_status dgc_geometry(dgc_mesh* mesh, void* stream);

/* Step a2, w = I u (Sec. 2.4, eq. for the L2 problem defining I):
 * (M^V)^-1 M^{U,V} applied to an hdiv vector.  u_hdiv: device [n_hdiv];
 * w_dg: device [n_dg], overwritten.  FP64. */
dgc_status dgc_transfer(dgc_mesh* mesh, const double* u_hdiv, double* w_dg, void* stream);

/* Step a8, g = I^T f (Sec. 2.4): the transpose of I, mapping a functional on
 * V_h (dg layout) to one on W_h (hdiv layout).  Facet entries are summed
 * over their (at most two) elements in a fixed order, owner first, so the
 * result is deterministic.  f_dg: device [n_dg]; g_hdiv: device [n_hdiv],
 * overwritten.  FP64. */
dgc_status dgc_transfer_T(dgc_mesh* mesh, const double* f_dg, double* g_hdiv, void* stream);

/* Diagnostics of a DG field v (device [n_dg]), the quantities of the conservation
 * and stability statements of Sec. 2.3: out[c] = sum_T int_T v_c dx for each of
 * the dim components (the mass, constant in time under a divergence-free wind
 * with no inflow), out[dim] = sum_T int_T |v|^2 dx (the energy, non-increasing
 * under the upwind flux) and out[dim + 1] = the number of non-finite
 * coefficients.  out: device [dim + 2], written asynchronously on `stream`.  The
 * sums run in a fixed two-pass tree order, so a result repeats bit for bit.  A
 * non-finite coefficient also marks the handle's status word: dgc_check then
 * returns DGC_ERR_NONFINITE (the check for a blown-up run after
 * dgc_rk_substeps).  All element shapes; FP64. */
dgc_status dgc_diagnostics(dgc_mesh* mesh, const double* v_dg, double* out, void* stream);

/* out = M^V v (inverse = 0) or (M^V)^-1 v (inverse = 1); M^V_T = |det J_T| Id
 * (Sec. 2.3, diagonal mass of an orthonormal basis).  device [n_dg] each;
 * out may equal v. */
dgc_status dgc_mass_apply(dgc_mesh* mesh, const double* v_dg, double* out_dg, int inverse, void* stream);

/* Steps a3-a6: out = (M^V)^-1 C^V(u) w, the upwind DG convection operator of
 * Sec. 2.3 with wind u in W_h (hdiv vector, exactly divergence-free for the
 * stability statement of Sec. 2.3 to hold) and zero inflow datum on the domain
 * boundary.  wind_hdiv: device [n_hdiv]; w_dg, out_dg: device [n_dg], must not
 * overlap.  prec selects the contraction precision (see dgc_prec; the result is
 * written in FP64). */
dgc_status dgc_conv_apply(dgc_mesh* mesh, const double* wind_hdiv, const double* w_dg, double* out_dg,
                          dgc_prec prec, void* stream);

/* Steps a3-a7 repeated: nsteps substeps of size ds of dv/ds = -(M^V)^-1 C^V(u) v
 * (the propagation problem of Sec. 3.2.2) by SSP-RK2 (Heun) or SSP-RK3
 * (Shu-Osher), wind frozen for the whole call.  v_dg: device [n_dg], FP64,
 * updated in place; the stage combinations are accumulated in FP64 whatever
 * prec is.  The launch sequence is captured in a CUDA graph cached on the
 * handle and replayed when the same arguments come again. */
dgc_status dgc_rk_substeps(dgc_mesh* mesh, const double* wind_hdiv, double* v_dg, double ds, int nsteps,
                           dgc_scheme scheme, dgc_prec prec, void* stream);

/* Many independent propagation problems (Sec. 3.2.2) in one call: instance i
 * advances states[i] (device [n_dg of meshes[i]], FP64, in place) by
 * nsteps[i] substeps of size ds[i] with the frozen wind winds[i] (device
 * [n_hdiv of meshes[i]]), exactly as dgc_rk_substeps would.  Meshes may
 * differ in size and order but must be distinct handles (each owns its
 * scratch).  All instances are captured into one CUDA graph whose branches
 * run concurrently; the graph is cached (keyed by every argument) and
 * replayed by later identical calls, and dropped when one of its meshes is
 * freed.  With DGC_TF32X3 or DGC_BF16X3 the affine-triangle instances of one
 * order share their stage launches: each stage is one launch of the persistent
 * kernel over the element tiles of all of them (those whose nsteps is not yet
 * reached), so the results equal the single calls' bit for bit.  The first
 * call uploads the per-instance stage arguments to device memory that the
 * cached graph owns.  meshes, winds, states, ds, nsteps: host arrays of n_inst
 * entries.
 * With DGC_TF32X3 or DGC_BF16X3, instances whose order the tensor-core path does not cover
 * (see dgc_prec) run their contractions in FP32 on CUDA cores. */
dgc_status dgc_batch_rk_substeps(int n_inst, dgc_mesh* const* meshes, const double* const* winds,
                                 double* const* states, const double* ds, const int* nsteps, dgc_scheme scheme,
                                 dgc_prec prec, void* stream);

/* Implicit convection step of the modified fractional-step-theta scheme
 * (Sec. 3.3.2): solves  v + tau (M^V)^-1 C^V(u) v = g  by explicit Euler steps
 * in pseudo-time (a Richardson iteration),
 *   rho_i = g - v_i - tau (M^V)^-1 C^V v_i,     v_{i+1} = v_i + ds rho_i,
 * stopped at the first i with ||rho_i|| <= reduction * ||rho_0|| or at
 * i = max_iter; ||x|| = sqrt(sum_T |det J_T| sum x^2), the L2 norm of the DG
 * function.  wind_hdiv: device [n_hdiv] (frozen u); g_dg: device [n_dg];
 * v_dg: device [n_dg], FP64, in: v_0 (initial guess), out: the returned v_i;
 * it must not overlap g_dg.  tau > 0 and ds in (0, 2) finite, reduction >= 0,
 * max_iter >= 0.  iters_dev: device int32[1], receives i; res_dev: device
 * [max_iter + 1] or NULL, receives ||rho_0|| .. ||rho_i|| (later entries
 * untouched).  prec selects the precision of the operator evaluation as in
 * dgc_conv_apply; residual, norm and update are FP64.  The iteration runs on
 * the device (a CUDA graph with a conditional WHILE node, cached on the handle
 * and replayed for identical arguments): nothing synchronizes, and iters_dev /
 * res_dev are valid once `stream` reaches the end of the call.  A non-finite
 * residual norm stops the iteration and makes the next dgc_check return
 * DGC_ERR_NONFINITE.  A stable ds is 1 / (1 + beta^2) with
 * beta = tau (2k+1) max|u| / (shortest edge). */
dgc_status dgc_richardson(dgc_mesh* mesh, const double* wind_hdiv, const double* g_dg, double* v_dg, double tau,
                          double ds, double reduction, int max_iter, dgc_prec prec, int32_t* iters_dev,
                          double* res_dev, void* stream);

/* The OIFS right-hand side M^{V,U} Q I u of Sec. 3.2 in one call:
 *   out = I^T M^V Q I u,
 * Q = nsteps SSP-RK substeps of size ds of the propagation problem (Sec. 3.2.2)
 * as in dgc_rk_substeps.  The convection velocity is wind_hdiv, frozen, when
 * wind_prev_hdiv is NULL; otherwise it is extrapolated linearly from wind_hdiv
 * (time t^n) and wind_prev_hdiv (time t^n - dt_prev) to the midpoint of each
 * substep, (1 + th_j) u^n - th_j u^{n-1} with th_j = (j + 1/2) ds / dt_prev,
 * and frozen within the substep.  u_hdiv, wind_hdiv, wind_prev_hdiv: device
 * [n_hdiv]; out_hdiv: device [n_hdiv], overwritten, must not overlap u_hdiv.
 * nsteps >= 0 (0 gives I^T M^V I u), ds > 0, dt_prev > 0 with wind_prev_hdiv.
 * The launch sequence is captured in a CUDA graph cached on the handle. */
dgc_status dgc_oifs_rhs(dgc_mesh* mesh, const double* u_hdiv, const double* wind_hdiv, const double* wind_prev_hdiv,
                        double dt_prev, double* out_hdiv, double ds, int nsteps, dgc_scheme scheme, dgc_prec prec,
                        void* stream);

/* The convection operator on W_h, C^U(u) w = I^T C^V(u) I w (Sec. 2.4), as one
 * call: out_hdiv = I^T M^V ((M^V)^-1 C^V(wind)) I u_hdiv.  wind_hdiv, u_hdiv:
 * device [n_hdiv]; out_hdiv: device [n_hdiv], overwritten, must not overlap
 * u_hdiv; prec as in dgc_conv_apply. */
dgc_status dgc_conv_apply_hdiv(dgc_mesh* mesh, const double* wind_hdiv, const double* u_hdiv, double* out_hdiv,
                               dgc_prec prec, void* stream);

/* Extrapolated convection velocity as a linear combination of earlier exactly
 * divergence-free velocities (Sec. 3.2.2): out = sum_t coefs[t] fields[t].
 * fields: host array of n_terms device pointers [n_hdiv]; coefs: host
 * [n_terms]; 1 <= n_terms <= 8; out_hdiv: device [n_hdiv], may equal one of
 * the fields (the combination is elementwise). */
dgc_status dgc_wind_extrapolate(dgc_mesh* mesh, int n_terms, const double* const* fields, const double* coefs,
                                double* out_hdiv, void* stream);

/* Autotuner of the CUDA-core stage kernel (every order of both element types,
 * DGC_FP64 and DGC_FP32): times one stage on this mesh with its wind for each
 * candidate block shape (64, 128, 192, 256 threads; reps timed launches each)
 * and keeps the fastest for this (dim, k, prec) in a process-wide table that
 * every later launch on any mesh of that kind uses.  Results do not depend on
 * the choice (each element is computed independently).  Drops the cached
 * graphs of this mesh (they hold the old shape).  *block_out (host, may be
 * NULL) receives the choice, 0 for the tensor-core precisions (one fixed tile shape, nothing
 * to tune).  1 <= reps <= 1000.  Synchronizes `stream`. */
dgc_status dgc_autotune(dgc_mesh* mesh, const double* wind_hdiv, dgc_prec prec, int reps, int* block_out,
                        void* stream);

/* Points at which callers evaluate input fields, host [count][dim]:
 * kind 0: the element-wise equispaced P^{k+1} Lagrange nodes used by
 *         dgc_wind_from_potential ([E][n_lagrange][dim]);
 * kind 1: the points of the projection rule used by dgc_project
 *         ([E][n_proj][dim]);
 * kind 2: the points of dgc_hdiv_interpolate ([E][n_dofpts][dim]): the facet
 *         DOF points of local facets 0..dim, then the interior points.
 * Writes count = rows when xyz is NULL. */
dgc_status dgc_point_coords(const dgc_mesh* mesh, int kind, double* xyz, int64_t* count);

/* Exactly divergence-free wind: the BDM_k DOFs of the curl of the P^{k+1}
 * Lagrange interpolant of a stream function (dim 2) or of the three
 * components of a vector potential (dim 3).  pot: device [E][n_lagrange]
 * (dim 2) or [E][n_lagrange][3] (dim 3) values at the kind-0 points;
 * u_hdiv: device [n_hdiv], overwritten.  (Input construction for the frozen,
 * discretely divergence-free wind of Sec. 3.2.2.) */
dgc_status dgc_wind_from_potential(dgc_mesh* mesh, const double* pot, double* u_hdiv, void* stream);

/* BDM_k interpolant in W_h of a physical vector field given at the kind-2
 * points: facet moments against the facet basis (taken from the facet's
 * owner element), interior moments against N_{k-1}.  vals: device
 * [E][n_dofpts][dim]; u_hdiv: device [n_hdiv], overwritten.  (Input
 * construction: the H(div)-conforming velocity of Sec. 2.1.1.) */
dgc_status dgc_hdiv_interpolate(dgc_mesh* mesh, const double* vals, double* u_hdiv, void* stream);

/* L2 projection onto V_h of a field given at the kind-1 points:
 * vals: device [E][n_proj][dim]; w_dg: device [n_dg], overwritten. */
dgc_status dgc_project(dgc_mesh* mesh, const double* vals, double* w_dg, void* stream);

/* max |u(x_q)| over the volume quadrature points (degree 3k-1 rule) of all
 * elements.  Synchronizes `stream`; result in *out (host). */
dgc_status dgc_max_wind_speed(dgc_mesh* mesh, const double* wind_hdiv, double* out, void* stream);

/* Checkpoint of a DG state (not part of the paper: restart support).  The blob
 * is host memory: a header (magic "DGCS", version 1, dim, k, n_elem, n_dg, the
 * caller's time t and step count, FNV-1a 64 checksum of the payload) followed
 * by the FP64 state in the DG layout.  dgc_state_save: with blob == NULL
 * writes the needed size to *size; otherwise *size is the blob's capacity on
 * input and the bytes written on output.  dgc_state_load: checks magic,
 * version, the mesh's dim / k / n_elem and the checksum (DGC_ERR_ARG on any
 * mismatch, nothing written), then copies the state to v_dg (device [n_dg])
 * and returns t and step (each pointer may be NULL).  Both synchronize
 * `stream`.  A run resumed from a saved state continues bit for bit. */
dgc_status dgc_state_save(const dgc_mesh* mesh, const double* v_dg, double t, int64_t step, void* blob,
                          int64_t* size, void* stream);
dgc_status dgc_state_load(const dgc_mesh* mesh, const void* blob, int64_t size, double* v_dg, double* t,
                          int64_t* step, void* stream);

/* Device-side status of the handle: synchronizes `stream`, returns
 * DGC_ERR_BOUNDS if a gather index was out of range (only the checked build,
 * libdgconv_checked.so, tests them; the message names the first such index),
 * else DGC_ERR_TIMEOUT if a bounded wait inside a kernel gave up since the last
 * check, else DGC_ERR_NONFINITE if dgc_richardson met a non-finite residual
 * norm or dgc_diagnostics a non-finite coefficient, else DGC_OK; a reported
 * word is cleared. */
dgc_status dgc_check(dgc_mesh* mesh, void* stream);

/* Shortest element edge of the mesh (host value, from the upload). */
dgc_status dgc_min_edge(const dgc_mesh* mesh, double* out);

/* Maximum scratch of dgc_transfer_T_noalloc, in doubles (16 MiB). */
#define DGC_NOALLOC_SCRATCH_DOUBLES 2097152LL

/* g = I^T f exactly as dgc_transfer_T, for callers that cannot allocate
 * device memory when they call: applications that reserve all their device
 * memory at start-up, and host loops that must not block on the device-wide
 * synchronisation a cudaMalloc or cudaFree implies (dgc_transfer_T allocates its
 * facet scratch on the handle at its first call).
 * The paper has no counterpart; this is a library service.
 * Scratch: a fixed file-scope device array of DGC_NOALLOC_SCRATCH_DOUBLES
 * doubles, held on every GPU that loads the library until the process exits.
 * The mesh must need at most that many: n_elem * (facets per element) * n_fm
 * doubles, with 3 facets per triangle, 4 per tetrahedron or parallelogram and
 * 6 per parallelepiped; larger meshes get DGC_ERR_ARG and a message, and
 * nothing is launched.  The call performs no allocation (no cudaMalloc /
 * cudaFree).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) for that device; make that first call before any
 * stream capture.  All calls share the one array, so calls that overlap on the
 * GPU (different streams, or different handles concurrently) race; serialise
 * them.  Every scratch entry a call reads is written by the same call first.
 * Arguments, layouts and errors as dgc_transfer_T. */
dgc_status dgc_transfer_T_noalloc(dgc_mesh* mesh, const double* f_dg, double* g_hdiv, void* stream);

/* Host-only introspection (no GPU needed) -------------------------------- */

/* Reference table `name` of the (dim, k) element, host double array.
 * Names: "Bv" [QV][N] basis at the volume points, "Gv" [QV][N][dim] reference
 * gradients, "wv" [QV] volume weights, "xv" [QV][dim] volume points, "wf" [QF]
 * and "sf" [QF][dim-1] the facet rule, "Ef" [dim+1][n_fm][N] traces on the facet
 * basis, "Qt" [QF][n_fm] facet basis at the facet points, "Cb" [N_W][N_W]
 * the BDM_k basis on the vector Dubiner basis.  Writes *count = entries; out
 * may be NULL to query the size. */
dgc_status dgc_table(int dim, int k, const char* name, double* out, int64_t* count);

/* Reference table `name` of the order-k parallelogram element (the square
 * [0,1]^2), host double array: "Bv" [QV][N] basis at the volume points
 * (q = p m + q', m = floor(3k/2) + 1 Gauss points per direction), "Gv"
 * [QV][N][2] reference gradients, "wv" [QV], "xv" [QV][2], "wf" [m], "sf" [m]
 * the 1D rule, "Bf" [4][m][N] the basis at the facet points, "Cb" [2N][2N] the
 * W_h basis on the vector tensor basis (column j: local basis function j),
 * "q1L" / "q1D" [m][k+1] l_a and l_a' at the Gauss points, "q1E" [2][k+1]
 * l_a(0) and l_a(1).  Writes *count = entries; out may be NULL to query the
 * size. */
dgc_status dgc_quad_table(int k, const char* name, double* out, int64_t* count);

/* Host connectivity exactly as dgc_mesh_upload_quad builds it: facet_id,
 * nbr ((e' << 3) | (rev << 2) | f', rev = 1 when the neighbour's local facet
 * parameter runs the other way; -1 on the boundary), orient (+1 owner /
 * boundary, -1 otherwise) and flip (1 when the local facet parameter runs
 * from the higher to the lower global vertex id), each [n_elem][4]; any output
 * may be NULL. */
dgc_status dgc_quad_connectivity(int n_vert, int n_elem, const int32_t* elems, int32_t* facet_id, int32_t* nbr,
                                 int8_t* orient, int8_t* flip, int32_t* n_facets);

/* Reference table `name` of the order-k parallelepiped element (the cube
 * [0,1]^3), host double array: "Bv" [QV][N] basis at the volume points
 * (q = (p m + q') m + q'', m = floor(3k/2) + 1), "wv" [QV], "xv" [QV][3], "wf"
 * [m^2] the face rule, "Bf" [6][m^2][N] the basis at the face points, "Cb"
 * [3N][3N] the W_h basis on the vector tensor basis, "q1L" / "q1D" [m][k+1],
 * "q1E" [2][k+1].  Writes *count = entries; out may be NULL. */
dgc_status dgc_hex_table(int k, const char* name, double* out, int64_t* count);

/* Host connectivity exactly as dgc_mesh_upload_hex builds it: facet_id, nbr
 * ((e' << 3) | f', -1 on the boundary), orient and fcode (T | o1 << 1 | o2 << 2:
 * the local corner (o1, o2) of the face's global origin, T = 1 when the global
 * s1 runs along the local s2), each [n_elem][6]; any output may be NULL. */
dgc_status dgc_hex_connectivity(int n_vert, int n_elem, const int32_t* elems, int32_t* facet_id, int32_t* nbr,
                                int8_t* orient, int8_t* fcode, int32_t* n_facets);

/* Host connectivity exactly as dgc_mesh_upload builds it: facet_id
 * [n_elem][dim+1], nbr [n_elem][dim+1] ((neighbour << 2) | neighbour's local
 * facet, or -1 on the boundary), orient [n_elem][dim+1] (+1 owner/boundary,
 * -1 otherwise), *n_facets.  Local facet f is opposite the f-th smallest
 * vertex id of the element. */
dgc_status dgc_connectivity(int dim, int n_vert, int n_elem, const int32_t* elems, int32_t* facet_id,
                            int32_t* nbr, int8_t* orient, int32_t* n_facets);

/* Copy the last error message of the calling thread into buf (len bytes,
 * NUL-terminated).  Synchronizes nothing. */
dgc_status dgc_last_error(char* buf, int len);

#ifdef __cplusplus
}
#endif

#endif /* DGCONV_H */
