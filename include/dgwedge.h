/*
 * dgwedge -- nodal discontinuous Galerkin for the first-order acoustic wave
 * equation on hybrid meshes of vertically mapped wedges and tetrahedra,
 * following Chan, Wang, Hewett & Warburton, "Reduced storage nodal
 * discontinuous Galerkin methods on semi-structured prismatic meshes".
 *
 * C ABI.  Plain pointers and sizes only.  Every call returns a dg_status
 * (0 = success); no exception, abort or device trap ever crosses this
 * boundary.  dg_last_error() gives a one-line description of the last failure
 * on a context.
 *
 * Problem (Section 2, eq. (1)):
 *   (1/kappa) dp/dt + div u = 0,   rho du/dt + grad p = 0,   kappa = rho c^2,
 * with rho and c constant per element, strong DG form with penalty fluxes
 *   F_p = 1/2 (tau_p [p] - n.[u]),  F_u = 1/2 (tau_u [u].n - [p]),
 *   tau_p = 1/{rho c}, tau_u = {rho c} (upwind) or tau = 0 (central),
 * where [x] = x_neighbour - x_own and {rho c} is the two-sided average.
 * Boundary ghosts: Dirichlet (p+ = -p-, u+ = u-, Section 2) or rigid wall
 * (p+ = p-, u+ = u- - 2 (n.u-) n).
 *
 * Discretisation: degree-N nodal bases (Section 3.1).  Wedges use the exact,
 * Jacobian-weighted mass matrix M^k = M^{tri,k} (x) M^1D (Section 4.2), with all
 * geometric factors recomputed from the six vertices on every evaluation
 * (Lemma 3.1); nothing per element is stored but vertex ids, neighbour ids and
 * material.  Time integration: five-stage fourth-order low-storage
 * Runge-Kutta (Carpenter & Kennedy 1994), res <- a_s res + dt f(q),
 * q <- q + b_s res.
 *
 * Canonical field layout (used by dg_set_fields, dg_get_fields, dg_rhs and
 * dg_node_coords): q[4][total_nodes], fields (p, u_x, u_y, u_z); nodes ordered
 * element by element in input order, each element contiguous:
 *   wedge: node n = j * Nt + i, j = 0..N the GLL index along the extruded
 *          (vertex 0 -> vertex 3) direction, i the triangle node;
 *   triangle node order: for b = 0..N, for a = 0..N-b  (barycentric weights
 *          (N-a-b, a, b)/N on vertices (0, 1, 2) before warping);
 *   tet:   for c = 0..N, for b = 0..N-c, for a = 0..N-b-c  (weights
 *          (N-a-b-c, a, b, c)/N on vertices (0, 1, 2, 3) before warping).
 * Nodes are Warp & Blend points (tet) and the tet's face points x GLL (wedge).
 * Element type sizes: wedge Np = (N+1)^2 (N+2)/2, tet Np = (N+1)(N+2)(N+3)/6.
 *
 * Memory: the library allocates no device memory.  The caller allocates one
 * mesh blob and three field buffers (sizes from dg_device_bytes) and passes
 * them to dg_bind; it keeps ownership.  Host arrays passed in are copied.
 * Work is issued asynchronously on the stream given to dg_bind.
 *
 * Call order: dg_mesh_create -> dg_set_order -> [dg_set_material]
 *   -> [dg_set_shots] -> [dg_add_source] -> [dg_set_options] -> [dg_set_mass_mode] -> dg_device_bytes -> dg_bind -> dg_set_fields
 *   -> dg_step / dg_rhs / dg_energy / dg_get_fields.
 * Setters after dg_bind return DG_ERR_STATE.  Several contexts may live in one
 * process; contexts with different (N, precision) must not run concurrently
 * on one device (operator tables live in device constant memory and are
 * reloaded, in stream order, when the configuration changes).
 */
#ifndef DGWEDGE_H
#define DGWEDGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx;

typedef enum dg_status {
  DG_OK = 0,
  DG_ERR_ARG = -1,       /* null pointer, size or enum out of range              */
  DG_ERR_MESH = -2,      /* invalid mesh: not vertically mapped, J <= 0, a face
                            shared by more than two elements, bad vertex id      */
  DG_ERR_ORDER = -3,     /* N outside 1..4                                       */
  DG_ERR_CUDA = -4,      /* a CUDA runtime call failed (message has the name)    */
  DG_ERR_STATE = -5,     /* call out of order                                    */
  DG_ERR_TIMEOUT = -6,   /* a bounded device-side wait ran out                   */
  DG_ERR_NONFINITE = -7  /* non-finite value found in the state                  */
} dg_status;

enum { DG_TET = 4, DG_WEDGE = 6 };
enum { DG_BC_DIRICHLET = 0, DG_BC_RIGID = 1 };
enum { DG_FLUX_UPWIND = 0, DG_FLUX_CENTRAL = 1 };
enum { DG_F32 = 0, DG_F64 = 1 };
enum { DG_MASS_ONTHEFLY = 0, DG_MASS_STORED = 1 };
enum { DG_OPS_FP32 = 0, DG_OPS_TF32X3 = 1, DG_OPS_TF32 = 2, DG_OPS_BF16 = 3 };
enum { DG_SHOTS_OUTER = 0, DG_SHOTS_INNER = 1 };

/* Create a mesh context from vertices and element-to-vertex lists
 * (Section 2.1 "triangulation of the domain"; Section 3.2 vertex maps).
 *   VX    [nverts][3] vertex coordinates (x, y, z).
 *   EToV  [nelem][6]  vertex ids.  Wedge: (b0, b1, b2, t0, t1, t2), bottom
 *         triangle counter-clockwise seen from +z, t_a above b_a with equal x
 *         and y (vertically mapped, Section 3.2) and z(t_a) > z(b_a).  Tet: the
 *         first four entries with positive orientation, the rest ignored.
 *   etype [nelem] DG_WEDGE or DG_TET.
 * Faces are matched by vertex sets; unmatched faces are domain boundary.
 * Errors: DG_ERR_ARG, DG_ERR_MESH (message names the element). */
int dg_mesh_create(dg_ctx** out, int64_t nverts, const double* VX, int64_t nelem,
                   const int64_t* EToV, const uint8_t* etype);

/* Polynomial degree N in 1..5 (Section 3; the paper's experiments run 1..5).  Builds the reference operators
 * (GLL line, Warp & Blend triangle/tet, Section 3.1; Kronecker factors of
 * Section 4.2) and the face-node orientation maps. */
int dg_set_order(dg_ctx* ctx, int N);

/* Per-element c^2 and rho (host arrays of length nelem, copied; both > 0),
 * the piecewise-constant coefficients of the acoustic system (Section 2:
 * kappa = rho c^2 multiplies the pressure equation, 1/rho the velocity
 * equations, and the upwind penalties use the impedance rho c).
 * Default: c^2 = rho = 1. */
int dg_set_material(dg_ctx* ctx, const double* c2, const double* rho);

/* Point source in the pressure equation (not in the paper; the seismic
 * workloads need one): the element containing (x, y, z) (lowest id on ties)
 * gets rhs_p += amp * R(t) * kappa_k (M^k)^{-1} l(x_s), where l(x_s) are its
 * Lagrange basis functions at the point, M^k its exact mass matrix and
 * R(t) = (1 - 2a) exp(-a), a = (pi f0 (t - t0))^2 a Ricker wavelet evaluated
 * at each Runge-Kutta stage time.  At most 4096 (source, shot) pairs; after dg_set_order and
 * before dg_bind.  Errors: DG_ERR_ARG (point outside the mesh, f0 <= 0),
 * DG_ERR_STATE. */
int dg_add_source(dg_ctx* ctx, double x, double y, double z, double f0, double t0, double amp);

/* Shots: S independent states on the same mesh and material (seismic shots,
 * ensembles), advanced together by every dg_step / dg_rhs launch.  Field
 * arrays of dg_set_fields / dg_get_fields / dg_rhs then hold S canonical
 * states one after another ([S][4][total_nodes]); dg_energy returns the sum
 * over shots.  Inside the library the element tables are laid out shot-major
 * (shot s of element i is element s K + i of the type's list), so the stage
 * kernels see one larger mesh; each shot's result equals that of a one-shot
 * context bit for bit.  After dg_set_order, before dg_bind; default 1.
 * Errors: DG_ERR_ARG (shots < 1, shots x elements of a type >= 2^30, a source
 * already placed on a later shot), DG_ERR_STATE. */
int dg_set_shots(dg_ctx* ctx, int64_t shots);

/* As dg_add_source, for one shot only (dg_add_source places the source in
 * every shot).  Errors as dg_add_source, and DG_ERR_ARG for a shot index
 * outside [0, shots). */
int dg_add_shot_source(dg_ctx* ctx, int64_t shot, double x, double y, double z, double f0, double t0, double amp);

/* How the shots of dg_set_shots are laid out in the stage kernels' element
 * blocks (32 consecutive virtual elements, one per lane).  DG_SHOTS_OUTER
 * (default): shot-major, virtual element s K + i, so a block holds 32
 * elements of one shot and keeps the column-order reuse of vertical traces.
 * DG_SHOTS_INNER: virtual element i S + s, so a block holds the shots of one
 * or a few elements; every lane of a warp then reads the same neighbour
 * element, for all shots at once, in one contiguous record (the shot-lane
 * layout), while vertical traces leave the block.  Results are identical
 * bit for bit either way; the field layout of dg_set_fields etc. does not
 * change.  Before dg_bind.  Errors: DG_ERR_ARG (unknown order), DG_ERR_STATE. */
int dg_set_shot_order(dg_ctx* ctx, int order);

/* Shots per block group (no counterpart in the paper; the layout choice of
 * the batched form): shots in groups of G (1 <= G, G divides the shot count;
 * call after dg_set_shots), virtual element (s / G) K G + i G + s % G, so a
 * 32-lane block holds 32 / G elements of G shots each (G >= 32: the G shots
 * of one element span G / 32 blocks).  G = 1 is DG_SHOTS_OUTER, G = shots
 * is DG_SHOTS_INNER.  Results are identical bit for bit for every G; the
 * canonical field layout does not change.  Before dg_bind.  dg_autotune_layout
 * picks G by timing.  Errors: DG_ERR_ARG (G does not divide the shots),
 * DG_ERR_STATE. */
int dg_set_shot_group(dg_ctx* ctx, int64_t group);

/* Boundary condition (DG_BC_*), flux (DG_FLUX_*), arithmetic precision
 * (DG_F32: fields and arithmetic in float; DG_F64: double).
 * Default: rigid walls, upwind, DG_F32. */
int dg_set_options(dg_ctx* ctx, int bc, int flux, int precision);

/* How the stage applies (M^{tri,k})^{-1}, the inverse of the Jacobian-weighted
 * triangle mass matrix M^{tri,k} = sum_a J_a M_a of each wedge (Section 4.2;
 * the wedge mass matrix is M^{tri,k} (x) M^1D):
 *   DG_MASS_ONTHEFLY  the stage factors M^{tri,k} = L L^T from the element's
 *                     vertices every time (nothing per element is stored);
 *   DG_MASS_STORED    the factor is computed once in double precision at
 *                     dg_bind and kept in the mesh blob, (N+1)(N+2)/2 x
 *                     ((N+1)(N+2)/2 + 1) / 2 reals per wedge, which the stage
 *                     reads with the state.  Section 4.3 stores the related
 *                     triangular lift (M^{tri,k})^{-1} M^tri per element.
 * Both give the same operator up to rounding.  Default: DG_MASS_STORED.
 * Before dg_bind.  Errors: DG_ERR_ARG (unknown mode), DG_ERR_STATE. */
int dg_set_mass_mode(dg_ctx* ctx, int mode);

/* How the wedge stage applies the shared reference triangle mass matrix of
 * Section 4.2, M^tri, in the weak-form accumulation (per slice, 4 fields:
 * W_j = M^tri G_j) -- the Nt x Nt matrix common to every element, applied to
 * a whole 32-element block slice by slice (the per-element geometric factors
 * of Lemma 3.1, the per-element mass inverse and the strong D_r, D_s part stay
 * FP32 on the CUDA cores):
 *   DG_OPS_FP32    FP32 fused multiply-adds on the CUDA cores (default);
 *   DG_OPS_TF32X3  tensor cores, each operand split into two TF32 numbers
 *                  (three products, FP32 accumulation): about FP32 accuracy;
 *   DG_OPS_TF32    tensor cores, TF32 operands, FP32 accumulation;
 *   DG_OPS_BF16    tensor cores, BF16 operands, FP32 accumulation.
 * Fields, fluxes, the rest of the stage and the update stay FP32.  Needs the
 * DG_F32 precision (DG_ERR_ARG otherwise); applies to every stage launch of
 * the context (steps, dg_rhs, the adjoint).  Call after dg_set_options and
 * before dg_bind; the tet stage is unaffected.  The paper's kernels use FP32
 * CUDA cores only (Section 6.3); the variants trade operator accuracy for
 * tensor-core throughput. */
int dg_set_op_precision(dg_ctx* ctx, int mode);

/* Node counts: total wedge nodes and total tet nodes; the canonical layout
 * holds wedge_nodes + tet_nodes nodes. */
int dg_num_nodes(const dg_ctx* ctx, int64_t* wedge_nodes, int64_t* tet_nodes);

/* Physical node coordinates, host array xyz[3][total_nodes] (canonical
 * order), computed from the vertex maps.  Needs dg_set_order. */
int dg_node_coords(const dg_ctx* ctx, double* xyz);

/* For every element (input order), face and face node: the canonical index
 * of the coincident node of the neighbouring element, or -1 on the domain
 * boundary.  Face order: wedge (bottom t=-1, top t=+1, quads over triangle
 * edges (0,1), (1,2), (2,0)); tet (vertices (0,1,2), (0,1,3), (1,2,3),
 * (0,2,3)).  Face nodes in element node order.  `out` holds
 * sum_k sum_f nfacenodes(k, f) entries; *count receives that number (pass
 * out = NULL to query it).  Host only. */
int dg_face_neighbors(const dg_ctx* ctx, int64_t* out, int64_t* count);

/* Reference operator by name, row-major doubles, host only (diagnostics):
 * "tri.r", "tri.s" (nodes), "tri.Dr", "tri.Ds", "tri.M", "tri.M0", "tri.M1",
 * "tri.M2" (barycentric-weighted masses int l_i l_j lambda_a), "line.r",
 * "line.D", "line.M", "line.ell0", "line.ellN", "line.Ma", "line.Mb",
 * "tet.r", "tet.s", "tet.t", "tet.Dr", "tet.Ds", "tet.Dt", "tet.M", "tet.LIFT".
 * *rows, *cols receive the shape; pass out = NULL to query it. */
int dg_reference_operator(const dg_ctx* ctx, const char* name, double* out,
                          int64_t* rows, int64_t* cols);

/* Device sizes for the current mesh, order and precision: the mesh blob
 * (connectivity, vertices, material, operator scratch) and one field buffer
 * (packed state of all elements, padded to 32-element blocks). */
int dg_device_bytes(const dg_ctx* ctx, size_t* mesh_bytes, size_t* field_bytes);

/* Bind caller-owned device memory (256-byte aligned) and a cudaStream_t
 * (NULL = legacy default stream), upload the mesh blob and operator tables,
 * and zero the state.  q0/q1 are the two state buffers the Runge-Kutta stages
 * alternate between, res the low-storage residual.  The current device must be
 * the one that owns the buffers; dg_bind records it, and every later call that
 * issues GPU work makes that device current for its duration and restores the
 * caller's current device before returning. */
int dg_bind(dg_ctx* ctx, void* d_mesh, void* d_q0, void* d_q1, void* d_res, void* stream);

/* Set / read the state in the canonical layout ([4][total_nodes] of float or
 * double per precision).  on_device != 0: a device pointer, else host.  Host
 * transfers synchronise the stream; device ones are asynchronous.  A host
 * buffer in pinned, device-mapped memory (cudaHostAlloc / cudaHostRegister, as
 * cudaPointerGetAttributes reports it) is read or written by the layout kernel
 * directly over the CPU-GPU link; pageable memory goes through a bulk copy and
 * the state buffer not in use.  Either way the buffer must hold the whole
 * state.  dg_set_fields resets the simulation time to 0 and the residual to 0. */
int dg_set_fields(dg_ctx* ctx, const void* q, int on_device);
int dg_get_fields(dg_ctx* ctx, void* q, int on_device);

/* Semi-discrete right-hand side dq/dt = rhs(q, t) (Section 2.1) at the
 * current simulation time t (sources), canonical
 * layout, device pointers (d_q may equal d_rhs).  Uses the inactive state
 * buffer and the residual buffer as scratch: call between steps only.  The
 * current state is not modified.  Asynchronous. */
int dg_rhs(dg_ctx* ctx, const void* d_q, void* d_rhs);

/* Advance the bound state by nsteps LSRK45 steps of size dt (dt > 0,
 * nsteps >= 0): the five-stage, two-register low-storage Runge-Kutta scheme
 * of Carpenter and Kennedy (1994), the explicit integrator family of the
 * paper's experiments (Section 6.2; the paper itself runs multirate AB3),
 * res <- a_s res + dt rhs(q, t_n + c_s dt), q <- q + b_s res per stage.
 * One fused kernel per element type per stage, replayed from
 * a CUDA graph.  Asynchronous; launch errors are returned, device-side errors
 * (bounded waits) surface at the next synchronising call. */
int dg_step(dg_ctx* ctx, double dt, int64_t nsteps);

/* Per-element-type timing of the fused stage (diagnostic, not in the paper):
 * launches the wedge stage kernel nrep times, then the tet stage kernel nrep
 * times, on the bound stream, each as a full Runge-Kutta stage of the
 * current state with coefficients a = 1, b = 0 and dt = 0 (the state is not
 * changed; the residual is rewritten with itself plus 0 * rhs), and returns
 * the mean device time per launch in microseconds from CUDA events (0 for a
 * type the mesh does not have).  Synchronous.  Errors: DG_ERR_ARG (nrep < 1,
 * null outputs), DG_ERR_STATE (before dg_set_fields), DG_ERR_CUDA. */
int dg_stage_times(dg_ctx* ctx, int nrep, double* us_wedge, double* us_tet);

/* Launch autotuner (diagnostic plus configuration, not in the paper): times
 * the wedge stage (as dg_stage_times, nrep launches each) in every launch
 * variant this context can run -- 1 or 2 element blocks of 32 wedges per CTA
 * (2 only for N = 3 in DG_F32), and, when the context stores the mass
 * factors, reading them or recomputing them in the stage; with the stored
 * factor, FP32 fields and FP32 operator applies also the stage split over
 * field pairs (two threads per element and slice, for more resident warps)
 * -- and keeps the fastest for later dg_step / dg_rhs calls.  *variant =
 * 2 * blocks_per_cta + (1 if the factor is recomputed) + (8 if split), *us =
 * its mean microseconds per launch.
 * All variants compute the same operator up to rounding.  Synchronous.
 * Errors: DG_ERR_ARG, DG_ERR_STATE (before dg_bind), DG_ERR_CUDA. */
int dg_autotune(dg_ctx* ctx, int nrep, int* variant, double* us);

/* Select a launch variant directly (encoded as dg_autotune reports it), e.g.
 * to reapply a tuned choice without timing.  "Factor recomputed" is ignored
 * when the context does not store the factor (it recomputes anyway).  The
 * step graphs are captured again at the next dg_step.  Errors: DG_ERR_ARG
 * (unknown variant, or one this context cannot run). */
int dg_set_launch_variant(dg_ctx* ctx, int variant);

/* Layout autotuner of the batched form (not in the paper; the paper tunes
 * its kernels' elements per block, Section 6.2): re-lays out the bound
 * context's element tables for every shots-per-group choice G of
 * dg_set_shot_group (1, 2, 4, ... and the shot count, each dividing it),
 * times one stage of each element type (nrep launches, as dg_stage_times)
 * and keeps the G with the shortest total.  *group = that G, *us = its
 * microseconds per stage.  The state buffers and the simulation time are
 * reset to zero: call it after dg_bind and before dg_set_fields.  The
 * operator is the same for every G (bit for bit).  Synchronous.
 * Errors: DG_ERR_ARG, DG_ERR_STATE (before dg_bind), DG_ERR_CUDA. */
int dg_autotune_layout(dg_ctx* ctx, int nrep, int64_t* group, double* us);

/* ---------------------------------------------------------------- receivers
 * Pressure receivers (not in the paper; the inversion workloads need them):
 * p sampled at (x, y, z) by the Lagrange basis of the containing element
 * (lowest id on ties).  After dg_set_order, before dg_bind.  Returns the
 * receiver index (>= 0) or DG_ERR_ARG (outside the mesh, more than 65536),
 * DG_ERR_STATE. */
int dg_add_receiver(dg_ctx* ctx, double x, double y, double z);

/* Pressure of the current state at every receiver: device array
 * d_out[shots][receivers] (reals of the context precision).  Async on the
 * bound stream.  Errors: DG_ERR_ARG, DG_ERR_STATE. */
int dg_sample(dg_ctx* ctx, void* d_out);

/* Copy of the current packed state (dg_device_bytes' field_bytes) to / from a
 * caller device buffer, for checkpoints.  dg_load_state also sets the
 * simulation time to t.  Both are asynchronous on the bound stream.
 * Errors: DG_ERR_ARG, DG_ERR_STATE. */
int dg_save_state(dg_ctx* ctx, void* d_dst);
int dg_load_state(dg_ctx* ctx, const void* d_src, double t);

/* ------------------------------------------------------------------ adjoint
 * Discrete adjoint of dg_step for the misfit J = 1/2 sum_n sum_r
 * (p_r(t_n) - d_r(t_n))^2 and its gradient with respect to the per-element
 * kappa = rho c^2 and rho (not in the paper).  The method's operator A splits
 * into a part that is skew-adjoint in the energy inner product (volume terms
 * and the p-u couplings of the fluxes) and the symmetric penalty, so A^T =
 * W P A P W^{-1} with W the energy mass (Section 4.1) and P = diag(1, -I)
 * (velocity sign flip); in the variable mu = P W^{-1} lambda the adjoint of
 * one LSRK45 step runs the forward stage with the update coefficients
 * reversed, and receiver residuals enter exactly like point sources.  Wedges
 * and tets (the gradient terms of a tet use its affine mass J M^tet and face
 * masses J_f M^tri); every shot shares the receivers.
 *
 * Workspace (dg_adjoint_bytes, caller-owned device memory): fourteen packed
 * fields, then FP64 sums per padded device element: d/dkappa and d/drho of
 * the wedges, of the tets, and five face sums per wedge (the penalty term of
 * a face between two wedges is evaluated once, by the lower-numbered wedge,
 * for both; dg_adjoint_gradient combines the face sums through z = rho c).
 *
 * Use: dg_adjoint_bytes -> allocate -> dg_adjoint_bind (zeroes everything)
 * -> for n = nsteps .. 1: dg_adjoint_inject(residuals of step n);
 * dg_load_state(q_{n-1}, t_{n-1}); dg_adjoint_step(dt) -> dg_adjoint_gradient.
 * dg_adjoint_step recomputes the forward step from the current state and
 * time (which it leaves unchanged), then applies the five adjoint stages and
 * accumulates the gradient terms.  Errors: DG_ERR_ARG, DG_ERR_STATE,
 * DG_ERR_CUDA; dg_adjoint_bind also DG_ERR_ORDER at N = 5 in DG_F64 (the
 * gradient kernel's shared memory exceeds a CTA's there). */
int dg_adjoint_bytes(const dg_ctx* ctx, size_t* bytes);
int dg_adjoint_bind(dg_ctx* ctx, void* d_work);
int dg_adjoint_reset(dg_ctx* ctx);
/* d_resid[shots][receivers] (device, context precision) */
int dg_adjoint_inject(dg_ctx* ctx, const void* d_resid);
int dg_adjoint_step(dg_ctx* ctx, double dt);

/* Stage records: a memory-for-time alternative to the recomputation inside
 * dg_adjoint_step (not in the paper).  A record of one step holds ten packed
 * fields (each dg_device_bytes' field_bytes, in this order): the step's input
 * state q_n, the stage states Q_1..Q_4 and the five stage right-hand sides
 * r_s = A Q_{s-1} + f(t_n + c_s dt).
 *   dg_step_record_bytes  bytes of one record (10 x field_bytes).
 *   dg_step_record        one LSRK45 step of the bound state, like dg_step with
 *                         nsteps = 1 (same result bit for bit), that also writes
 *                         the record of the step to d_rec (device memory,
 *                         caller-owned, 256-byte aligned, overwritten).  Async.
 *   dg_adjoint_step_recorded
 *                         dg_adjoint_step with the forward stages read from a
 *                         record that dg_step_record wrote for that step (same
 *                         result bit for bit); the bound state and time are
 *                         neither used nor changed.  d_rec is not modified.
 * Use: checkpoints every C steps in the forward pass; per segment, from the
 * last: dg_load_state(checkpoint), dg_step_record_chain into C records, then
 * for n = last .. first: dg_adjoint_inject, dg_adjoint_step_recorded(record n).
 * Errors: DG_ERR_ARG (null or misaligned d_rec, dt <= 0), DG_ERR_STATE
 * (unbound context or adjoint), DG_ERR_CUDA. */
int dg_step_record_bytes(const dg_ctx* ctx, size_t* bytes);
int dg_step_record(dg_ctx* ctx, double dt, void* d_rec);
/* dg_step_record over nsteps consecutive steps into the records d_recs[0 ..
 * nsteps - 1] (a host array of device pointers, each record distinct,
 * 256-byte aligned, dg_step_record_bytes bytes).  The last stage of step i
 * writes its result straight into slot 0 of record i + 1, so only the first
 * step copies the bound state; the records and the final state and time equal
 * those of nsteps dg_step_record calls bit for bit.  The bound state is only
 * written by the last step (receivers sampled in between see the first
 * step's input).  nsteps = 0 does nothing.  Errors as dg_step_record. */
int dg_step_record_chain(dg_ctx* ctx, double dt, int64_t nsteps, void* const* d_recs);
int dg_adjoint_step_recorded(dg_ctx* ctx, double dt, const void* d_rec);
/* set the adjoint state: mu_Q and the next stage input x (normally b_5 mu_Q),
 * canonical layout, host or device sources */
int dg_adjoint_set(dg_ctx* ctx, const void* mu_q, const void* x, int on_device);
/* the adjoint state in the variables mu = P W^{-1} lambda, canonical layout
 * ([shots][4][total_nodes]), host or device destination */
int dg_adjoint_get(dg_ctx* ctx, void* dst, int on_device);
/* dJ/dkappa and dJ/drho per element (input order, host arrays of nelem; tets
 * none), summed over shots.  Synchronous. */
int dg_adjoint_gradient(dg_ctx* ctx, double* g_kappa, double* g_rho);

/* Discrete energy E = 1/2 sum_k (p^T M^k p / kappa_k + rho_k sum_c u_c^T M^k u_c)
 * with the scheme's exact mass matrices (Section 4.1), accumulated in double.
 * Synchronises the stream.  Returns DG_ERR_NONFINITE if E is not finite and
 * DG_ERR_TIMEOUT if a device-side wait had run out since the last check. */
int dg_energy(dg_ctx* ctx, double* E);

/* Allocation-free discrete energy of a caller-provided state (no counterpart
 * in the paper; a service for callers that cannot allocate device memory at
 * the point of the call -- code running while a framework forbids
 * allocations, inside host callbacks, or with a locked memory pool).
 *   d_q  device pointer, canonical layout [shots][4][total_nodes] of the
 *        context's precision (as dg_save_state writes it; any state, not only
 *        the bound one); not modified.
 *   E    host pointer; receives the energy (same definition as dg_energy),
 *        summed over the shots.
 * The per-block partial sums live in a file-scope device array of 65536
 * doubles plus one total (512 KB, resident on every GPU that loads the
 * library until exit), so at most 65536 * 128 = 8388608 elements (wedges
 * and tets of all shots) are accepted; more return DG_ERR_ARG.  No
 * cudaMalloc, cudaFree or allocating library routine is called.  The call
 * runs on the device bound by dg_bind (made current for the call, the
 * caller's device restored afterwards).  The first call on a device looks up
 * the array's device address; make that first call before any stream
 * capture.  All calls share the array: calls that overlap on the GPU (other
 * streams, other contexts) race; each call fully rewrites the partials it
 * sums.  Synchronises the bound stream.
 * Errors: DG_ERR_ARG, DG_ERR_STATE (before dg_bind), DG_ERR_CUDA,
 * DG_ERR_NONFINITE, and DG_ERR_TIMEOUT if a device-side wait had run out
 * since the last check (as dg_energy). */
int dg_energy_static(dg_ctx* ctx, const void* d_q, double* E);

/* Synchronise the bound stream and report pending device-side errors. */
int dg_sync(dg_ctx* ctx);

/* Failure-path check of the bounded device-side waits (no counterpart in the
 * paper).  Enqueues on the bound stream one kernel that arms an mbarrier for
 * bytes no copy will deliver and waits on it with the stages' bounded wait
 * (a 64-poll budget instead of the stages' ~1 s), so the wait runs out, the
 * kernel sets the timeout bit of the device error word and returns -- what a
 * stage does when one of its bulk copies never lands.  Nothing faults or
 * hangs and the context stays usable: the next synchronising call (dg_sync,
 * dg_energy, ...) returns DG_ERR_TIMEOUT and clears the word.  Asynchronous.
 * Errors: DG_ERR_STATE (before dg_bind), DG_ERR_CUDA. */
int dg_expire_wait(dg_ctx* ctx);

/* Simulation time of the bound state (sum of dt over completed steps). */
int dg_time(const dg_ctx* ctx, double* t);

/* Stable time step dt = cfl * min_k 1 / (c_k (N+1)^2 max_f(area_f / vol_k)).
 * The paper bounds dt by trace and Markov constants without printing them
 * (Section 6); this is the library's explicit form of that bound. */
int dg_stable_dt(const dg_ctx* ctx, double cfl, double* dt);

/* Measured CUDA-core fused multiply-add throughput of the current device in
 * TFLOP/s (2 flops per FMA), precision DG_F32 or DG_F64 (no counterpart in
 * the paper: the arithmetic roofline that the stage kernels' flop rates are
 * reported against).  Runs a warm-up and one timed launch of independent FMA
 * chains on every SM, on `stream` (a cudaStream_t, NULL = legacy default),
 * timed with CUDA events; synchronous, about 10 ms.  Needs no context.
 * Errors: DG_ERR_ARG (null output, unknown precision), DG_ERR_CUDA. */
int dg_fma_peak(int precision, void* stream, double* tflops);

const char* dg_last_error(const dg_ctx* ctx);
void dg_destroy(dg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DGWEDGE_H */
