/*
 * pbf.h - C ABI of the GPU (sm_103a) library for the matrix-free thermal powder-bed-fusion
 * hot path of Proell, Munch, Kronbichler, Wall, Meier, arXiv 2302.05164.
 *
 * Conventions for every entry point
 *  - Returns a pbf_status. PBF_OK on success; otherwise pbf_last_error() gives a message
 *    (thread-local, valid until the next call on the same thread). No call aborts, traps or
 *    throws across the ABI.
 *  - Field arrays named *_dev are caller-owned DEVICE pointers (e.g. torch tensor data_ptr),
 *    FP64, contiguous, laid out [n_dofs][batch] with the instance index fastest. Input and
 *    output fields must not alias unless stated.
 *  - Host pointers (descriptors, tables, laser powers) are read only during the call.
 *  - pbf_stream is a cudaStream_t (0 = legacy default stream). Work is enqueued on it; a call
 *    synchronises only when it must return values computed on the device (stated below).
 *  - pbf_mesh and pbf_ctx are opaque, library-owned, and freed by their destroy calls.
 *  - After PBF_ECUDA a context refuses further work with PBF_ESTATE.
 */
#ifndef PBF_H
#define PBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PBF_OK = 0,
  PBF_EINVAL = 1,   /* invalid argument or descriptor */
  PBF_ENOMEM = 2,   /* host or device allocation failed */
  PBF_ECUDA = 3,    /* a CUDA runtime call failed */
  PBF_ENOCONV = 4,  /* an iterative solve missed its tolerance */
  PBF_ENAN = 5,     /* reserved for a check of the state for non-finite values (no call returns it) */
  PBF_ETIMEOUT = 6, /* a bounded device wait expired */
  PBF_EFAULT = 7,   /* reserved for device-side index checks (no call returns it) */
  PBF_ESTATE = 8    /* object is poisoned or out of date (mesh changed under a context) */
} pbf_status;

typedef void* pbf_stream; /* cudaStream_t */

const char* pbf_last_error(void);
const char* pbf_version(void);

/* ------------------------------------------------------------------------------------- */
/* Mesh (host). Paper Sec. 4.1: coarse hexahedral mesh of uniform trees, a-priori octree   */
/* refinement, 2:1 balance, Z-curve cell order, inactive cells above the active layer.    */
/* ------------------------------------------------------------------------------------- */

typedef struct pbf_mesh pbf_mesh;

enum { PBF_REGION_BALL = 0, PBF_REGION_BOX = 1 };

/* Refinement region: a leaf is refined to `level` while its box lies closer than `radius`
 * to the region core (the point a for a ball, the box [a, b] for a box). Squared distances
 * are compared in FP64, d2 < radius^2. */
typedef struct {
  int kind;
  int level;
  double a[3];
  double b[3];
  double radius;
} pbf_region;

/* Forest of ntree[0] x ntree[1] x ntree[2] axis-aligned trees of edge tree_h starting at
 * origin (metres). Q_degree Lagrange elements, degree 1 or 2, trees refined at most
 * max_level times (0 <= max_level <= 12). tree_exists (nullable) masks trees of a
 * boundary-fitted voxel mesh, [nz][ny][nx] with x fastest. Cells whose lower z lies at or
 * above active_top_z are inactive (no dofs). dirichlet_faces: bit 0 -x, 1 +x, 2 -y, 3 +y,
 * 4 -z, 5 +z faces of the tree brick carry T = T_dirichlet. Cells whose z-centre lies in
 * [powder_z0, powder_z1) get material 1 (powder), others material 0 (solid). */
typedef struct {
  double origin[3];
  int ntree[3];
  double tree_h[3];
  int degree;
  int max_level;
  const uint8_t* tree_exists;
  double active_top_z;
  uint32_t dirichlet_faces;
  int n_regions;
  const pbf_region* regions;
  double powder_z0, powder_z1;
} pbf_mesh_desc;

typedef struct {
  int64_t n_leaves;      /* all leaves, active or not */
  int64_t n_active;      /* active cells */
  int64_t n_dofs;        /* degrees of freedom (hanging nodes are not dofs) */
  int64_t n_hanging;     /* constrained (hanging) nodes */
  int64_t n_con_entries; /* entries of the flattened constraint rows */
  int64_t n_colours;     /* colours of the greedy cell colouring */
  int64_t n_top_faces;   /* active top faces (laser / objective surface) */
  int64_t nodes_per_cell;
  int64_t generation;    /* incremented by every topology change */
} pbf_mesh_info_t;

/* Host output buffers of pbf_mesh_export, sized from pbf_mesh_info_t; any may be NULL.
 *  leaves      [n_leaves][5]  anchor x, y, z on the lattice of finest cells, level, active
 *  material    [n_leaves]     0 solid, 1 powder
 *  cell_dofs   [n_active][nodes_per_cell] dof id, or -1-r for a node constrained by row r;
 *              local nodes lexicographic with x fastest
 *  con_ptr     [n_hanging+1], con_idx/con_w [n_con_entries]: constraint rows (masters sorted)
 *  hang_coord  [n_hanging][3], dof_coord [n_dofs][3]: node positions in units of
 *              (finest cell edge)/degree
 *  dirichlet   [n_dofs], colour [n_active], top [n_active] */
typedef struct {
  int64_t* leaves;
  uint8_t* material;
  int32_t* cell_dofs;
  int32_t* con_ptr;
  int32_t* con_idx;
  double* con_w;
  int64_t* hang_coord;
  int64_t* dof_coord;
  uint8_t* dirichlet;
  int32_t* colour;
  uint8_t* top;
} pbf_mesh_tables;

/* Builds the canonical mesh: refinement to region targets, full 2:1 balance, Morton order
 * within trees (trees lexicographic), activity, first-touch dof numbering, hanging-node
 * constraints (weights = Lagrange basis of the first coarse cell in cell order, chains
 * substituted, masters merged and sorted), Dirichlet flags, greedy colouring, top faces.
 * Host only. Errors: PBF_EINVAL (bad descriptor), PBF_ENOMEM. */
pbf_status pbf_mesh_create(const pbf_mesh_desc* desc, pbf_mesh** out);
pbf_status pbf_mesh_destroy(pbf_mesh* mesh);
pbf_status pbf_mesh_info(const pbf_mesh* mesh, pbf_mesh_info_t* out);
pbf_status pbf_mesh_export(const pbf_mesh* mesh, const pbf_mesh_tables* out);

/* Patch tables of the fused explicit step (the one-pass step of Sec. 4.2: a block loads its
 * cells' nodal values once, evaluates f and updates the state), built on the host as
 * pbf_ctx_create builds them for an FP32-operator context of batch 1. A patch is up to
 * cells_per_patch active cells consecutive in the Morton order of their anchors over the whole
 * brick, with at most 640 hanging-table entries unless it holds one cell; patches are numbered
 * by decreasing work (slots + 2 x hanging entries); each dof is owned by the first patch in
 * that numbering that lists it. Shared-memory positions are s(j) = j ^ ((j >> 5) & 31) of
 * slot index j.
 *  ptr    [n_patches]                          first entry of patch q in slot
 *  cnt    [n_patches][4]                       dof slots, all slots, hanging table begin, end
 *  slot   [n_slots]  per patch, ascending keys: dof d (bit 31 set where q owns d) for the
 *                    dofs of its cells and the masters of its hanging nodes, then one entry
 *                    (start << 5) | count per hanging row in ascending row order (start
 *                    relative to the patch's hanging table); zero-padded to a multiple of 4
 *  cell   [n_patches][cells_per_patch]          active cell of each lane, -1 past the end
 *  loc    [n_patches][nodes_per_cell][cells_per_patch]  s(slot index) of each lane's node
 *  hloc   [n_hent], hw [n_hent]                s(slot index) of each master, its weight
 * Sizes are outputs. With every array NULL the call only reports the sizes; otherwise the
 * sizes passed in must equal the mesh's (from a sizes-only call on the same mesh generation)
 * and each non-NULL array is filled. n_patches = 0 when the fused form does not apply (a
 * constraint row of more than 31 entries, or a patch of more than 65,536 slots). Host only.
 * Errors: PBF_EINVAL (null mesh or tables, sizes that differ), PBF_ENOMEM. */
typedef struct {
  int64_t n_patches, n_slots, n_hent;
  int32_t cells_per_patch, max_slots, max_hent;
  int32_t* ptr;
  int32_t* cnt;
  int32_t* slot;
  int32_t* cell;
  uint16_t* loc;
  uint16_t* hloc;
  float* hw;
} pbf_step_tables;
pbf_status pbf_mesh_step_tables(const pbf_mesh* mesh, pbf_step_tables* tables);

/* Layer activation (Sec. 4.1; initial condition of Sec. 2 for later-activated parts): raises
 * the activation height to z_new_top; newly active cells take `material`. Host topology
 * change only; it records a pending transfer (old dofs -> new dofs) that pbf_mesh_transfer
 * applies: nodes shared with the old active domain keep their value, new nodes get T_init.
 * Contexts created before the call return PBF_ESTATE until recreated. */
pbf_status pbf_mesh_activate_layer(pbf_mesh* mesh, double z_new_top, int material, double T_init);

/* Re-adaptation to a new region set (a-priori refinement around the scan, Sec. 4.1): the
 * mesh becomes the canonical mesh for the new regions (same trees and activation);
 * materials follow the old leaf holding each new leaf's anchor. Records a pending transfer
 * (field interpolation on the old mesh, i.e. prolongation / injection). */
pbf_status pbf_mesh_adapt(pbf_mesh* mesh, int n_regions, const pbf_region* regions);

/* Applies the pending transfer on the device: T_new_dev[new n_dofs][batch] from
 * T_old_dev[old n_dofs][batch]. Errors: PBF_ESTATE when no transfer is pending. */
pbf_status pbf_mesh_transfer(pbf_mesh* mesh, const double* T_old_dev, double* T_new_dev, int batch,
                             pbf_stream stream);

/* The pending transfer's map (the state moved onto a changed mesh, Sec. 4.1) on the host, for
 * inspection; pbf_mesh_transfer applies it. New dof i takes T_new[i] = sum over e in
 * [ptr[i], ptr[i+1]) of w[e] T_old[idx[e]], or `fill` when its row is empty (a dof outside
 * the old active domain).
 *  ptr [n_new + 1], idx [n_entries] (old dofs, ascending within a row), w [n_entries]
 * Sizes and fill are outputs. With every array NULL only they are reported; otherwise the
 * sizes passed in must equal the map's and each non-NULL array is filled. Host only. Errors:
 * PBF_EINVAL (null mesh or map, sizes that differ), PBF_ESTATE (no pending transfer). */
typedef struct {
  int64_t n_old, n_new, n_entries;
  double fill;
  int32_t* ptr;
  int32_t* idx;
  double* w;
} pbf_transfer_map;
pbf_status pbf_mesh_transfer_map(const pbf_mesh* mesh, pbf_transfer_map* map);

/* ------------------------------------------------------------------------------------- */
/* Context: device copy of the mesh tables, material and work space for `batch` instances */
/* ------------------------------------------------------------------------------------- */

typedef struct pbf_ctx pbf_ctx;

typedef enum { PBF_F64 = 0, PBF_F32OP = 1 } pbf_precision;

enum { PBF_LUMP_QUADRATURE = 0, PBF_LUMP_NODAL = 1 };

/* Material (Sec. 2 heat equation; configuration readings for k(T) and latent heat):
 * k(T) = k0 + (k1-k0) clamp((T-Tk0)/(Tk1-Tk0), 0, 1) (constant k0 when Tk1 <= Tk0),
 * multiplied by powder_k_scale on material-1 cells and by the per-instance scale s;
 * c_app(T) = c + latent/(sigma sqrt(2 pi)) exp(-(T-Tm)^2/(2 sigma^2)) (off when sigma <= 0).
 * T_ref: offset subtracted from T before the FP32 operator rounds it.
 * lumping (only matters with latent heat): PBF_LUMP_QUADRATURE, the row sum of the consistent
 * capacity C~_ii = sum_j C_ij (Sec. 3.2) with c_app at the quadrature points; PBF_LUMP_NODAL,
 * C~_ii = rho c_app(T_i) sum_j M_ij with the constant-coefficient mass M. For Q2 elements the
 * quadrature form can turn negative where c_app(T) peaks sharply inside a cell (the Q2 basis
 * is negative in parts of a cell); the nodal form stays positive. */
typedef struct {
  double rho, c;
  double k0, k1, Tk0, Tk1;
  double latent, Tm, sigma;
  double powder_k_scale;
  double T_dirichlet;
  double T_ref;
  int lumping;
} pbf_material;

/* Moving laser (Sec. 2 heat source). The spot moves linearly over segment k,
 * seg[k] = {x0, y0, x1, y1, t0, t1}, during t0 <= t < t1 with power power[instance][k]; no
 * segment active: no source. volumetric = 0: surface flux 2 eta P/(pi r^2) exp(-2 d^2/r^2)
 * on active top faces; volumetric = 1: the cylinder source 2 eta P/(pi r^2 h_powder)
 * exp(-2 d^2/r^2) for active_top_z - h_powder < z < active_top_z (Eq. heat_soruce_cylindrical,
 * W_eff = eta P). At most 64 segments. */
typedef struct {
  int n_seg;
  const double* seg;   /* host [n_seg][6] */
  const double* power; /* host [batch][n_seg] */
  double eta, radius;
  int volumetric;
  double h_powder;
} pbf_laser;

/* Uploads the mesh tables and the material; allocates work space for `batch` instances
 * (1 <= batch <= 1024). precision PBF_F64: operator in FP64; PBF_F32OP: operator arithmetic
 * and cell accumulation in FP32; within an explicit-step call the state T - T_ref is kept as
 * an unevaluated pair of FP32 numbers (about 48 bits) and updated without rounding error,
 * between calls it is the caller's FP64 array; CG vectors, dot products and adjoint
 * accumulation stay in FP64. */
pbf_status pbf_ctx_create(const pbf_mesh* mesh, const pbf_material* mat, pbf_precision prec, int batch,
                          pbf_ctx** out);
pbf_status pbf_ctx_destroy(pbf_ctx* ctx);

/* Per-instance conductivity scale s (host [batch]); default 1. */
pbf_status pbf_ctx_set_k_scale(pbf_ctx* ctx, const double* s_host);

/* Evaluates, at state T_dev and time t, the three parts of the semi-discrete right-hand
 * side (Eq. semi-discrete) and the row-sum lumped capacity (Sec. 3.2):
 *   fdiff_dev = -P^T sum_e int k(T_h) grad N . grad T_h   (Eq. diffusive_term_evaluation)
 *   fvol_dev  = P^T sum_e laser source against N (plus, with a surface loss set by
 *               pbf_ctx_set_surface_loss, the term -int_top N (q_rad + q_evap)(T_h) dA)
 *   C_dev     = P^T sum_e int rho c_app(T_h) N
 * Any output may be NULL. Outputs [n_dofs][batch] FP64. laser may be NULL (no source). */
pbf_status pbf_eval_residual(pbf_ctx* ctx, const double* T_dev, const pbf_laser* laser, double t,
                             double* fdiff_dev, double* fvol_dev, double* C_dev, pbf_stream stream);

/* nsteps forward-Euler steps T <- T + dt C~(T)^-1 f(T) on free dofs (Eq. forward_euler),
 * with the laser at t0 + n dt for step n; Dirichlet dofs hold T_dirichlet. In place on
 * T_dev [n_dofs][batch]. */
pbf_status pbf_explicit_step(pbf_ctx* ctx, double* T_dev, const pbf_laser* laser, double t0, double dt, int nsteps,
                             pbf_stream stream);

/* Largest eigenvalue of C~^-1 K_diff on free dofs by power iteration (Eq. explicit_time_step,
 * k frozen at k0 scaled by s of instance 0, plain c): x0_dev [n_dofs] start vector (NULL: a
 * built-in SplitMix64 vector), at most max_iter iterations, stop when successive Rayleigh
 * quotients differ by <= rtol relative. Writes lambda and dt_crit = 2/lambda. Synchronises. */
pbf_status pbf_estimate_dt(pbf_ctx* ctx, const double* x0_dev, int max_iter, double rtol, double* lambda_out,
                           double* dt_crit_out, int* iters_out, pbf_stream stream);

/* Allocation-free form of pbf_estimate_dt (the paper has no counterpart: it exists for
 * callers that cannot allocate device memory during the call, e.g. applications that
 * reserve nearly all device memory for their own pool allocator, or latency-bound loops
 * where cudaMalloc / cudaFree would stall the device). Same power iteration, with the
 * vectors passed in: x_dev [n_dofs] holds the start vector on entry and the last iterate on
 * return; y_dev [n_dofs] is overwritten (last K x). The partial sums of its reductions live
 * in a fixed static device array of 32,768 + 64 doubles (262,656 bytes) that every GPU
 * loading the library keeps until the process exits; meshes with more than 134,217,728 dofs
 * are rejected with PBF_EINVAL, and so are x_dev and y_dev when their ranges overlap. The
 * one-time set-up on a device happens in pbf_ctx_create (which may allocate): it looks up the
 * array's device address and runs the iteration once on temporary vectors, so that every
 * kernel of this call is loaded (the CUDA runtime loads kernels lazily on first launch, and
 * loading allocates device memory). Create the context before any stream capture. All calls
 * share the array and find the last call's contents in it; calls whose work overlaps on the
 * GPU race on it. No cudaMalloc, cudaFree or allocating library routine is called.
 * Synchronises. */
pbf_status pbf_estimate_dt_noalloc(pbf_ctx* ctx, double* x_dev, double* y_dev, int max_iter, double rtol,
                                   double* lambda_out, double* dt_crit_out, int* iters_out, pbf_stream stream);

/* Eigenvalue bounds of D^-1 A, A = C/dt + K (consistent capacity, linear material, Dirichlet
 * rows identity), D = diag(A), from the Lanczos tridiagonal of n_iter Jacobi-PCG steps on
 * A x = b, x0 = 0 (b_dev [n_dofs]; NULL: built-in SplitMix64 vector). out = {lmin, lmax}.
 * Synchronises. */
pbf_status pbf_cheb_bounds(pbf_ctx* ctx, double dt, const double* b_dev, int n_iter, double* out,
                           pbf_stream stream);

/* nsteps backward-Euler steps (Eq. backward_euler_nonlinear, no laser; the
 * capacity is the consistent one with the plain c, the latent heat's apparent capacity is
 * not part of it). Constant k: (C/dt + K) dT = f(T_n), T_{n+1} = T_n + dT, by CG with a
 * Chebyshev(cheb_degree)-Jacobi preconditioner on bounds {lmin, lmax} (NULL: pbf_cheb_bounds
 * with 30 steps, lmax x 1.1), FP64 dot products, stop at ||r||_2 <= rtol ||r_0||_2 on the CG
 * recurrence; iters_out (host, nullable) [nsteps] CG iterations. A T-dependent k, the phase
 * model or a surface loss: Newton's method, pbf_implicit_newton with newton_rtol = rtol, 50
 * corrections, lin_rtol = 1e-4 and lin_max = max_it, iters_out the BiCGStab iterations. Instance 0 only (batch
 * must be 1). Synchronises once per CG iteration. PBF_ENOCONV when a step missed rtol (T holds
 * the last iterate). */
pbf_status pbf_implicit_solve(pbf_ctx* ctx, double* T_dev, double dt, int nsteps, double rtol, int max_it,
                              int cheb_degree, const double* cheb_bounds, int* iters_out, pbf_stream stream);

/* Nonlinear backward Euler (Sec. 3.2, Eq. backward_euler_nonlinear, no laser) by
 * Newton-Raphson (Eqs. Newton_1, Newton_2): residual
 *   r(T) = C (T - T_n)/dt - f_diff(T) - f_RE(T_n)  on free dofs (T = T_D on Dirichlet dofs),
 * C the consistent capacity with the plain c, f_RE the context's surface loss (if set) at the
 * previous state; Jacobian J(T) w = C w/dt + int k(T) grad N . grad w + int k'(T) w grad N .
 * grad T (the L_e term of Eq. matrix_free_eval), k from the material ramp or, with the phase
 * model, k(T, r_c) with r_c = max(stored, g(T)) and k' along the branch of the max; after
 * each step the phase model stores r_c = max(r_c, g(T_{n+1})). From
 * T^0 = T_n each correction solves J(T^i) dT = -r(T^i) by BiCGStab to lin_rtol (relative to
 * ||r(T^i)||_2, at most lin_max iterations) with the Chebyshev(cheb_degree)-Jacobi
 * preconditioner of the linear operator C/dt + K(k0) on bounds {lmin, lmax} (NULL: estimated
 * as in pbf_implicit_solve), until ||r(T^i)||_2 <= newton_rtol ||r(T^0)||_2, or a correction
 * with ||dT||_2 <= 1e-13 ||T||_2 (the rounding level of T, below which the residual cannot be
 * reduced), or newton_max corrections. The residual is evaluated in FP64 and the Jacobian in the context's operator
 * precision: for an FP32-operator context this is FP64 iterative refinement of FP32-operator
 * solves, and it reaches the FP64 solution (also for a constant k). newton_iters_out and
 * lin_iters_out (host, nullable) [nsteps]: corrections and BiCGStab iterations per step;
 * rel_residual_out (nullable): the largest ||r||_2 / ||r_0||_2 reached over the steps.
 * Instance 0 only (batch 1). Synchronises twice per BiCGStab iteration. PBF_ENOCONV when a step
 * missed newton_rtol (T holds the last iterate). */
pbf_status pbf_implicit_newton(pbf_ctx* ctx, double* T_dev, double dt, int nsteps, double newton_rtol,
                               int newton_max, double lin_rtol, int lin_max, int cheb_degree,
                               const double* cheb_bounds, int* newton_iters_out, int* lin_iters_out,
                               double* rel_residual_out, pbf_stream stream);

/* Adjoint sweep of the explicit stepper for every instance (objective reading of the
 * configuration: J = (1/N) sum_{n=1..N} (M_n - T_target)^2, M_n = (sum_i w_i T_{n,i}^p /
 * sum_i w_i)^(1/p) over top-surface dofs, w_i = int_{top} N_i): forward nsteps from T0_dev
 * storing n_checkpoints states on a binomial (revolve) schedule, then the reverse recursion
 * lambda_n = lambda_{n+1} + dt (du/dT)^T lambda_{n+1} + dJ/dT_n, u = C~^-1 f. Gradients with
 * respect to the laser power of each segment and to the conductivity scale s. With a surface
 * loss, f includes it (at each step's state) and du/dT its face term -int N_i q'(T_h) N_j dA;
 * the power gradients take the laser's part of f_vol alone. With the phase model the history
 * r_n = max(r_{n-1}, g(T_n)) is a state of the stepper: every snapshot stores it with T, the
 * reverse pass carries its adjoint (through the max where the stored value wins, into lambda
 * through g'(T) where g wins), and the context's history is as on entry when the call returns
 * (one more history-sized buffer per snapshot, and one for the adjoint).
 * J_out host [batch]; grad_out host [batch][n_seg + 1] (dJ/dP_0..dJ/dP_{n_seg-1}, dJ/ds);
 * forward_steps_out (nullable): forward steps taken, including recomputation. Synchronises. */
pbf_status pbf_adjoint_sweep(pbf_ctx* ctx, const double* T0_dev, const pbf_laser* laser, double t0, double dt,
                             int nsteps, int n_checkpoints, double T_target, double p_exp, double* J_out,
                             double* grad_out, long long* forward_steps_out, pbf_stream stream);

/* Forward-step count of the binomial checkpoint schedule (Griewank and Walther, revolve)
 * for nsteps steps and n_snaps stored states; host only. */
pbf_status pbf_revolve_cost(int nsteps, int n_snaps, long long* forward_steps_out);

/* Explicit-step shapes of an FP32-operator context. 0-3: the per-cell residual kernel
 * (one thread per cell and instance, gather / atomic scatter; 0: 128 threads, 1: 128 threads
 * with 5 resident blocks per SM, 2: 6 blocks, 3: 64 threads with 10 blocks) followed by the
 * hanging-node and update kernels; 4: the fused step, one launch per step for one instance
 * with the constant or nodal capacity (patches of 64 cells, consecutive in the global Morton
 * order, staged in shared memory, the previous step's update applied while staging, the
 * state kept as an FP32 pair); 5: shape 4 launched with programmatic dependent launch; 6: the
 * fused step for all steps of a call in one persistent cooperative launch, with a grid
 * barrier between steps whose waits end after one second with PBF_ETIMEOUT (state undefined,
 * context still usable; when the resident blocks cover every patch, each keeps its patch
 * tables in shared memory for the whole call); shape 6 synchronises the stream; 7, 8, 9: the
 * fused step of shape 5 in its lean form (patch tables read through L1, only the staged values
 * and their sums in shared memory, the conductivity recomputed in each gradient direction),
 * compiled for 14, 12 and 10 resident blocks per SM. For a batch (batch > 1, constant or
 * nodal capacity, no surface loss or phase model, surface laser) shapes 4-9 run the batched
 * fused step: one launch per step for all instances, threads (cell, instance) with the
 * instance fastest, the previous step's update applied in the gather, the spot computed on
 * the device, a call's launches replayed as one CUDA graph when (nsteps, dt, T_dev) repeat.
 * The phase model and the surface loss run in the fused step of shapes 4 and 5 (shapes 6-9
 * then act as shape 5). Where no fused form applies (quadrature-point capacity; a batch with
 * an option or a volumetric source) shapes 4-9 run the per-cell form; with a volumetric
 * source shape 6 runs shape 5; residual-only evaluations of shapes 4-9 use shape 1.
 *
 * pbf_ctx_autotune times `reps` explicit steps of every applicable shape with dt = 0 on a
 * scratch copy of T_dev (not modified), with the laser of the last call, keeps the fastest in
 * the context and returns its index; us_per_step_out (nullable, 10 entries) receives each
 * shape's microseconds per step, -1 where it does not apply. FP64 contexts keep shape 0.
 * Allocates one scratch vector; synchronises. */
pbf_status pbf_ctx_autotune(pbf_ctx* ctx, const double* T_dev, int reps, int* variant_out, float* us_per_step_out,
                            pbf_stream stream);

/* History of the phase model across mesh changes (Sec. 4.1 coarsening rule, with the
 * consolidated fraction r_c of Eq. consolidated_fraction as the material history).
 *
 * pbf_ctx_history_cell_min: the smallest r_c of each active cell over its quadrature points
 * and instances, into rc_min_host [n_cells] (host); synchronises.
 * pbf_ctx_get_history / pbf_ctx_set_history: r_c as an FP64 device array
 * [(p+1)^3][n_cells][batch] (quadrature point index x fastest), read from or written to the
 * context (FP32-operator contexts round it).
 * pbf_mesh_adapt_gated: pbf_mesh_adapt with the coarsening restriction of Sec. 4.1: the eight
 * octants of a parent merge only if r_c lies at or above r_coarsen on all of them (the paper
 * uses 0.9). cell_rc_min (host, [n_active] of the mesh before the change, from
 * pbf_ctx_history_cell_min): every cell below r_coarsen keeps its parent's box refined to its
 * own level (a box region added to `regions`), so its family cannot merge.
 * pbf_ctx_transfer_history: after a mesh change (pbf_mesh_adapt, pbf_mesh_adapt_gated or
 * pbf_mesh_activate_layer), moves r_c from `from` (a context of the mesh before the change,
 * which may no longer be used otherwise) to `to` (a context of the changed mesh with the
 * phase model set; same batch, precision and degree): each quadrature point of a new cell
 * takes the value of the nearest (per axis) quadrature point of the first old active cell, in
 * cell order, whose closure holds it (a copy on refinement, injection on coarsening); points
 * outside the old active domain start as new cells do (0 in powder, 1 elsewhere). PBF_ESTATE
 * when `from` is not of the mesh before its last change. Synchronises.
 * pbf_mesh_history_map: the map pbf_ctx_transfer_history applies, on the host, for inspection:
 * map [n_active][(p+1)^3] (nullable; quadrature point index x fastest) receives, for each
 * quadrature point of the mesh, the old cell x (p+1)^3 + old point whose r_c it takes, or -1
 * (it starts at 0: powder) or -2 (it starts at 1); n_old_cells_out (nullable) the old mesh's
 * active cells. Host only. PBF_EINVAL for a null mesh, PBF_ESTATE when the mesh has not
 * changed since it was created. */
pbf_status pbf_mesh_history_map(const pbf_mesh* mesh, int64_t* n_old_cells_out, int32_t* map);
pbf_status pbf_ctx_history_cell_min(pbf_ctx* ctx, double* rc_min_host, pbf_stream stream);
pbf_status pbf_ctx_get_history(pbf_ctx* ctx, double* rc_dev, pbf_stream stream);
pbf_status pbf_ctx_set_history(pbf_ctx* ctx, const double* rc_dev, pbf_stream stream);
pbf_status pbf_mesh_adapt_gated(pbf_mesh* mesh, int n_regions, const pbf_region* regions, const double* cell_rc_min,
                                double r_coarsen);
pbf_status pbf_ctx_transfer_history(pbf_ctx* from, pbf_ctx* to, pbf_stream stream);

/* Selects an explicit-step shape directly (0..9, see pbf_ctx_autotune). */
pbf_status pbf_ctx_set_kernel_shape(pbf_ctx* ctx, int shape);

/* Radiation and evaporation on the free top surface (Sec. 2, Eqs. bc_rad_evap, bc_radiation,
 * bc_evaporation): on the active top faces the outward heat flux
 *   q_rad  = emissivity sigma_S (T^4 - T_amb^4)   (sigma_S = 5.670374419e-8 W m^-2 K^-4),
 *   q_evap = 0.82 C_P exp(-C_T (1/[T] - 1/T_v)) sqrt(C_M/[T]) (h_v + c_h ([T] - T_h0)) when
 *            [T] > T_v, with [T] = min(T, T_max),
 * enters the right-hand side as the boundary term -int_top N_i (q_rad + q_evap)(T_h) dA of the
 * weak form, (p+1)^2 Gauss points per face, evaluated at the state of each step (explicit, as
 * in the paper). emissivity = 0 or C_P = 0 switch a part off. */
typedef struct {
  double emissivity, T_amb;
  double C_P, C_T, C_M, T_v, h_v, c_h, T_h0, T_max;
} pbf_surface_loss;

/* Sets (q != NULL) or clears (NULL) the surface loss of a context for its later residual
 * evaluations (added to fvol_dev) and explicit steps. With a surface loss the explicit steps of
 * one instance run it inside the fused step kernel (shapes 4, 5; shapes 6-9 act as shape 5),
 * batches run the per-cell form with a face kernel; the implicit solves evaluate it at the
 * previous state (Newton's method); pbf_adjoint_sweep includes its linearisation. Bad
 * parameters: PBF_EINVAL. Host only. */
pbf_status pbf_ctx_set_surface_loss(pbf_ctx* ctx, const pbf_surface_loss* q);

/* Phase-dependent conductivity with history (Sec. 2, Eqs. liquid_fraction,
 * consolidated_fraction, phase_fractions, material_parameter_interp): liquid fraction
 * g(T) = clamp((T - T_s)/(T_l - T_s), 0, 1); consolidated fraction r_c per quadrature point and
 * instance, starting at 0 in powder cells (material 1) and 1 elsewhere; k(T, r_c) =
 * (1 - r_c) k_p + g k_m + (r_c - g) k_s, times the instance's conductivity scale (the material's
 * k(T) and powder scale are not used). Each explicit step uses and stores
 * r_c = max(stored r_c, g(T_n)) at its state; residual evaluations use that maximum without
 * storing it. */
typedef struct {
  double T_s, T_l, k_p, k_m, k_s;
} pbf_phase;

/* Sets (ph != NULL; the history restarts from the cell materials) or clears (NULL) the phase
 * model of a context. With it the explicit steps of one instance read and store r_c inside the
 * fused step kernel (shapes 4, 5; shapes 6-9 act as shape 5), batches run the per-cell form;
 * the implicit solves use it (Newton's method, storing r_c after each step), and
 * pbf_adjoint_sweep differentiates it with its history. PBF_EINVAL for bad parameters or the
 * quadrature-point capacity. Allocates the history once
 * ((p+1)^3 n_cells batch values); synchronises. */
pbf_status pbf_ctx_set_phase(pbf_ctx* ctx, const pbf_phase* ph);

/* Test hook for the time-out path of shape 6 (no counterpart in the paper): while
 * extra_blocks > 0 the persistent form's grid barrier waits for that many blocks more than
 * were launched, so its first wait runs out (after one second) and the call returns
 * PBF_ETIMEOUT. 0 restores normal operation. */
pbf_status pbf_ctx_set_barrier_test(pbf_ctx* ctx, int extra_blocks);

/* Kernel timing of the dominant (cell operator) kernel: when enabled, CUDA events bracket
 * every cell-operator launch on its stream (the fused step kernel under shapes 4/5);
 * pbf_ctx_kernel_time returns the summed elapsed milliseconds and the launch count since the
 * last reset (synchronises). */
pbf_status pbf_ctx_set_timing(pbf_ctx* ctx, int enable);
pbf_status pbf_ctx_kernel_time(pbf_ctx* ctx, double* ms_out, long long* launches_out);

/* The exact conversions of the FP32-operator form, exposed for testing: IEEE-754 binary64 to
 * binary32 rounding to nearest (ties to even; magnitudes below 2^-126 flush to signed zero;
 * inputs finite with magnitude < 2^128), and the exact binary32 to binary64 widening
 * (subnormals flush to signed zero). Device arrays of n elements; enqueued on stream. */
pbf_status pbf_round_to_f32(const double* x_dev, float* y_dev, int64_t n, pbf_stream stream);
pbf_status pbf_widen_to_f64(const float* x_dev, double* y_dev, int64_t n, pbf_stream stream);

/* Counts of kernels launched by this context since creation (all kinds). */
pbf_status pbf_ctx_launch_count(pbf_ctx* ctx, long long* launches_out);

#ifdef __cplusplus
}
#endif

#endif /* PBF_H */
