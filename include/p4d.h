/*
 * p4d.h -- C ABI of the GB300 (sm_103a) block-preconditioned Newton-Krylov
 * hot path of the pseudo-4D Doyle-Fuller-Newman (P4D DFN) battery model
 * (Roy et al., "Scalable Preconditioners for the Pseudo-4D DFN Lithium-ion
 * Battery Model", arXiv 2602.07225).
 *
 * Problem (paper sections 2-4): the backward-Euler step of the coupled
 * electrode-level Q1 finite-element equations for phi_s, phi_e, c_e
 * (eqs. phis-weak, phie-weak, ce-weak) and the per-particle radial finite
 * differences for c_s (eqs. L1, L2, L0, LR, FD), linked by Butler-Volmer
 * kinetics, is solved by Newton's method; every Newton linear system
 * J(u) delta = -R(u) (section 4, eq. blocks) is solved by FGMRES,
 * right-preconditioned by the block preconditioner of section 4
 * (eqs. PJ / PGS): the particle blocks are inverted exactly per electrode
 * node and eliminated onto the electrode fields by a Schur complement; the
 * electrode-level blocks get one geometric multigrid V-cycle each.
 *
 * Geometry: a structured tensor-product hex mesh of nx*ny*nz elements.
 * Node (i,j,k), 0<=i<=nx, ..., has index i + (nx+1)*(j + (ny+1)*k); element
 * (i,j,k) has index i + nx*(j + ny*k).  The anode sits on the z = 0 side
 * (grounded face Gamma_n, Dirichlet phi_s = 0 on the faces flagged in
 * gamma_n), the cathode on the z = Lz side (applied current on the faces
 * flagged in gamma_p).
 *
 * Unknown vector ("full layout", FP64, length ndof = 3*nnode + nelec*nc):
 *   [ phi_s(nnode) | phi_e(nnode) | c_e(nnode) | c_s(nelec, nc) ]
 * c_s is stored node-major: particle of electrode node e (0 <= e < nelec,
 * electrode nodes numbered in increasing node index), radial node i
 * (0 = centre, nc-1 = surface) at 3*nnode + e*nc + i.  phi_s carries an
 * identity row at every node that is not an electrode node or that lies on
 * Gamma_n; those values are read as 0 by every other row.
 *
 * Conventions
 *  - Memory: pointers marked [host] are host memory, [device] are device
 *    memory of the current CUDA device.  The caller owns every pointer it
 *    passes; the library only reads/writes them during the call (or, for
 *    asynchronous calls, until the handle's stream reaches that point).
 *    The library owns its workspace, allocated in p4d_setup and freed in
 *    p4d_destroy (a batch's, in p4d_batch_create and p4d_batch_destroy); no
 *    other call allocates device memory.
 *  - Streams: work is issued on the stream given to p4d_setup (NULL = the
 *    legacy default stream).  p4d_fgmres_solve / p4d_adjoint_solve
 *    synchronize that stream before returning; the other calls are
 *    asynchronous unless stated.
 *  - Errors: every call returns a p4d_status; no device traps.  On
 *    P4D_ERR_CUDA the handle should be destroyed.
 *  - Threads: a handle is used by one host thread at a time; distinct
 *    handles are independent.
 *  - Devices: a handle lives on the device current at p4d_setup; a call that
 *    launches work with another device current returns INVALID_ARG.
 */
#ifndef P4D_H
#define P4D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct p4d_ctx* p4d_handle;

typedef enum {
  P4D_OK = 0,
  P4D_ERR_INVALID_ARG = 1,   /* bad sizes, null pointers, unsupported option */
  P4D_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  P4D_ERR_OOM = 3,           /* device allocation failed (p4d_setup only) */
  P4D_ERR_NOT_CONVERGED = 4, /* Krylov or Newton hit maxit; output = best iterate */
  P4D_ERR_BREAKDOWN = 5,     /* Krylov breakdown before convergence */
  P4D_ERR_NONFINITE = 6,     /* NaN/Inf met in a residual or Krylov scalar */
  P4D_ERR_DOMAIN = 7,        /* c_surf outside (0, c_max) or c_e <= 0 */
  P4D_ERR_TIMEOUT = 8        /* a bounded device-side wait expired */
} p4d_status;

/* Mesh and material layout (all [host]; copied during p4d_setup). */
typedef struct {
  int32_t nx, ny, nz;              /* elements per axis, each >= 1 */
  const double* hx;                /* [nx] element widths along x (m) */
  const double* hy;                /* [ny] */
  const double* hz;                /* [nz] */
  const uint8_t* region;           /* [nelem] 0 anode, 1 separator, 2 cathode, 3 electrolyte-only */
  const double* eps;               /* [nelem] porosity eps (electrolyte volume fraction) */
  const double* eps_s;             /* [nelem] active-material volume fraction (0 off-electrode) */
  const double* Rs;                /* [nnode] particle radius (m), read at electrode nodes */
  const double* Ds;                /* [nnode] solid diffusivity (m^2/s), read at electrode nodes */
  const uint8_t* gamma_p;          /* [nx*ny] 1 = face (i,j) of the z = Lz boundary carries i_app */
  const uint8_t* gamma_n;          /* [nx*ny] 1 = face (i,j) of the z = 0 boundary is grounded */
  const double* rgrid;             /* [nc] radial nodes / R_s, rgrid[0] = 0, rgrid[nc-1] = 1, increasing */
  int32_t nc;                      /* radial nodes per particle, 3 <= nc <= 32 */
  const double* sigma_e;           /* optional [nelem] bulk solid conductivity per element (S/m);
                                      NULL: sigma_n / sigma_p by region.  sigma_eff = eps_s^b sigma */
  const double* Ds_e;              /* optional [nelem] solid diffusivity per element; when given, the
                                      particle of an electrode node uses the volume-weighted mean over
                                      its electrode elements and Ds is ignored */
  double shell_sigma_t_p;          /* current-collector foil on the z = Lz face as a thin shell: surface
                                      conductance sigma_foil * thickness (S), 0 = none.  Adds the 2D Q1
                                      stiffness of the face to the phi_s rows between active nodes (a
                                      stand-in for the collector layers of the paper's jelly roll, section 5) */
  double shell_sigma_t_n;          /* the same on the z = 0 face (anode foil) */
} p4d_mesh;

/* Physics and solver options. */
typedef struct {
  /* constants (paper Appendix "Model Parameters") */
  double F, R, T, tplus, brug, De, kappa;
  double sigma_n, sigma_p, k_n, k_p, cmax_n, cmax_p, alpha;
  double ocp_n[2], ocp_p[2];       /* linear OCP U(theta) = c0 + c1*theta per electrode */
  double dt;                       /* backward-Euler step (s) */
  double i_app;                    /* applied current density on Gamma_p (A/m^2), < 0 for discharge */
  double diffpot_sign;             /* sign of the diffusion-potential term of eq. phie-weak (+1 as printed) */
  /* solver */
  int32_t precision;    /* 0: FP64 preconditioner; 1: FP32 preconditioner; 2: FP32 with BF16 coarse-level stencils */
  int32_t combine;      /* 0: block Jacobi (eq. PJ); 1: block Gauss-Seidel (eq. PGS) */
  int32_t order[3];     /* BGS order over {0 phi_s, 1 phi_e, 2 c_e}; default {1, 0, 2} */
  int32_t restart;      /* FGMRES restart length m, 1 <= m <= 128 (paper: 30; 100 for the jelly roll) */
  int32_t maxit;        /* maximum FGMRES iterations per solve */
  int32_t mode;         /* 0: FULL (Krylov on all unknowns); 1: REDUCED (Krylov on the Schur system) */
  int32_t cheb_degree;  /* Chebyshev smoothing steps before and after the coarse correction (>= 1) */
  int32_t coarse_max;   /* coarsen while a level has more than this many nodes (>= 8); a
                           level coarsens by two the axes with >= 2 elements whose
                           mean element size is at most twice the smallest of them
                           (weakly coupled axes of anisotropic elements stay fine) */
  double cheb_ratio;    /* Chebyshev interval [lam/ratio, lam] on D^-1 A */
  double rtol;          /* relative residual target of FGMRES in the scaled norm */
  int32_t profile;      /* 1: time phases and kernel classes of each solve with CUDA events
                           (fields ms_* / n_* of p4d_info); 0: off */
  int32_t ocp_model;    /* 0: the linear OCP of ocp_n / ocp_p; 1: the paper's open-circuit
                           potential curves (Appendix "Model Parameters": graphite anode,
                           LiCoO2 cathode with theta~ = 1.062 theta), U and dU/dtheta in the
                           kinetics of the residual and the Jacobian */
  int32_t transport_model; /* 0: constant kappa and De; 1: the paper's kappa(c_e), D_e(c_e)
                           (eqs. kappa_app, De_app with their Arrhenius factors at T), per
                           element at the element mean of the nodal c_e; kappa and De are then
                           ignored, and the multigrid preconditioner uses the laws at
                           c_e = 1000 mol/m^3.  Fixed at p4d_setup */
  int32_t cgs_refine;   /* second classical Gram-Schmidt pass of each Arnoldi step:
                           0 never (the GMRES settings of the paper's Appendix "Solver
                           parameters" keep the default classical Gram-Schmidt without
                           refinement), 1 when the first pass leaves ||w|| < 0.7 ||w_0||
                           (default), 2 always */
  int32_t mf_zchunk;    /* node planes per block of the matrix-free level-0 kernel (the
                           z depth of its tile; 0 = 8, at most 64).  Fixed at p4d_setup */
} p4d_params;

/* A linearization state.  All [device], FP64; cs / cs_prev are [nelec][nc]. */
typedef struct {
  const double *phis, *phie, *ce, *cs;
  const double *ce_prev, *cs_prev;   /* previous backward-Euler time level */
} p4d_state;

/* Solve report ([host], written when the solve returns). */
typedef struct {
  int32_t iters;          /* FGMRES iterations (preconditioner applications) */
  int32_t restarts;       /* restart cycles started */
  int32_t status;         /* p4d_status of the solve */
  int32_t reorth;         /* iterations that needed a second Gram-Schmidt pass */
  double rel_res;         /* final ||s.(b - J x)|| / ||s.b|| (true residual, scaled norm) */
  double rel_res_block[4];/* the same restricted to phi_s, phi_e, c_e, c_s rows */
  double ms_total;        /* device time of the solve (CUDA events) */
  /* filled when p4d_params.profile = 1 (device time, CUDA events on the handle's stream): */
  double ms_precond;      /* preconditioner applications */
  double ms_jvp;          /* operator applications inside the Krylov loop */
  double ms_ortho;        /* Gram-Schmidt passes, norms and Givens updates */
  double ms_smooth0;      /* level-0 Chebyshev steps that apply the stencil (all hierarchies) */
  int32_t n_smooth0;      /* number of those launches */
  int32_t n_jvp;          /* number of operator applications timed in ms_jvp */
  double rel_res_unscaled;          /* final ||b - J x||_2 / ||b||_2, unscaled, full system */
  double rel_res_block_unscaled[4]; /* ||(b - J x)_f|| / ||b_f|| per field phi_s, phi_e, c_e, c_s */
  int32_t nsolves;        /* linear solves behind this report (1; p4d_newton_solve: all of its solves) */
  int32_t iters_total;    /* FGMRES iterations summed over those solves */
} p4d_info;

/* Fill *p with the defaults (paper constants, BJ, FP32 preconditioner,
   restart 30, rtol 1e-8, REDUCED mode, Chebyshev degree 2, ratio 10,
   linear OCP, constant transport coefficients). */
void p4d_params_default(p4d_params* p);

/* Build a handle for one cell (paper sections 3-4): validates the mesh,
   classifies nodes (electrode nodes = nodes of anode/cathode elements;
   anode and cathode elements must not share a node), assembles the fixed
   Q1 stiffness/mass stencils, plans the multigrid hierarchy and allocates
   all workspace.  If state != NULL the Jacobian is linearized at it (as
   p4d_jacobian_update).  stream: a cudaStream_t or NULL.
   Errors: INVALID_ARG (sizes, options, anode/cathode contact; kernels use
   32-bit indices, so 27 N_n and N_E N_c must stay below 2^31), OOM, CUDA. */
p4d_status p4d_setup(const p4d_mesh* mesh, const p4d_params* params, const p4d_state* state,
                     void* stream, p4d_handle* out);

/* Release all device memory of the handle (NULL is ignored). */
void p4d_destroy(p4d_handle h);

/* Sizes: nodes, electrode nodes, total unknowns, radial nodes ([host] outputs, any may be NULL). */
p4d_status p4d_get_sizes(p4d_handle h, int64_t* nnode, int64_t* nelec, int64_t* ndof, int32_t* nc);

/* Node index of every electrode node, increasing ([host] int32 array of nelec). */
p4d_status p4d_electrode_nodes(p4d_handle h, int32_t* out);

/* Change solver options (combine, order, restart, maxit, rtol, cheb_ratio,
   cheb_degree, mode, profile, cgs_refine) and the kinetics constants.
   precision, coarse_max, mf_zchunk and the parameters assembled at setup
   (dt, F, brug, De, kappa, sigma_n, sigma_p, transport_model) cannot
   change (INVALID_ARG). */
p4d_status p4d_set_params(p4d_handle h, const p4d_params* params);

/* Nonlinear residual R(u) (paper section 4, block residual [R_phis; R_phie;
   R_ce; R_cs]) at `state` into r_out [device, ndof].  DOMAIN if a
   concentration leaves the kinetics domain (r_out then undefined).
   Synchronizes the stream (to report DOMAIN). */
p4d_status p4d_residual(p4d_handle h, const p4d_state* state, double* r_out);

/* Linearize at `state` (paper section 4, eq. blocks): Butler-Volmer
   derivatives per electrode node, particle tridiagonals and their Schur
   scalars, the Jacobi scaling, the Schur-corrected multigrid operators of
   every level and the coarsest-level inverses.  Synchronizes the stream
   (to report DOMAIN). */
p4d_status p4d_jacobian_update(p4d_handle h, const p4d_state* state);

/* y = J x (transpose = 0) or y = J^T x (transpose = 1), unscaled, full
   layout, [device] x and y of ndof doubles, x != y.  Requires a prior
   p4d_jacobian_update. */
p4d_status p4d_jvp(p4d_handle h, const double* x, double* y, int transpose);

/* z = P^-1 r, the block preconditioner of section 4 in the unscaled full
   layout (transpose = 1: P^-T, used by the adjoint), [device] r, z of ndof
   doubles, r != z. */
p4d_status p4d_precond_apply(p4d_handle h, const double* r, double* z, int transpose);

/* Solve J x = b by right-preconditioned FGMRES(m) to
   ||s.(b - J x)|| <= rtol ||s.b||, [device] b and x (in: initial guess,
   out: solution) of ndof doubles.  s is a Jacobi scaling with per-field
   balancing: s_i = w_f / sqrt(J_ii) for row i of field f, with
   w_f = 1 / max(||(b / sqrt(diag J))_f||, floor_f) and
   floor_f = (1e-14 / rtol) ||(sqrt(diag J) u)_f|| (u the linearization
   state), so every field's residual block counts equally unless its
   right-hand side is at the rounding level of its own terms.  info may be
   NULL.  Returns OK, NOT_CONVERGED (x = last iterate), BREAKDOWN or
   NONFINITE. */
p4d_status p4d_fgmres_solve(p4d_handle h, const double* b, double* x, p4d_info* info);

/* Adjoint solve J^T lam = g with the transposed block preconditioner,
   same conventions as p4d_fgmres_solve. */
p4d_status p4d_adjoint_solve(p4d_handle h, const double* g, double* lam, p4d_info* info);

/* ---- Many cells solved together (independent electrode cells of uneven
   sizes, each like the interpenetrating gyroid cell of section 5.1, Case IV).
   A batch drives the FGMRES solves of its cells in lockstep: the restart
   cycles start together, and the Arnoldi steps of Krylov column k of every
   cell form one CUDA graph in which each cell's step sits under a
   conditional node whose flag a device kernel sets from the host's
   per-cell convergence mask, so the GPU runs all cells' steps concurrently
   and the host launches one graph and reads the cells' residual estimates
   once per column.  Each cell keeps its own options, restart length and
   stream (its non-Arnoldi work runs there); results and iteration counts
   are those of p4d_fgmres_solve on each cell alone. */
typedef struct p4d_batch_ctx* p4d_batch;

/* Group ncells distinct handles of the current device (not owned: destroy
   the batch before its cells).  Allocates the batch's own small workspace
   (a stream, per-cell flags and status pairs), freed by p4d_batch_destroy.
   Errors: INVALID_ARG (NULL or repeated handle, ncells <= 0), OOM, CUDA. */
p4d_status p4d_batch_create(const p4d_handle* cells, int32_t ncells, p4d_batch* out);

/* J_i x_i = b_i for every cell i: [host] arrays b, x of ncells [device]
   pointers with each cell's conventions of p4d_fgmres_solve; info: NULL or
   ncells entries.  Every cell must be linearized, with profile = 0.
   Synchronizes every cell's stream.  Returns OK when every cell converged,
   else the status of the first cell that did not (each cell's own status is
   in info[i].status). */
p4d_status p4d_batch_fgmres_solve(p4d_batch b, const double* const* rhs, double* const* x, p4d_info* info);

/* J_i^T lam_i = g_i for every cell, as p4d_batch_fgmres_solve. */
p4d_status p4d_batch_adjoint_solve(p4d_batch b, const double* const* g, double* const* lam, p4d_info* info);

/* Release the batch (NULL is ignored); the cells are untouched. */
void p4d_batch_destroy(p4d_batch b);

/* ---- Slab domain decomposition of one cell (paper section 5, the strong
   and weak scaling runs partition the cell over MPI ranks).  The cell is
   cut along z into slabs; slab p owns a contiguous range of node planes
   and is built as its own handle from the sub-mesh of the elements between
   `ghosts` node planes below and above that range (clipped at the cell's
   faces): the lowest `ghosts` local planes of every slab but the first and
   the highest `ghosts` of every slab but the last are ghost planes, owned
   by the neighbour.  The slab meshes and states are the cell's restricted
   to those elements and nodes; Gamma_n and the z = 0 foil belong to the
   first slab only, Gamma_p and the z = Lz foil to the last.  An operator
   application exchanges the ghost planes of its input with the owners
   (pack, transfer, unpack); every inner product sums the slabs' owned-row
   partial sums.  In this library all slabs of a decomposition live on one
   GPU and one stream (a transfer is a device-to-device copy; the sum runs
   over the slabs' staged partials); with one slab per rank the same steps
   are a send/recv pair per message and an allreduce. */
typedef struct p4d_dd_ctx* p4d_dd;

/* Halo messages of nparts slabs with nplanes[p] local node planes each and
   `ghosts` ghost planes per interior side ([host], no device work, callable
   without a GPU): writes 4 int32 per message to plan (if not NULL): source
   slab, first source plane, destination slab, first destination plane
   (`ghosts` consecutive planes each), and returns the number of messages,
   2 (nparts - 1); -1 when nparts < 1, ghosts < 1, or a slab owns no plane
   or (nparts > 1) fewer planes than ghosts. */
int32_t p4d_dd_halo_plan(int32_t nparts, const int32_t* nplanes, int32_t ghosts, int32_t* plan);

/* Group the slab handles parts[0..nparts) (bottom to top, 1 <= nparts <=
   32, `ghosts` ghost planes per interior side; not owned: destroy the
   decomposition before them).  They must share the device, the stream, nx,
   ny and nc.  Allocates the message buffers, one right-hand-side copy and
   two coarse-space work vectors per slab.  Errors: INVALID_ARG (NULL or
   repeated handle, mismatch, a plan p4d_dd_halo_plan rejects), OOM, CUDA.
   The calls below return INVALID_ARG when the slabs' device is not the
   current device. */
p4d_status p4d_dd_create(const p4d_handle* parts, int32_t nparts, int32_t ghosts, p4d_dd* out);

/* Coarse space of the two-level preconditioner (default 2): 0 none (block
   Jacobi across the slabs), 1 one constant per slab and block (phi_s of
   each electrode, phi_e, c_e), 2 also one linear-in-z function per slab and
   block.  The correction Z A_c^-1 Z^T, with the Galerkin matrix A_c = Z^T J Z
   of the REDUCED operator, is added to every slab preconditioner's output;
   A_c (at most 8 per slab) is built at p4d_dd_jacobian_update and solved in
   FP64 redundantly on every slab.  Takes effect at the next update; a
   singular A_c leaves the correction off. */
p4d_status p4d_dd_set_coarse(p4d_dd dd, int32_t modes);

/* Linearize every slab at states[p] (each the cell's state restricted to
   the slab, ghost planes included), then set the norm floor of the Krylov
   weights from the owned rows of all slabs and build the coarse space (one
   decomposed JVP per coarse basis vector).  Synchronizes the stream. */
p4d_status p4d_dd_jacobian_update(p4d_dd dd, const p4d_state* states);

/* y = J x on the owned rows of every slab ([host] arrays of [device] slab
   vectors in the full layout).  The ghost planes of x[p] (phi_s, phi_e,
   c_e) are overwritten with the owners' values first; the ghost rows of
   y[p] (and the particle rows of the ghost planes' electrode nodes) are
   zero.  Asynchronous. */
p4d_status p4d_dd_jvp(p4d_dd dd, double* const* x, double* const* y);

/* J x = b for the whole cell by FGMRES over the slabs (REDUCED mode only,
   every slab with the same rtol, restart, maxit and cgs_refine, profile
   off).  b[p], x[p] as p4d_fgmres_solve per slab; the ghost rows of b are
   ignored, the owned rows of x are the solution (its ghost planes hold the
   owners' values).  The preconditioner is restricted additive Schwarz
   over the slabs: each slab applies its own block preconditioner to the
   Krylov vector on its owned and ghost rows (the owners' values) and keeps
   its owned rows; with ghosts = 1 the ghost rows are zero instead (block
   Jacobi across the slabs); plus the coarse correction of p4d_dd_set_coarse.  The
   converged solution is the cell's.  info (one report for the cell) as p4d_fgmres_solve.
   Synchronizes the stream. */
p4d_status p4d_dd_fgmres_solve(p4d_dd dd, const double* const* b, double* const* x, p4d_info* info);

/* Release the decomposition (NULL is ignored); the slabs are untouched. */
void p4d_dd_destroy(p4d_dd dd);

/* Largest number of electrode nodes p4d_jvp_noalloc accepts (size of its
   fixed scratch array: 2^20 doubles = 8 MiB per GPU that loads the library). */
#define P4D_NOALLOC_MAX_NELEC (1 << 20)

/* y = J x or J^T x like p4d_jvp, for callers that must not allocate device
   memory at the time of the call: code running under CUDA stream capture,
   where cudaMalloc would break the capture, or code whose device memory is
   owned entirely by a framework's pool or a fixed arena.  The paper has no
   counterpart; this is a deployment variant of p4d_jvp.  It calls no
   cudaMalloc/cudaFree and no allocating library routine: the only scratch
   the JVP needs (one coupling scalar per electrode node) lives in a fixed
   device array of P4D_NOALLOC_MAX_NELEC doubles that every GPU loading the
   library keeps until the process exits.  The first call on each device
   looks up that array's device address (cudaGetSymbolAddress); make that
   first call before any stream capture.  All calls share the one array, so
   calls whose kernels overlap on the GPU (several streams or handles at
   once) race; nothing in it needs to start at zero (each entry is written
   before it is read within a call).  Not available with transport_model 1
   (INVALID_ARG: those products need per-element scratch of the handle).
   The result agrees with p4d_jvp's to
   rounding (the non-transposed product forms phi_e + (gamma/c_e) c_e inside
   the stencil loop rather than in a separate pass).  Returns INVALID_ARG
   when the handle has more than P4D_NOALLOC_MAX_NELEC electrode nodes, when
   x == y, before a p4d_jacobian_update, or when the current device is not
   the one the handle was set up on; otherwise as p4d_jvp. */
p4d_status p4d_jvp_noalloc(p4d_handle h, const double* x, double* y, int transpose);

/* Newton's method for one backward-Euler step (paper section 4: the
   monolithic residual R = [R_phis; R_phie; R_ce; R_cs] = 0, every linear
   system solved by p4d_fgmres_solve).  phis, phie, ce, cs [device, updated
   in place] hold the initial guess and receive the solution; ce_prev,
   cs_prev [device] are the previous time level.  The residual is measured
   in the Jacobi-scaled norm ||D^-1/2 R|| (D = diag J at the initial
   guess).  Full Newton steps (the paper uses its nonlinear solver's
   default, basic, line search); a step is halved (at most 8 times) only
   while the trial state leaves the kinetics' domain or gives a non-finite
   residual.  Converged when ||D^-1/2 R|| <= rtol ||D^-1/2 R_0|| or when a
   full Newton step is at most rtol times the state in every field (the
   residual has a rounding floor); NOT_CONVERGED after maxit iterations.
   iters and info may be NULL; info describes the last linear solve, except
   nsolves and iters_total, which count all of the step's linear solves.  Returns OK,
   NOT_CONVERGED, DOMAIN or a linear-solve failure.  Leaves the handle
   linearized at the last accepted iterate but one. */
p4d_status p4d_newton_solve(p4d_handle h, double* phis, double* phie, double* ce, double* cs,
                            const double* ce_prev, const double* cs_prev, double rtol, int32_t maxit,
                            int32_t* iters, p4d_info* info);

/* Weights q of the terminal voltage V = q . u (full layout, [device] ndof
   doubles): the mean of phi_s over the applied-current face Gamma_p
   (bilinear face weights; phi_s = 0 on the grounded face). */
p4d_status p4d_voltage_weights(p4d_handle h, double* q);

/* Terminal voltage V = q . u = the mean of phi_s over Gamma_p (the
   objective of the adjoint, paper section 3's sensitivity motivation),
   from phis [device, nnode doubles] into v [device, one double].
   Asynchronous on the handle's stream.  Errors: INVALID_ARG (NULL, or no
   applied-current face). */
p4d_status p4d_terminal_voltage(p4d_handle h, const double* phis, double* v);

/* Accumulate g_p += -lam^T dR/dp at `state` (the residual of one
   backward-Euler step, paper section 4) for the per-element parameters
   p = sigma (bulk solid conductivity), D_s (solid diffusivity, through the
   volume-weighted node means) and eps (porosity, through kappa_eff,
   D_e,eff and the electrolyte mass); eps_s is held fixed.  lam [device,
   ndof]; g_sigma, g_Ds, g_eps [device, nelem], each may be NULL. */
p4d_status p4d_param_grad(p4d_handle h, const p4d_state* state, const double* lam, double* g_sigma,
                          double* g_Ds, double* g_eps);

/* Adjoint coupling to the previous time level: out = -(dR_n/du_{n-1})^T lam
   (only the c_e mass and the particle accumulation terms depend on the
   previous state), [device] ndof doubles. */
p4d_status p4d_adjoint_prev(p4d_handle h, const double* lam, double* out);

/* Number of CUDA kernels the library has launched in this process so far
   (instrumentation for benchmarks; thread-safe, never reset). */
long long p4d_launch_count(void);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (2 flops
   per FMA; eight independent dependent-FMA chains per thread over 8 blocks
   of 256 threads per SM, best of three timed launches on the legacy default
   stream, which it synchronizes).  The denominator of the FP64 kernels'
   roofline fractions (instrumentation for benchmarks, like
   p4d_launch_count).  Errors: INVALID_ARG (NULL), CUDA. */
p4d_status p4d_fp64_fma_rate(double* tflops);

/* Human-readable name of a status. */
const char* p4d_status_string(p4d_status s);

#ifdef __cplusplus
}
#endif
#endif /* P4D_H */
