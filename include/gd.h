/*
 * gd.h -- C ABI of the GB300 (sm_103a) gradient-enhanced damage library.
 *
 * The library computes the monolithic Newton iteration of the gradient-enhanced
 * damage model with input-convex neural network (ICNN) constitutive laws of
 * arxiv 2604.03411 (Wilkinson, Amiri-Hezaveh, Buganza Tepole): per quadrature
 * point the deformation gradient, C - I without cancellation, the invariants,
 * the ICNN strain energy with first and second derivatives, the ICNN yield
 * function with the local damage/history update, the degraded stress and the
 * non-local fluxes; per element the coupled residual and consistent tangent,
 * scattered into a CSR matrix through a precomputed slot map; and the global
 * Newton iteration with a Krylov solver on the device, preconditioned by node-block
 * Jacobi plus an aggregation coarse level.
 *
 * Conventions
 *  - Every call returns gd_status; after a non-OK status gd_last_error() gives a
 *    message and the handle stays usable at its last committed load step.
 *  - Unless stated otherwise, array arguments of gd_create/gd_set_state/
 *    gd_get_fields are HOST pointers, copied during the call (the caller keeps
 *    ownership).  Arguments documented as "device" are borrowed for the duration
 *    of the call only and must be resident on the handle's device.
 *  - All device work is issued on gd_options.cuda_stream (NULL: the legacy
 *    default stream).  Calls that return results to host memory synchronise
 *    that stream.
 *  - One handle must not be used from two host threads at once.
 *  - Sizes: nnz of the global matrix must stay below 2^31 (int32 column
 *    indices and slot map); larger meshes are rejected with GD_ERR_ARG.
 *
 * Degrees of freedom are node-major: dof (node n, component c) has index
 * n * ndof + c, ndof = dim + 1, components 0..dim-1 are the displacement and
 * component dim is the non-local damage phi (Sec. 3.1, Table kernel_inputs).
 */
#ifndef GD_H
#define GD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gd_status {
    GD_OK = 0,
    GD_ERR_ARG = 1,            /* invalid argument or size                          */
    GD_ERR_MESH = 2,           /* bad connectivity, node id, or Jacobian <= 0       */
    GD_ERR_CUDA = 3,           /* a CUDA runtime call failed                        */
    GD_ERR_OOM = 4,            /* device allocation failed                          */
    GD_ERR_NOT_CONVERGED = 5,  /* Newton did not converge after all step cuts       */
    GD_ERR_NAN = 6,            /* non-finite residual                               */
    GD_ERR_KRYLOV = 7,         /* Krylov breakdown or iteration cap                 */
    GD_ERR_LOCAL_SOLVE = 8,    /* local kappa update hit its iteration cap          */
    GD_ERR_TIMEOUT = 9,        /* a bounded device wait gave up                     */
    GD_ERR_STATE = 10          /* call not valid in the handle's current state      */
} gd_status;

enum { GD_ENERGY_ICNN_RAW = 0,   /* psi-ICNN of (I1-3, I2-3, J-1)                          */
       GD_ENERGY_ICNN_ISO = 1,   /* psi-ICNN of (I1G-3, I2G-3, J-1), Eq. (dd_0)            */
       GD_ENERGY_NEO_HOOKE = 2 };/* closed-form compressible Neo-Hookean, Sec. 4.1         */
enum { GD_FP64 = 0, GD_MIXED = 1 };
enum { GD_BICGSTAB = 0, GD_GMRES = 1 };
enum { GD_ASM_RESIDUAL = 0, GD_ASM_TANGENT = 1 };
enum { GD_INNER_AUTO = 0, GD_INNER_FP64 = 1, GD_INNER_REFINED = 2 };
enum { GD_MONOLITHIC = 0, GD_STAGGERED = 1, GD_STAGGERED_ITERATED = 2 };
enum { GD_ICNN_AUTO = 0, GD_ICNN_CUDA_CORES = 1, GD_ICNN_BF16 = 2, GD_ICNN_BF16X3 = 3 };

/* Mesh and boundary data (Sec. 3.1, Table kernel_inputs; Dirichlet data of the
 * incremental load, Sec. 3.2).
 *   dim 2: plane-strain bilinear Q4, 2x2 Gauss, nodes counter-clockwise;
 *   dim 3: trilinear HEX8, 2x2x2 Gauss, nodes (-,-,-) (+,-,-) (+,+,-) (-,+,-) then z = +.
 * Quadrature points are ordered lexicographically, reference coordinate xi fastest.
 * Prescribed dof (bc_node[i], bc_comp[i]) takes bc_scale[i] * load(t); bc_comp < dim
 * (phi has the natural zero-flux condition on the whole boundary, Sec. 2.1).
 * The reaction of a step is the sum of the internal force components react_comp
 * over react_node, taken before the prescribed rows are eliminated. */
typedef struct gd_mesh {
    int32_t dim;
    int64_t n_nodes, n_elems;
    const double *coords;      /* [n_nodes * dim]  reference coordinates              */
    const int32_t *conn;       /* [n_elems * nen]  nen = 4 (dim 2) or 8 (dim 3)       */
    int64_t n_bc;
    const int32_t *bc_node;    /* [n_bc] */
    const int8_t *bc_comp;     /* [n_bc] */
    const double *bc_scale;    /* [n_bc] */
    int64_t n_react;
    const int32_t *react_node; /* [n_react] */
    int32_t react_comp;
} gd_mesh;

/* Two-layer softplus ICNN with input skips (Sec. 4.2, Eqs. (dd_0), (Gq_NN)).
 * params packs W1[w][n_in] b1[w] W2[w][w] A2[w][n_in] b2[w] w3[w] a3[n_in]:
 *   N(x) = w3 . sp(W2 sp(W1 x + b1) + A2 x + b2) + a3 . x,  sp = softplus.
 * W1, W2, A2, w3, a3 must be >= 0 (convex, non-decreasing); biases are free.
 * n_in = 3 for the energy network, 1 for the yield network.  width 0 for the
 * yield network selects G(q) = q (the closed-form loading function of
 * Eq. (ostwald_potential)); widths up to 64. */
typedef struct gd_icnn {
    int32_t n_in;
    int32_t width;
    const double *params;
} gd_icnn;

/* Constants of Sec. 4: f_d(kappa) = exp(-eta_d <kappa - kappa_d>_+) (Eq. (degradation_function)),
 * gradient energy c_d/2 gradphi.C^-1.gradphi, penalty beta_d/2 (phi - kappa)^2,
 * q = psi_e + gamma_d beta_d (phi - kappa) / (eta_d f_d(kappa)) (Eq. (ostwald_potential)).
 * Energy psi_e = mu_e [N(x) - N(0) - n (J-1)] + lambda_e (J + 1/J - 2)^2 with n fixed
 * by S(C = I) = 0; for GD_ENERGY_NEO_HOOKE mu_e, lambda_e are the Lame constants.
 * eta_d must be > 0. */
typedef struct gd_material {
    double mu_e, lambda_e, eta_d, kappa_d, beta_d, c_d, gamma_d;
    int32_t energy;
} gd_material;

/* Quasi-static incremental load (Sec. 3.2): step s prescribes bc_scale * load[s]. */
typedef struct gd_load_path {
    int32_t n_steps;
    const double *load;        /* [n_steps] */
} gd_load_path;

typedef struct gd_options {
    int32_t precision;         /* GD_FP64 or GD_MIXED                                  */
    double newton_rtol;        /* ||R_free|| <= max(rtol max(||R0_free||, ||R_fixed||), atol);
                                  raised to 1e-5 in GD_MIXED (FP32 element math), where an
                                  iterate whose residual the line search cannot lower any
                                  more and that is below 1e-4 of that scale is accepted    */
    double newton_atol;
    int32_t newton_max;        /* Newton iterations per step                           */
    int32_t line_search_max;   /* backtracking halvings per Newton direction           */
    int32_t krylov;            /* GD_BICGSTAB (default): the persistent two-level BiCGStab, and
                                  for an FP64 solve it does not finish (breakdown, stagnation,
                                  krylov_max) GMRES(gmres_m) takes over; GD_GMRES: every FP64
                                  solve by restarted GMRES(gmres_m), right-preconditioned by
                                  node-block Jacobi (FP32 inner solves stay BiCGStab)          */
    double krylov_rtol;        /* floor of the relative residual of each Newton solve (the
                                  solve stops at max(krylov_rtol, min(1e-2, 0.1 tol/||R||)),
                                  tol the Newton tolerance); gd_solve uses it directly       */
    int32_t krylov_max;
    int32_t gmres_m;           /* GMRES restart length, 1..64 (default 50)              */
    int32_t local_max;         /* local kappa iterations (the paper caps at 100, Sec. 5.3) */
    int32_t checkpoint_every;  /* adjoint checkpoint interval in load steps            */
    int32_t max_step_cuts;     /* nested load-step halvings after a failed step        */
    void *cuda_stream;         /* cudaStream_t or NULL                                 */
    int32_t inner_solve;       /* GD_INNER_AUTO (default): FP64 BiCGStab in GD_FP64; in GD_MIXED
                                  FP32 BiCGStab (FP64 dots) for directions that need at most
                                  1e-5 relative accuracy, FP64 otherwise.  GD_INNER_FP64: FP64
                                  BiCGStab always.  GD_INNER_REFINED: FP32 BiCGStab cycles
                                  refined by FP64 residuals b - K x until the FP64 tolerance
                                  is met.  A failed FP32 solve falls back to FP64.          */
    int32_t coarse;            /* target number of coarse unknowns of the two-level
                                  preconditioner M^-1 = D^-1 + P (P^T K P)^-1 P^T (D the
                                  node-block diagonal, P constants and rigid rotations on
                                  aggregates of the node graph); default 1536, at most 3072,
                                  0 = node-block Jacobi only.  The preconditioner changes the
                                  iteration count, not the solution.  A batch with a coarse
                                  level (aggregates never span two specimens) solves its
                                  union system in one recurrence instead of per-specimen
                                  recurrences.                                              */
    int32_t scheme;            /* GD_MONOLITHIC (default, Sec. 3.2): kappa is updated inside
                                  every Newton iteration and its sensitivity enters the
                                  tangent.  GD_STAGGERED (Sec. 3.2, single specimens): the
                                  history is advanced apart from the nodal solve: Newton on
                                  the (u, phi) equilibrium with kappa held at the committed
                                  kappa_n, then one local update at the converged fields; the
                                  step is accepted without a coupled test, so the update lags
                                  the nodal solve by one step (first order in the load
                                  step), and the step's reaction is that of the equilibrium.
                                  GD_STAGGERED_ITERATED (single specimens): the same two
                                  stages alternate within the step until the residual with
                                  the updated kappa meets the Newton test; the converged step
                                  solves the monolithic equations (the alternation converges
                                  linearly, slowly for a stiff penalty beta_d).             */
    int32_t stagger_max;       /* GD_STAGGERED_ITERATED: alternations per load step before the
                                  step counts as failed (default 100)                       */
    int32_t asm_grid_max;      /* cap on the CTAs of the persistent element-kernel grid (0, the
                                  default: SMs x resident CTAs).  A small cap makes every warp
                                  take several element batches in turn; results do not depend
                                  on it beyond the order of the atomic additions.            */
    int32_t krylov_row_cache;  /* shared-memory copy of each Krylov block's matrix rows:
                                  0 (default) column lists and values where they fit, else
                                  column lists only; 1 column lists only; 2 none (every
                                  product reads the rows from global memory).  Changes the
                                  speed, not the iterates.                                  */
    int32_t icnn_mma;          /* arithmetic of the networks' second layers in GD_MIXED (Sec. 4.2
                                  ICNNs; the layer is a dense contraction over the points of a
                                  thread block):
                                  GD_ICNN_CUDA_CORES  FP32 on the CUDA cores;
                                  GD_ICNN_BF16        tensor cores, BF16 operands, FP32
                                                      accumulation;
                                  GD_ICNN_BF16X3      tensor cores, every operand split into
                                                      a BF16 high part and a BF16 residual,
                                                      three products accumulated in FP32
                                                      (about 16 significant bits);
                                  GD_ICNN_AUTO (0, the default) GD_ICNN_BF16X3 for a single
                                  specimen, GD_ICNN_CUDA_CORES for batches.  The tensor-core
                                  modes need a single specimen (GD_ERR_ARG for batches).
                                  Ignored in GD_FP64.                                        */
} gd_options;

typedef struct gd_newton_report {
    int32_t converged;
    int32_t iterations;        /* Newton directions taken                               */
    int32_t krylov_iterations; /* summed over the step                                  */
    int32_t line_search_cuts;
    int32_t local_failures;
    int32_t loading_points;    /* qps on the loading branch at convergence              */
    int32_t step_cuts;
    int32_t assemblies;        /* element-kernel launches in the step                   */
    double residual0, residual, reaction, max_damage;
    double assembly_ms;        /* device time of those launches (CUDA events)           */
    double krylov_ms;          /* device time of the linear solves                      */
    int64_t yield_evals;       /* yield-network evaluations of the local solves (all launches) */
    int64_t kernel_launches;   /* device kernels this library launched for the step     */
    int32_t krylov_fp32_iterations; /* iterations of FP32 inner solves (the rest ran in FP64) */
    int32_t noise_passes;      /* GD_MIXED: FP64 reference passes run to measure the noise floor */
    double noise;              /* GD_MIXED: rounding-noise level of ||R_free|| at the last Newton
                                  test (the test does not go below twice it); 0 in GD_FP64      */
    double noise_ms;           /* device time of the FP64 reference passes (in the step time, not
                                  in assembly_ms)                                              */
} gd_newton_report;

typedef struct gd_path_report {
    int32_t steps_done;
    int32_t total_newton;
    int32_t total_krylov;
    int32_t step_cuts;
    int32_t assemblies;
    double assembly_ms;        /* device time of the assembly kernels (CUDA events)     */
    double krylov_ms;          /* device time of the linear solves                      */
    double total_ms;
} gd_path_report;

typedef struct gd_handle gd_handle;

/* Fills *opt with the defaults: FP64, newton_rtol 1e-10, newton_atol 1e-12,
 * newton_max 25, line_search_max 12, BiCGStab with krylov_rtol 1e-12 and
 * krylov_max 20000, local_max 100, checkpoint_every 5, max_step_cuts 4,
 * default stream, coarse 1536, monolithic scheme (stagger_max 100), no element
 * grid cap, automatic Krylov row cache, automatic network arithmetic. */
void gd_default_options(gd_options *opt);

/* Creates a problem (Sec. 3.1 kernel inputs, Sec. 3.2 load path): copies and
 * validates the mesh (node ids, positive Jacobians at every qp), builds the CSR
 * pattern of the node graph with ndof x ndof blocks, the per-element slot map
 * and the Dirichlet masks, stages the ICNN weights and their normalising
 * constants N(0), n, N_k(0), 1/N_k'(0) on the device, and zeroes the state
 * (u = 0, phi = 0, kappa = 0).  The handle owns all device memory.
 * Errors: GD_ERR_ARG (null/size/width), GD_ERR_MESH, GD_ERR_OOM, GD_ERR_CUDA. */
gd_status gd_create(const gd_mesh *mesh, const gd_icnn *psi, const gd_icnn *yield,
                    const gd_material *mat, const gd_load_path *path, const gd_options *opt,
                    gd_handle **out);

/* Batched specimens (many independent problems in one handle): n_spec meshes,
 * energy networks, yield networks and load paths (arrays of n_spec structs; psi
 * may be NULL for GD_ENERGY_NEO_HOOKE), one material and one set of options.
 * The meshes are laid end to end into one block-diagonal system (nodes and
 * elements of specimen s follow those of specimens 0..s-1), every assembly is a
 * single persistent launch over the elements of all specimens, each element
 * reading its own specimen's network weights, and one Newton iteration advances
 * all specimens together: each specimen has its own convergence test
 * ||R_free,s|| <= max(rtol max(||R0_free,s||, ||R_fixed,s||), atol) and its own
 * line-search step, and a converged specimen is held fixed while the others
 * iterate.  Load step k of the batch takes step k of every path; a specimen whose
 * path is shorter holds its last load.  A failed step is halved for every
 * specimen.  The dim, and the widths' upper bound (64), are common; widths may
 * differ between specimens.  gd_newton_step and gd_run_load_path advance the
 * batch (reactions [n_steps * n_spec], step-major; see gd_batch_layout for
 * n_steps), gd_get_fields/gd_set_state/gd_assemble/gd_solve work on the union;
 * gd_set_params and gd_backward return GD_ERR_STATE.  This batching (one
 * handle, per-specimen weights) is a throughput layout with no counterpart in
 * the paper, which treats one specimen at a time (Sec. 5).
 * Errors: as gd_create, with the specimen index in the message. */
gd_status gd_create_batch(int32_t n_spec, const gd_mesh *meshes, const gd_icnn *psi, const gd_icnn *yield,
                          const gd_material *mat, const gd_load_path *paths, const gd_options *opt,
                          gd_handle **out);

/* Layout of a handle's specimens (a single-specimen handle is a batch of one):
 * node_off and elem_off [n_spec + 1] (host, may be NULL) receive the first node
 * and element of every specimen, n_steps the number of load steps of the batch
 * (the longest path). */
gd_status gd_batch_layout(gd_handle *h, int32_t *n_spec, int64_t *node_off, int64_t *elem_off, int32_t *n_steps);

/* Replaces the network weights (same widths) from host or device memory
 * (cudaMemcpyDefault) and recomputes the normalising constants on the device. */
gd_status gd_set_params(gd_handle *h, const double *theta_psi, const double *theta_yield);

/* CSR pattern of the global matrix: n_rows = n_nodes * ndof rows; the block of
 * node n has ndof consecutive rows with identical column lists (every dof of
 * every neighbour node, neighbours ascending).  rowptr [n_rows + 1] and colidx
 * [nnz] are host buffers (either may be NULL to query the sizes only). */
gd_status gd_csr_pattern(gd_handle *h, int64_t *n_rows, int64_t *nnz, int32_t *rowptr, int32_t *colidx);

/* Host-only helper (no GPU needed): validates the mesh exactly as gd_create
 * does and returns the CSR pattern described at gd_csr_pattern plus the slot
 * map that the assembly kernel scatters through: slot [n_elems * nen * nen],
 * slot[(e*nen + a)*nen + b] = position in colidx/values of the entry (row dof 0
 * of node conn[e][a], column dof 0 of node conn[e][b]); the entry of row dof i,
 * column dof k is at slot + i * rowlen + k with rowlen = rowptr[r+1] - rowptr[r]
 * of that node's first row r.  Any output may be NULL (query sizes first). */
gd_status gd_build_pattern(const gd_mesh *mesh, int64_t *n_rows, int64_t *nnz, int32_t *rowptr, int32_t *colidx,
                           int32_t *slot);

/* One assembly pass (Sec. 3.1 residual, Sec. 3.2 monolithic tangent), every
 * pointer on the device:
 *   dofs        [n_nodes*ndof] FP64  current u and phi
 *   kappa_n     [n_elems*nq]   FP64  committed history (NULL: the handle's)
 *   R           [n_nodes*ndof] FP64  out: assembled residual (all dofs, no elimination)
 *   csr_vals    [nnz] out: consistent tangent values (FP64 in GD_FP64 precision,
 *               FP32 in GD_MIXED), NULL or mode GD_ASM_RESIDUAL to skip the tangent
 *   kappa_trial [n_elems*nq]   FP64  out: kappa_{n+1} at every qp (may be NULL)
 *   loading     [n_elems*nq]   int8  out: 1 where the qp is on the loading branch (may be NULL)
 * Returns GD_ERR_LOCAL_SOLVE when a local solve hit local_max (outputs still written). */
gd_status gd_assemble(gd_handle *h, const double *dofs, const double *kappa_n, double *R,
                      void *csr_vals, double *kappa_trial, int8_t *loading, int32_t mode);

/* y = K x with the tangent of the handle's last assembly (the one used by the
 * most recent Newton direction, or by gd_assemble when csr_vals was NULL there):
 * x, y device FP64 [n_nodes*ndof]; with free_only != 0 prescribed rows return
 * x and prescribed columns are skipped (the eliminated operator of the Newton
 * system).  Works on the handle's stream; does not synchronise. */
gd_status gd_spmv(gd_handle *h, const double *x, double *y, int32_t free_only);

/* Solves K x = b on the free dofs (the eliminated Newton system) with BiCGStab,
 * preconditioned by node-block Jacobi plus the handle's coarse level when it has
 * one (opt.coarse; recomputed from csr_vals for the call) (opt.krylov_rtol /
 * krylov_max).  csr_vals: device
 * tangent values in the handle's precision from gd_assemble, or NULL for the
 * tangent of the handle's last Newton iteration.  b, x device FP64
 * [n_nodes*ndof]; prescribed dofs of x are returned as 0.  iterations and
 * rel_residual (host, may be NULL) report the solve.  Synchronises the stream.
 * Errors: GD_ERR_KRYLOV when the tolerance is not reached. */
gd_status gd_solve(gd_handle *h, const void *csr_vals, const double *b, double *x, int32_t *iterations,
                   double *rel_residual);

/* Coarse space of the handle's two-level preconditioner (see gd_options.coarse):
 * number of aggregates and of coarse unknowns (0 and 0 when it is off).  Host
 * only.  Errors: GD_ERR_ARG. */
gd_status gd_coarse_info(gd_handle *h, int32_t *n_aggregates, int32_t *n_coarse);

/* The aggregates the two-level preconditioner would build for `mesh` (host only,
 * no device needed): greedy breadth-first aggregates of about target_nodes
 * connected nodes over the node graph of gd_build_pattern's pattern, those below
 * a quarter of the target joined to their smallest neighbour.  agg (host,
 * [n_nodes]) receives every node's aggregate in [0, *n_aggregates).
 * Errors: GD_ERR_ARG, GD_ERR_MESH (as gd_build_pattern). */
gd_status gd_coarse_aggregates(const gd_mesh *mesh, int32_t target_nodes, int32_t *agg, int32_t *n_aggregates);

/* The coarse basis the two-level preconditioner would build for `mesh` with
 * aggregates of about target_nodes nodes (host only, no device needed).  agg
 * [n_nodes] and *n_aggregates as gd_coarse_aggregates; coff [n_nodes + 1] receives
 * the first coarse unknown of every aggregate (coff[a + 1] - coff[a] columns kept
 * for aggregate a, at most *n_modes); P [n_nodes * ndof * n_modes] (row-major
 * [node][dof][mode]) the basis values: per aggregate, the constant field of each
 * nodal unknown and the rigid rotations of the displacement, zero on prescribed
 * dofs, orthonormalised over the aggregate (columns beyond coff[a + 1] - coff[a]
 * are zero).  *n_modes = ndof + 1 in 2D, ndof + 3 in 3D.
 * Errors: GD_ERR_ARG, GD_ERR_MESH (as gd_build_pattern). */
gd_status gd_coarse_basis(const gd_mesh *mesh, int32_t target_nodes, int32_t *agg, int32_t *n_aggregates,
                          int32_t *coff, float *P, int32_t *n_modes);

/* Largest system (n_nodes * ndof) that gd_solve_noalloc accepts. */
#define GD_NOALLOC_MAX_DOFS 131072

/* Krylov solve that allocates no device memory (the paper has no counterpart;
 * this exists for callers that cannot call cudaMalloc -- applications whose own
 * pool owns all of the device memory, runtimes that forbid allocation after
 * start-up).
 * Solves K x = b on the free dofs of a caller-provided node-block CSR system
 * (the layout of gd_csr_pattern, ndof 3 or 4, FP64 values: every node's rows
 * share one ascending column list, and that list holds the node's own ndof x
 * ndof diagonal block, whose inverse preconditions the solve) with the persistent
 * BiCGStab of gd_solve and node-block Jacobi alone (no coarse level: it would
 * need work space of its own).  All arrays are device pointers owned
 * by the caller: rowptr [n_nodes*ndof + 1], colidx, vals [nnz], fixed
 * [n_nodes*ndof] (1 = prescribed dof), b, x [n_nodes*ndof]; prescribed dofs of x
 * come back as 0.  iterations and rel_residual (host, may be NULL) report the
 * solve.  Work runs on `stream` (a cudaStream_t, NULL for the legacy default
 * stream); the call copies its result words to host memory and synchronises
 * `stream` before it returns.
 * Work space: one fixed device array inside the library, sized for
 * GD_NOALLOC_MAX_DOFS dofs (about 13.7 MB), held by every GPU that loads the
 * library until the process exits; larger systems are rejected with GD_ERR_ARG.
 * The first call on a device looks up the array's device address (with that
 * device current).  Every call on a device shares the one array and rewrites all of it that it reads, so
 * calls that overlap on the GPU (other streams, other host threads) race: run
 * them one after another.  Errors: GD_ERR_ARG, GD_ERR_CUDA, GD_ERR_KRYLOV; the
 * message is available from gd_last_error(NULL) on the calling thread. */
gd_status gd_solve_noalloc(int32_t ndof, int64_t n_nodes, const int32_t *rowptr, const int32_t *colidx,
                           const double *vals, const uint8_t *fixed, const double *b, double *x, double rtol,
                           int32_t max_it, void *stream, int32_t *iterations, double *rel_residual);

/* Launch shapes chosen by gd_autotune and the times it measured. */
typedef struct gd_tune_report {
    int32_t asm_warps;           /* warps per CTA of the element kernel (2, 4 or 8)            */
    int32_t krylov_ctas_per_sm;  /* CTAs per SM of the cooperative Krylov grid                 */
    double asm_ms[3];            /* element-kernel pass (tangent) with 2, 4, 8 warps; -1: does
                                    not fit in shared memory                                    */
    double krylov_us[4];         /* Krylov iteration time with 1..4 CTAs per SM; -1: not
                                    co-resident                                                 */
    int32_t krylov_up;           /* node groups per lane in the Krylov products (1, 2 or 4)     */
    double krylov_us_up[3];      /* iteration time with 1, 2, 4 node groups at the chosen grid  */
    int32_t krylov_lanes;        /* lanes per node of 3D solves with FP32 vectors (32, 8 or 4)  */
    double krylov_us_lanes[3];   /* iteration time with 32, 8, 4 lanes per node; -1: not timed */
} gd_tune_report;

/* Times the element kernel (one tangent pass at the committed state) for each CTA
 * width and the Krylov solve (a fixed 40-iteration run on that tangent, in the
 * handle's inner-solve precision) for each grid size, and keeps the fastest
 * shapes for the handle's later calls (the paper has no counterpart: a launch
 * tuning step).  Results do not depend on the choice beyond summation order.
 * rep may be NULL.  Uses the handle's work buffers; the committed state is
 * unchanged.  Errors: GD_ERR_CUDA. */
gd_status gd_autotune(gd_handle *h, gd_tune_report *rep);

/* Advances the next load step of the path to convergence (monolithic Newton,
 * Sec. 3.2, with a line search and nested step halving on failure; or the step of
 * the handle's staggered scheme); commits kappa and the fields on success.  rep
 * may be NULL. */
gd_status gd_newton_step(gd_handle *h, gd_newton_report *rep);

/* Runs every remaining step of the load path; reaction [n_steps] (host, may be
 * NULL; [n_steps * n_spec] step-major for a batch) receives the reaction of each
 * step.  rep may be NULL. */
gd_status gd_run_load_path(gd_handle *h, double *reaction, gd_path_report *rep);

/* Gradient of a loss of the reaction curve with respect to the network weights
 * through the whole load path (discrete adjoint with checkpoints every
 * checkpoint_every steps and recomputation in between).
 *   dL_dreaction [n_steps] host; dL_dtheta [n_psi + n_yield] host out.
 * The adjoint differentiates the monolithic step equations: GD_ERR_STATE for a
 * handle with scheme GD_STAGGERED (whose lagged steps solve other equations).
 * GD_MIXED: the segments are recomputed in mixed precision as the forward ran; the
 * adjoint systems use the FP64 element kernel's tangent at those states and FP64
 * solves, so the gradient is the FP64 model's at the mixed path (its error against
 * the FP64 path's gradient follows the mixed states' error; one extra FP64 value
 * array of nnz entries is allocated on the first call). */
gd_status gd_backward(gd_handle *h, const double *dL_dreaction, double *dL_dtheta);

/* Copies the committed fields to host: dofs [n_nodes*ndof], kappa [n_elems*nq]
 * and the damage d = 1 - f_d(kappa) = 1 - exp(-eta_d <kappa - kappa_d>_+) at every
 * quadrature point [n_elems*nq] (Eq. (degradation_function)); any may be NULL. */
gd_status gd_get_fields(gd_handle *h, double *dofs, double *kappa, double *damage);

/* Overwrites the committed state from host arrays and sets the next step index.
 * dofs, kappa as in gd_get_fields (NULL keeps the handle's).  dofs_prev (may be
 * NULL) is the converged state one step before `dofs` (needs next_step >= 1) and
 * dofs_prev2 (may be NULL) the one two steps before (needs dofs_prev and next_step
 * >= 2).  The next step's initial guess extrapolates from the states given: the
 * quadratic through all three where the path is monotone (as an uninterrupted run
 * does), the last increment linearly with dofs_prev alone, else `dofs` itself; the
 * converged states agree to the Newton tolerance either way.  With dofs_prev (a
 * continuation) the coarse level of the preconditioner and the mixed-precision
 * residual-noise estimate are kept -- the coarse inverse is recomputed when a
 * solve slows down or fails with it, the noise estimate at its usual interval;
 * without it (a new start) both are recomputed at the next solve.  gd_get_state
 * gives the arrays that continue the path. */
gd_status gd_set_state(gd_handle *h, const double *dofs, const double *dofs_prev, const double *dofs_prev2,
                       const double *kappa, int32_t next_step);

/* Copies the committed state to host: dofs, dofs_prev and dofs_prev2 (the states
 * one and two committed steps earlier, the predictor's other points)
 * [n_nodes*ndof], kappa [n_elems*nq]; any may be NULL.  next_step (may be NULL)
 * receives the index of the next load step.  gd_set_state(dofs, dofs_prev,
 * dofs_prev2, kappa, next_step) restores it. */
gd_status gd_get_state(gd_handle *h, double *dofs, double *dofs_prev, double *dofs_prev2, double *kappa,
                       int32_t *next_step);

/* Message for the last non-OK status of this handle (or of gd_create when h is NULL). */
const char *gd_last_error(const gd_handle *h);

/* Frees every device and host resource of the handle (NULL is a no-op). */
void gd_destroy(gd_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* GD_H */
