// gd_internal.cuh -- internal declarations shared by the translation units of
// the CUDA library (handle layout, kernel argument blocks, launchers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gd.h"

namespace gd {

constexpr int kMaxWidth = 64;   // widest supported ICNN layer

// Network constants computed on the device from the weights (Sec. 4.2):
// psi: N(0) and the normalising coefficient n of -n (J - 1) that keeps
// S(C = I) = 0; yield: N_k(0) and s = 1 / N_k'(0) so that G(0) = 0, G'(0) = 1.
struct NetConst {
    double psi_N0, psi_n, y_N0, y_s;
};

// One ICNN on the device: packed parameters (gd_icnn layout) plus a
// transposed copy of the square layer W2 so that both the forward pass
// (lane = output unit) and the reverse pass (lane = input unit) read
// consecutive addresses.
struct DevNet {
    int n_in = 0, width = 0, n_params = 0;
    double *p = nullptr;     // [n_params]
    double *W2T = nullptr;   // [width * width], W2T[j * w + k] = W2[k * w + j]
    float *pf = nullptr;     // FP32 copies for the mixed-precision kernel
    float *W2Tf = nullptr;
};

struct MatConst {
    double mu_e, lambda_e, eta_d, kappa_d, beta_d, c_d, gamma_d;
    double qcoef;            // gamma_d * beta_d / eta_d (0 when gamma_d or beta_d is 0)
    int energy;
    int local_max;
};

struct AsmArgs {
    int64_t n_elems;
    const int32_t *conn;
    const double *X;
    const double *dofs;
    const double *kappa_n;
    double *R;               // may be null
    double *Rabs;            // may be null (mixed kernels): per dof, the summed magnitudes of the terms of
                             // the element residual rows (the scale of their FP32 rounding)
    double *vals;            // FP64 values (may be null)
    float *vals32;           // FP32 values (mixed mode, may be null)
    double *kappa_new;       // may be null
    const double *kappa_guess;   // may be null: a nearby solution of the local update (the last Newton
                                 // iterate's kappa), where the local solve starts
    const double *kappa_fixed;   // may be null: a frozen history (staggered scheme): every point takes
                                 // this kappa, no local update and no kappa sensitivity in the tangent
    int8_t *loading;         // may be null
    const int32_t *slot;     // [E * nen * nen] CSR position of (row node a dof 0, col node b dof 0)
    const int32_t *rowptr;   // [n_dofs + 1]
    DevNet psi, yld;
    const NetConst *netc;    // [n_spec]
    MatConst mat;
    int tangent;
    int *counters;           // [0] local-solve failures, [1] loading points, [2] yield-network evaluations
    // batched specimens (null for a single specimen): specimen of every element and
    // the per-specimen networks; netc is then indexed by specimen
    const int32_t *elem_spec;
    const DevNet *psi_tab, *yld_tab;
    int wmax;                // widest network over all specimens
};

// adjoint element kernel (gd_adjoint.cu)
struct AdjArgs {
    int64_t n_elems;
    const int32_t *conn;
    const double *X;
    const double *dofs;        // d_n
    const double *kappa_prev;  // kappa_{n-1}
    const double *kappa_cur;   // kappa_n
    const double *w;           // nodal adjoint weights (mode 1)
    const double *kbar;        // dL/dkappa_n
    double *kbar_prev;         // out (mode 1): dL/dkappa_{n-1}
    double *rhs;               // out (mode 0): (dkappa/dd)^T kbar, accumulated
    double *theta_bar;         // out (mode 1): packed [psi | yield] gradient, accumulated
    double *glob;              // out (mode 1): weights of N(0), n, N_k(0), N_k'(0), accumulated
    DevNet psi, yld;
    const NetConst *netc;
    MatConst mat;
    int mode;
};

// a stored state of the load path (for the adjoint's recomputation)
struct Checkpoint {
    int commit = 0;                 // number of commits before this state
    double *dofs = nullptr, *dofs_prev = nullptr, *kappa = nullptr;
    double load_prev = 0.0, load_prevprev = 0.0;
    bool have_prev = false;
};

// Tensor-core element kernel (gd_asm_tc.cu): byte layout of the per-handle weight
// blob that every CTA copies into shared memory: the layer-2 tiles of both networks
// in the canonical K-major BF16 layout (energy W2 for the forward columns, W2^T for
// the reverse column, yield V2; with split operands each tile is followed by its
// residual tile), then FP32 vectors (energy W1 b1 A2 b2 w3 a3, yield V1 c1 B2 c2 v3 b3).
struct TcLayout {
    int we = 0, wy = 0;          // widths (0: no network)
    int wpe = 0, wpy = 0;        // widths padded to 16
    int split = 0;               // 1: high and residual BF16 parts (three products)
    int off_w2f = 0, off_w2r = 0, off_v2f = 0, off_e32 = 0, off_y32 = 0;
    int bytes = 0;               // multiple of 16
};
struct TcArgs {
    TcLayout L;
    const uint8_t *blob;
    int *status;                 // set to 1 when a bounded wait gave up
    float tol_r, tol_br;         // local-solve stopping tests (residual, bracket) relative to max(1, kappa)
    int ncols;                   // tensor-memory columns per CTA
    int tiles_off, tile_bytes, warp_off, warp_floats, bar_off;   // shared-memory layout
    // weights in shared memory: W2 at 0 (fwd_bytes), one slot (slot_bytes) at s_slot for
    // W2^T or V2, the FP32 vectors at s_e32 / s_y32 (vec_bytes from the blob's off_e32)
    int fwd_bytes, rev_bytes, v2_bytes, s_slot, slot_bytes, s_e32, s_y32, vec_bytes;
    int slot_mode;               // 0: none, 1: W2^T resident, 2: V2 resident, 3: W2^T then V2 per batch
};
struct TcLaunch {
    TcLayout L;
    const uint8_t *blob = nullptr;
    int *status = nullptr;
    int grid_max = 0;
};
TcLayout tc_layout(int we, int wy, bool split);
cudaError_t tc_build_blob(const DevNet &psi, const DevNet &yld, const TcLayout &L, uint8_t *blob, cudaStream_t s);
cudaError_t launch_assemble_tc(int dim, const AsmArgs &a, const TcLaunch &c, cudaStream_t s);

// launch shape of the element kernels (chosen by gd_autotune): warps per CTA
// (2, 4 or 8) and a cap on resident CTAs per SM for the persistent grid (0: none)
struct AsmTune {
    int warps = 4;
    int cta_per_sm = 0;
    bool exact = false;      // true: fail instead of falling back to a narrower CTA that fits
    int grid_max = 0;        // cap on the persistent grid's CTAs (gd_options.asm_grid_max; 0: none)
};
// Batched specimens: the Krylov grid's blocks take contiguous node chunks and
// every specimen runs its own BiCGStab recurrences (own scalars, own stopping
// test) inside one cooperative launch.
constexpr int kMaxSpecPerBlock = 32;
struct BatchKrylov {
    const int32_t *node_spec = nullptr;   // [n_nodes] specimen of every node
    const int32_t *blk_fs = nullptr;      // [blocks] first specimen overlapping block b
    const int32_t *blk_ns = nullptr;      // [blocks] specimens overlapping block b (<= kMaxSpecPerBlock)
    const int32_t *spec_b0 = nullptr;     // [n_spec] first block overlapping specimen s
    const int32_t *spec_b1 = nullptr;     // [n_spec] last block overlapping specimen s
    const double *rtol = nullptr;         // [n_spec] relative tolerance of every specimen
    int *active_cnt = nullptr;            // [2] device counters (zeroed by the launcher)
    double *red = nullptr;                // [5][blocks][J] block partials
    double *out = nullptr;                // [n_spec][3] iterations, relative residual, status
    int64_t chunk = 0;                    // nodes per block
    int J = 0;                            // max specimens per block
    int n_spec = 0;
};
// Two-level preconditioner (gd_coarse.cu): aggregation coarse space of the node
// graph, M^-1 = D^-1 + P Ac^-1 P^T with Ac = P^T A P.
constexpr int kCoarseMax = 3072;     // most coarse unknowns (the inversion keeps 16 rows of them in shared memory)
struct CoarseSpace {
    int nm = 0;                   // basis slots per aggregate: ndof constants + rotations (4 in 2D, 7 in 3D)
    int n_agg = 0;
    int nc = 0;                   // coarse unknowns (the kept basis columns of all aggregates)
    int32_t *agg = nullptr;       // [n_nodes] aggregate of every node
    int32_t *coff = nullptr;      // [n_agg + 1] first coarse unknown of every aggregate
    int32_t *node_co = nullptr;   // [n_nodes] 8 x first coarse unknown + count of the node's aggregate
    float *P = nullptr;           // [n_nodes][ndof][nm] basis values (zero beyond the kept columns)
    double *Ac = nullptr;         // [nc][nc] Galerkin matrix
    float *X32 = nullptr;         // [nc][nc] its inverse
    double *X64 = nullptr;        // [nc][nc] the same values in FP64
    double *rc = nullptr;         // [2][nc] restriction sums (FP32 solves use them as float storage)
    double *cc = nullptr;         // [nc] coarse solution (likewise)
    int *status = nullptr;        // device: 0 when X holds the inverse
};
struct Handle {
    // sizes
    int dim = 0, nen = 0, nq = 0, ndof = 0;
    int64_t n_nodes = 0, n_elems = 0, n_dofs = 0, nnz = 0;
    // device mesh and pattern
    double *X = nullptr;
    int32_t *conn = nullptr;
    int32_t *slot = nullptr;
    int32_t *rowptr = nullptr;
    int32_t *colidx = nullptr;
    uint8_t *fixed = nullptr;        // [n_dofs] 1 = prescribed
    int32_t *bc_dof = nullptr;
    double *bc_scale = nullptr;
    int64_t n_bc = 0;
    int32_t *react_dof = nullptr;
    int64_t n_react = 0;
    // host copies of the pattern (for gd_csr_pattern)
    std::vector<int32_t> h_rowptr, h_colidx;
    // constitutive data
    DevNet psi, yld;
    NetConst *netc = nullptr;                            // [n_spec]
    MatConst mat{};
    // batched specimens
    int n_spec = 1;
    int wmax = 0;
    int32_t *elem_spec = nullptr;                        // [n_elems] (null: one specimen)
    DevNet *psi_tab = nullptr, *yld_tab = nullptr;       // [n_spec] device tables
    std::vector<DevNet> h_psi_tab, h_yld_tab;            // host copies (own the parameter buffers)
    std::vector<std::vector<double>> paths;              // per-specimen load paths
    int n_steps_max = 0;
    int32_t *node_spec = nullptr, *bc_spec = nullptr;    // [n_nodes], [n_bc] (batches only)
    int64_t *react_off = nullptr;                        // [n_spec + 1] device (batches only)
    int64_t *node_off = nullptr;                         // [n_spec + 1] device (batches only)
    std::vector<int64_t> h_node_off, h_elem_off;         // [n_spec + 1]
    std::vector<int64_t> spec_nbc;                       // prescribed dofs per specimen
    double *d_load = nullptr;                            // [2 n_spec] device loads / reactions (batches only)
    double *d_pw = nullptr;                              // [3 n_spec] predictor weights (batches only)
    double *d_norm = nullptr, *d_coef = nullptr;         // [2 n_spec], [n_spec] device (batches only)
    // per-specimen Krylov layout (batches whose specimens are not too small for the grid)
    bool bk_ok = false;
    BatchKrylov bk;
    int32_t *bk_i32 = nullptr;                           // device storage of the layout arrays
    double *bk_f64 = nullptr;
    int *bk_cnt = nullptr;
    std::vector<double> bk_out;                          // host copy of the per-specimen results
    std::vector<double> last_reac;                       // per-specimen reactions of the last commit
    gd_options opt{};
    cudaStream_t stream = nullptr;
    std::vector<double> load;
    // state
    double *dofs = nullptr, *kappa = nullptr;            // committed
    double *dofs_prev = nullptr;                         // state before the last committed step
    double load_prev = 0.0, load_prevprev = 0.0;         // step coordinates t of the last two commits
    bool have_prev = false;
    // the state before dofs_prev and its step coordinate (quadratic predictor)
    double *dofs_pp = nullptr;
    double load_ppp = 0.0;
    bool have_pp = false;
    int next_step = 0;
    // work arrays
    double *w_dofs = nullptr, *w_trial = nullptr;
    double *R = nullptr, *R_trial = nullptr;
    double *Rabs = nullptr;                              // GD_MIXED: sum of |element residual rows| (noise scale)
    double *vals = nullptr, *vals_trial = nullptr;       // FP64 (or FP32 bit storage in mixed mode)
    double *kappa_trial = nullptr, *kappa_trial2 = nullptr;
    int8_t *loading = nullptr, *loading2 = nullptr;
    int *counters = nullptr;                             // device [8]
    // Krylov workspace (FP64 vectors of n_dofs)
    double *kv[11] = {};                                 // Krylov: 0..7 and 10; Newton: 8, 9
    double *diag = nullptr;
    double *binv = nullptr;                              // node-block Jacobi inverses
    float *vals_f32 = nullptr;                           // FP32 tangent copy for the inner solve (FP64 mode)
    double *kx = nullptr;                                // FP32 iterate storage
    int krylov_grid = 0;
    int krylov_grid32 = 0;                               // single-system solves with FP32 vectors
    double *red = nullptr;                               // device reduction buffers
    double *scal = nullptr;                              // device scalars
    int red_blocks = 0;
    // launch shapes (gd_autotune)
    AsmTune asm_tune;
    int krylov_cpsm = 2;
    int krylov_cpsm32 = 4;
    // GD_MIXED: measured FP32 residual noise per unit force scale, and load steps until
    // it is measured again
    std::vector<double> noise_ratio;
    int noise_age = 0;
    int krylov_up = 0;                                   // 0: the precision's default
    int krylov_lanes = 0;                                // 3D FP32 solves: lanes per node (0: 32)
    double *gm_ws = nullptr;                             // GMRES work space (allocated on first use)
    double *gm_binv = nullptr;                           // its node-block inverses (FP64)
    long long gmres_iterations = 0;                      // GMRES iterations run by this handle
    long long noise_passes = 0;                          // GD_MIXED FP64 reference passes run
    double noise_ms = 0.0;                               // their device time
    double last_noise = 0.0;                             // noise level of the last Newton test
    int krylov_lmax = 0;                                 // longest CSR row
    CoarseSpace coarse;                                  // two-level preconditioner (nc = 0: off)
    // tensor-core networks of the mixed element kernel (icnn_mma): mode and weight blob
    int icnn_mode = 0;                                   // GD_ICNN_CUDA_CORES, GD_ICNN_BF16 or GD_ICNN_BF16X3
    TcLayout tc;
    uint8_t *tc_blob = nullptr;
    // staggered scheme: the frozen history of the current equilibrium solve (null: none)
    // and its storage
    const double *kappa_fix = nullptr;
    double *kappa_stag = nullptr;
    // reuse of the coarse inverse across solves: solves since it was computed (-1: none
    // valid), the kind of matrix it belongs to, and the convergence rate of that solve
    int coarse_age = -1, coarse_kind = -1;
    double coarse_rate = 0.0;
    // timing
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, kv0 = nullptr, kv1 = nullptr;
    double assembly_ms = 0.0, krylov_ms = 0.0;
    int assemblies = 0;
    long long launches = 0;                              // kernels launched by this handle
    // record of the forward path for the adjoint
    bool rec_on = false;
    bool replaying = false;
    int rec_start_step = 0;
    std::vector<double> rec_load;                        // load of every commit
    std::vector<int> rec_step;                           // path step finished by the commit, or -1
    std::vector<Checkpoint> ckpts;
    // adjoint work space (allocated by the first gd_backward)
    int32_t *perm_T = nullptr;
    // GD_MIXED adjoint: FP64 tangent of the FP64 element kernel at the mixed path's states,
    // and the switch that makes the solvers read FP64 values in a mixed handle
    double *vals64 = nullptr;
    bool adj_fp64 = false;
    double *vals_T = nullptr, *adj_v[6] = {}, *kbar = nullptr, *kbar2 = nullptr, *theta_bar = nullptr,
           *glob = nullptr, *seg = nullptr;
    int seg_cap = 0;
    std::string err;
    int num_sms = 0;
};

// records a message for gd_last_error(NULL) on this thread and returns st
gd_status set_error(gd_status st, const std::string &msg);

// launchers (return the launch status)
cudaError_t launch_prep_nets(const DevNet &psi, const DevNet &yld, int energy, NetConst *out, cudaStream_t s);
cudaError_t launch_transpose(const DevNet &net, cudaStream_t s);
cudaError_t launch_assemble_fp64(int dim, const AsmArgs &a, int num_sms, cudaStream_t s, const AsmTune &t = AsmTune());
cudaError_t launch_assemble_fp32(int dim, const AsmArgs &a, int num_sms, cudaStream_t s, const AsmTune &t = AsmTune());
cudaError_t launch_adjoint(int dim, const AdjArgs &a, int num_sms, cudaStream_t s);
cudaError_t launch_adjoint_globals(const DevNet &psi, const DevNet &yld, int energy, const double *glob,
                                   double *theta_bar, cudaStream_t s);
// FP32 copies of a network's parameters and transposed W2
cudaError_t launch_net_to_float(const DevNet &net, cudaStream_t s);

// solver kernels (gd_solver.cu)
struct SolverCtx {
    int64_t n;                  // rows
    int64_t n_nodes;
    int ndof;
    const int32_t *rowptr;
    const int32_t *colidx;
    const double *vals;
    const float *vals32 = nullptr;  // FP32 values (mixed mode); used instead of vals when set
    const uint8_t *fixed;
    cudaStream_t stream;
    double *red;                // [2 * blocks * 4]
    double *scal;               // [64]
    int blocks;
    long long *launches;        // host counter of kernel launches (may be null)
};
// y = A x; free_only: prescribed rows copy x, prescribed columns skipped
cudaError_t launch_spmv(const SolverCtx &c, const double *x, double *y, int free_only);
// Solves A x = b on the free dofs (A = vals with prescribed rows/cols removed);
// x is overwritten; returns iterations (>= 0) or -1 on breakdown / cap.
cudaError_t launch_norm2_free(const SolverCtx &c, const double *v, double *out_dev, double *out_fixed_dev);
cudaError_t launch_axpy_free(const SolverCtx &c, double *y, const double *x, double alpha);
// r = b - y on free dofs (0 on prescribed), *out_norm = ||r|| (device)
cudaError_t launch_residual(const SolverCtx &c, const double *b, const double *y, double *r, double *out_norm);
cudaError_t launch_predictor(int64_t n, double *out, const double *cur, const double *prev, double factor,
                             const int32_t *bc_dof, const double *bc_scale, int64_t n_bc, double load,
                             cudaStream_t s);
// out = w0 x0 + w1 x1 + w2 x2, then the prescribed dofs set to bc_scale * load
cudaError_t launch_predictor3(int64_t n, double *out, const double *x0, const double *x1, const double *x2,
                              const double (&w)[3], const int32_t *bc_dof, const double *bc_scale, int64_t n_bc,
                              double load, cudaStream_t s);
cudaError_t launch_reaction(const double *R, const int32_t *react_dof, int64_t n_react, double *out,
                            cudaStream_t s);
cudaError_t launch_gather(const double *in, const int32_t *perm, double *out, int64_t n, cudaStream_t s);
// out = w0 cur + w1 prev + w2 pp per specimen (w [3 n_spec]), then the prescribed dofs
cudaError_t launch_predictor_batch(int64_t n, int ndof, double *out, const double *cur, const double *prev,
                                   const double *pp, const double *w, const int32_t *node_spec, const int32_t *bc_dof,
                                   const double *bc_scale, const int32_t *bc_spec, const double *load, int64_t n_bc,
                                   cudaStream_t s);
cudaError_t launch_norms_batch(const double *R, const uint8_t *fixed, const int64_t *node_off, int ndof, int n_spec,
                               double *out, cudaStream_t s);
cudaError_t launch_scale_spec(int64_t n, int ndof, double *out, const double *in, const double *coef,
                              const int32_t *node_spec, const uint8_t *fixed, int accumulate, cudaStream_t s);
cudaError_t launch_fill(double *v, double val, int64_t n, cudaStream_t s);
cudaError_t launch_damage_field(const double *kappa, int64_t n, double eta_d, double kappa_d, double *out,
                                cudaStream_t s);
cudaError_t launch_reaction_batch(const double *R, const int32_t *react_dof, const int64_t *off, int n_spec,
                                  double *out, cudaStream_t s);
cudaError_t launch_adj_rhs(int64_t n, const double *sv, const double *y, double fbar, const uint8_t *fixed,
                           double *out, cudaStream_t s);
cudaError_t launch_axpby(int64_t n, double *out, const double *x, double b, const double *y, cudaStream_t s);
cudaError_t launch_damage_max(const double *kappa, int64_t n, double eta_d, double kappa_d, double *out,
                              cudaStream_t s);

int coarse_modes(int dim);
// greedy breadth-first aggregates of about `target` nodes over the node graph of
// the node-block CSR pattern; aggregates below target/4 join their smallest
// neighbour.  Returns the number of aggregates, agg[i] in [0, n).
int32_t coarse_aggregate(int64_t n_nodes, int ndof, const std::vector<int32_t> &rowptr,
                         const std::vector<int32_t> &colidx, int target, std::vector<int32_t> &agg);
// orthonormal basis per aggregate (constants per nodal unknown, rigid rotations of
// the displacement; zero on prescribed dofs); P [n_nodes][ndof][nm], coff [n_agg + 1]
void coarse_basis(int dim, int64_t n_nodes, const double *coords, const uint8_t *fixed,
                  const std::vector<int32_t> &agg, int32_t n_agg, std::vector<float> &P, std::vector<int32_t> &coff);
// Ac = P^T A P for the tangent values vals, X32 = Ac^-1 (and X64 when want_x64)
// lmax: the longest row (columns); rows up to 256 columns take the shared-memory kernel
cudaError_t coarse_setup(const CoarseSpace &cs, int ndof, int64_t n_nodes, const int32_t *rowptr,
                         const int32_t *colidx, const void *vals, bool fp32_vals, bool want_x64, int num_sms,
                         cudaStream_t s, int lmax = 0);

// persistent cooperative Krylov solve (gd_krylov.cu)
struct KrylovCtx {
    int64_t n_nodes;
    int ndof;
    const int32_t *rowptr, *colidx;
    const uint8_t *fixed;
    double *binv;               // [n_nodes * ndof * ndof]
    double *work[9];            // [n_nodes * ndof] each
    double *work_x;             // iterate when the vectors are FP32
    double *red;                // [8 * blocks]
    double *out;                // [3] device: iterations, relative residual, status
    cudaStream_t stream;
    int blocks;                 // cooperative grid size (all blocks co-resident)
    int num_sms;
    int up = 0;                 // node groups per product round: 1, 2 or 4 (0: 1)
    int lmax = 0;               // longest row (0: rows are not copied to shared memory)
    const CoarseSpace *coarse = nullptr;   // two-level preconditioner (single systems; null: Jacobi only)
    bool coarse_refresh = true;            // recompute P^T A P and its inverse before the solve
    int row_cache = 0;                     // gd_options.krylov_row_cache: 0 automatic, 1 column lists only, 2 none
    int lanes = 0;                         // lanes per node of the 3D FP32-vector solve: 4, 8 or 32 (0: 32)
};
cudaError_t krylov_solve_batch(const KrylovCtx &c, const BatchKrylov &L, const void *vals, bool fp32_vals,
                               const double *b, double *x, int max_it, bool fp32_vectors);
// cooperative grid of the Krylov kernels: SMs x co-resident CTAs per SM (at most cap)
int krylov_blocks(int ndof, bool fp32_vals, int num_sms, int cap = 2);
// the same for the single-system kernels with FP32 vectors (built for four CTAs per SM)
int krylov_blocks_fp32(int ndof, int num_sms, int cap = 4);
// Solves K x = b on the free dofs; the result and statistics land in x and c.out.
// fp32_vectors: the iteration runs on FP32 values and vectors (dot products stay FP64).
cudaError_t krylov_solve(const KrylovCtx &c, const void *vals, bool fp32_vals, const double *b, double *x,
                         double rtol, int max_it, bool fp32_vectors = false);
cudaError_t narrow_to_float(const double *in, float *out, int64_t n, cudaStream_t s);
// node-block inverses [n_nodes][ndof][ndof] of the eliminated matrix (identity on prescribed dofs)
cudaError_t launch_block_inverse(int ndof, int64_t n_nodes, const int32_t *rowptr, const int32_t *colidx,
                                 const void *vals, bool fp32_vals, const uint8_t *fixed, double *binv, int num_sms,
                                 cudaStream_t s);

// restarted, right-preconditioned GMRES(m) (gd_gmres.cu)
cudaError_t gmres_solve(const SolverCtx &c, const double *binv, const double *b, double *x, double rtol, int m,
                        int max_it, double *ws, int &iters, double &rel, bool &converged);
size_t gmres_workspace_doubles(int64_t n, int m, int nb);
int gmres_max_m();

}  // namespace gd
