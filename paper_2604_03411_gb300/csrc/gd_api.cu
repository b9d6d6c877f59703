// gd_api.cu -- C ABI of the library: handle creation (mesh validation, CSR
// pattern of the node graph, per-element slot map, Dirichlet masks, network
// staging), the assembly entry point and the device Newton iteration over the
// quasi-static load path (Sec. 3.2 of arxiv 2604.03411: monolithic scheme,
// warm start from the last converged step, incremental loading).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gd_internal.cuh"

struct gd_handle {
    gd::Handle h;
};

namespace {

thread_local std::string g_create_error;

gd_status fail(gd::Handle *H, gd_status st, const std::string &msg)
{
    if (H) H->err = msg;
    else g_create_error = msg;
    return st;
}

#define GD_CUDA(H, call)                                                                                   \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) {                                                                           \
            (void)cudaGetLastError(); /* consume a non-sticky error: it must not fail the next call */     \
            return fail((H), e_ == cudaErrorMemoryAllocation ? GD_ERR_OOM : GD_ERR_CUDA,                   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                               \
        }                                                                                                  \
    } while (0)

// counters[3] is set by the tensor-core element kernel when one of its bounded waits
// gave up (the kernel then frees its tensor memory and returns)
#define GD_TC_CHECK(H, hc)                                                                                 \
    do {                                                                                                   \
        if ((hc)[3]) return fail((H), GD_ERR_TIMEOUT, "tensor-core element kernel: a bounded wait gave up"); \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
}

void dfree(void *p)
{
    if (p) cudaFree(p);
}

// sign of node a along reference axis k (HEX8 node order; Q4 uses the first four)
double sgn(int a, int k)
{
    int b = (k == 0) ? ((a & 3) == 1 || (a & 3) == 2) : (k == 1 ? ((a & 3) >= 2) : (a >= 4));
    return b ? 1.0 : -1.0;
}

// det of dX/dxi at every Gauss point must be positive
bool element_ok(int dim, const double *Xe)
{
    const int nen = dim == 2 ? 4 : 8;
    const double g = 1.0 / std::sqrt(3.0);
    for (int q = 0; q < nen; ++q) {
        double xi[3] = {(q & 1) ? g : -g, (q & 2) ? g : -g, (q & 4) ? g : -g};
        double Jm[3][3] = {{0}};
        for (int a = 0; a < nen; ++a) {
            double f[3], dN[3];
            for (int k = 0; k < dim; ++k) f[k] = 0.5 * (1.0 + sgn(a, k) * xi[k]);
            for (int k = 0; k < dim; ++k) {
                double v = 0.5 * sgn(a, k);
                for (int l = 0; l < dim; ++l)
                    if (l != k) v *= f[l];
                dN[k] = v;
            }
            for (int J = 0; J < dim; ++J)
                for (int k = 0; k < dim; ++k) Jm[J][k] += Xe[a * dim + J] * dN[k];
        }
        double det = dim == 2 ? Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0]
                              : Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) -
                                    Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) +
                                    Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
        if (!(det > 0.0)) return false;
    }
    return true;
}

void free_ckpts(gd::Handle &H);

void free_handle(gd::Handle &H)
{
    void *ptrs[] = {H.X, H.conn, H.slot, H.rowptr, H.colidx, H.fixed, H.bc_dof, H.bc_scale, H.react_dof,
                    H.psi.p, H.psi.W2T, H.yld.p, H.yld.W2T, H.psi.pf, H.psi.W2Tf, H.yld.pf, H.yld.W2Tf, H.netc, H.dofs, H.kappa, H.dofs_prev, H.dofs_pp, H.w_dofs,
                    H.w_trial, H.R, H.R_trial, H.vals, H.vals_trial, H.kappa_trial, H.kappa_trial2, H.loading,
                    H.loading2, H.counters, H.diag, H.binv, H.vals_f32, H.kx, H.red, H.scal};
    for (void *p : ptrs) dfree(p);
    for (double *p : H.kv) dfree(p);
    free_ckpts(H);
    dfree(H.perm_T);
    dfree(H.vals_T);
    dfree(H.vals64);
    for (double *p : H.adj_v) dfree(p);
    dfree(H.kbar);
    dfree(H.kbar2);
    dfree(H.theta_bar);
    dfree(H.glob);
    dfree(H.seg);
    dfree(H.elem_spec);
    dfree(H.node_spec);
    dfree(H.bc_spec);
    dfree(H.react_off);
    dfree(H.node_off);
    dfree(H.d_load);
    dfree(H.d_norm);
    dfree(H.d_coef);
    dfree(H.d_pw);
    dfree(H.kappa_stag);
    dfree(H.bk_i32);
    dfree(H.bk_f64);
    dfree(H.bk_cnt);
    dfree(H.psi_tab);
    dfree(H.yld_tab);
    dfree(H.tc_blob);
    dfree(H.Rabs);
    dfree(H.gm_ws);
    dfree(H.gm_binv);
    {
        gd::CoarseSpace &c = H.coarse;
        void *cp[] = {c.agg, c.coff, c.node_co, c.P, c.Ac, c.X32, c.X64, c.rc, c.cc, c.status};
        for (void *p : cp) dfree(p);
    }
    for (gd::DevNet &n : H.h_psi_tab) {
        dfree(n.p); dfree(n.W2T); dfree(n.pf); dfree(n.W2Tf);
    }
    for (gd::DevNet &n : H.h_yld_tab) {
        dfree(n.p); dfree(n.W2T); dfree(n.pf); dfree(n.W2Tf);
    }
    if (H.ev0) cudaEventDestroy(H.ev0);
    if (H.ev1) cudaEventDestroy(H.ev1);
    if (H.kv0) cudaEventDestroy(H.kv0);
    if (H.kv1) cudaEventDestroy(H.kv1);
}

gd::SolverCtx solver_ctx(gd::Handle &H, const double *vals)
{
    gd::SolverCtx c;
    c.n = H.n_dofs;
    c.n_nodes = H.n_nodes;
    c.ndof = H.ndof;
    c.rowptr = H.rowptr;
    c.colidx = H.colidx;
    c.vals = vals;
    c.fixed = H.fixed;
    c.stream = H.stream;
    c.red = H.red;
    c.scal = H.scal;
    c.blocks = H.red_blocks;
    c.launches = &H.launches;
    return c;
}

gd::AsmArgs asm_args(gd::Handle &H, const double *dofs, const double *kappa_n, double *R, void *vals,
                     double *kappa_out, int8_t *loading, int tangent)
{
    gd::AsmArgs a;
    a.n_elems = H.n_elems;
    a.conn = H.conn;
    a.X = H.X;
    a.dofs = dofs;
    a.kappa_n = kappa_n;
    a.R = R;
    a.Rabs = nullptr;
    a.vals = (tangent && H.opt.precision == GD_FP64) ? (double *)vals : nullptr;
    a.vals32 = (tangent && H.opt.precision == GD_MIXED) ? (float *)vals : nullptr;
    a.kappa_new = kappa_out;
    a.kappa_guess = nullptr;
    a.kappa_fixed = H.kappa_fix;
    a.loading = loading;
    a.slot = H.slot;
    a.rowptr = H.rowptr;
    a.psi = H.psi;
    a.yld = H.yld;
    a.netc = H.netc;
    a.mat = H.mat;
    a.tangent = tangent && vals != nullptr;
    a.counters = H.counters;
    a.elem_spec = H.elem_spec;
    a.psi_tab = H.psi_tab;
    a.yld_tab = H.yld_tab;
    a.wmax = H.wmax;
    return a;
}

// one assembly pass with timing; counters[0] = local failures, [1] = loading points
// guess: a nearby solution of the local updates (the current Newton iterate's kappa),
// where the local solves of the loading points start; null: at kappa_n
gd_status assemble_pass(gd::Handle &H, const double *dofs, const double *kappa_n, double *R, void *vals,
                        double *kappa_out, int8_t *loading, int tangent, bool force_fp64 = false,
                        const double *guess = nullptr, double *rabs = nullptr)
{
    const size_t vbytes = H.opt.precision == GD_FP64 ? sizeof(double) : sizeof(float);
    if (force_fp64) tangent = 0;
    if (R) GD_CUDA(&H, cudaMemsetAsync(R, 0, sizeof(double) * H.n_dofs, H.stream));
    if (tangent && vals) GD_CUDA(&H, cudaMemsetAsync(vals, 0, vbytes * H.nnz, H.stream));
    GD_CUDA(&H, cudaMemsetAsync(H.counters, 0, sizeof(int) * 8, H.stream));
    GD_CUDA(&H, cudaEventRecord(H.ev0, H.stream));
    gd::AsmArgs a = asm_args(H, dofs, kappa_n, R, vals, kappa_out, loading, tangent);
    a.kappa_guess = guess;
    if (rabs && !force_fp64 && H.opt.precision == GD_MIXED) {
        GD_CUDA(&H, cudaMemsetAsync(rabs, 0, sizeof(double) * H.n_dofs, H.stream));
        a.Rabs = rabs;
    }
    if (H.opt.precision == GD_FP64 || force_fp64) {
        GD_CUDA(&H, gd::launch_assemble_fp64(H.dim, a, H.num_sms, H.stream, H.asm_tune));
    } else if (H.icnn_mode == GD_ICNN_BF16 || H.icnn_mode == GD_ICNN_BF16X3) {
        gd::TcLaunch c;
        c.L = H.tc;
        c.blob = H.tc_blob;
        c.status = H.counters + 3;
        c.grid_max = H.asm_tune.grid_max;
        GD_CUDA(&H, gd::launch_assemble_tc(H.dim, a, c, H.stream));
    } else {
        GD_CUDA(&H, gd::launch_assemble_fp32(H.dim, a, H.num_sms, H.stream, H.asm_tune));
    }
    ++H.launches;
    GD_CUDA(&H, cudaEventRecord(H.ev1, H.stream));
    ++H.assemblies;
    return GD_OK;
}

// FP64 residual and tangent of the FP64 element kernel into vals64 (FP64 values in
// the handle's pattern), whatever the handle's precision: the adjoint of a GD_MIXED path
gd_status assemble_tangent_fp64(gd::Handle &H, const double *dofs, const double *kappa_n, double *R, double *vals64,
                                double *kappa_out, int8_t *loading)
{
    GD_CUDA(&H, cudaMemsetAsync(R, 0, sizeof(double) * H.n_dofs, H.stream));
    GD_CUDA(&H, cudaMemsetAsync(vals64, 0, sizeof(double) * H.nnz, H.stream));
    GD_CUDA(&H, cudaMemsetAsync(H.counters, 0, sizeof(int) * 8, H.stream));
    GD_CUDA(&H, cudaEventRecord(H.ev0, H.stream));
    gd::AsmArgs a = asm_args(H, dofs, kappa_n, R, nullptr, kappa_out, loading, 0);
    a.vals = vals64;
    a.vals32 = nullptr;
    a.tangent = 1;
    GD_CUDA(&H, gd::launch_assemble_fp64(H.dim, a, H.num_sms, H.stream, H.asm_tune));
    ++H.launches;
    GD_CUDA(&H, cudaEventRecord(H.ev1, H.stream));
    ++H.assemblies;
    return GD_OK;
}

double elapsed_ms(gd::Handle &H)
{
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, H.ev0, H.ev1) != cudaSuccess) return 0.0;
    return ms;
}

struct NormPair {
    double free_, fixed_;
};

gd_status norms(gd::Handle &H, const double *R, NormPair &out)
{
    gd::SolverCtx c = solver_ctx(H, nullptr);
    GD_CUDA(&H, gd::launch_norm2_free(c, R, H.scal + 16, H.scal + 17));
    double h[2];
    GD_CUDA(&H, cudaMemcpyAsync(h, H.scal + 16, 2 * sizeof(double), cudaMemcpyDeviceToHost, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    out.free_ = h[0];
    out.fixed_ = h[1];
    return GD_OK;
}

// K x = b with the persistent Krylov kernel on `vals`; timing accumulated in H.krylov_ms
// accept: a solve that stops at its iteration cap or on a breakdown is still
// returned as GD_OK when its relative residual is at most `accept` (default: rtol,
// i.e. strict); a non-finite residual is always an error.
// The coarse inverse of the two-level preconditioner is kept for the next solves of
// the same kind of matrix (the Newton tangent changes little from one solve to the
// next, and a slightly stale coarse level is still a good one): it is recomputed
// after kCoarseReuse solves, for another kind of matrix, and as soon as a solve
// converges at under 0.7 times the rate (log reduction per iteration) of the solve
// that computed it.  kind: the Newton tangent, its transpose (adjoint), or a
// caller's matrix (always recomputed, and not kept).
constexpr int kCoarseReuse = 8;
enum MatKind { kTangent = 0, kTransposed = 1, kCallerMatrix = 2 };

// FP64-vector GMRES(gmres_m) on `vals` (the handle's precision: FP64 values, or FP32
// values with FP64 vectors in GD_MIXED); work space allocated on first use.
gd_status gmres(gd::Handle &H, const void *vals, const double *b, double *x, int &iters, double &rel, double rtol,
                bool &converged)
{
    const bool fp32_vals = H.opt.precision == GD_MIXED && !H.adj_fp64;
    const int m = std::max(1, std::min(H.opt.gmres_m, gd::gmres_max_m()));
    gd::SolverCtx c = solver_ctx(H, nullptr);
    if (fp32_vals) c.vals32 = (const float *)vals;
    else c.vals = (const double *)vals;
    if (!H.gm_ws) {
        GD_CUDA(&H, dalloc(&H.gm_ws, gd::gmres_workspace_doubles(H.n_dofs, gd::gmres_max_m(), c.blocks)));
        GD_CUDA(&H, dalloc(&H.gm_binv, (size_t)H.n_nodes * H.ndof * H.ndof));
    }
    GD_CUDA(&H, gd::launch_block_inverse(H.ndof, H.n_nodes, H.rowptr, H.colidx, vals, fp32_vals, H.fixed, H.gm_binv,
                                         H.num_sms, H.stream));
    GD_CUDA(&H, gd::gmres_solve(c, H.gm_binv, b, x, rtol, m, H.opt.krylov_max, H.gm_ws, iters, rel, converged));
    H.gmres_iterations += iters;
    H.launches += 8 + 8LL * iters;
    return GD_OK;
}

gd_status krylov(gd::Handle &H, const void *vals, const double *b, double *x, int &iters, double &rel,
                 double rtol, bool inner_fp32 = false, double accept = -1.0, int kind = kTangent)
{
    if (H.opt.krylov == GD_GMRES && !inner_fp32) {
        // every FP64 solve by GMRES(m)
        GD_CUDA(&H, cudaEventRecord(H.kv0, H.stream));
        bool conv = false;
        gd_status st = gmres(H, vals, b, x, iters, rel, rtol, conv);
        if (st) return st;
        GD_CUDA(&H, cudaEventRecord(H.kv1, H.stream));
        GD_CUDA(&H, cudaEventSynchronize(H.kv1));
        float kms = 0.0f;
        cudaEventElapsedTime(&kms, H.kv0, H.kv1);
        H.krylov_ms += kms;
        if (!conv && !(std::isfinite(rel) && rel <= std::max(accept, rtol)))
            return fail(&H, GD_ERR_KRYLOV, "GMRES stopped at relative residual " + std::to_string(rel));
        return GD_OK;
    }
    gd::KrylovCtx kc;
    kc.n_nodes = H.n_nodes;
    kc.ndof = H.ndof;
    kc.rowptr = H.rowptr;
    kc.colidx = H.colidx;
    kc.fixed = H.fixed;
    kc.binv = H.binv;
    for (int k = 0; k < 8; ++k) kc.work[k] = H.kv[k];
    kc.work[8] = H.kv[10];
    kc.work_x = H.kx;
    kc.red = H.red;
    kc.out = H.scal + 24;
    kc.stream = H.stream;
    // the FP32-vector kernels run on a grid of their own (built for more CTAs per SM)
    kc.blocks = (inner_fp32 && H.krylov_grid32 > 0) ? H.krylov_grid32 : H.krylov_grid;
    kc.num_sms = H.num_sms;
    kc.up = H.krylov_up;
    kc.lmax = H.krylov_lmax;
    kc.row_cache = H.opt.krylov_row_cache;
    kc.lanes = H.krylov_lanes;
    kc.coarse = H.coarse.nc > 0 ? &H.coarse : nullptr;
    bool refresh =
        kind == kCallerMatrix || H.coarse_age < 0 || H.coarse_kind != kind || H.coarse_age >= kCoarseReuse;
    kc.coarse_refresh = refresh;
    GD_CUDA(&H, cudaEventRecord(H.kv0, H.stream));
    bool fp32_vals = H.opt.precision == GD_MIXED && !H.adj_fp64;
    if (inner_fp32 && !fp32_vals) {
        GD_CUDA(&H, gd::narrow_to_float((const double *)vals, H.vals_f32, H.nnz, H.stream));
        ++H.launches;
        vals = H.vals_f32;
        fp32_vals = true;
    }
    GD_CUDA(&H, gd::krylov_solve(kc, vals, fp32_vals, b, x, rtol, H.opt.krylov_max, inner_fp32));
    H.launches += kc.coarse ? 4 : 2;
    double kout[3];
    GD_CUDA(&H, cudaMemcpyAsync(kout, H.scal + 24, 3 * sizeof(double), cudaMemcpyDeviceToHost, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    if (kc.coarse && !refresh && kout[2] != 0.0) {
        // a reused coarse inverse (from another state of the path) may no longer fit:
        // recompute it and solve again
        kc.coarse_refresh = true;
        refresh = true;
        GD_CUDA(&H, gd::krylov_solve(kc, vals, fp32_vals, b, x, rtol, H.opt.krylov_max, inner_fp32));
        H.launches += 4;
        GD_CUDA(&H, cudaMemcpyAsync(kout, H.scal + 24, 3 * sizeof(double), cudaMemcpyDeviceToHost, H.stream));
        GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    }
    GD_CUDA(&H, cudaEventRecord(H.kv1, H.stream));
    GD_CUDA(&H, cudaEventSynchronize(H.kv1));
    float kms = 0.0f;
    cudaEventElapsedTime(&kms, H.kv0, H.kv1);
    H.krylov_ms += kms;
    iters = (int)kout[0];
    rel = kout[1];
    if (kc.coarse) {
        const double rate = (iters > 0 && rel > 0.0 && std::isfinite(rel)) ? -std::log(rel) / iters : 0.0;
        if (kind == kCallerMatrix) {
            H.coarse_age = -1;
        } else if (refresh) {
            H.coarse_age = 1;
            H.coarse_kind = kind;
            H.coarse_rate = rate;
        } else {
            ++H.coarse_age;
            if (rate < 0.7 * H.coarse_rate) H.coarse_age = -1;
        }
    }
    if (kout[2] != 0.0 && !(kout[2] != 2.0 && std::isfinite(rel) && rel <= std::max(accept, rtol))) {
        if (!inner_fp32) {
            // an FP64 solve that BiCGStab did not finish (breakdown, stagnation, the
            // iteration cap): GMRES(m) from zero, which minimises the residual and
            // cannot break down before convergence
            int git = 0;
            double grel = 1.0;
            bool conv = false;
            gd_status st = gmres(H, vals, b, x, git, grel, rtol, conv);
            if (st) return st;
            iters += git;
            if (conv || (std::isfinite(grel) && grel <= std::max(accept, rtol))) {
                rel = grel;
                return GD_OK;
            }
        }
        return fail(&H, GD_ERR_KRYLOV, "BiCGStab stopped (status " + std::to_string((int)kout[2]) +
                                           ", relative residual " + std::to_string(rel) + ")");
    }
    return GD_OK;
}

// K x = b to relative tolerance eta by mixed-precision iterative refinement:
// FP32 BiCGStab cycles on the FP32 tangent copy, each followed by the FP64
// residual r = b - K x with the FP64 tangent (GB300's FP64 rate makes the FP32
// iteration several times cheaper, and the FP64 residual keeps the result at
// FP64 accuracy).  Returns GD_ERR_KRYLOV when a cycle breaks down.
gd_status krylov_refined(gd::Handle &H, const double *b, double *x, double eta, int &iters, double &rel)
{
    gd::SolverCtx c = solver_ctx(H, H.vals);
    // scratch: residual in R_trial, correction in w_trial (both rewritten by the line search after the solve)
    double *res = H.R_trial, *dx = H.w_trial, *y = H.diag;
    GD_CUDA(&H, cudaMemsetAsync(x, 0, sizeof(double) * H.n_dofs, H.stream));
    GD_CUDA(&H, cudaMemcpyAsync(res, b, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToDevice, H.stream));
    double bn = 0.0, rn = 0.0;
    {
        GD_CUDA(&H, gd::launch_norm2_free(c, b, H.scal + 30, nullptr));
        GD_CUDA(&H, cudaMemcpyAsync(&bn, H.scal + 30, sizeof(double), cudaMemcpyDeviceToHost, H.stream));
        GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    }
    iters = 0;
    rel = 1.0;
    if (bn == 0.0) {
        rel = 0.0;
        return GD_OK;
    }
    for (int cycle = 0; cycle < 12; ++cycle) {
        int kit = 0;
        double krel = 0.0;
        // each cycle reduces the FP64 residual by about the FP32 solve's tolerance
        const double inner = std::max(1e-4, std::min(1e-2, 0.5 * eta * bn / std::max(rn > 0.0 ? rn : bn, 1e-300)));
        gd_status st = krylov(H, H.vals, res, dx, kit, krel, inner, true, 0.5);
        iters += kit;
        if (st) return st;
        GD_CUDA(&H, gd::launch_axpy_free(c, x, dx, 1.0));
        GD_CUDA(&H, gd::launch_spmv(c, x, y, 1));
        GD_CUDA(&H, gd::launch_residual(c, b, y, res, H.scal + 31));
        H.launches += 1;
        GD_CUDA(&H, cudaMemcpyAsync(&rn, H.scal + 31, sizeof(double), cudaMemcpyDeviceToHost, H.stream));
        GD_CUDA(&H, cudaStreamSynchronize(H.stream));
        rel = rn / bn;
        if (!std::isfinite(rel)) return fail(&H, GD_ERR_KRYLOV, "refined solve produced a non-finite residual");
        if (rel <= eta) return GD_OK;
    }
    return fail(&H, GD_ERR_KRYLOV, "refined solve did not reach its tolerance");
}

// Newton direction K delta = rhs to relative tolerance eta (policy: gd_options.inner_solve).
// GD_MIXED solves directions that need at most 1e-5 relative accuracy with FP32
// values and vectors (FP64 dot products); GD_INNER_REFINED refines FP32 cycles by
// FP64 residuals; any FP32 solve that breaks down falls back to the FP64 solve.  The
// FP64 residual of the assembly decides convergence, so FP64 parity is unaffected.
gd_status solve_direction(gd::Handle &H, const double *rhs, double *delta, double eta, gd_newton_report &rep)
{
    int kit = 0;
    double rel = 0.0;
    gd_status st = GD_ERR_KRYLOV;
    if (H.opt.inner_solve != GD_INNER_FP64) {
        if (H.opt.inner_solve == GD_INNER_REFINED) {
            st = krylov_refined(H, rhs, delta, eta, kit, rel);
        } else if (H.opt.precision == GD_MIXED && eta >= 1e-5) {
            st = krylov(H, H.vals, rhs, delta, kit, rel, eta, true, 0.1);
        }
        rep.krylov_iterations += kit;
        rep.krylov_fp32_iterations += kit;
    }
    if (st) {
        // an FP64 solve that stalls (iteration cap, breakdown) after a tenfold reduction
        // still gives a descent direction for the line search: inexact Newton
        st = krylov(H, H.vals, rhs, delta, kit, rel, eta, false, 0.1);
        rep.krylov_iterations += kit;
    }
    return st;
}

gd_status norms_batch(gd::Handle &H, const double *R, std::vector<double> &nf, std::vector<double> &nx);

// FP64 solve whose TRUE relative residual ||b - K x|| / ||b|| (free dofs) reaches
// rtol: the recursively updated BiCGStab residual drifts from the true one by
// rounding, so the true residual is formed after each solve and corrected by
// further solves (at most four).  vals are FP64 values on the handle's pattern.
gd_status krylov_true(gd::Handle &H, const double *vals, const double *b, double *x, double rtol)
{
    gd::SolverCtx c = solver_ctx(H, vals);
    double *res = H.R_trial, *dx = H.kv[8], *y = H.diag;
    int kit = 0;
    double rel = 0.0;
    const int kind = vals == H.vals_T ? kTransposed : kTangent;
    gd_status st = krylov(H, vals, b, x, kit, rel, rtol, false, std::max(rtol, 1e-10), kind);
    if (st) return st;
    double bn = 0.0;
    GD_CUDA(&H, gd::launch_norm2_free(c, b, H.scal + 30, nullptr));
    GD_CUDA(&H, cudaMemcpyAsync(&bn, H.scal + 30, sizeof(double), cudaMemcpyDeviceToHost, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    if (bn == 0.0) return GD_OK;
    for (int pass = 0; pass < 4; ++pass) {
        GD_CUDA(&H, gd::launch_spmv(c, x, y, 1));
        GD_CUDA(&H, gd::launch_residual(c, b, y, res, H.scal + 31));
        H.launches += 1;
        double rn = 0.0;
        GD_CUDA(&H, cudaMemcpyAsync(&rn, H.scal + 31, sizeof(double), cudaMemcpyDeviceToHost, H.stream));
        GD_CUDA(&H, cudaStreamSynchronize(H.stream));
        if (!std::isfinite(rn)) return fail(&H, GD_ERR_NAN, "non-finite residual in a refined solve");
        if (rn <= std::max(rtol, 1e-15) * bn) return GD_OK;
        st = krylov(H, vals, res, dx, kit, rel, std::max(rtol * bn / rn, 1e-13), false, 0.5, kind);
        if (st) return st;
        GD_CUDA(&H, gd::launch_axpy_free(c, x, dx, 1.0));
    }
    return GD_OK;       // best effort: the last correction was applied
}

// Per-specimen BiCGStab on the batch system: specimen s stops at ||r_s|| <=
// eta[s] ||b_s||.  iters = the largest count over the specimens.
gd_status krylov_batch(gd::Handle &H, const std::vector<double> &eta, const double *b, double *x, int &iters,
                       bool inner_fp32, double accept)
{
    gd::KrylovCtx kc;
    kc.n_nodes = H.n_nodes;
    kc.ndof = H.ndof;
    kc.rowptr = H.rowptr;
    kc.colidx = H.colidx;
    kc.fixed = H.fixed;
    kc.binv = H.binv;
    for (int k = 0; k < 8; ++k) kc.work[k] = H.kv[k];
    kc.work[8] = H.kv[10];
    kc.work_x = H.kx;
    kc.red = H.red;
    kc.out = H.scal + 24;
    kc.stream = H.stream;
    kc.blocks = H.krylov_grid;
    kc.num_sms = H.num_sms;
    kc.up = H.krylov_up;
    kc.lmax = H.krylov_lmax;
    const int S = H.n_spec;
    GD_CUDA(&H, cudaMemcpyAsync((void *)H.bk.rtol, eta.data(), sizeof(double) * S, cudaMemcpyHostToDevice, H.stream));
    GD_CUDA(&H, cudaEventRecord(H.kv0, H.stream));
    const void *vals = H.vals;
    bool fp32_vals = H.opt.precision == GD_MIXED && !H.adj_fp64;
    if (inner_fp32 && !fp32_vals) {
        GD_CUDA(&H, gd::narrow_to_float((const double *)vals, H.vals_f32, H.nnz, H.stream));
        ++H.launches;
        vals = H.vals_f32;
        fp32_vals = true;
    }
    GD_CUDA(&H, gd::krylov_solve_batch(kc, H.bk, vals, fp32_vals, b, x, H.opt.krylov_max, inner_fp32));
    H.launches += 2;
    GD_CUDA(&H, cudaEventRecord(H.kv1, H.stream));
    H.bk_out.resize((size_t)3 * S);
    GD_CUDA(&H, cudaMemcpyAsync(H.bk_out.data(), H.bk.out, sizeof(double) * 3 * S, cudaMemcpyDeviceToHost, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    float kms = 0.0f;
    cudaEventElapsedTime(&kms, H.kv0, H.kv1);
    H.krylov_ms += kms;
    iters = 0;
    for (int s = 0; s < S; ++s) {
        if (eta[s] < 0.0) continue;                   // skipped specimen
        iters = std::max(iters, (int)H.bk_out[3 * s]);
        const double rel = H.bk_out[3 * s + 1], status = H.bk_out[3 * s + 2];
        if (status != 0.0 && !(status != 2.0 && std::isfinite(rel) && rel <= std::max(accept, eta[s])))
            return fail(&H, GD_ERR_KRYLOV, "BiCGStab of specimen " + std::to_string(s) + " stopped (status " +
                                               std::to_string((int)status) + ", relative residual " +
                                               std::to_string(rel) + ")");
    }
    return GD_OK;
}

// Newton directions of a batch with per-specimen tolerances (policy as solve_direction):
// in GD_MIXED the specimens whose tolerance allows it are solved in FP32 first, and
// only the specimens that need it (tighter tolerance, or an FP32 solve that did not
// reach a tenfold reduction) are then solved in FP64, the others kept as they are.
gd_status solve_direction_batch(gd::Handle &H, const double *rhs, double *delta, const std::vector<double> &eta,
                                gd_newton_report &rep)
{
    const int S = H.n_spec;
    int kit = 0;
    std::vector<double> todo = eta;
    bool any64 = true;
    if (H.opt.inner_solve == GD_INNER_AUTO && H.opt.precision == GD_MIXED) {
        std::vector<double> e32(S, -1.0);
        bool any32 = false;
        for (int s = 0; s < S; ++s)
            if (eta[s] >= 1e-5) {
                e32[s] = eta[s];
                any32 = true;
            }
        if (any32) {
            // every specimen is solved or skipped; failures are collected, not returned
            gd_status st = krylov_batch(H, e32, rhs, delta, kit, true, 1e300);
            if (st) return st;
            rep.krylov_iterations += kit;
            rep.krylov_fp32_iterations += kit;
            any64 = false;
            for (int s = 0; s < S; ++s) {
                const double rel = H.bk_out[3 * s + 1], status = H.bk_out[3 * s + 2];
                const bool ok = e32[s] >= 0.0 && (status == 0.0 || (status != 2.0 && std::isfinite(rel) && rel <= 0.1));
                todo[s] = ok ? -1.0 : eta[s];
                any64 = any64 || !ok;
            }
        }
    }
    if (!any64) return GD_OK;
    gd_status st = krylov_batch(H, todo, rhs, delta, kit, false, 0.1);
    rep.krylov_iterations += kit;
    return st;
}

// GD_MIXED: rounding noise of the FP32 residual at the current iterate, measured
// as ||R_fp32 - R_fp64|| on the free dofs (one residual-only FP64 pass), per
// specimen.  Near equilibrium the residual is a sum of element forces that cancel,
// so its FP32 rounding error, not the Newton iteration, sets how small it can get;
// the Newton test is not asked to go below twice this level.
gd_status mixed_noise(gd::Handle &H, const double *R32, std::vector<double> &noise)
{
    // the FP64 pass holds the history at the mixed pass's kappa of this iterate (no local
    // solve): the rounding of the element evaluation is the noise, the local solve's
    // tolerance adds a negligible part (measured on the 64^3 cube path: the two differ
    // by under 1 %), and the frozen pass costs about half as much
    const double *keep = H.kappa_fix;
    H.kappa_fix = H.kappa_trial;
    gd_status st = assemble_pass(H, H.w_dofs, H.kappa, H.R_trial, nullptr, nullptr, nullptr, 0, true, H.kappa_trial);
    H.kappa_fix = keep;
    if (st) return st;
    gd::SolverCtx c = solver_ctx(H, nullptr);
    double *diff = H.kv[9];
    GD_CUDA(&H, gd::launch_residual(c, H.R_trial, R32, diff, H.scal + 32));
    H.launches += 2;
    noise.assign(H.n_spec, 0.0);
    if (H.n_spec == 1) {
        GD_CUDA(&H, cudaMemcpyAsync(noise.data(), H.scal + 32, sizeof(double), cudaMemcpyDeviceToHost, H.stream));
        GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    } else {
        std::vector<double> nx;
        if ((st = norms_batch(H, diff, noise, nx))) return st;     // synchronises the stream
    }
    H.noise_ms += elapsed_ms(H);        // the pass's events have completed
    ++H.noise_passes;
    return GD_OK;
}

// GD_MIXED noise level for the Newton test.  The rounding noise of the residual
// scales with the magnitudes of the terms that cancel in it, so it is measured by the
// FP64 pass of mixed_noise on the first Newton solve (and after every new start of the
// state) and every kNoiseEvery solves, and in between taken as the measured ratio to
// the specimen's scale: the norm of the per-dof sums of the term magnitudes that the
// mixed kernels accumulate beside R (|P_ij n_j| J w in the displacement rows;
// |c_d C^-1 grad phi . grad N| J w + beta_d (|phi| + |kappa|) |N| J w in the damage rows,
// whose phi - kappa cancels in FP32 however small the element residual gets).
// The FP64 pass costs as much as several mixed passes.  A Newton solve whose line
// search stalls on an estimate it did not measure itself measures it again (force =
// true).
constexpr int kNoiseEvery = 8;

gd_status noise_estimate(gd::Handle &H, const double *R, const std::vector<double> &scale,
                         std::vector<double> &noise, bool &measured, bool force = false)
{
    const int S = H.n_spec;
    measured = false;
    if (force || H.noise_age <= 0 || (int)H.noise_ratio.size() != S) {
        measured = true;
        gd_status st = mixed_noise(H, R, noise);
        if (st) return st;
        H.noise_ratio.assign(S, 0.0);
        for (int s = 0; s < S; ++s) H.noise_ratio[s] = scale[s] > 0.0 ? noise[s] / scale[s] : 0.0;
        H.noise_age = kNoiseEvery;
        return GD_OK;
    }
    noise.assign(S, 0.0);
    for (int s = 0; s < S; ++s) noise[s] = H.noise_ratio[s] * scale[s];
    --H.noise_age;
    return GD_OK;
}

// Newton iteration for one load value starting from H.w_dofs (already predicted,
// prescribed dofs set).  On return H.w_dofs/H.R/H.kappa_trial hold the last iterate.
gd_status newton(gd::Handle &H, gd_newton_report &rep)
{
    gd_status st = assemble_pass(H, H.w_dofs, H.kappa, H.R, H.vals, H.kappa_trial, H.loading, 1, false, nullptr,
                                 H.Rabs);
    if (st) return st;
    NormPair nr;
    if ((st = norms(H, H.R, nr))) return st;
    H.assembly_ms += elapsed_ms(H);
    int hc[4];
    GD_CUDA(&H, cudaMemcpy(hc, H.counters, 4 * sizeof(int), cudaMemcpyDeviceToHost));
    GD_TC_CHECK(&H, hc);
    rep.yield_evals += hc[2];
    double nrm = nr.free_;
    const double r0 = std::max(nr.free_, nr.fixed_);
    double noise = 0.0;
    bool fresh = false;     // noise measured at an iterate of this solve
    std::vector<double> sc(1, nr.fixed_ > 0.0 ? nr.fixed_ : r0);
    if (H.opt.precision == GD_MIXED) {
        NormPair na;
        if ((st = norms(H, H.Rabs, na))) return st;
        if (na.free_ > 0.0) sc[0] = na.free_;
        std::vector<double> nz;
        if ((st = noise_estimate(H, H.R, sc, nz, fresh))) return st;
        noise = nz[0];
    }
    double ntol = std::max(std::max(H.opt.newton_rtol * r0, H.opt.newton_atol), 2.0 * noise);
    rep.residual0 = nrm;
    rep.local_failures = hc[0];
    rep.loading_points = hc[1];
    double *delta = H.kv[8], *rhs = H.kv[9];
    for (int it = 0; it <= H.opt.newton_max; ++it) {
        rep.iterations = it;
        rep.residual = nrm;
        if (!std::isfinite(nrm)) return fail(&H, GD_ERR_NAN, "non-finite residual in the Newton iteration");
        H.last_noise = noise;
        if (nrm <= ntol) {
            rep.converged = 1;
            return GD_OK;
        }
        if (it == H.opt.newton_max) break;
        // K delta = -R on the free dofs (one persistent cooperative launch)
        gd::SolverCtx c = solver_ctx(H, H.vals);
        GD_CUDA(&H, cudaMemsetAsync(rhs, 0, sizeof(double) * H.n_dofs, H.stream));
        GD_CUDA(&H, gd::launch_axpy_free(c, rhs, H.R, -1.0));
        // inexact Newton: the linear solve only needs to reach a tenth of the Newton
        // tolerance relative to the current residual (floor krylov_rtol, cap 1e-2)
        const double eta = std::min(1e-2, std::max(H.opt.krylov_rtol, 0.1 * ntol / nrm));
        if ((st = solve_direction(H, rhs, delta, eta, rep))) return st;
        // backtracking line search on ||R_free|| (GD_MIXED near its noise floor: at most
        // two halvings, a decrease below the noise cannot be measured)
        double alpha = 1.0, nt = 0.0;
        bool decreased = false;
        int ls_max = (H.opt.precision == GD_MIXED && nrm <= 8.0 * noise) ? std::min(2, H.opt.line_search_max)
                                                                         : H.opt.line_search_max;
        bool at_floor = false;
        for (int ls = 0; ls <= ls_max; ++ls) {
            if (ls == 1 && H.opt.precision == GD_MIXED && !fresh) {
                // the full step did not lower ||R_free||.  Within 8 times the estimated
                // noise the iterate is at the floor of the mode; further away, measure the
                // noise at this iterate before halving (the pass overwrites R_trial,
                // recomputed below)
                if (nrm <= 8.0 * noise) {
                    at_floor = true;
                    break;
                }
                std::vector<double> nz;
                if ((st = noise_estimate(H, H.R, sc, nz, fresh, true))) return st;
                noise = nz[0];
                ntol = std::max(ntol, 2.0 * noise);
                if (nrm <= 8.0 * noise) ls_max = std::max(1, std::min(2, H.opt.line_search_max));
            }
            GD_CUDA(&H, cudaMemcpyAsync(H.w_trial, H.w_dofs, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToDevice,
                                        H.stream));
            GD_CUDA(&H, gd::launch_axpy_free(c, H.w_trial, delta, alpha));
            if ((st = assemble_pass(H, H.w_trial, H.kappa, H.R_trial, H.vals_trial, H.kappa_trial2, H.loading2, 1, false,
                                     H.kappa_trial)))
                return st;
            if ((st = norms(H, H.R_trial, nr))) return st;
            H.assembly_ms += elapsed_ms(H);
            GD_CUDA(&H, cudaMemcpy(hc, H.counters, 4 * sizeof(int), cudaMemcpyDeviceToHost));
    GD_TC_CHECK(&H, hc);
            rep.yield_evals += hc[2];
            nt = nr.free_;
            decreased = std::isfinite(nt) && nt <= (1.0 - 1e-4 * alpha) * nrm;
            if (decreased || ls == ls_max) break;
            alpha *= 0.5;
            ++rep.line_search_cuts;
        }
        if (at_floor) {
            // the current iterate (H.w_dofs, H.R, H.kappa_trial) stands
            rep.iterations = it + 1;
            rep.residual = nrm;
            rep.converged = 1;
            H.last_noise = noise;
            return GD_OK;
        }
        std::swap(H.w_dofs, H.w_trial);
        std::swap(H.R, H.R_trial);
        std::swap(H.vals, H.vals_trial);
        std::swap(H.kappa_trial, H.kappa_trial2);
        std::swap(H.loading, H.loading2);
        rep.local_failures = hc[0];
        rep.loading_points = hc[1];
        nrm = nt;
        // GD_MIXED: when no step of the line search lowers ||R_free|| any more and it is
        // within four times the measured FP32 noise, the iterate is converged to the
        // precision of the mode
        if (!decreased && H.opt.precision == GD_MIXED && std::isfinite(nrm) && nrm <= 4.0 * noise) {
            rep.iterations = it + 1;
            rep.residual = nrm;
            rep.converged = 1;
            H.last_noise = noise;
            return GD_OK;
        }
    }
    rep.converged = 0;
    return GD_OK;
}

// per-specimen ||R_free|| and ||R_fixed|| (batches)
gd_status norms_batch(gd::Handle &H, const double *R, std::vector<double> &nf, std::vector<double> &nx)
{
    const int S = H.n_spec;
    GD_CUDA(&H, gd::launch_norms_batch(R, H.fixed, H.node_off, H.ndof, S, H.d_norm, H.stream));
    ++H.launches;
    std::vector<double> h((size_t)2 * S);
    GD_CUDA(&H, cudaMemcpyAsync(h.data(), H.d_norm, sizeof(double) * 2 * S, cudaMemcpyDeviceToHost, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    nf.resize(S);
    nx.resize(S);
    for (int s = 0; s < S; ++s) {
        nf[s] = h[2 * s];
        nx[s] = h[2 * s + 1];
    }
    return GD_OK;
}

gd_status set_coef(gd::Handle &H, const std::vector<double> &coef)
{
    GD_CUDA(&H, cudaMemcpyAsync(H.d_coef, coef.data(), sizeof(double) * H.n_spec, cudaMemcpyHostToDevice, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    return GD_OK;
}

// Newton iteration of a batch of independent specimens in one block-diagonal
// system.  Each specimen keeps its own convergence test (its own force scale),
// its own line-search step length and, once converged, stays where it is (zero
// right-hand side, zero step) while the others continue.  The linear solve of the
// union system is tight enough that every unconverged block meets its own
// inexact-Newton tolerance.
gd_status newton_batch(gd::Handle &H, gd_newton_report &rep)
{
    const int S = H.n_spec;
    gd_status st = assemble_pass(H, H.w_dofs, H.kappa, H.R, H.vals, H.kappa_trial, H.loading, 1, false, nullptr,
                                 H.Rabs);
    if (st) return st;
    std::vector<double> nf, nx, nt, ntx;
    if ((st = norms_batch(H, H.R, nf, nx))) return st;
    H.assembly_ms += elapsed_ms(H);
    int hc[4];
    GD_CUDA(&H, cudaMemcpy(hc, H.counters, 4 * sizeof(int), cudaMemcpyDeviceToHost));
    GD_TC_CHECK(&H, hc);
    rep.yield_evals += hc[2];
    std::vector<double> r0(S), ntol(S), coef(S), alpha(S);
    std::vector<char> done(S, 0), accepted(S, 0);
    auto total = [&](const std::vector<double> &v) {
        double t = 0.0;
        for (double x : v) t += x * x;
        return std::sqrt(t);
    };
    std::vector<double> noise(S, 0.0), sc(S);
    bool fresh = false;     // noise measured at an iterate of this solve
    for (int s = 0; s < S; ++s) sc[s] = nx[s] > 0.0 ? nx[s] : nf[s];
    if (H.opt.precision == GD_MIXED) {
        std::vector<double> af, ax;
        if ((st = norms_batch(H, H.Rabs, af, ax))) return st;
        for (int s = 0; s < S; ++s)
            if (af[s] > 0.0) sc[s] = af[s];
        if ((st = noise_estimate(H, H.R, sc, noise, fresh))) return st;
    }
    for (int s = 0; s < S; ++s) {
        r0[s] = std::max(nf[s], nx[s]);
        ntol[s] = std::max(std::max(H.opt.newton_rtol * r0[s], H.opt.newton_atol), 2.0 * noise[s]);
    }
    rep.residual0 = total(nf);
    rep.local_failures = hc[0];
    rep.loading_points = hc[1];
    double *delta = H.kv[8], *rhs = H.kv[9];
    for (int it = 0; it <= H.opt.newton_max; ++it) {
        rep.iterations = it;
        rep.residual = total(nf);
        H.last_noise = noise.empty() ? 0.0 : *std::max_element(noise.begin(), noise.end());
        if (!std::isfinite(rep.residual)) return fail(&H, GD_ERR_NAN, "non-finite residual in the Newton iteration");
        bool all = true;
        for (int s = 0; s < S; ++s) {
            if (nf[s] <= ntol[s]) done[s] = 1;
            all = all && done[s];
        }
        if (all) {
            rep.converged = 1;
            return GD_OK;
        }
        if (it == H.opt.newton_max) break;
        // right-hand side -R on the unconverged specimens only
        double bn2 = 0.0, need = 1e300;
        std::vector<double> eta_s(S, 1.0);
        for (int s = 0; s < S; ++s) {
            coef[s] = done[s] ? 0.0 : -1.0;
            if (done[s]) continue;
            bn2 += nf[s] * nf[s];
            eta_s[s] = std::min(1e-2, std::max(H.opt.krylov_rtol, 0.1 * ntol[s] / nf[s]));
            need = std::min(need, eta_s[s] * nf[s]);
        }
        if ((st = set_coef(H, coef))) return st;
        GD_CUDA(&H, gd::launch_scale_spec(H.n_dofs, H.ndof, rhs, H.R, H.d_coef, H.node_spec, H.fixed, 0, H.stream));
        ++H.launches;
        if (H.bk_ok && H.opt.inner_solve != GD_INNER_REFINED && H.coarse.nc == 0) {
            // every specimen runs its own recurrences to its own tolerance
            if ((st = solve_direction_batch(H, rhs, delta, eta_s, rep))) return st;
        } else {
            // one union solve (the two-level preconditioner's coarse level has aggregates in
            // every specimen): ||r_s|| <= ||r|| <= eta ||b|| with eta = min_s eta_s ||b_s|| / ||b||
            const double eta = std::max(1e-14, need / std::sqrt(bn2));
            if ((st = solve_direction(H, rhs, delta, eta, rep))) return st;
        }
        // backtracking line search per specimen on its own ||R_free||
        bool near_floor = H.opt.precision == GD_MIXED;
        for (int s = 0; s < S; ++s) {
            alpha[s] = done[s] ? 0.0 : 1.0;
            accepted[s] = done[s];
            if (!done[s] && nf[s] > 8.0 * noise[s]) near_floor = false;
        }
        int ls_max = near_floor ? std::min(2, H.opt.line_search_max) : H.opt.line_search_max;
        for (int ls = 0; ls <= ls_max; ++ls) {
            if (ls == 1 && H.opt.precision == GD_MIXED && !fresh) {
                // a full step lowered no ||R_free|| of some specimen: measure the noise
                // at this iterate before halving (the pass overwrites R_trial and the
                // right-hand side, both recomputed before they are read again)
                if ((st = noise_estimate(H, H.R, sc, noise, fresh, true))) return st;
                near_floor = true;
                for (int s = 0; s < S; ++s) {
                    ntol[s] = std::max(ntol[s], 2.0 * noise[s]);
                    if (!accepted[s] && nf[s] > 8.0 * noise[s]) near_floor = false;
                }
                if (near_floor) ls_max = std::max(1, std::min(2, H.opt.line_search_max));
            }
            if ((st = set_coef(H, alpha))) return st;
            GD_CUDA(&H, cudaMemcpyAsync(H.w_trial, H.w_dofs, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToDevice,
                                        H.stream));
            GD_CUDA(&H, gd::launch_scale_spec(H.n_dofs, H.ndof, H.w_trial, delta, H.d_coef, H.node_spec, H.fixed, 1,
                                              H.stream));
            ++H.launches;
            if ((st = assemble_pass(H, H.w_trial, H.kappa, H.R_trial, H.vals_trial, H.kappa_trial2, H.loading2, 1, false,
                                     H.kappa_trial)))
                return st;
            if ((st = norms_batch(H, H.R_trial, nt, ntx))) return st;
            H.assembly_ms += elapsed_ms(H);
            GD_CUDA(&H, cudaMemcpy(hc, H.counters, 4 * sizeof(int), cudaMemcpyDeviceToHost));
    GD_TC_CHECK(&H, hc);
            rep.yield_evals += hc[2];
            bool all_acc = true;
            for (int s = 0; s < S; ++s) {
                if (!accepted[s] && std::isfinite(nt[s]) && nt[s] <= (1.0 - 1e-4 * alpha[s]) * nf[s]) accepted[s] = 1;
                all_acc = all_acc && accepted[s];
            }
            if (all_acc || ls == ls_max) break;
            for (int s = 0; s < S; ++s)
                if (!accepted[s]) alpha[s] *= 0.5;
            ++rep.line_search_cuts;
        }
        std::swap(H.w_dofs, H.w_trial);
        std::swap(H.R, H.R_trial);
        std::swap(H.vals, H.vals_trial);
        std::swap(H.kappa_trial, H.kappa_trial2);
        std::swap(H.loading, H.loading2);
        rep.local_failures = hc[0];
        rep.loading_points = hc[1];
        // GD_MIXED: a specimen whose residual no step can lower any more and that is
        // within four times its measured FP32 noise is converged to the precision of the mode
        for (int s = 0; s < S; ++s) {
            if (!accepted[s] && H.opt.precision == GD_MIXED && std::isfinite(nt[s]) && nt[s] <= 4.0 * noise[s])
                ntol[s] = std::max(ntol[s], nt[s]);
        }
        nf = nt;
    }
    rep.converged = 0;
    return GD_OK;
}

gd_status linear_predictor(gd::Handle &H);

// load of specimen s at step coordinate t: piecewise linear through 0 at t = 0
// and the path values at t = 1..n (held after the last step)
double path_load(const gd::Handle &H, int s, double t)
{
    const std::vector<double> &P = H.paths[s];
    const int n = (int)P.size();
    if (n == 0 || t <= 0.0) return 0.0;
    if (t >= n) return P[n - 1];
    const int k = (int)std::floor(t);
    const double a = k == 0 ? 0.0 : P[k - 1], b = P[k];
    return a + (t - k) * (b - a);
}

// initial guess for step coordinate t: the last converged state plus the previous
// increment scaled to this one (per specimen), prescribed dofs at their loads
gd_status predict(gd::Handle &H, double t)
{
    if (H.n_spec == 1) {
        const double Lt = path_load(H, 0, t), L1 = path_load(H, 0, H.load_prev), L2 = path_load(H, 0, H.load_prevprev);
        const double dl = L1 - L2;
        const bool extrap = H.have_prev && dl != 0.0;
        // three converged states on a monotone stretch of the path: the quadratic through
        // them (Lagrange in the load), else the line through the last two
        if (extrap && H.have_pp) {
            const double L3 = path_load(H, 0, H.load_ppp);
            const bool mono = (Lt > L1 && L1 > L2 && L2 > L3) || (Lt < L1 && L1 < L2 && L2 < L3);
            if (mono) {
                const double w[3] = {(Lt - L2) * (Lt - L3) / ((L1 - L2) * (L1 - L3)),
                                     (Lt - L1) * (Lt - L3) / ((L2 - L1) * (L2 - L3)),
                                     (Lt - L1) * (Lt - L2) / ((L3 - L1) * (L3 - L2))};
                GD_CUDA(&H, gd::launch_predictor3(H.n_dofs, H.w_dofs, H.dofs, H.dofs_prev, H.dofs_pp, w, H.bc_dof,
                                                  H.bc_scale, H.n_bc, Lt, H.stream));
                H.launches += H.n_bc > 0 ? 2 : 1;
                return GD_OK;
            }
        }
        GD_CUDA(&H, gd::launch_predictor(H.n_dofs, H.w_dofs, H.dofs, extrap ? H.dofs_prev : nullptr,
                                         extrap ? (Lt - L1) / dl : 0.0, H.bc_dof, H.bc_scale, H.n_bc, Lt, H.stream));
        H.launches += H.n_bc > 0 ? 2 : 1;
        return extrap ? GD_OK : linear_predictor(H);
    }
    // per specimen: the quadratic through its last three states on a monotone stretch of
    // its path, else the line through the last two, else the last state
    std::vector<double> hl((size_t)H.n_spec), hw((size_t)3 * H.n_spec);
    for (int s = 0; s < H.n_spec; ++s) {
        const double Lt = path_load(H, s, t), L1 = path_load(H, s, H.load_prev), L2 = path_load(H, s, H.load_prevprev);
        const double L3 = path_load(H, s, H.load_ppp), dl = L1 - L2;
        double *w = hw.data() + 3 * s;
        hl[s] = Lt;
        w[0] = 1.0;
        w[1] = w[2] = 0.0;
        if (H.have_prev && dl != 0.0) {
            const double f = (Lt - L1) / dl;
            w[0] = 1.0 + f;
            w[1] = -f;
        }
        if (H.have_prev && H.have_pp && ((Lt > L1 && L1 > L2 && L2 > L3) || (Lt < L1 && L1 < L2 && L2 < L3))) {
            w[0] = (Lt - L2) * (Lt - L3) / ((L1 - L2) * (L1 - L3));
            w[1] = (Lt - L1) * (Lt - L3) / ((L2 - L1) * (L2 - L3));
            w[2] = (Lt - L1) * (Lt - L2) / ((L3 - L1) * (L3 - L2));
        }
    }
    GD_CUDA(&H, cudaMemcpyAsync(H.d_load, hl.data(), sizeof(double) * H.n_spec, cudaMemcpyHostToDevice, H.stream));
    GD_CUDA(&H, cudaMemcpyAsync(H.d_pw, hw.data(), sizeof(double) * 3 * H.n_spec, cudaMemcpyHostToDevice, H.stream));
    GD_CUDA(&H, gd::launch_predictor_batch(H.n_dofs, H.ndof, H.w_dofs, H.dofs, H.have_prev ? H.dofs_prev : nullptr,
                                           H.have_pp ? H.dofs_pp : nullptr, H.d_pw, H.node_spec, H.bc_dof, H.bc_scale,
                                           H.bc_spec, H.d_load, H.n_bc, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));     // hl is pageable host memory
    H.launches += H.n_bc > 0 ? 2 : 1;
    return H.have_prev ? GD_OK : linear_predictor(H);
}

// First step of a path (no previous increment to extrapolate): the prescribed
// increment d_bc on the committed state plus the free-dof response of the
// committed state's tangent, K_ff delta = -K_f. d_bc (one assembly, one loose
// solve).  Without it the whole increment sits in the first column of elements
// at the loaded boundary, whose strain at the first Newton iterate is many times
// the nominal one, and the iteration needs dozens of damped steps and halvings.
gd_status linear_predictor(gd::Handle &H)
{
    double *dbc = H.diag, *y = H.kv[8], *rhs = H.kv[9];
    GD_CUDA(&H, gd::launch_axpby(H.n_dofs, dbc, H.w_dofs, -1.0, H.dofs, H.stream));
    ++H.launches;
    gd_status st = assemble_pass(H, H.dofs, H.kappa, H.R_trial, H.vals, H.kappa_trial2, H.loading2, 1);
    if (st) return st;
    H.assembly_ms += elapsed_ms(H);
    gd::SolverCtx c = solver_ctx(H, H.opt.precision == GD_FP64 ? H.vals : nullptr);
    if (H.opt.precision != GD_FP64) c.vals32 = (const float *)H.vals;
    GD_CUDA(&H, gd::launch_spmv(c, dbc, y, 0));      // K d_bc (all rows and columns)
    GD_CUDA(&H, cudaMemsetAsync(rhs, 0, sizeof(double) * H.n_dofs, H.stream));
    GD_CUDA(&H, gd::launch_axpy_free(c, rhs, y, -1.0));
    int kit = 0;
    double rel = 0.0;
    // a loose solve is enough for an initial guess; a failed one leaves w as it is
    if (krylov(H, H.vals, rhs, y, kit, rel, 1e-3, H.opt.precision == GD_MIXED, 0.5) == GD_OK)
        GD_CUDA(&H, gd::launch_axpy_free(c, H.w_dofs, y, 1.0));
    return GD_OK;
}

void free_ckpts(gd::Handle &H)
{
    for (auto &c : H.ckpts) {
        dfree(c.dofs);
        dfree(c.dofs_prev);
        dfree(c.kappa);
    }
    H.ckpts.clear();
}

// stores the handle's committed state as a checkpoint after `commits` commits
gd_status save_ckpt(gd::Handle &H, int commits)
{
    gd::Checkpoint c;
    c.commit = commits;
    GD_CUDA(&H, dalloc(&c.dofs, (size_t)H.n_dofs));
    GD_CUDA(&H, dalloc(&c.dofs_prev, (size_t)H.n_dofs));
    GD_CUDA(&H, dalloc(&c.kappa, (size_t)(H.n_elems * H.nq)));
    GD_CUDA(&H, cudaMemcpyAsync(c.dofs, H.dofs, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToDevice, H.stream));
    GD_CUDA(&H, cudaMemcpyAsync(c.dofs_prev, H.dofs_prev, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToDevice,
                                H.stream));
    GD_CUDA(&H, cudaMemcpyAsync(c.kappa, H.kappa, sizeof(double) * H.n_elems * H.nq, cudaMemcpyDeviceToDevice,
                                H.stream));
    c.load_prev = H.load_prev;
    c.load_prevprev = H.load_prevprev;
    c.have_prev = H.have_prev;
    H.ckpts.push_back(c);
    return GD_OK;
}

gd_status restore_ckpt(gd::Handle &H, const gd::Checkpoint &c)
{
    GD_CUDA(&H, cudaMemcpyAsync(H.dofs, c.dofs, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToDevice, H.stream));
    GD_CUDA(&H, cudaMemcpyAsync(H.dofs_prev, c.dofs_prev, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToDevice,
                                H.stream));
    GD_CUDA(&H, cudaMemcpyAsync(H.kappa, c.kappa, sizeof(double) * H.n_elems * H.nq, cudaMemcpyDeviceToDevice,
                                H.stream));
    H.load_prev = c.load_prev;
    H.load_prevprev = c.load_prevprev;
    H.have_prev = c.have_prev;
    H.have_pp = false;                       // checkpoints keep two states
    return GD_OK;
}

gd_status commit(gd::Handle &H, double target, gd_newton_report &rep)
{
    // reaction at the converged state, then shift the history
    GD_CUDA(&H, gd::launch_reaction(H.R, H.react_dof, H.n_react, H.scal + 20, H.stream));
    GD_CUDA(&H, gd::launch_damage_max(H.kappa_trial, H.n_elems * H.nq, H.mat.eta_d, H.mat.kappa_d, H.scal + 21,
                                      H.stream));
    H.launches += 2;
    rep.kernel_launches += 2;
    double h[2];
    GD_CUDA(&H, cudaMemcpyAsync(h, H.scal + 20, 2 * sizeof(double), cudaMemcpyDeviceToHost, H.stream));
    if (H.n_spec > 1) {
        GD_CUDA(&H, gd::launch_reaction_batch(H.R, H.react_dof, H.react_off, H.n_spec, H.d_load, H.stream));
        ++H.launches;
        H.last_reac.resize(H.n_spec);
        GD_CUDA(&H, cudaMemcpyAsync(H.last_reac.data(), H.d_load, sizeof(double) * H.n_spec, cudaMemcpyDeviceToHost,
                                    H.stream));
    }
    {
        // dofs_pp <- dofs_prev <- dofs <- converged iterate; the oldest buffer becomes scratch
        double *old_pp = H.dofs_pp;
        H.dofs_pp = H.dofs_prev;
        H.dofs_prev = H.dofs;
        H.dofs = H.w_dofs;
        H.w_dofs = old_pp;
        H.have_pp = H.have_prev;
        H.load_ppp = H.load_prevprev;
    }
    std::swap(H.kappa, H.kappa_trial);
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    rep.reaction = h[0];
    rep.max_damage = h[1];
    if (H.n_spec == 1) H.last_reac.assign(1, h[0]);
    H.load_prevprev = H.load_prev;
    H.load_prev = target;
    H.have_prev = true;
    if (H.rec_on && !H.replaying) {
        H.rec_load.push_back(target);
        H.rec_step.push_back(-1);
        const int k = H.opt.checkpoint_every > 0 ? H.opt.checkpoint_every : 1;
        if ((int)H.rec_load.size() % k == 0) return save_ckpt(H, (int)H.rec_load.size());
    }
    return GD_OK;
}

// Staggered scheme of Sec. 3.2 (gd_options.scheme = GD_STAGGERED): the history is
// advanced apart from the nodal solve.  Newton on the (u, phi) equilibrium with kappa
// held at the committed kappa_n, then one local update at the converged fields (its
// loading test against kappa_n).  The step takes no coupled test: the update lags the
// nodal solve by one step.  The update's residual goes to the scratch R_trial, so H.R
// keeps the equilibrium residual and the step's reaction is that equilibrium's.
gd_status newton_staggered(gd::Handle &H, gd_newton_report &rep)
{
    H.kappa_fix = H.kappa;
    gd_status st = newton(H, rep);
    H.kappa_fix = nullptr;
    if (st || !rep.converged) return st;
    if ((st = assemble_pass(H, H.w_dofs, H.kappa, H.R_trial, nullptr, H.kappa_trial, H.loading, 0))) return st;
    H.assembly_ms += elapsed_ms(H);
    int hc[4];
    GD_CUDA(&H, cudaMemcpy(hc, H.counters, 4 * sizeof(int), cudaMemcpyDeviceToHost));
    GD_TC_CHECK(&H, hc);
    rep.yield_evals += hc[2];
    rep.local_failures = hc[0];
    rep.loading_points = hc[1];
    return GD_OK;
}

// Iterated staggered scheme (GD_STAGGERED_ITERATED): Newton on the (u, phi) equilibrium
// with the history frozen, then the local update at the converged fields; the two alternate
// until the residual with the updated history meets the Newton test (then the step
// solves the same equations as the monolithic scheme).  The loading test of every
// local update is against the committed history kappa_n, as in the monolithic scheme.
gd_status newton_staggered_iterated(gd::Handle &H, gd_newton_report &rep)
{
    const size_t nq_bytes = sizeof(double) * (size_t)(H.n_elems * H.nq);
    GD_CUDA(&H, cudaMemcpyAsync(H.kappa_stag, H.kappa, nq_bytes, cudaMemcpyDeviceToDevice, H.stream));
    gd_status st = GD_OK;
    double r0 = -1.0;
    for (int s = 0; s < H.opt.stagger_max; ++s) {
        gd_newton_report sub{};
        H.kappa_fix = H.kappa_stag;
        st = newton(H, sub);
        H.kappa_fix = nullptr;
        rep.iterations += sub.iterations;
        rep.krylov_iterations += sub.krylov_iterations;
        rep.krylov_fp32_iterations += sub.krylov_fp32_iterations;
        rep.line_search_cuts += sub.line_search_cuts;
        rep.yield_evals += sub.yield_evals;
        if (s == 0) rep.residual0 = sub.residual0;
        if (st) return st;
        if (!sub.converged) {
            rep.residual = sub.residual;
            rep.converged = 0;
            return GD_OK;
        }
        // the fields already met the Newton test with this history (which the update
        // computed from them): a fixed point to that test (in GD_MIXED, to its noise floor)
        if (s > 0 && sub.iterations == 0) {
            rep.residual = sub.residual;
            rep.converged = 1;
            return GD_OK;
        }
        // local update at the converged fields, and the residual with it
        if ((st = assemble_pass(H, H.w_dofs, H.kappa, H.R, nullptr, H.kappa_trial, H.loading, 0))) return st;
        NormPair nr;
        if ((st = norms(H, H.R, nr))) return st;
        H.assembly_ms += elapsed_ms(H);
        int hc[4];
        GD_CUDA(&H, cudaMemcpy(hc, H.counters, 4 * sizeof(int), cudaMemcpyDeviceToHost));
    GD_TC_CHECK(&H, hc);
        rep.yield_evals += hc[2];
        rep.local_failures = hc[0];
        rep.loading_points = hc[1];
        if (r0 < 0.0) r0 = std::max(std::max(sub.residual0, nr.free_), nr.fixed_);
        rep.residual = nr.free_;
        const double tol = std::max(H.opt.newton_rtol * r0, H.opt.newton_atol);
        if (!std::isfinite(nr.free_)) return fail(&H, GD_ERR_NAN, "non-finite residual in the staggered scheme");
        if (nr.free_ <= tol) {
            rep.converged = 1;
            return GD_OK;
        }
        GD_CUDA(&H, cudaMemcpyAsync(H.kappa_stag, H.kappa_trial, nq_bytes, cudaMemcpyDeviceToDevice, H.stream));
    }
    rep.converged = 0;
    return GD_OK;
}

gd_status advance(gd::Handle &H, double target, int depth, gd_newton_report &rep)
{
    gd_status sp = predict(H, target);
    if (sp) return sp;
    gd_newton_report sub{};
    const double a0 = H.assembly_ms, k0 = H.krylov_ms, z0 = H.noise_ms;
    const int n0 = H.assemblies;
    const long long l0 = H.launches, p0 = H.noise_passes;
    H.last_noise = 0.0;
    gd_status st = H.n_spec > 1                      ? newton_batch(H, sub)
                   : H.opt.scheme == GD_STAGGERED          ? newton_staggered(H, sub)
                   : H.opt.scheme == GD_STAGGERED_ITERATED ? newton_staggered_iterated(H, sub)
                                                           : newton(H, sub);
    rep.assembly_ms += H.assembly_ms - a0;
    rep.krylov_ms += H.krylov_ms - k0;
    rep.assemblies += H.assemblies - n0;
    rep.yield_evals += sub.yield_evals;
    rep.krylov_fp32_iterations += sub.krylov_fp32_iterations;
    rep.kernel_launches += H.launches - l0;
    rep.noise_ms += H.noise_ms - z0;
    rep.noise_passes += (int32_t)(H.noise_passes - p0);
    rep.noise = H.last_noise;
    rep.iterations += sub.iterations;
    rep.krylov_iterations += sub.krylov_iterations;
    rep.line_search_cuts += sub.line_search_cuts;
    rep.residual0 = sub.residual0;
    rep.residual = sub.residual;
    rep.local_failures = sub.local_failures;
    rep.loading_points = sub.loading_points;
    const bool ok = st == GD_OK && sub.converged;
    if (!ok && depth < H.opt.max_step_cuts && (st == GD_OK || st == GD_ERR_NAN || st == GD_ERR_KRYLOV)) {
        ++rep.step_cuts;
        const double mid = 0.5 * (H.load_prev + target);
        if ((st = advance(H, mid, depth + 1, rep))) return st;
        return advance(H, target, depth + 1, rep);
    }
    if (st) return st;
    if (!sub.converged) {
        char msg[160];
        snprintf(msg, sizeof(msg), "Newton did not converge (|R_free| %.3e after %d iterations, first %.3e)",
                 sub.residual, sub.iterations, sub.residual0);
        return fail(&H, GD_ERR_NOT_CONVERGED, msg);
    }
    rep.converged = 1;
    return commit(H, target, rep);
}


struct Pattern {
    std::vector<uint8_t> fixed;
    std::vector<int32_t> bc_dof, react, rowptr, colidx, slot;
    int64_t nnz = 0;
};

// Validates the mesh and builds the CSR pattern of the node graph (ndof x ndof
// blocks, neighbours ascending), the per-element slot map and the Dirichlet
// masks.  Host only.
gd_status build_pattern(const gd_mesh *mesh, Pattern &P)
{
    if (!mesh) return fail(nullptr, GD_ERR_ARG, "mesh is null");
    if (mesh->dim != 2 && mesh->dim != 3) return fail(nullptr, GD_ERR_ARG, "dim must be 2 or 3");
    if (mesh->n_nodes <= 0 || mesh->n_elems < 0 || !mesh->coords || (mesh->n_elems > 0 && !mesh->conn))
        return fail(nullptr, GD_ERR_ARG, "empty or null mesh arrays");
    if (mesh->n_bc < 0 || (mesh->n_bc > 0 && (!mesh->bc_node || !mesh->bc_comp || !mesh->bc_scale)))
        return fail(nullptr, GD_ERR_ARG, "boundary arrays");
    if (mesh->n_react < 0 || (mesh->n_react > 0 && !mesh->react_node))
        return fail(nullptr, GD_ERR_ARG, "reaction arrays");
    if (mesh->react_comp < 0 || mesh->react_comp >= mesh->dim) return fail(nullptr, GD_ERR_ARG, "react_comp");
    const int dim = mesh->dim, nen = dim == 2 ? 4 : 8, ndof = dim + 1;
    const int64_t NN = mesh->n_nodes, NE = mesh->n_elems;
    // connectivity and Jacobians
    for (int64_t e = 0; e < NE; ++e) {
        double Xe[24];
        for (int a = 0; a < nen; ++a) {
            int32_t n = mesh->conn[e * nen + a];
            if (n < 0 || n >= NN) return fail(nullptr, GD_ERR_MESH, "element " + std::to_string(e) + " has a bad node id");
            for (int J = 0; J < dim; ++J) Xe[a * dim + J] = mesh->coords[(int64_t)n * dim + J];
        }
        if (!element_ok(dim, Xe))
            return fail(nullptr, GD_ERR_MESH, "element " + std::to_string(e) + " has a non-positive Jacobian");
    }
    // prescribed dofs
    P.fixed.assign((size_t)(NN * ndof), 0);
    P.bc_dof.resize((size_t)mesh->n_bc);
    for (int64_t i = 0; i < mesh->n_bc; ++i) {
        int32_t n = mesh->bc_node[i];
        int c = mesh->bc_comp[i];
        if (n < 0 || n >= NN || c < 0 || c >= dim) return fail(nullptr, GD_ERR_ARG, "bad boundary entry " + std::to_string(i));
        int64_t d = (int64_t)n * ndof + c;
        if (P.fixed[d]) return fail(nullptr, GD_ERR_ARG, "dof prescribed twice (boundary entry " + std::to_string(i) + ")");
        P.fixed[d] = 1;
        P.bc_dof[i] = (int32_t)d;
    }
    P.react.resize((size_t)mesh->n_react);
    for (int64_t i = 0; i < mesh->n_react; ++i) {
        int32_t n = mesh->react_node[i];
        if (n < 0 || n >= NN) return fail(nullptr, GD_ERR_ARG, "bad reaction node");
        P.react[i] = (int32_t)((int64_t)n * ndof + mesh->react_comp);
    }
    // node graph: node -> elements, then sorted unique neighbour lists
    std::vector<int64_t> ne_ptr((size_t)NN + 1, 0);
    for (int64_t e = 0; e < NE; ++e)
        for (int a = 0; a < nen; ++a) ne_ptr[mesh->conn[e * nen + a] + 1]++;
    for (int64_t n = 0; n < NN; ++n) ne_ptr[n + 1] += ne_ptr[n];
    std::vector<int64_t> ne_list((size_t)ne_ptr[NN]);
    {
        std::vector<int64_t> fill(ne_ptr.begin(), ne_ptr.end() - 1);
        for (int64_t e = 0; e < NE; ++e)
            for (int a = 0; a < nen; ++a) ne_list[fill[mesh->conn[e * nen + a]]++] = e;
    }
    std::vector<int64_t> nb_ptr((size_t)NN + 1, 0);
    std::vector<int32_t> nb_list;
    nb_list.reserve((size_t)NN * (dim == 2 ? 9 : 27));
    std::vector<int32_t> tmp;
    for (int64_t n = 0; n < NN; ++n) {
        tmp.clear();
        tmp.push_back((int32_t)n);
        for (int64_t k = ne_ptr[n]; k < ne_ptr[n + 1]; ++k) {
            int64_t e = ne_list[k];
            for (int a = 0; a < nen; ++a) tmp.push_back(mesh->conn[e * nen + a]);
        }
        std::sort(tmp.begin(), tmp.end());
        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
        nb_list.insert(nb_list.end(), tmp.begin(), tmp.end());
        nb_ptr[n + 1] = (int64_t)nb_list.size();
    }
    // CSR over dofs
    const int64_t n_dofs = NN * ndof;
    int64_t nnz = 0;
    for (int64_t n = 0; n < NN; ++n) nnz += (nb_ptr[n + 1] - nb_ptr[n]) * ndof * ndof;
    if (nnz >= (int64_t)1 << 31 || n_dofs >= (int64_t)1 << 31)
        return fail(nullptr, GD_ERR_ARG, "matrix too large for int32 indices");
    P.nnz = nnz;
    P.rowptr.resize((size_t)n_dofs + 1);
    P.colidx.resize((size_t)nnz);
    {
        int64_t pos = 0;
        for (int64_t n = 0; n < NN; ++n) {
            for (int i = 0; i < ndof; ++i) {
                P.rowptr[n * ndof + i] = (int32_t)pos;
                for (int64_t k = nb_ptr[n]; k < nb_ptr[n + 1]; ++k)
                    for (int c = 0; c < ndof; ++c) P.colidx[pos++] = nb_list[k] * ndof + c;
            }
        }
        P.rowptr[n_dofs] = (int32_t)pos;
    }
    // slot map: position of (row node a dof 0, column node b dof 0)
    P.slot.resize((size_t)(NE * nen * nen));
    for (int64_t e = 0; e < NE; ++e)
        for (int a = 0; a < nen; ++a) {
            const int32_t na = mesh->conn[e * nen + a];
            const int32_t *b0 = nb_list.data() + nb_ptr[na], *b1 = nb_list.data() + nb_ptr[na + 1];
            for (int b = 0; b < nen; ++b) {
                const int32_t nbn = mesh->conn[e * nen + b];
                const int64_t idx = std::lower_bound(b0, b1, nbn) - b0;
                P.slot[(e * nen + a) * nen + b] = (int32_t)(P.rowptr[(int64_t)na * ndof] + idx * ndof);
            }
        }
    return GD_OK;
}

}  // namespace

gd_status gd::set_error(gd_status st, const std::string &msg)
{
    g_create_error = msg;
    return st;
}

extern "C" {

void gd_default_options(gd_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = GD_FP64;
    o->newton_rtol = 1e-10;
    o->newton_atol = 1e-12;
    o->newton_max = 25;
    o->line_search_max = 12;
    o->krylov = GD_BICGSTAB;
    o->krylov_rtol = 1e-12;
    o->krylov_max = 20000;
    o->gmres_m = 50;
    o->local_max = 100;
    o->checkpoint_every = 5;
    o->max_step_cuts = 4;
    o->cuda_stream = nullptr;
    o->coarse = 1536;
    o->scheme = GD_MONOLITHIC;
    o->stagger_max = 100;
}

const char *gd_last_error(const gd_handle *h) { return h ? h->h.err.c_str() : g_create_error.c_str(); }

void gd_destroy(gd_handle *h)
{
    if (!h) return;
    free_handle(h->h);
    delete h;
}

static gd_status validate_net(const gd_icnn *n, int n_in, bool allow_zero, const char *name)
{
    if (!n) return fail(nullptr, GD_ERR_ARG, std::string(name) + " network is null");
    if (n->n_in != n_in) return fail(nullptr, GD_ERR_ARG, std::string(name) + " network must have n_in = " + std::to_string(n_in));
    if (n->width < (allow_zero ? 0 : 1) || n->width > gd::kMaxWidth)
        return fail(nullptr, GD_ERR_ARG, std::string(name) + " network width out of range");
    if (n->width > 0 && !n->params) return fail(nullptr, GD_ERR_ARG, std::string(name) + " network params null");
    return GD_OK;
}

static int net_params(int n_in, int w) { return w * n_in + w + w * w + w * n_in + w + w + n_in; }

static gd_status stage_net(gd::Handle &H, gd::DevNet &d, int n_in, int w, const double *params)
{
    d.n_in = n_in;
    d.width = w;
    d.n_params = w > 0 ? net_params(n_in, w) : 0;
    if (w == 0) return GD_OK;
    GD_CUDA(&H, dalloc(&d.p, d.n_params));
    GD_CUDA(&H, dalloc(&d.W2T, (size_t)w * w));
    GD_CUDA(&H, dalloc(&d.pf, d.n_params));
    GD_CUDA(&H, dalloc(&d.W2Tf, (size_t)w * w));
    GD_CUDA(&H, cudaMemcpyAsync(d.p, params, sizeof(double) * d.n_params, cudaMemcpyDefault, H.stream));
    GD_CUDA(&H, gd::launch_transpose(d, H.stream));
    GD_CUDA(&H, gd::launch_net_to_float(d, H.stream));
    return GD_OK;
}

// Per-specimen Krylov layout of a batch for the current cooperative grid: block b
// owns nodes [b chunk, (b+1) chunk); its first specimen and count, every
// specimen's first and last block, and the partial and result buffers.  Batches
// whose blocks would overlap more than kMaxSpecPerBlock specimens use the union
// solve instead (bk_ok = false).
gd_status build_batch_krylov(gd::Handle &H)
{
    dfree(H.bk_i32);
    dfree(H.bk_f64);
    dfree(H.bk_cnt);
    H.bk_i32 = nullptr;
    H.bk_f64 = nullptr;
    H.bk_cnt = nullptr;
    H.bk_ok = false;
    const int nb = H.krylov_grid, S = H.n_spec;
    const int64_t NN = H.n_nodes;
    const int64_t chunk = (NN + nb - 1) / nb;
    std::vector<int32_t> ns_of((size_t)NN);
    for (int s = 0; s < S; ++s)
        for (int64_t n = H.h_node_off[s]; n < H.h_node_off[s + 1]; ++n) ns_of[n] = s;
    std::vector<int32_t> lay((size_t)2 * nb + 2 * S, 0);
    int J = 0;
    for (int b = 0; b < nb; ++b) {
        const int64_t n0 = (int64_t)b * chunk, n1 = std::min<int64_t>(n0 + chunk, NN);
        if (n0 >= n1) continue;
        lay[b] = ns_of[n0];
        lay[nb + b] = ns_of[n1 - 1] - ns_of[n0] + 1;
        J = std::max(J, (int)lay[nb + b]);
    }
    for (int s = 0; s < S; ++s) {
        lay[2 * nb + s] = (int32_t)(H.h_node_off[s] / chunk);
        lay[2 * nb + S + s] = (int32_t)((H.h_node_off[s + 1] - 1) / chunk);
    }
    if (J > gd::kMaxSpecPerBlock) return GD_OK;
    GD_CUDA(&H, dalloc(&H.bk_i32, lay.size()));
    GD_CUDA(&H, cudaMemcpy(H.bk_i32, lay.data(), sizeof(int32_t) * lay.size(), cudaMemcpyHostToDevice));
    GD_CUDA(&H, dalloc(&H.bk_f64, (size_t)S + (size_t)5 * nb * J + (size_t)3 * S));
    GD_CUDA(&H, dalloc(&H.bk_cnt, 2));
    gd::BatchKrylov &L = H.bk;
    L.node_spec = H.node_spec;
    L.blk_fs = H.bk_i32;
    L.blk_ns = H.bk_i32 + nb;
    L.spec_b0 = H.bk_i32 + 2 * nb;
    L.spec_b1 = H.bk_i32 + 2 * nb + S;
    L.rtol = H.bk_f64;
    L.red = H.bk_f64 + S;
    L.out = H.bk_f64 + S + (size_t)5 * nb * J;
    L.active_cnt = H.bk_cnt;
    L.chunk = chunk;
    L.J = J;
    L.n_spec = S;
    H.bk_ok = true;
    return GD_OK;
}

// The meshes of a batch laid end to end: node, element, boundary and reaction
// numbering shifted by the counts of the specimens before; per-specimen
// reaction dofs carry each specimen's own react_comp.
struct Union {
    std::vector<double> coords, bc_scale;
    std::vector<int32_t> conn, bc_node, react_node;
    std::vector<int8_t> bc_comp;
    std::vector<int64_t> node_off, elem_off, bc_off, react_off;
    std::vector<int32_t> react_comp;
    gd_mesh mesh{};
};

static gd_status build_union(int32_t n_spec, const gd_mesh *meshes, Union &U)
{
    const int dim = meshes[0].dim;
    if (dim != 2 && dim != 3) return fail(nullptr, GD_ERR_ARG, "dim must be 2 or 3");
    const int nen = dim == 2 ? 4 : 8;
    U.node_off.assign(1, 0);
    U.elem_off.assign(1, 0);
    U.bc_off.assign(1, 0);
    U.react_off.assign(1, 0);
    for (int s = 0; s < n_spec; ++s) {
        const gd_mesh &m = meshes[s];
        const std::string tag = "specimen " + std::to_string(s) + ": ";
        if (m.dim != dim) return fail(nullptr, GD_ERR_ARG, tag + "all specimens must have the same dim");
        if (m.n_nodes <= 0 || m.n_elems < 0 || !m.coords || (m.n_elems > 0 && !m.conn))
            return fail(nullptr, GD_ERR_ARG, tag + "empty or null mesh arrays");
        if (m.n_bc < 0 || (m.n_bc > 0 && (!m.bc_node || !m.bc_comp || !m.bc_scale)))
            return fail(nullptr, GD_ERR_ARG, tag + "boundary arrays");
        if (m.n_react < 0 || (m.n_react > 0 && !m.react_node)) return fail(nullptr, GD_ERR_ARG, tag + "reaction arrays");
        if (m.react_comp < 0 || m.react_comp >= dim) return fail(nullptr, GD_ERR_ARG, tag + "react_comp");
        const int64_t off = U.node_off.back();
        for (int64_t i = 0; i < m.n_elems * nen; ++i)
            if (m.conn[i] < 0 || m.conn[i] >= m.n_nodes) return fail(nullptr, GD_ERR_MESH, tag + "bad node id in conn");
        for (int64_t i = 0; i < m.n_bc; ++i)
            if (m.bc_node[i] < 0 || m.bc_node[i] >= m.n_nodes) return fail(nullptr, GD_ERR_ARG, tag + "bad boundary node");
        for (int64_t i = 0; i < m.n_react; ++i)
            if (m.react_node[i] < 0 || m.react_node[i] >= m.n_nodes)
                return fail(nullptr, GD_ERR_ARG, tag + "bad reaction node");
        if (off + m.n_nodes >= ((int64_t)1 << 31) / (dim + 1)) return fail(nullptr, GD_ERR_ARG, "batch too large");
        U.coords.insert(U.coords.end(), m.coords, m.coords + m.n_nodes * dim);
        for (int64_t i = 0; i < m.n_elems * nen; ++i) U.conn.push_back((int32_t)(m.conn[i] + off));
        for (int64_t i = 0; i < m.n_bc; ++i) {
            U.bc_node.push_back((int32_t)(m.bc_node[i] + off));
            U.bc_comp.push_back(m.bc_comp[i]);
            U.bc_scale.push_back(m.bc_scale[i]);
        }
        for (int64_t i = 0; i < m.n_react; ++i) U.react_node.push_back((int32_t)(m.react_node[i] + off));
        U.react_comp.push_back(m.react_comp);
        U.node_off.push_back(off + m.n_nodes);
        U.elem_off.push_back(U.elem_off.back() + m.n_elems);
        U.bc_off.push_back(U.bc_off.back() + m.n_bc);
        U.react_off.push_back(U.react_off.back() + m.n_react);
    }
    gd_mesh &M = U.mesh;
    M.dim = dim;
    M.n_nodes = U.node_off.back();
    M.n_elems = U.elem_off.back();
    M.coords = U.coords.data();
    M.conn = U.conn.data();
    M.n_bc = U.bc_off.back();
    M.bc_node = U.bc_node.data();
    M.bc_comp = U.bc_comp.data();
    M.bc_scale = U.bc_scale.data();
    M.n_react = U.react_off.back();
    M.react_node = U.react_node.data();
    M.react_comp = meshes[0].react_comp;
    return GD_OK;
}

static gd_status create_impl(int32_t n_spec, const gd_mesh *meshes, const gd_icnn *psis, const gd_icnn *ylds,
                      const gd_material *mat, const gd_load_path *paths, const gd_options *opt, gd_handle **out)
{
    if (!out) return fail(nullptr, GD_ERR_ARG, "out is null");
    *out = nullptr;
    if (n_spec < 1) return fail(nullptr, GD_ERR_ARG, "n_spec must be at least 1");
    if (!meshes || !mat || !paths) return fail(nullptr, GD_ERR_ARG, "mesh, material or load path is null");
    if (mat->energy < 0 || mat->energy > 2) return fail(nullptr, GD_ERR_ARG, "unknown energy kind");
    if (!(mat->eta_d > 0.0)) return fail(nullptr, GD_ERR_ARG, "eta_d must be positive");
    gd_status st;
    for (int s = 0; s < n_spec; ++s) {
        const gd_load_path *path = paths + s;
        if (path->n_steps < 0 || (path->n_steps > 0 && !path->load)) return fail(nullptr, GD_ERR_ARG, "load path");
        if (mat->energy != GD_ENERGY_NEO_HOOKE && (st = validate_net(psis ? psis + s : nullptr, 3, false, "energy")))
            return st;
        if ((st = validate_net(ylds ? ylds + s : nullptr, 1, true, "yield"))) return st;
    }
    const gd_icnn *psi = psis, *yield = ylds;
    const gd_load_path *path = paths;
    Union U;
    const gd_mesh *mesh = meshes;
    if (n_spec > 1) {
        if ((st = build_union(n_spec, meshes, U))) return st;
        mesh = &U.mesh;
    }
    gd_options o;
    if (opt) o = *opt;
    else gd_default_options(&o);
    if (o.precision != GD_FP64 && o.precision != GD_MIXED) return fail(nullptr, GD_ERR_ARG, "precision");
    // FP32 element math resolves the residual to ~1e-5 of its scale
    if (o.precision == GD_MIXED && o.newton_rtol < 1e-5) o.newton_rtol = 1e-5;
    if (o.newton_max < 0 || o.krylov_max < 1 || o.local_max < 1 || o.line_search_max < 0)
        return fail(nullptr, GD_ERR_ARG, "iteration caps");
    if (o.inner_solve < GD_INNER_AUTO || o.inner_solve > GD_INNER_REFINED)
        return fail(nullptr, GD_ERR_ARG, "inner_solve");
    if (o.coarse < 0 || o.coarse > gd::kCoarseMax) return fail(nullptr, GD_ERR_ARG, "coarse must be in [0, 3072]");
    if (o.scheme != GD_MONOLITHIC && o.scheme != GD_STAGGERED && o.scheme != GD_STAGGERED_ITERATED)
        return fail(nullptr, GD_ERR_ARG, "scheme");
    if (o.scheme != GD_MONOLITHIC && n_spec > 1)
        return fail(nullptr, GD_ERR_ARG, "the staggered schemes need one specimen");
    if (o.scheme == GD_STAGGERED_ITERATED && o.stagger_max < 1)
        return fail(nullptr, GD_ERR_ARG, "the iterated staggered scheme needs stagger_max >= 1");
    if (o.asm_grid_max < 0) return fail(nullptr, GD_ERR_ARG, "asm_grid_max must be >= 0");
    if (o.krylov_row_cache < 0 || o.krylov_row_cache > 2)
        return fail(nullptr, GD_ERR_ARG, "krylov_row_cache must be 0, 1 or 2");
    if (o.icnn_mma < GD_ICNN_AUTO || o.icnn_mma > GD_ICNN_BF16X3) return fail(nullptr, GD_ERR_ARG, "icnn_mma");
    if (o.krylov != GD_BICGSTAB && o.krylov != GD_GMRES) return fail(nullptr, GD_ERR_ARG, "krylov");
    if (o.gmres_m < 1 || o.gmres_m > gd::gmres_max_m()) return fail(nullptr, GD_ERR_ARG, "gmres_m must be in [1, 64]");
    if (n_spec > 1 && o.precision == GD_MIXED && (o.icnn_mma == GD_ICNN_BF16 || o.icnn_mma == GD_ICNN_BF16X3))
        return fail(nullptr, GD_ERR_ARG, "the tensor-core networks need a single specimen (one weight set per launch)");

    const int dim = mesh->dim, nen = dim == 2 ? 4 : 8, ndof = dim + 1;
    const int64_t NN = mesh->n_nodes, NE = mesh->n_elems;
    Pattern P;
    if ((st = build_pattern(mesh, P))) return st;
    if (n_spec > 1)                          // each specimen's own reaction component
        for (int s = 0; s < n_spec; ++s)
            for (int64_t j = U.react_off[s]; j < U.react_off[s + 1]; ++j)
                P.react[j] = (int32_t)((int64_t)U.react_node[j] * ndof + U.react_comp[s]);
    std::vector<uint8_t> &fixed = P.fixed;
    std::vector<int32_t> &bc_dof = P.bc_dof, &react = P.react, &slot = P.slot;
    const int64_t n_dofs = NN * ndof, nnz = P.nnz;
    gd_handle *hh = new gd_handle();
    gd::Handle &H = hh->h;
    H.h_rowptr.swap(P.rowptr);
    H.h_colidx.swap(P.colidx);
    for (size_t r = 0; r + 1 < H.h_rowptr.size(); ++r)
        H.krylov_lmax = std::max(H.krylov_lmax, H.h_rowptr[r + 1] - H.h_rowptr[r]);
    H.dim = dim;
    H.nen = nen;
    H.nq = nen;
    H.ndof = ndof;
    H.n_nodes = NN;
    H.n_elems = NE;
    H.n_dofs = n_dofs;
    H.nnz = nnz;
    H.opt = o;
    H.asm_tune.grid_max = o.asm_grid_max;
    H.stream = (cudaStream_t)o.cuda_stream;
    H.load.assign(path->load, path->load + path->n_steps);
    H.n_spec = n_spec;
    H.paths.resize(n_spec);
    for (int s = 0; s < n_spec; ++s) {
        H.paths[s].assign(paths[s].load, paths[s].load + paths[s].n_steps);
        H.n_steps_max = std::max(H.n_steps_max, paths[s].n_steps);
    }
    H.mat.mu_e = mat->mu_e;
    H.mat.lambda_e = mat->lambda_e;
    H.mat.eta_d = mat->eta_d;
    H.mat.kappa_d = mat->kappa_d;
    H.mat.beta_d = mat->beta_d;
    H.mat.c_d = mat->c_d;
    H.mat.gamma_d = mat->gamma_d;
    H.mat.qcoef = (mat->gamma_d != 0.0 && mat->beta_d != 0.0) ? mat->gamma_d * mat->beta_d / mat->eta_d : 0.0;
    H.mat.energy = mat->energy;
    H.mat.local_max = o.local_max;
    H.n_bc = mesh->n_bc;
    H.n_react = mesh->n_react;

    auto bail = [&](gd_status s) {
        g_create_error = H.err;
        gd_destroy(hh);
        return s;
    };
#define GD_CREATE_CUDA(call)                                                                               \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) {                                                                           \
            (void)cudaGetLastError();                                                                      \
            H.err = std::string(#call) + ": " + cudaGetErrorString(e_);                                    \
            return bail(e_ == cudaErrorMemoryAllocation ? GD_ERR_OOM : GD_ERR_CUDA);                       \
        }                                                                                                  \
    } while (0)

    int dev = 0;
    GD_CREATE_CUDA(cudaGetDevice(&dev));
    GD_CREATE_CUDA(cudaDeviceGetAttribute(&H.num_sms, cudaDevAttrMultiProcessorCount, dev));
    GD_CREATE_CUDA(cudaEventCreate(&H.ev0));
    GD_CREATE_CUDA(cudaEventCreate(&H.ev1));
    GD_CREATE_CUDA(cudaEventCreate(&H.kv0));
    GD_CREATE_CUDA(cudaEventCreate(&H.kv1));
    GD_CREATE_CUDA(dalloc(&H.X, (size_t)(NN * dim)));
    GD_CREATE_CUDA(dalloc(&H.conn, (size_t)(NE * nen)));
    GD_CREATE_CUDA(dalloc(&H.slot, slot.size()));
    GD_CREATE_CUDA(dalloc(&H.rowptr, H.h_rowptr.size()));
    GD_CREATE_CUDA(dalloc(&H.colidx, H.h_colidx.size()));
    GD_CREATE_CUDA(dalloc(&H.fixed, fixed.size()));
    GD_CREATE_CUDA(dalloc(&H.bc_dof, bc_dof.size()));
    GD_CREATE_CUDA(dalloc(&H.bc_scale, bc_dof.size()));
    GD_CREATE_CUDA(dalloc(&H.react_dof, react.size()));
    GD_CREATE_CUDA(cudaMemcpy(H.X, mesh->coords, sizeof(double) * NN * dim, cudaMemcpyHostToDevice));
    if (NE > 0) {
        GD_CREATE_CUDA(cudaMemcpy(H.conn, mesh->conn, sizeof(int32_t) * NE * nen, cudaMemcpyHostToDevice));
        GD_CREATE_CUDA(cudaMemcpy(H.slot, slot.data(), sizeof(int32_t) * slot.size(), cudaMemcpyHostToDevice));
    }
    GD_CREATE_CUDA(cudaMemcpy(H.rowptr, H.h_rowptr.data(), sizeof(int32_t) * H.h_rowptr.size(), cudaMemcpyHostToDevice));
    if (nnz > 0)
        GD_CREATE_CUDA(cudaMemcpy(H.colidx, H.h_colidx.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
    GD_CREATE_CUDA(cudaMemcpy(H.fixed, fixed.data(), fixed.size(), cudaMemcpyHostToDevice));
    if (!bc_dof.empty()) {
        GD_CREATE_CUDA(cudaMemcpy(H.bc_dof, bc_dof.data(), sizeof(int32_t) * bc_dof.size(), cudaMemcpyHostToDevice));
        GD_CREATE_CUDA(cudaMemcpy(H.bc_scale, mesh->bc_scale, sizeof(double) * bc_dof.size(), cudaMemcpyHostToDevice));
    }
    if (!react.empty())
        GD_CREATE_CUDA(cudaMemcpy(H.react_dof, react.data(), sizeof(int32_t) * react.size(), cudaMemcpyHostToDevice));
    // networks
    if (n_spec == 1) {
        if (mat->energy != GD_ENERGY_NEO_HOOKE) {
            if ((st = stage_net(H, H.psi, 3, psi->width, psi->params))) return bail(st);
        }
        if ((st = stage_net(H, H.yld, 1, yield->width, yield->params))) return bail(st);
        GD_CREATE_CUDA(dalloc(&H.netc, 1));
        GD_CREATE_CUDA(gd::launch_prep_nets(H.psi, H.yld, H.mat.energy, H.netc, H.stream));
        H.wmax = std::max(H.psi.width, H.yld.width);
        // tensor-core networks: the weight blob the element kernel stages per CTA
        H.icnn_mode = o.icnn_mma == GD_ICNN_AUTO ? GD_ICNN_BF16X3 : o.icnn_mma;
        if (o.precision == GD_MIXED && H.icnn_mode != GD_ICNN_CUDA_CORES) {
            H.tc = gd::tc_layout(H.psi.width, H.yld.width, H.icnn_mode == GD_ICNN_BF16X3);
            GD_CREATE_CUDA(dalloc(&H.tc_blob, (size_t)H.tc.bytes));
            GD_CREATE_CUDA(gd::tc_build_blob(H.psi, H.yld, H.tc, H.tc_blob, H.stream));
        }
    } else {
        H.icnn_mode = GD_ICNN_CUDA_CORES;
        // per-specimen networks in device tables indexed by the element's specimen
        H.h_psi_tab.resize(n_spec);
        H.h_yld_tab.resize(n_spec);
        GD_CREATE_CUDA(dalloc(&H.netc, (size_t)n_spec));
        for (int s = 0; s < n_spec; ++s) {
            if (mat->energy != GD_ENERGY_NEO_HOOKE) {
                if ((st = stage_net(H, H.h_psi_tab[s], 3, psis[s].width, psis[s].params))) return bail(st);
            }
            if ((st = stage_net(H, H.h_yld_tab[s], 1, ylds[s].width, ylds[s].params))) return bail(st);
            GD_CREATE_CUDA(gd::launch_prep_nets(H.h_psi_tab[s], H.h_yld_tab[s], H.mat.energy, H.netc + s, H.stream));
            H.wmax = std::max(H.wmax, std::max(H.h_psi_tab[s].width, H.h_yld_tab[s].width));
        }
        GD_CREATE_CUDA(dalloc(&H.psi_tab, (size_t)n_spec));
        GD_CREATE_CUDA(dalloc(&H.yld_tab, (size_t)n_spec));
        GD_CREATE_CUDA(cudaMemcpy(H.psi_tab, H.h_psi_tab.data(), sizeof(gd::DevNet) * n_spec, cudaMemcpyHostToDevice));
        GD_CREATE_CUDA(cudaMemcpy(H.yld_tab, H.h_yld_tab.data(), sizeof(gd::DevNet) * n_spec, cudaMemcpyHostToDevice));
        // specimen maps
        std::vector<int32_t> es((size_t)NE), ns((size_t)NN), bs((size_t)mesh->n_bc);
        for (int s = 0; s < n_spec; ++s) {
            for (int64_t e = U.elem_off[s]; e < U.elem_off[s + 1]; ++e) es[e] = s;
            for (int64_t n = U.node_off[s]; n < U.node_off[s + 1]; ++n) ns[n] = s;
            for (int64_t i = U.bc_off[s]; i < U.bc_off[s + 1]; ++i) bs[i] = s;
            H.spec_nbc.push_back(U.bc_off[s + 1] - U.bc_off[s]);
        }
        H.h_node_off = U.node_off;
        H.h_elem_off = U.elem_off;
        GD_CREATE_CUDA(dalloc(&H.elem_spec, es.size()));
        GD_CREATE_CUDA(dalloc(&H.node_spec, ns.size()));
        GD_CREATE_CUDA(dalloc(&H.bc_spec, bs.size()));
        GD_CREATE_CUDA(dalloc(&H.react_off, U.react_off.size()));
        GD_CREATE_CUDA(dalloc(&H.node_off, U.node_off.size()));
        GD_CREATE_CUDA(dalloc(&H.d_load, (size_t)2 * n_spec));
        GD_CREATE_CUDA(dalloc(&H.d_norm, (size_t)2 * n_spec));
        GD_CREATE_CUDA(dalloc(&H.d_coef, (size_t)n_spec));
        GD_CREATE_CUDA(dalloc(&H.d_pw, (size_t)3 * n_spec));
        if (NE > 0) GD_CREATE_CUDA(cudaMemcpy(H.elem_spec, es.data(), sizeof(int32_t) * es.size(), cudaMemcpyHostToDevice));
        GD_CREATE_CUDA(cudaMemcpy(H.node_spec, ns.data(), sizeof(int32_t) * ns.size(), cudaMemcpyHostToDevice));
        if (!bs.empty()) GD_CREATE_CUDA(cudaMemcpy(H.bc_spec, bs.data(), sizeof(int32_t) * bs.size(), cudaMemcpyHostToDevice));
        GD_CREATE_CUDA(cudaMemcpy(H.react_off, U.react_off.data(), sizeof(int64_t) * U.react_off.size(),
                                  cudaMemcpyHostToDevice));
        GD_CREATE_CUDA(cudaMemcpy(H.node_off, U.node_off.data(), sizeof(int64_t) * U.node_off.size(),
                                  cudaMemcpyHostToDevice));
    }
    // state and work arrays
    const size_t nq_tot = (size_t)(NE * nen);
    double **vec_d[] = {&H.dofs, &H.dofs_prev, &H.w_dofs, &H.w_trial, &H.R, &H.R_trial, &H.diag};
    for (double **p : vec_d) GD_CREATE_CUDA(dalloc(p, (size_t)n_dofs));
    if (o.precision == GD_MIXED) GD_CREATE_CUDA(dalloc(&H.Rabs, (size_t)n_dofs));
    GD_CREATE_CUDA(dalloc(&H.dofs_pp, (size_t)n_dofs));
    for (double *&p : H.kv) GD_CREATE_CUDA(dalloc(&p, (size_t)n_dofs));
    GD_CREATE_CUDA(dalloc(&H.kappa, nq_tot));
    GD_CREATE_CUDA(dalloc(&H.kappa_trial, nq_tot));
    GD_CREATE_CUDA(dalloc(&H.kappa_trial2, nq_tot));
    GD_CREATE_CUDA(dalloc(&H.loading, nq_tot));
    GD_CREATE_CUDA(dalloc(&H.loading2, nq_tot));
    if (o.scheme == GD_STAGGERED_ITERATED) GD_CREATE_CUDA(dalloc(&H.kappa_stag, nq_tot));
    GD_CREATE_CUDA(dalloc(&H.vals, (size_t)nnz));
    GD_CREATE_CUDA(dalloc(&H.vals_trial, (size_t)nnz));
    GD_CREATE_CUDA(dalloc(&H.counters, 8));
    GD_CREATE_CUDA(dalloc(&H.binv, (size_t)(NN * ndof * ndof)));
    GD_CREATE_CUDA(dalloc(&H.vals_f32, (size_t)nnz));
    GD_CREATE_CUDA(dalloc(&H.kx, (size_t)n_dofs));
    H.krylov_grid = gd::krylov_blocks(ndof, o.precision == GD_MIXED, H.num_sms);
    H.krylov_grid32 = gd::krylov_blocks_fp32(ndof, H.num_sms, H.krylov_cpsm32);
    if (H.krylov_grid < 1) {
        H.err = "no cooperative grid fits on this device";
        return bail(GD_ERR_CUDA);
    }
    if (n_spec > 1) {
        gd_status sb = build_batch_krylov(H);
        if (sb) return bail(sb);
    }
    if (o.coarse > 0) {
        // two-level preconditioner: aggregates sized so the coarse unknowns come near
        // the target (larger aggregates when the kept modes exceed the cap)
        gd::CoarseSpace &C = H.coarse;
        C.nm = gd::coarse_modes(dim);
        std::vector<int32_t> agg, coff;
        std::vector<float> Pc;
        int target = (int)std::max<int64_t>(4, (NN * C.nm + o.coarse - 1) / o.coarse);
        int32_t na = 0;
        for (int tries = 0; tries < 8; ++tries) {
            na = gd::coarse_aggregate(NN, ndof, H.h_rowptr, H.h_colidx, target, agg);
            gd::coarse_basis(dim, NN, mesh->coords, fixed.data(), agg, na, Pc, coff);
            if (coff[na] <= gd::kCoarseMax) break;
            target = target * 3 / 2 + 1;
        }
        if (coff[na] > gd::kCoarseMax) {
            H.err = "coarse space larger than 3072 unknowns";
            return bail(GD_ERR_ARG);
        }
        C.n_agg = na;
        C.nc = coff[na];
        if (C.nc > 0) {
            const size_t nc = (size_t)C.nc;
            GD_CREATE_CUDA(dalloc(&C.agg, agg.size()));
            GD_CREATE_CUDA(dalloc(&C.coff, coff.size()));
            GD_CREATE_CUDA(dalloc(&C.node_co, agg.size()));
            GD_CREATE_CUDA(dalloc(&C.P, Pc.size()));
            GD_CREATE_CUDA(dalloc(&C.Ac, nc * nc));
            GD_CREATE_CUDA(dalloc(&C.X32, nc * nc));
            GD_CREATE_CUDA(dalloc(&C.X64, nc * nc));
            GD_CREATE_CUDA(dalloc(&C.rc, 2 * nc));
            GD_CREATE_CUDA(dalloc(&C.cc, nc));
            GD_CREATE_CUDA(dalloc(&C.status, 1));
            GD_CREATE_CUDA(cudaMemcpy(C.agg, agg.data(), sizeof(int32_t) * agg.size(), cudaMemcpyHostToDevice));
            GD_CREATE_CUDA(cudaMemcpy(C.coff, coff.data(), sizeof(int32_t) * coff.size(), cudaMemcpyHostToDevice));
            std::vector<int32_t> nco(agg.size());
            for (size_t i = 0; i < agg.size(); ++i) nco[i] = coff[agg[i]] * 8 + (coff[agg[i] + 1] - coff[agg[i]]);
            GD_CREATE_CUDA(cudaMemcpy(C.node_co, nco.data(), sizeof(int32_t) * nco.size(), cudaMemcpyHostToDevice));
            GD_CREATE_CUDA(cudaMemcpy(C.P, Pc.data(), sizeof(float) * Pc.size(), cudaMemcpyHostToDevice));
        }
    }
    H.red_blocks = 4 * H.num_sms;                    // room for Krylov grids up to 4 CTAs per SM
    GD_CREATE_CUDA(dalloc(&H.red, (size_t)8 * H.red_blocks));
    GD_CREATE_CUDA(dalloc(&H.scal, 64));
    GD_CREATE_CUDA(cudaMemsetAsync(H.dofs, 0, sizeof(double) * n_dofs, H.stream));
    GD_CREATE_CUDA(cudaMemsetAsync(H.dofs_prev, 0, sizeof(double) * n_dofs, H.stream));
    GD_CREATE_CUDA(cudaMemsetAsync(H.kappa, 0, sizeof(double) * nq_tot, H.stream));
    GD_CREATE_CUDA(cudaStreamSynchronize(H.stream));
    *out = hh;
#undef GD_CREATE_CUDA
    return GD_OK;
}

gd_status gd_create(const gd_mesh *mesh, const gd_icnn *psi, const gd_icnn *yield, const gd_material *mat,
                    const gd_load_path *path, const gd_options *opt, gd_handle **out)
{
    if (!mesh || !path) {
        if (out) *out = nullptr;
        return fail(nullptr, GD_ERR_ARG, "mesh, material or load path is null");
    }
    return create_impl(1, mesh, psi, yield, mat, path, opt, out);
}

gd_status gd_create_batch(int32_t n_spec, const gd_mesh *meshes, const gd_icnn *psi, const gd_icnn *yield,
                          const gd_material *mat, const gd_load_path *paths, const gd_options *opt, gd_handle **out)
{
    return create_impl(n_spec, meshes, psi, yield, mat, paths, opt, out);
}

gd_status gd_batch_layout(gd_handle *h, int32_t *n_spec, int64_t *node_off, int64_t *elem_off, int32_t *n_steps)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (n_spec) *n_spec = H.n_spec;
    if (n_steps) *n_steps = H.n_steps_max;
    for (int s = 0; s <= H.n_spec; ++s) {
        const bool one = H.n_spec == 1;
        if (node_off) node_off[s] = one ? (s ? H.n_nodes : 0) : H.h_node_off[s];
        if (elem_off) elem_off[s] = one ? (s ? H.n_elems : 0) : H.h_elem_off[s];
    }
    return GD_OK;
}

gd_status gd_build_pattern(const gd_mesh *mesh, int64_t *n_rows, int64_t *nnz, int32_t *rowptr, int32_t *colidx,
                           int32_t *slot)
{
    Pattern P;
    gd_status st = build_pattern(mesh, P);
    if (st) return st;
    if (n_rows) *n_rows = (int64_t)P.rowptr.size() - 1;
    if (nnz) *nnz = P.nnz;
    if (rowptr) std::memcpy(rowptr, P.rowptr.data(), sizeof(int32_t) * P.rowptr.size());
    if (colidx) std::memcpy(colidx, P.colidx.data(), sizeof(int32_t) * P.colidx.size());
    if (slot) std::memcpy(slot, P.slot.data(), sizeof(int32_t) * P.slot.size());
    return GD_OK;
}

gd_status gd_set_params(gd_handle *h, const double *theta_psi, const double *theta_yield)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (H.n_spec > 1) return fail(&H, GD_ERR_STATE, "a batch keeps the networks given to gd_create_batch");
    if (theta_psi && H.psi.width > 0) {
        GD_CUDA(&H, cudaMemcpyAsync(H.psi.p, theta_psi, sizeof(double) * H.psi.n_params, cudaMemcpyDefault, H.stream));
        GD_CUDA(&H, gd::launch_transpose(H.psi, H.stream));
        GD_CUDA(&H, gd::launch_net_to_float(H.psi, H.stream));
    }
    if (theta_yield && H.yld.width > 0) {
        GD_CUDA(&H, cudaMemcpyAsync(H.yld.p, theta_yield, sizeof(double) * H.yld.n_params, cudaMemcpyDefault, H.stream));
        GD_CUDA(&H, gd::launch_transpose(H.yld, H.stream));
        GD_CUDA(&H, gd::launch_net_to_float(H.yld, H.stream));
    }
    GD_CUDA(&H, gd::launch_prep_nets(H.psi, H.yld, H.mat.energy, H.netc, H.stream));
    if (H.tc_blob) GD_CUDA(&H, gd::tc_build_blob(H.psi, H.yld, H.tc, H.tc_blob, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    H.coarse_age = -1;                       // new networks, new tangents
    H.noise_age = 0;                         // and a new rounding noise of the mixed residual
    return GD_OK;
}

gd_status gd_csr_pattern(gd_handle *h, int64_t *n_rows, int64_t *nnz, int32_t *rowptr, int32_t *colidx)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (n_rows) *n_rows = H.n_dofs;
    if (nnz) *nnz = H.nnz;
    if (rowptr) std::memcpy(rowptr, H.h_rowptr.data(), sizeof(int32_t) * H.h_rowptr.size());
    if (colidx) std::memcpy(colidx, H.h_colidx.data(), sizeof(int32_t) * H.h_colidx.size());
    return GD_OK;
}

gd_status gd_coarse_info(gd_handle *h, int32_t *n_aggregates, int32_t *n_coarse)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "handle is null");
    if (n_aggregates) *n_aggregates = h->h.coarse.nc > 0 ? h->h.coarse.n_agg : 0;
    if (n_coarse) *n_coarse = h->h.coarse.nc;
    return GD_OK;
}

gd_status gd_coarse_aggregates(const gd_mesh *mesh, int32_t target_nodes, int32_t *agg, int32_t *n_aggregates)
{
    if (!agg || !n_aggregates) return fail(nullptr, GD_ERR_ARG, "output arrays are null");
    if (target_nodes < 1) return fail(nullptr, GD_ERR_ARG, "target_nodes must be positive");
    Pattern P;
    gd_status st = build_pattern(mesh, P);
    if (st) return st;
    std::vector<int32_t> a;
    *n_aggregates = gd::coarse_aggregate(mesh->n_nodes, mesh->dim + 1, P.rowptr, P.colidx, target_nodes, a);
    std::memcpy(agg, a.data(), sizeof(int32_t) * a.size());
    return GD_OK;
}

gd_status gd_coarse_basis(const gd_mesh *mesh, int32_t target_nodes, int32_t *agg, int32_t *n_aggregates,
                          int32_t *coff, float *P, int32_t *n_modes)
{
    if (!agg || !n_aggregates || !coff || !P || !n_modes) return fail(nullptr, GD_ERR_ARG, "output arrays are null");
    if (target_nodes < 1) return fail(nullptr, GD_ERR_ARG, "target_nodes must be positive");
    Pattern pat;
    gd_status st = build_pattern(mesh, pat);
    if (st) return st;
    std::vector<int32_t> a, co;
    std::vector<float> Pv;
    const int32_t na = gd::coarse_aggregate(mesh->n_nodes, mesh->dim + 1, pat.rowptr, pat.colidx, target_nodes, a);
    gd::coarse_basis(mesh->dim, mesh->n_nodes, mesh->coords, pat.fixed.data(), a, na, Pv, co);
    std::memcpy(agg, a.data(), sizeof(int32_t) * a.size());
    std::memcpy(coff, co.data(), sizeof(int32_t) * co.size());
    std::memcpy(P, Pv.data(), sizeof(float) * Pv.size());
    *n_aggregates = na;
    *n_modes = gd::coarse_modes(mesh->dim);
    return GD_OK;
}

gd_status gd_assemble(gd_handle *h, const double *dofs, const double *kappa_n, double *R, void *csr_vals,
                      double *kappa_trial, int8_t *loading, int32_t mode)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (!dofs) return fail(&H, GD_ERR_ARG, "dofs is null");
    const int tangent = (mode == GD_ASM_TANGENT && csr_vals) ? 1 : 0;
    gd_status st = assemble_pass(H, dofs, kappa_n ? kappa_n : H.kappa, R, csr_vals, kappa_trial, loading, tangent);
    if (st) return st;
    int hc[4];
    GD_CUDA(&H, cudaMemcpyAsync(hc, H.counters, sizeof(hc), cudaMemcpyDeviceToHost, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    GD_TC_CHECK(&H, hc);
    H.assembly_ms += elapsed_ms(H);
    if (hc[0] > 0) return fail(&H, GD_ERR_LOCAL_SOLVE, std::to_string(hc[0]) + " local solves hit local_max");
    return GD_OK;
}

gd_status gd_spmv(gd_handle *h, const double *x, double *y, int32_t free_only)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (!x || !y) return fail(&H, GD_ERR_ARG, "null vector");
    if (H.opt.precision != GD_FP64) return fail(&H, GD_ERR_ARG, "gd_spmv needs FP64 values");
    gd::SolverCtx c = solver_ctx(H, H.vals);
    GD_CUDA(&H, gd::launch_spmv(c, x, y, free_only));
    return GD_OK;
}

gd_status gd_solve(gd_handle *h, const void *csr_vals, const double *b, double *x, int32_t *iterations,
                   double *rel_residual)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (!b || !x) return fail(&H, GD_ERR_ARG, "null vector");
    int it = 0;
    double rel = 0.0;
    gd_status st = krylov(H, csr_vals ? csr_vals : H.vals, b, x, it, rel, H.opt.krylov_rtol, false, -1.0,
                          csr_vals ? kCallerMatrix : kTangent);
    if (iterations) *iterations = it;
    if (rel_residual) *rel_residual = rel;
    return st;
}

gd_status gd_autotune(gd_handle *h, gd_tune_report *rep)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    gd_tune_report r{};
    for (double &v : r.asm_ms) v = -1.0;
    for (double &v : r.krylov_us) v = -1.0;
    // element kernel: one tangent pass at the committed state per CTA width
    const gd::AsmTune keep = H.asm_tune;
    const int widths[3] = {2, 4, 8};
    double best = 1e300;
    gd::AsmTune pick = keep;
    for (int wi = 0; wi < 3; ++wi) {
        H.asm_tune.warps = widths[wi];
        H.asm_tune.cta_per_sm = 0;
        H.asm_tune.exact = true;
        double tmin = 1e300;
        bool ok = true;
        for (int rep_i = 0; rep_i < 3 && ok; ++rep_i) {
            if (assemble_pass(H, H.dofs, H.kappa, H.R_trial, H.vals_trial, H.kappa_trial2, H.loading2, 1)) {
                ok = false;
                break;
            }
            GD_CUDA(&H, cudaStreamSynchronize(H.stream));
            if (rep_i > 0) tmin = std::min(tmin, elapsed_ms(H));   // the first pass warms up
        }
        cudaGetLastError();
        if (!ok) continue;
        r.asm_ms[wi] = tmin;
        if (tmin < best) {
            best = tmin;
            pick = H.asm_tune;
        }
    }
    pick.exact = false;
    H.asm_tune = pick;
    r.asm_warps = pick.warps;
    // Krylov: a fixed number of iterations on that tangent per grid size
    std::swap(H.vals, H.vals_trial);                 // the tangent just assembled
    const int keep_grid = H.krylov_grid, keep_max = H.opt.krylov_max;
    const bool fp32 = H.opt.precision == GD_MIXED && H.opt.inner_solve == GD_INNER_AUTO;
    const int iters = 40;
    H.opt.krylov_max = iters;
    double kbest = 1e300;
    int kpick = H.krylov_cpsm;
    gd_status st = GD_OK;
    // right-hand side: ones on the free dofs (the committed residual may be zero)
    GD_CUDA(&H, gd::launch_fill(H.kv[9], 1.0, H.n_dofs, H.stream));
    ++H.launches;
    const int keep_grid32 = H.krylov_grid32;
    int kpick32 = H.krylov_cpsm32;
    for (int cap = 1; cap <= 4; ++cap) {
        // the solve timed here runs with FP32 vectors in GD_MIXED: tune that grid
        const int grid = fp32 ? gd::krylov_blocks_fp32(H.ndof, H.num_sms, cap)
                              : gd::krylov_blocks(H.ndof, H.opt.precision == GD_MIXED, H.num_sms, cap);
        if (grid != cap * H.num_sms) continue;       // not co-resident at this width
        if ((size_t)grid > (size_t)4 * H.num_sms) continue;
        if (grid > H.red_blocks) continue;           // beyond the reduction buffers
        if (fp32) H.krylov_grid32 = grid;
        else H.krylov_grid = grid;
        double tmin = 1e300;
        for (int rep_i = 0; rep_i < 2; ++rep_i) {
            int kit = 0;
            double rel = 0.0;
            const double k0 = H.krylov_ms;
            st = krylov(H, H.vals, H.kv[9], H.kv[8], kit, rel, 1e-300, fp32, 1e300);
            if (st) break;
            if (rep_i > 0 && kit > 0) tmin = std::min(tmin, (H.krylov_ms - k0) * 1e3 / kit);
        }
        if (st) break;
        r.krylov_us[cap - 1] = tmin;
        if (tmin < kbest) {
            kbest = tmin;
            if (fp32) kpick32 = cap;
            else kpick = cap;
        }
    }
    if (fp32) {
        H.krylov_cpsm32 = kpick32;
        H.krylov_grid32 = gd::krylov_blocks_fp32(H.ndof, H.num_sms, kpick32);
        if (H.krylov_grid32 < 1) H.krylov_grid32 = keep_grid32;
        H.krylov_grid = keep_grid;
        r.krylov_ctas_per_sm = kpick32;
    } else {
        H.krylov_cpsm = kpick;
        H.krylov_grid = gd::krylov_blocks(H.ndof, H.opt.precision == GD_MIXED, H.num_sms, kpick);
        if (H.krylov_grid < 1) H.krylov_grid = keep_grid;
        r.krylov_ctas_per_sm = kpick;
    }
    // node groups per product round at the chosen grid (the two-level kernel: 1 or 2)
    const int ups[3] = {1, 2, 4};
    double ubest = 1e300;
    int upick = H.krylov_up;
    for (double &v : r.krylov_us_up) v = -1.0;
    for (int ui = 0; ui < (H.coarse.nc > 0 ? 2 : 3) && st == GD_OK; ++ui) {
        H.krylov_up = ups[ui];
        double tmin = 1e300;
        for (int rep_i = 0; rep_i < 2; ++rep_i) {
            int kit = 0;
            double rel = 0.0;
            const double k0 = H.krylov_ms;
            st = krylov(H, H.vals, H.kv[9], H.kv[8], kit, rel, 1e-300, fp32, 1e300);
            if (st) break;
            if (rep_i > 0 && kit > 0) tmin = std::min(tmin, (H.krylov_ms - k0) * 1e3 / kit);
        }
        r.krylov_us_up[ui] = st ? -1.0 : tmin;
        if (!st && tmin < ubest) {
            ubest = tmin;
            upick = ups[ui];
        }
    }
    H.krylov_up = upick;
    r.krylov_up = upick ? upick : 1;
    // lanes per node of the 3D FP32 solve (32: a warp per node; 8 or 4: four or
    // eight nodes per warp, more lanes busy in the vector phases)
    const int lanes[3] = {32, 8, 4};
    double lbest = 1e300;
    int lpick = H.krylov_lanes;
    for (double &v : r.krylov_us_lanes) v = -1.0;
    for (int li = 0; li < 3 && st == GD_OK && H.ndof == 4 && fp32; ++li) {
        H.krylov_lanes = lanes[li];
        double tmin = 1e300;
        for (int rep_i = 0; rep_i < 2; ++rep_i) {
            int kit = 0;
            double rel = 0.0;
            const double k0 = H.krylov_ms;
            st = krylov(H, H.vals, H.kv[9], H.kv[8], kit, rel, 1e-300, fp32, 1e300);
            if (st) break;
            if (rep_i > 0 && kit > 0) tmin = std::min(tmin, (H.krylov_ms - k0) * 1e3 / kit);
        }
        r.krylov_us_lanes[li] = st ? -1.0 : tmin;
        if (!st && tmin < lbest) {
            lbest = tmin;
            lpick = lanes[li];
        }
    }
    H.krylov_lanes = lpick;
    r.krylov_lanes = lpick ? lpick : 32;
    std::swap(H.vals, H.vals_trial);
    H.opt.krylov_max = keep_max;
    if (st) return st;
    if (H.n_spec > 1 && (st = build_batch_krylov(H))) return st;
    if (rep) *rep = r;
    return GD_OK;
}

gd_status gd_newton_step(gd_handle *h, gd_newton_report *rep)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (H.next_step >= H.n_steps_max) return fail(&H, GD_ERR_STATE, "load path already finished");
    if (!H.rec_on) {
        // record the path from here on for gd_backward
        free_ckpts(H);
        H.rec_load.clear();
        H.rec_step.clear();
        H.rec_start_step = H.next_step;
        gd_status s0 = save_ckpt(H, 0);
        if (s0) return s0;
        H.rec_on = true;
    }
    gd_newton_report r{};
    gd_status st = advance(H, (double)(H.next_step + 1), 0, r);
    if (rep) *rep = r;
    if (st) {
        H.rec_on = false;                   // a failed step ends the record
        return st;
    }
    if (H.rec_on && !H.rec_step.empty()) H.rec_step.back() = H.next_step;
    ++H.next_step;
    return GD_OK;
}

gd_status gd_run_load_path(gd_handle *h, double *reaction, gd_path_report *rep)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    gd_path_report pr{};
    const double a0 = H.assembly_ms, k0 = H.krylov_ms;
    const int as0 = H.assemblies;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaEventRecord(t0, H.stream);
    gd_status st = GD_OK;
    while (H.next_step < H.n_steps_max) {
        gd_newton_report r{};
        const int s = H.next_step;
        st = gd_newton_step(h, &r);
        pr.total_newton += r.iterations;
        pr.total_krylov += r.krylov_iterations;
        pr.step_cuts += r.step_cuts;
        if (st) break;
        if (reaction)
            for (int i = 0; i < H.n_spec; ++i) reaction[(size_t)s * H.n_spec + i] = H.last_reac[i];
        ++pr.steps_done;
    }
    cudaEventRecord(t1, H.stream);
    cudaEventSynchronize(t1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    pr.total_ms = ms;
    pr.assembly_ms = H.assembly_ms - a0;
    pr.krylov_ms = H.krylov_ms - k0;
    pr.assemblies = H.assemblies - as0;
    if (rep) *rep = pr;
    return st;
}

gd_status gd_get_fields(gd_handle *h, double *dofs, double *kappa, double *damage)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    const int64_t nq_tot = H.n_elems * H.nq;
    if (dofs) GD_CUDA(&H, cudaMemcpyAsync(dofs, H.dofs, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToHost, H.stream));
    if (kappa)
        GD_CUDA(&H, cudaMemcpyAsync(kappa, H.kappa, sizeof(double) * nq_tot, cudaMemcpyDeviceToHost, H.stream));
    if (damage && nq_tot > 0) {
        // H.kappa_trial2 is scratch between Newton steps
        GD_CUDA(&H, gd::launch_damage_field(H.kappa, nq_tot, H.mat.eta_d, H.mat.kappa_d, H.kappa_trial2, H.stream));
        ++H.launches;
        GD_CUDA(&H, cudaMemcpyAsync(damage, H.kappa_trial2, sizeof(double) * nq_tot, cudaMemcpyDeviceToHost, H.stream));
    }
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    return GD_OK;
}

gd_status gd_set_state(gd_handle *h, const double *dofs, const double *dofs_prev, const double *dofs_prev2,
                       const double *kappa, int32_t next_step)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (next_step < 0 || next_step > H.n_steps_max) return fail(&H, GD_ERR_ARG, "next_step out of range");
    if (dofs_prev && next_step < 1) return fail(&H, GD_ERR_ARG, "dofs_prev needs next_step >= 1");
    if (dofs_prev2 && (!dofs_prev || next_step < 2))
        return fail(&H, GD_ERR_ARG, "dofs_prev2 needs dofs_prev and next_step >= 2");
    if (dofs) GD_CUDA(&H, cudaMemcpyAsync(H.dofs, dofs, sizeof(double) * H.n_dofs, cudaMemcpyHostToDevice, H.stream));
    if (dofs_prev)
        GD_CUDA(&H, cudaMemcpyAsync(H.dofs_prev, dofs_prev, sizeof(double) * H.n_dofs, cudaMemcpyHostToDevice, H.stream));
    if (dofs_prev2)
        GD_CUDA(&H, cudaMemcpyAsync(H.dofs_pp, dofs_prev2, sizeof(double) * H.n_dofs, cudaMemcpyHostToDevice, H.stream));
    if (kappa)
        GD_CUDA(&H, cudaMemcpyAsync(H.kappa, kappa, sizeof(double) * H.n_elems * H.nq, cudaMemcpyHostToDevice, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    H.next_step = next_step;
    H.rec_on = false;
    // A continuation (the state one step back given) keeps the coarse inverse and the
    // mixed-precision noise estimate: the first is recomputed by its own
    // convergence-rate test (and after a failed solve), the second at its usual
    // interval.  A state without that history starts a path anew: both are dropped
    // (an inverse formed at a damaged state preconditions the undamaged one badly).
    if (!dofs_prev) {
        H.coarse_age = -1;
        H.noise_age = 0;
    }
    H.have_prev = dofs_prev != nullptr;
    H.have_pp = dofs_prev2 != nullptr;
    H.load_prev = (double)next_step;
    H.load_prevprev = dofs_prev ? (double)(next_step - 1) : H.load_prev;
    H.load_ppp = dofs_prev2 ? (double)(next_step - 2) : H.load_prevprev;
    return GD_OK;
}

gd_status gd_get_state(gd_handle *h, double *dofs, double *dofs_prev, double *dofs_prev2, double *kappa,
                       int32_t *next_step)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (dofs) GD_CUDA(&H, cudaMemcpyAsync(dofs, H.dofs, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToHost, H.stream));
    if (dofs_prev)
        GD_CUDA(&H, cudaMemcpyAsync(dofs_prev, H.dofs_prev, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToHost, H.stream));
    if (dofs_prev2)
        GD_CUDA(&H, cudaMemcpyAsync(dofs_prev2, H.dofs_pp, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToHost, H.stream));
    if (kappa)
        GD_CUDA(&H, cudaMemcpyAsync(kappa, H.kappa, sizeof(double) * H.n_elems * H.nq, cudaMemcpyDeviceToHost, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    if (next_step) *next_step = H.next_step;
    return GD_OK;
}

gd_status gd_backward(gd_handle *h, const double *dL_dreaction, double *dL_dtheta)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (!dL_dreaction || !dL_dtheta) return fail(&H, GD_ERR_ARG, "null argument");
    if (H.n_spec > 1) return fail(&H, GD_ERR_STATE, "gd_backward takes a single-specimen handle");
    if (H.opt.scheme == GD_STAGGERED)
        return fail(&H, GD_ERR_STATE, "gd_backward differentiates the monolithic step equations, which the "
                                      "staggered scheme's lagged steps do not solve");
    if (!H.rec_on || H.rec_load.empty() || H.ckpts.empty())
        return fail(&H, GD_ERR_STATE, "no recorded load path: run gd_newton_step / gd_run_load_path first");
    const int M = (int)H.rec_load.size();
    const int64_t nq_tot = H.n_elems * H.nq;
    const int kseg = H.opt.checkpoint_every > 0 ? H.opt.checkpoint_every : 1;
    const int n_theta = H.psi.n_params + H.yld.n_params;
    const bool mixed = H.opt.precision == GD_MIXED;
    if (mixed && !H.vals64) GD_CUDA(&H, dalloc(&H.vals64, (size_t)H.nnz));
    // --- work space ---
    if (!H.perm_T) {
        std::vector<int32_t> perm((size_t)H.nnz);
        for (int64_t r = 0; r < H.n_dofs; ++r)
            for (int32_t p = H.h_rowptr[r]; p < H.h_rowptr[r + 1]; ++p) {
                const int32_t c = H.h_colidx[p];
                const int32_t *b0 = H.h_colidx.data() + H.h_rowptr[c], *b1 = H.h_colidx.data() + H.h_rowptr[c + 1];
                perm[p] = (int32_t)(H.h_rowptr[c] + (std::lower_bound(b0, b1, (int32_t)r) - b0));
            }
        GD_CUDA(&H, dalloc(&H.perm_T, (size_t)H.nnz));
        GD_CUDA(&H, cudaMemcpy(H.perm_T, perm.data(), sizeof(int32_t) * H.nnz, cudaMemcpyHostToDevice));
        GD_CUDA(&H, dalloc(&H.vals_T, (size_t)H.nnz));
        for (double *&p : H.adj_v) GD_CUDA(&H, dalloc(&p, (size_t)H.n_dofs));
        GD_CUDA(&H, dalloc(&H.kbar, (size_t)nq_tot));
        GD_CUDA(&H, dalloc(&H.kbar2, (size_t)nq_tot));
        GD_CUDA(&H, dalloc(&H.theta_bar, (size_t)(n_theta > 0 ? n_theta : 1)));
        GD_CUDA(&H, dalloc(&H.glob, 4));
    }
    if (H.seg_cap < kseg + 1) {
        dfree(H.seg);
        H.seg = nullptr;
        GD_CUDA(&H, dalloc(&H.seg, (size_t)(kseg + 1) * (H.n_dofs + nq_tot)));
        H.seg_cap = kseg + 1;
    }
    double *er = H.adj_v[0], *y = H.adj_v[1], *S = H.adj_v[2], *rhs = H.adj_v[3], *lam = H.adj_v[4],
           *w = H.adj_v[5];
    // reaction indicator e_r
    {
        std::vector<double> e((size_t)H.n_dofs, 0.0);
        std::vector<int32_t> rd((size_t)H.n_react);
        if (H.n_react > 0)
            GD_CUDA(&H, cudaMemcpy(rd.data(), H.react_dof, sizeof(int32_t) * H.n_react, cudaMemcpyDeviceToHost));
        for (int32_t d : rd) e[d] += 1.0;
        GD_CUDA(&H, cudaMemcpy(er, e.data(), sizeof(double) * H.n_dofs, cudaMemcpyHostToDevice));
    }
    // save the committed end state, restored at the end
    gd::Checkpoint end;
    {
        gd_status s0 = save_ckpt(H, M);
        if (s0) return s0;
        end = H.ckpts.back();
        H.ckpts.pop_back();
    }
    const int end_step = H.next_step;
    GD_CUDA(&H, cudaMemsetAsync(H.kbar, 0, sizeof(double) * nq_tot, H.stream));
    GD_CUDA(&H, cudaMemsetAsync(H.theta_bar, 0, sizeof(double) * (n_theta > 0 ? n_theta : 1), H.stream));
    GD_CUDA(&H, cudaMemsetAsync(H.glob, 0, sizeof(double) * 4, H.stream));
    gd_status st = GD_OK;
    H.replaying = true;
    for (int ci = (int)H.ckpts.size() - 1; ci >= 0 && st == GD_OK; --ci) {
        const int c0 = H.ckpts[ci].commit;
        const int c1 = (ci + 1 < (int)H.ckpts.size()) ? H.ckpts[ci + 1].commit : M;
        if (c1 <= c0) continue;
        // recompute the segment's states from its checkpoint
        if ((st = restore_ckpt(H, H.ckpts[ci]))) break;
        auto seg_d = [&](int i) { return H.seg + (size_t)i * (H.n_dofs + nq_tot); };
        auto seg_k = [&](int i) { return seg_d(i) + H.n_dofs; };
        GD_CUDA(&H, cudaMemcpyAsync(seg_d(0), H.dofs, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToDevice, H.stream));
        GD_CUDA(&H, cudaMemcpyAsync(seg_k(0), H.kappa, sizeof(double) * nq_tot, cudaMemcpyDeviceToDevice, H.stream));
        for (int c = c0 + 1; c <= c1 && st == GD_OK; ++c) {
            const double target = H.rec_load[c - 1];
            if ((st = predict(H, target))) break;
            gd_newton_report sub{};
            st = newton(H, sub);
            if (st == GD_OK && !sub.converged)
                st = fail(&H, GD_ERR_NOT_CONVERGED, "recomputation of load commit " + std::to_string(c) + " failed");
            if (st) break;
            gd_newton_report cr{};
            if ((st = commit(H, target, cr))) break;
            GD_CUDA(&H, cudaMemcpyAsync(seg_d(c - c0), H.dofs, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToDevice,
                                        H.stream));
            GD_CUDA(&H, cudaMemcpyAsync(seg_k(c - c0), H.kappa, sizeof(double) * nq_tot, cudaMemcpyDeviceToDevice,
                                        H.stream));
        }
        if (st) break;
        // reverse sweep through the segment
        for (int c = c1; c > c0 && st == GD_OK; --c) {
            const int step = H.rec_step[c - 1];
            const double fbar = step >= 0 ? dL_dreaction[step - H.rec_start_step] : 0.0;
            const double *d_c = seg_d(c - c0), *k_c = seg_k(c - c0), *k_p = seg_k(c - c0 - 1);
            // tangent at the converged state of commit c (GD_MIXED: the FP64 element
            // kernel's tangent at the mixed path's state; the adjoint systems are FP64)
            if (mixed) {
                if ((st = assemble_tangent_fp64(H, d_c, k_p, H.R_trial, H.vals64, H.kappa_trial2, H.loading2)))
                    break;
                GD_CUDA(&H, gd::launch_gather(H.vals64, H.perm_T, H.vals_T, H.nnz, H.stream));
            } else {
                if ((st = assemble_pass(H, d_c, k_p, H.R_trial, H.vals, H.kappa_trial2, H.loading2, 1))) break;
                GD_CUDA(&H, gd::launch_gather(H.vals, H.perm_T, H.vals_T, H.nnz, H.stream));
            }
            // source (dkappa/dd)^T kbar
            GD_CUDA(&H, cudaMemsetAsync(S, 0, sizeof(double) * H.n_dofs, H.stream));
            gd::AdjArgs A;
            A.n_elems = H.n_elems;
            A.conn = H.conn;
            A.X = H.X;
            A.dofs = d_c;
            A.kappa_prev = k_p;
            A.kappa_cur = k_c;
            A.w = nullptr;
            A.kbar = H.kbar;
            A.kbar_prev = nullptr;
            A.rhs = S;
            A.theta_bar = H.theta_bar;
            A.glob = H.glob;
            A.psi = H.psi;
            A.yld = H.yld;
            A.netc = H.netc;
            A.mat = H.mat;
            A.mode = 0;
            GD_CUDA(&H, gd::launch_adjoint(H.dim, A, H.num_sms, H.stream));
            // y = K^T e_r
            gd::SolverCtx cT = solver_ctx(H, H.vals_T);
            if (fbar != 0.0) GD_CUDA(&H, gd::launch_spmv(cT, er, y, 0));
            GD_CUDA(&H, gd::launch_adj_rhs(H.n_dofs, S, fbar != 0.0 ? y : nullptr, fbar, H.fixed, rhs, H.stream));
            // K^T lambda = rhs on the free dofs (FP64, refined against the true residual)
            H.adj_fp64 = true;
            st = krylov_true(H, H.vals_T, rhs, lam, H.opt.krylov_rtol);
            H.adj_fp64 = false;
            if (st) break;
            GD_CUDA(&H, gd::launch_axpby(H.n_dofs, w, lam, fbar, er, H.stream));
            A.mode = 1;
            A.w = w;
            A.kbar_prev = H.kbar2;
            A.rhs = nullptr;
            GD_CUDA(&H, gd::launch_adjoint(H.dim, A, H.num_sms, H.stream));
            std::swap(H.kbar, H.kbar2);
        }
    }
    H.replaying = false;
    if (st == GD_OK) {
        GD_CUDA(&H, gd::launch_adjoint_globals(H.psi, H.yld, H.mat.energy, H.glob, H.theta_bar, H.stream));
        if (n_theta > 0)
            GD_CUDA(&H, cudaMemcpyAsync(dL_dtheta, H.theta_bar, sizeof(double) * n_theta, cudaMemcpyDeviceToHost,
                                        H.stream));
    }
    // back to the end of the path
    gd_status s2 = restore_ckpt(H, end);
    dfree(end.dofs);
    dfree(end.dofs_prev);
    dfree(end.kappa);
    H.next_step = end_step;
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    return st ? st : s2;
}

}  // extern "C"
