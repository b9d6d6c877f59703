// gd_api.cu -- C ABI of the library: handle creation (mesh validation, CSR
// pattern of the node graph, per-element slot map, Dirichlet masks, network
// staging), the assembly entry point and the device Newton iteration over the
// quasi-static load path (Sec. 3.2 of arxiv 2604.03411: monolithic scheme,
// warm start from the last converged step, incremental loading).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
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
        if (e_ != cudaSuccess)                                                                             \
            return fail((H), e_ == cudaErrorMemoryAllocation ? GD_ERR_OOM : GD_ERR_CUDA,                   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                               \
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

void free_handle(gd::Handle &H)
{
    void *ptrs[] = {H.X, H.conn, H.slot, H.rowptr, H.colidx, H.fixed, H.bc_dof, H.bc_scale, H.react_dof,
                    H.psi.p, H.psi.W2T, H.yld.p, H.yld.W2T, H.psi.pf, H.psi.W2Tf, H.yld.pf, H.yld.W2Tf, H.netc, H.dofs, H.kappa, H.dofs_prev, H.w_dofs,
                    H.w_trial, H.R, H.R_trial, H.vals, H.vals_trial, H.kappa_trial, H.kappa_trial2, H.loading,
                    H.loading2, H.counters, H.diag, H.binv, H.red, H.scal};
    for (void *p : ptrs) dfree(p);
    for (double *p : H.kv) dfree(p);
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
    a.vals = (tangent && H.opt.precision == GD_FP64) ? (double *)vals : nullptr;
    a.vals32 = (tangent && H.opt.precision == GD_MIXED) ? (float *)vals : nullptr;
    a.kappa_new = kappa_out;
    a.loading = loading;
    a.slot = H.slot;
    a.rowptr = H.rowptr;
    a.psi = H.psi;
    a.yld = H.yld;
    a.netc = H.netc;
    a.mat = H.mat;
    a.tangent = tangent && vals != nullptr;
    a.counters = H.counters;
    return a;
}

// one assembly pass with timing; counters[0] = local failures, [1] = loading points
gd_status assemble_pass(gd::Handle &H, const double *dofs, const double *kappa_n, double *R, void *vals,
                        double *kappa_out, int8_t *loading, int tangent)
{
    const size_t vbytes = H.opt.precision == GD_FP64 ? sizeof(double) : sizeof(float);
    if (R) GD_CUDA(&H, cudaMemsetAsync(R, 0, sizeof(double) * H.n_dofs, H.stream));
    if (tangent && vals) GD_CUDA(&H, cudaMemsetAsync(vals, 0, vbytes * H.nnz, H.stream));
    GD_CUDA(&H, cudaMemsetAsync(H.counters, 0, sizeof(int) * 8, H.stream));
    GD_CUDA(&H, cudaEventRecord(H.ev0, H.stream));
    gd::AsmArgs a = asm_args(H, dofs, kappa_n, R, vals, kappa_out, loading, tangent);
    if (H.opt.precision == GD_FP64) GD_CUDA(&H, gd::launch_assemble_fp64(H.dim, a, H.num_sms, H.stream));
    else GD_CUDA(&H, gd::launch_assemble_fp32(H.dim, a, H.num_sms, H.stream));
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
gd_status krylov(gd::Handle &H, const void *vals, const double *b, double *x, int &iters, double &rel,
                 double rtol)
{
    gd::KrylovCtx kc;
    kc.n_nodes = H.n_nodes;
    kc.ndof = H.ndof;
    kc.rowptr = H.rowptr;
    kc.colidx = H.colidx;
    kc.fixed = H.fixed;
    kc.binv = H.binv;
    for (int k = 0; k < 8; ++k) kc.work[k] = H.kv[k];
    kc.red = H.red;
    kc.out = H.scal + 24;
    kc.stream = H.stream;
    kc.blocks = H.krylov_grid;
    kc.num_sms = H.num_sms;
    GD_CUDA(&H, cudaEventRecord(H.kv0, H.stream));
    GD_CUDA(&H, gd::krylov_solve(kc, vals, H.opt.precision == GD_MIXED, b, x, rtol, H.opt.krylov_max));
    H.launches += 2;
    GD_CUDA(&H, cudaEventRecord(H.kv1, H.stream));
    double kout[3];
    GD_CUDA(&H, cudaMemcpyAsync(kout, H.scal + 24, 3 * sizeof(double), cudaMemcpyDeviceToHost, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    float kms = 0.0f;
    cudaEventElapsedTime(&kms, H.kv0, H.kv1);
    H.krylov_ms += kms;
    iters = (int)kout[0];
    rel = kout[1];
    if (kout[2] != 0.0)
        return fail(&H, GD_ERR_KRYLOV, "BiCGStab stopped (status " + std::to_string((int)kout[2]) +
                                           ", relative residual " + std::to_string(rel) + ")");
    return GD_OK;
}

// Newton iteration for one load value starting from H.w_dofs (already predicted,
// prescribed dofs set).  On return H.w_dofs/H.R/H.kappa_trial hold the last iterate.
gd_status newton(gd::Handle &H, gd_newton_report &rep)
{
    gd_status st = assemble_pass(H, H.w_dofs, H.kappa, H.R, H.vals, H.kappa_trial, H.loading, 1);
    if (st) return st;
    NormPair nr;
    if ((st = norms(H, H.R, nr))) return st;
    H.assembly_ms += elapsed_ms(H);
    int hc[3];
    GD_CUDA(&H, cudaMemcpy(hc, H.counters, 3 * sizeof(int), cudaMemcpyDeviceToHost));
    rep.yield_evals += hc[2];
    double nrm = nr.free_;
    const double r0 = std::max(nr.free_, nr.fixed_);
    rep.residual0 = nrm;
    rep.local_failures = hc[0];
    rep.loading_points = hc[1];
    double *delta = H.kv[8], *rhs = H.kv[9];
    for (int it = 0; it <= H.opt.newton_max; ++it) {
        rep.iterations = it;
        rep.residual = nrm;
        if (!std::isfinite(nrm)) return fail(&H, GD_ERR_NAN, "non-finite residual in the Newton iteration");
        if (nrm <= std::max(H.opt.newton_rtol * r0, H.opt.newton_atol)) {
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
        const double ntol = std::max(H.opt.newton_rtol * r0, H.opt.newton_atol);
        const double eta = std::min(1e-2, std::max(H.opt.krylov_rtol, 0.1 * ntol / nrm));
        int kit = 0;
        double rel = 0.0;
        st = krylov(H, H.vals, rhs, delta, kit, rel, eta);
        rep.krylov_iterations += kit;
        if (st) return st;
        // backtracking line search on ||R_free||
        double alpha = 1.0, nt = 0.0;
        for (int ls = 0; ls <= H.opt.line_search_max; ++ls) {
            GD_CUDA(&H, cudaMemcpyAsync(H.w_trial, H.w_dofs, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToDevice,
                                        H.stream));
            GD_CUDA(&H, gd::launch_axpy_free(c, H.w_trial, delta, alpha));
            if ((st = assemble_pass(H, H.w_trial, H.kappa, H.R_trial, H.vals_trial, H.kappa_trial2, H.loading2, 1)))
                return st;
            if ((st = norms(H, H.R_trial, nr))) return st;
            H.assembly_ms += elapsed_ms(H);
            GD_CUDA(&H, cudaMemcpy(hc, H.counters, 3 * sizeof(int), cudaMemcpyDeviceToHost));
            rep.yield_evals += hc[2];
            nt = nr.free_;
            if ((std::isfinite(nt) && nt <= (1.0 - 1e-4 * alpha) * nrm) || ls == H.opt.line_search_max) break;
            alpha *= 0.5;
            ++rep.line_search_cuts;
        }
        std::swap(H.w_dofs, H.w_trial);
        std::swap(H.R, H.R_trial);
        std::swap(H.vals, H.vals_trial);
        std::swap(H.kappa_trial, H.kappa_trial2);
        std::swap(H.loading, H.loading2);
        rep.local_failures = hc[0];
        rep.loading_points = hc[1];
        nrm = nt;
    }
    rep.converged = 0;
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
    std::swap(H.dofs_prev, H.dofs);
    std::swap(H.dofs, H.w_dofs);            // dofs <- converged iterate
    std::swap(H.kappa, H.kappa_trial);
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    rep.reaction = h[0];
    rep.max_damage = h[1];
    H.load_prevprev = H.load_prev;
    H.load_prev = target;
    H.have_prev = true;
    return GD_OK;
}

gd_status advance(gd::Handle &H, double target, int depth, gd_newton_report &rep)
{
    // predictor: last converged state plus the previous increment scaled to this one
    const double dl = H.load_prev - H.load_prevprev;
    const bool extrap = H.have_prev && dl != 0.0;
    const double factor = extrap ? (target - H.load_prev) / dl : 0.0;
    GD_CUDA(&H, gd::launch_predictor(H.n_dofs, H.w_dofs, H.dofs, extrap ? H.dofs_prev : nullptr, factor, H.bc_dof,
                                     H.bc_scale, H.n_bc, target, H.stream));
    H.launches += H.n_bc > 0 ? 2 : 1;
    gd_newton_report sub{};
    const double a0 = H.assembly_ms, k0 = H.krylov_ms;
    const int n0 = H.assemblies;
    const long long l0 = H.launches;
    gd_status st = newton(H, sub);
    rep.assembly_ms += H.assembly_ms - a0;
    rep.krylov_ms += H.krylov_ms - k0;
    rep.assemblies += H.assemblies - n0;
    rep.yield_evals += sub.yield_evals;
    rep.kernel_launches += H.launches - l0;
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
    if (!sub.converged)
        return fail(&H, GD_ERR_NOT_CONVERGED,
                    "Newton did not converge (residual " + std::to_string(sub.residual) + ")");
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

gd_status gd_create(const gd_mesh *mesh, const gd_icnn *psi, const gd_icnn *yield, const gd_material *mat,
                    const gd_load_path *path, const gd_options *opt, gd_handle **out)
{
    if (!out) return fail(nullptr, GD_ERR_ARG, "out is null");
    *out = nullptr;
    if (!mesh || !mat || !path) return fail(nullptr, GD_ERR_ARG, "mesh, material or load path is null");
    if (mat->energy < 0 || mat->energy > 2) return fail(nullptr, GD_ERR_ARG, "unknown energy kind");
    if (!(mat->eta_d > 0.0)) return fail(nullptr, GD_ERR_ARG, "eta_d must be positive");
    if (path->n_steps < 0 || (path->n_steps > 0 && !path->load)) return fail(nullptr, GD_ERR_ARG, "load path");
    gd_status st;
    if (mat->energy != GD_ENERGY_NEO_HOOKE && (st = validate_net(psi, 3, false, "energy"))) return st;
    if ((st = validate_net(yield, 1, true, "yield"))) return st;
    gd_options o;
    if (opt) o = *opt;
    else gd_default_options(&o);
    if (o.precision != GD_FP64 && o.precision != GD_MIXED) return fail(nullptr, GD_ERR_ARG, "precision");
    // FP32 element math resolves the residual to ~1e-5 of its scale
    if (o.precision == GD_MIXED && o.newton_rtol < 1e-5) o.newton_rtol = 1e-5;
    if (o.newton_max < 0 || o.krylov_max < 1 || o.local_max < 1 || o.line_search_max < 0)
        return fail(nullptr, GD_ERR_ARG, "iteration caps");

    const int dim = mesh->dim, nen = dim == 2 ? 4 : 8, ndof = dim + 1;
    const int64_t NN = mesh->n_nodes, NE = mesh->n_elems;
    Pattern P;
    if ((st = build_pattern(mesh, P))) return st;
    std::vector<uint8_t> &fixed = P.fixed;
    std::vector<int32_t> &bc_dof = P.bc_dof, &react = P.react, &slot = P.slot;
    const int64_t n_dofs = NN * ndof, nnz = P.nnz;
    gd_handle *hh = new gd_handle();
    gd::Handle &H = hh->h;
    H.h_rowptr.swap(P.rowptr);
    H.h_colidx.swap(P.colidx);
    H.dim = dim;
    H.nen = nen;
    H.nq = nen;
    H.ndof = ndof;
    H.n_nodes = NN;
    H.n_elems = NE;
    H.n_dofs = n_dofs;
    H.nnz = nnz;
    H.opt = o;
    H.stream = (cudaStream_t)o.cuda_stream;
    H.load.assign(path->load, path->load + path->n_steps);
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
    if (mat->energy != GD_ENERGY_NEO_HOOKE) {
        if ((st = stage_net(H, H.psi, 3, psi->width, psi->params))) return bail(st);
    }
    if ((st = stage_net(H, H.yld, 1, yield->width, yield->params))) return bail(st);
    GD_CREATE_CUDA(dalloc(&H.netc, 1));
    GD_CREATE_CUDA(gd::launch_prep_nets(H.psi, H.yld, H.mat.energy, H.netc, H.stream));
    // state and work arrays
    const size_t nq_tot = (size_t)(NE * nen);
    double **vec_d[] = {&H.dofs, &H.dofs_prev, &H.w_dofs, &H.w_trial, &H.R, &H.R_trial, &H.diag};
    for (double **p : vec_d) GD_CREATE_CUDA(dalloc(p, (size_t)n_dofs));
    for (double *&p : H.kv) GD_CREATE_CUDA(dalloc(&p, (size_t)n_dofs));
    GD_CREATE_CUDA(dalloc(&H.kappa, nq_tot));
    GD_CREATE_CUDA(dalloc(&H.kappa_trial, nq_tot));
    GD_CREATE_CUDA(dalloc(&H.kappa_trial2, nq_tot));
    GD_CREATE_CUDA(dalloc(&H.loading, nq_tot));
    GD_CREATE_CUDA(dalloc(&H.loading2, nq_tot));
    GD_CREATE_CUDA(dalloc(&H.vals, (size_t)nnz));
    GD_CREATE_CUDA(dalloc(&H.vals_trial, (size_t)nnz));
    GD_CREATE_CUDA(dalloc(&H.counters, 8));
    GD_CREATE_CUDA(dalloc(&H.binv, (size_t)(NN * ndof * ndof)));
    H.krylov_grid = gd::krylov_blocks(ndof, o.precision == GD_MIXED, H.num_sms);
    if (H.krylov_grid < 1) {
        H.err = "no cooperative grid fits on this device";
        return bail(GD_ERR_CUDA);
    }
    H.red_blocks = 2 * H.num_sms;
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
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
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

gd_status gd_assemble(gd_handle *h, const double *dofs, const double *kappa_n, double *R, void *csr_vals,
                      double *kappa_trial, int8_t *loading, int32_t mode)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (!dofs) return fail(&H, GD_ERR_ARG, "dofs is null");
    const int tangent = (mode == GD_ASM_TANGENT && csr_vals) ? 1 : 0;
    gd_status st = assemble_pass(H, dofs, kappa_n ? kappa_n : H.kappa, R, csr_vals, kappa_trial, loading, tangent);
    if (st) return st;
    int hc[2];
    GD_CUDA(&H, cudaMemcpyAsync(hc, H.counters, sizeof(hc), cudaMemcpyDeviceToHost, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
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
    gd_status st = krylov(H, csr_vals ? csr_vals : H.vals, b, x, it, rel, H.opt.krylov_rtol);
    if (iterations) *iterations = it;
    if (rel_residual) *rel_residual = rel;
    return st;
}

gd_status gd_newton_step(gd_handle *h, gd_newton_report *rep)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (H.next_step >= (int)H.load.size()) return fail(&H, GD_ERR_STATE, "load path already finished");
    gd_newton_report r{};
    gd_status st = advance(H, H.load[H.next_step], 0, r);
    if (rep) *rep = r;
    if (st) return st;
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
    while (H.next_step < (int)H.load.size()) {
        gd_newton_report r{};
        const int s = H.next_step;
        st = gd_newton_step(h, &r);
        pr.total_newton += r.iterations;
        pr.total_krylov += r.krylov_iterations;
        pr.step_cuts += r.step_cuts;
        if (st) break;
        if (reaction) reaction[s] = r.reaction;
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

gd_status gd_get_fields(gd_handle *h, double *dofs, double *kappa)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (dofs) GD_CUDA(&H, cudaMemcpyAsync(dofs, H.dofs, sizeof(double) * H.n_dofs, cudaMemcpyDeviceToHost, H.stream));
    if (kappa)
        GD_CUDA(&H, cudaMemcpyAsync(kappa, H.kappa, sizeof(double) * H.n_elems * H.nq, cudaMemcpyDeviceToHost, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    return GD_OK;
}

gd_status gd_set_state(gd_handle *h, const double *dofs, const double *kappa, int32_t next_step)
{
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    gd::Handle &H = h->h;
    if (next_step < 0 || next_step > (int)H.load.size()) return fail(&H, GD_ERR_ARG, "next_step out of range");
    if (dofs) GD_CUDA(&H, cudaMemcpyAsync(H.dofs, dofs, sizeof(double) * H.n_dofs, cudaMemcpyHostToDevice, H.stream));
    if (kappa)
        GD_CUDA(&H, cudaMemcpyAsync(H.kappa, kappa, sizeof(double) * H.n_elems * H.nq, cudaMemcpyHostToDevice, H.stream));
    GD_CUDA(&H, cudaStreamSynchronize(H.stream));
    H.next_step = next_step;
    H.have_prev = false;
    H.load_prev = next_step > 0 ? H.load[next_step - 1] : 0.0;
    H.load_prevprev = H.load_prev;
    return GD_OK;
}

gd_status gd_backward(gd_handle *h, const double *dL_dreaction, double *dL_dtheta)
{
    (void)dL_dreaction;
    (void)dL_dtheta;
    if (!h) return fail(nullptr, GD_ERR_ARG, "null handle");
    return fail(&h->h, GD_ERR_STATE, "gd_backward: the adjoint is not built into this library yet");
}

}  // extern "C"
