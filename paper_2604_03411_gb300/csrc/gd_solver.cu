// gd_solver.cu -- device linear algebra for the global Newton iteration:
// CSR SpMV over the node-block pattern, Jacobi preconditioning, FP64
// reductions and a Jacobi-preconditioned BiCGStab (van der Vorst, 1992) whose
// scalars live in device memory so that an iteration needs no host round trip.
//
// The paper solves every Newton system with a direct LU factorisation and
// warm-starts each load step from the last converged state (Sec. 3.2); here
// the linear systems are solved iteratively on the device.  Prescribed
// displacement components are eliminated implicitly: Krylov vectors are zero
// on prescribed dofs and the operator acts as the identity there.
#include <cuda_runtime.h>

#include <cmath>

#include "gd_internal.cuh"

namespace gd {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block reduction of up to 4 values; thread 0 writes red[slot_k * nb + blockIdx.x]
template <int K>
__device__ __forceinline__ void block_partials(double (&v)[K], double *red, const int (&slot)[K], int nb)
{
    __shared__ double sh[K][kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = warp_sum(v[k]);
        if (lane == 0) sh[k][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = (lane < kThreads / 32) ? sh[k][lane] : 0.0;
            s = warp_sum(s);
            if (lane == 0) red[slot[k] * nb + blockIdx.x] = s;
        }
    }
}

// every block sums the nb partials of a slot (deterministic order)
__device__ __forceinline__ double sum_partials(const double *red, int slot, int nb)
{
    __shared__ double sh[kThreads / 32];
    __shared__ double res;
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += red[slot * nb + i];
    s = warp_sum(s);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = (lane < (int)(blockDim.x / 32)) ? sh[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) res = t;
    }
    __syncthreads();
    return res;
}

// plain y = A x (free_only: prescribed rows y = x, prescribed columns skipped)
template <int NDOF, class V>
__global__ void __launch_bounds__(kThreads) spmv_plain_kernel(int64_t n_nodes, const int32_t *__restrict__ rowptr,
                                                              const int32_t *__restrict__ colidx,
                                                              const V *__restrict__ vals,
                                                              const uint8_t *__restrict__ fixed,
                                                              const double *__restrict__ x, double *__restrict__ y,
                                                              int free_only)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    for (int64_t nd = warp0; nd < n_nodes; nd += nwarps) {
        const int64_t r0 = nd * NDOF;
        const int32_t base = rowptr[r0];
        const int32_t len = rowptr[r0 + 1] - base;
        double acc[NDOF];
#pragma unroll
        for (int i = 0; i < NDOF; ++i) acc[i] = 0.0;
        for (int j = lane; j < len; j += 32) {
            const int32_t c = colidx[base + j];
            const double xv = (free_only && fixed[c]) ? 0.0 : x[c];
#pragma unroll
            for (int i = 0; i < NDOF; ++i) acc[i] += (double)vals[base + (int64_t)i * len + j] * xv;
        }
#pragma unroll
        for (int i = 0; i < NDOF; ++i) acc[i] = warp_sum(acc[i]);
        if (lane < NDOF) {
            double v = 0.0;
#pragma unroll
            for (int i = 0; i < NDOF; ++i)
                if (i == lane) v = acc[i];
            const int64_t r = r0 + lane;
            if (free_only && fixed[r]) v = x[r];
            y[r] = v;
        }
    }
}

// partial slots in red[] of the vector kernels: 5, 6 norms and residuals
enum { S_MISC = 5 };

__global__ void __launch_bounds__(kThreads) norm_free_kernel(int64_t n, const double *__restrict__ v,
                                                             const uint8_t *__restrict__ fixed, double *red, int nb)
{
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x = v[i];
        if (fixed[i]) b += x * x; else a += x * x;
    }
    double v2[2] = {a, b};
    const int sl[2] = {S_MISC, S_MISC + 1};
    block_partials<2>(v2, red, sl, nb);
}

__global__ void norm_finish_kernel(const double *red, int nb, double *out_free, double *out_fixed)
{
    double a = sum_partials(red, S_MISC, nb);
    double b = sum_partials(red, S_MISC + 1, nb);
    if (threadIdx.x == 0) {
        *out_free = sqrt(a);
        if (out_fixed) *out_fixed = sqrt(b);
    }
}

__global__ void axpy_free_kernel(int64_t n, double *y, const double *x, double alpha, const uint8_t *fixed)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!fixed[i]) y[i] += alpha * x[i];
}

// out = cur + factor (cur - prev) (prev null: out = cur), then prescribed dofs = scale * load
__global__ void predictor_kernel(int64_t n, double *out, const double *cur, const double *prev, double factor)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = prev ? cur[i] + factor * (cur[i] - prev[i]) : cur[i];
}
// quadratic extrapolation through three converged states: out = w0 x0 + w1 x1 + w2 x2
__global__ void predictor3_kernel(int64_t n, double *out, const double *x0, const double *x1, const double *x2,
                                  double w0, double w1, double w2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = w0 * x0[i] + w1 * x1[i] + w2 * x2[i];
}
__global__ void set_bc_kernel(double *out, const int32_t *bc_dof, const double *bc_scale, int64_t n_bc, double load)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_bc; i += (int64_t)gridDim.x * blockDim.x)
        out[bc_dof[i]] = bc_scale[i] * load;
}

// batched specimens: per-specimen extrapolation factor and prescribed load
// batched specimens: per-specimen weights of the current, previous and earlier state
// (w[3 s + 0..2]; an absent state has weight 0)
__global__ void predictor_batch_kernel(int64_t n, int ndof, double *out, const double *cur, const double *prev,
                                       const double *pp, const double *w, const int32_t *node_spec)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double *ws = w + 3 * node_spec[i / ndof];
        double v = ws[0] == 1.0 ? cur[i] : ws[0] * cur[i];
        if (prev && ws[1] != 0.0) v += ws[1] * prev[i];
        if (pp && ws[2] != 0.0) v += ws[2] * pp[i];
        out[i] = v;
    }
}
__global__ void set_bc_batch_kernel(double *out, const int32_t *bc_dof, const double *bc_scale, const int32_t *bc_spec,
                                    const double *load, int64_t n_bc)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_bc; i += (int64_t)gridDim.x * blockDim.x)
        out[bc_dof[i]] = bc_scale[i] * load[bc_spec[i]];
}
// one block per specimen: sum of R over its reaction dofs [off[s], off[s+1])
__global__ void reaction_batch_kernel(const double *R, const int32_t *react_dof, const int64_t *off, double *out)
{
    const int s = blockIdx.x;
    double acc = 0.0;
    for (int64_t j = off[s] + threadIdx.x; j < off[s + 1]; j += blockDim.x) acc += R[react_dof[j]];
    __shared__ double sh[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) out[s] = t;
    }
}

// one block per specimen: ||R|| over its free and its prescribed dofs
// (dofs [node_off[s] * ndof, node_off[s + 1] * ndof))
__global__ void norms_batch_kernel(const double *R, const uint8_t *fixed, const int64_t *node_off, int ndof,
                                   double *out)
{
    const int s = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int64_t i = node_off[s] * ndof + threadIdx.x; i < node_off[s + 1] * ndof; i += blockDim.x) {
        const double r = R[i];
        if (fixed[i]) b += r * r;
        else a += r * r;
    }
    __shared__ double sa[32], sb[32];
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool in = threadIdx.x < blockDim.x / 32;
        a = warp_sum(in ? sa[threadIdx.x] : 0.0);
        b = warp_sum(in ? sb[threadIdx.x] : 0.0);
        if (threadIdx.x == 0) {
            out[2 * s] = sqrt(a);
            out[2 * s + 1] = sqrt(b);
        }
    }
}

// free dofs: out = coef[spec] * in (accumulate = 0) or out += coef[spec] * in
// (accumulate = 1); prescribed dofs: 0 (accumulate = 0) or unchanged
__global__ void scale_spec_kernel(int64_t n, int ndof, double *out, const double *in, const double *coef,
                                  const int32_t *node_spec, const uint8_t *fixed, int accumulate)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = fixed[i] ? 0.0 : coef[node_spec[i / ndof]] * in[i];
        out[i] = accumulate ? out[i] + v : v;
    }
}

__global__ void reaction_kernel(const double *R, const int32_t *react_dof, int64_t n_react, double *out)
{
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n_react; i += blockDim.x) s += R[react_dof[i]];
    __shared__ double sh[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) *out = t;
    }
}

// d = 1 - f_d(kappa) = 1 - exp(-eta_d <kappa - kappa_d>_+) at every quadrature point
__global__ void damage_field_kernel(const double *kappa, int64_t n, double eta_d, double kappa_d, double *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double k = kappa[i];
        out[i] = k > kappa_d ? -expm1(-eta_d * (k - kappa_d)) : 0.0;
    }
}

__global__ void damage_max_kernel(const double *kappa, int64_t n, double eta_d, double kappa_d, double *out)
{
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, kappa[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < (int)(blockDim.x / 32); ++i) m = fmax(m, sh[i]);
        *out = m > kappa_d ? -expm1(-eta_d * (m - kappa_d)) : 0.0;
    }
}

inline void count(const SolverCtx &c, int n = 1)
{
    if (c.launches) *c.launches += n;
}

__global__ void gather_kernel(const double *in, const int32_t *perm, double *out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}
// out = -(fbar y + s) on free dofs, 0 on prescribed dofs
__global__ void adj_rhs_kernel(int64_t n, const double *s, const double *y, double fbar, const uint8_t *fixed,
                               double *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = fixed[i] ? 0.0 : -(fbar * (y ? y[i] : 0.0) + s[i]);
}
// r = b - y on free dofs, 0 on prescribed dofs; partial ||r||^2
__global__ void __launch_bounds__(kThreads) resid_kernel(int64_t n, const double *b, const double *y,
                                                         const uint8_t *fixed, double *r, double *red, int nb)
{
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = fixed[i] ? 0.0 : b[i] - y[i];
        r[i] = v;
        s += v * v;
    }
    double v2[2] = {s, 0.0};
    const int sl[2] = {S_MISC, S_MISC + 1};
    block_partials<2>(v2, red, sl, nb);
}

// out = x + b y
__global__ void axpby_kernel(int64_t n, double *out, const double *x, double b, const double *y)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = x[i] + b * y[i];
}

int vec_grid(int64_t n, int nb) { return (int)((n + kThreads - 1) / kThreads < nb ? (n + kThreads - 1) / kThreads : nb); }

}  // namespace

cudaError_t launch_spmv(const SolverCtx &c, const double *x, double *y, int free_only)
{
    count(c);
    if (c.ndof == 3)
        if (c.vals32)
            spmv_plain_kernel<3, float><<<c.blocks, kThreads, 0, c.stream>>>(c.n_nodes, c.rowptr, c.colidx, c.vals32,
                                                                            c.fixed, x, y, free_only);
        else
            spmv_plain_kernel<3, double><<<c.blocks, kThreads, 0, c.stream>>>(c.n_nodes, c.rowptr, c.colidx, c.vals,
                                                                             c.fixed, x, y, free_only);
    else if (c.vals32)
        spmv_plain_kernel<4, float><<<c.blocks, kThreads, 0, c.stream>>>(c.n_nodes, c.rowptr, c.colidx, c.vals32,
                                                                        c.fixed, x, y, free_only);
    else
        spmv_plain_kernel<4, double><<<c.blocks, kThreads, 0, c.stream>>>(c.n_nodes, c.rowptr, c.colidx, c.vals,
                                                                         c.fixed, x, y, free_only);
    return cudaGetLastError();
}

cudaError_t launch_norm2_free(const SolverCtx &c, const double *v, double *out_dev, double *out_fixed_dev)
{
    count(c, 2);
    norm_free_kernel<<<c.blocks, kThreads, 0, c.stream>>>(c.n, v, c.fixed, c.red, c.blocks);
    norm_finish_kernel<<<1, kThreads, 0, c.stream>>>(c.red, c.blocks, out_dev, out_fixed_dev);
    return cudaGetLastError();
}

cudaError_t launch_axpy_free(const SolverCtx &c, double *y, const double *x, double alpha)
{
    count(c);
    axpy_free_kernel<<<vec_grid(c.n, c.blocks), kThreads, 0, c.stream>>>(c.n, y, x, alpha, c.fixed);
    return cudaGetLastError();
}

cudaError_t launch_predictor(int64_t n, double *out, const double *cur, const double *prev, double factor,
                             const int32_t *bc_dof, const double *bc_scale, int64_t n_bc, double load, cudaStream_t s)
{
    int g = (int)((n + kThreads - 1) / kThreads);
    if (g > 1024) g = 1024;
    predictor_kernel<<<g, kThreads, 0, s>>>(n, out, cur, prev, factor);
    if (n_bc > 0) {
        int gb = (int)((n_bc + kThreads - 1) / kThreads);
        if (gb > 1024) gb = 1024;
        set_bc_kernel<<<gb, kThreads, 0, s>>>(out, bc_dof, bc_scale, n_bc, load);
    }
    return cudaGetLastError();
}

cudaError_t launch_predictor3(int64_t n, double *out, const double *x0, const double *x1, const double *x2,
                              const double (&w)[3], const int32_t *bc_dof, const double *bc_scale, int64_t n_bc,
                              double load, cudaStream_t s)
{
    int g = (int)((n + kThreads - 1) / kThreads);
    if (g > 1024) g = 1024;
    predictor3_kernel<<<g, kThreads, 0, s>>>(n, out, x0, x1, x2, w[0], w[1], w[2]);
    if (n_bc > 0) {
        int gb = (int)((n_bc + kThreads - 1) / kThreads);
        if (gb > 1024) gb = 1024;
        set_bc_kernel<<<gb, kThreads, 0, s>>>(out, bc_dof, bc_scale, n_bc, load);
    }
    return cudaGetLastError();
}

cudaError_t launch_residual(const SolverCtx &c, const double *b, const double *y, double *r, double *out_norm)
{
    count(c, 2);
    resid_kernel<<<c.blocks, kThreads, 0, c.stream>>>(c.n, b, y, c.fixed, r, c.red, c.blocks);
    norm_finish_kernel<<<1, kThreads, 0, c.stream>>>(c.red, c.blocks, out_norm, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_gather(const double *in, const int32_t *perm, double *out, int64_t n, cudaStream_t s)
{
    gather_kernel<<<1024, 256, 0, s>>>(in, perm, out, n);
    return cudaGetLastError();
}

cudaError_t launch_adj_rhs(int64_t n, const double *sv, const double *y, double fbar, const uint8_t *fixed, double *out,
                           cudaStream_t s)
{
    adj_rhs_kernel<<<512, 256, 0, s>>>(n, sv, y, fbar, fixed, out);
    return cudaGetLastError();
}

cudaError_t launch_axpby(int64_t n, double *out, const double *x, double b, const double *y, cudaStream_t s)
{
    axpby_kernel<<<512, 256, 0, s>>>(n, out, x, b, y);
    return cudaGetLastError();
}

cudaError_t launch_predictor_batch(int64_t n, int ndof, double *out, const double *cur, const double *prev,
                                   const double *pp, const double *w, const int32_t *node_spec, const int32_t *bc_dof,
                                   const double *bc_scale, const int32_t *bc_spec, const double *load, int64_t n_bc,
                                   cudaStream_t s)
{
    predictor_batch_kernel<<<1024, kThreads, 0, s>>>(n, ndof, out, cur, prev, pp, w, node_spec);
    if (n_bc > 0) set_bc_batch_kernel<<<256, kThreads, 0, s>>>(out, bc_dof, bc_scale, bc_spec, load, n_bc);
    return cudaGetLastError();
}

cudaError_t launch_norms_batch(const double *R, const uint8_t *fixed, const int64_t *node_off, int ndof, int n_spec,
                               double *out, cudaStream_t s)
{
    norms_batch_kernel<<<n_spec, 256, 0, s>>>(R, fixed, node_off, ndof, out);
    return cudaGetLastError();
}

cudaError_t launch_scale_spec(int64_t n, int ndof, double *out, const double *in, const double *coef,
                              const int32_t *node_spec, const uint8_t *fixed, int accumulate, cudaStream_t s)
{
    scale_spec_kernel<<<1024, kThreads, 0, s>>>(n, ndof, out, in, coef, node_spec, fixed, accumulate);
    return cudaGetLastError();
}

__global__ void fill_kernel(double *v, double val, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = val;
}

cudaError_t launch_fill(double *v, double val, int64_t n, cudaStream_t s)
{
    fill_kernel<<<256, kThreads, 0, s>>>(v, val, n);
    return cudaGetLastError();
}

cudaError_t launch_reaction_batch(const double *R, const int32_t *react_dof, const int64_t *off, int n_spec, double *out,
                                  cudaStream_t s)
{
    reaction_batch_kernel<<<n_spec, 256, 0, s>>>(R, react_dof, off, out);
    return cudaGetLastError();
}

cudaError_t launch_reaction(const double *R, const int32_t *react_dof, int64_t n_react, double *out, cudaStream_t s)
{
    reaction_kernel<<<1, 1024, 0, s>>>(R, react_dof, n_react, out);
    return cudaGetLastError();
}

cudaError_t launch_damage_max(const double *kappa, int64_t n, double eta_d, double kappa_d, double *out,
                              cudaStream_t s)
{
    damage_max_kernel<<<1, 1024, 0, s>>>(kappa, n, eta_d, kappa_d, out);
    return cudaGetLastError();
}

cudaError_t launch_damage_field(const double *kappa, int64_t n, double eta_d, double kappa_d, double *out,
                                cudaStream_t s)
{
    damage_field_kernel<<<256, kThreads, 0, s>>>(kappa, n, eta_d, kappa_d, out);
    return cudaGetLastError();
}

}  // namespace gd
