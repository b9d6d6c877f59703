// gd_krylov.cu -- the Newton system solve as ONE persistent cooperative kernel:
// node-block-Jacobi preconditioned BiCGStab (van der Vorst, 1992).
//
// The paper solves each Newton system with a direct LU factorisation (Sec. 3.2);
// on the device an iterative solve is used instead.  All blocks of a
// cooperative launch are co-resident, so phases are separated by grid-wide
// barriers instead of kernel launches.  Dot products are written as per-block
// partials; after a barrier every block sums all partials in the same fixed
// order, so every block holds bit-identical scalars and takes the same branch
// (deterministic, no atomics, no host round trip).  The loop ends on the device
// when ||r|| <= rtol ||b||, on breakdown, or after max_it iterations.
//
// Prescribed dofs: Krylov vectors are zero there and the operator is the
// identity there (the eliminated Newton system).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "gd_internal.cuh"

namespace cg = cooperative_groups;

namespace gd {
namespace {

constexpr int kThreads = 256;

template <class V>
struct KArgs {
    int64_t n_nodes;
    const int32_t *rowptr, *colidx;
    const V *vals;
    const uint8_t *fixed;
    const double *binv;       // [n_nodes][NDOF][NDOF] inverse diagonal node blocks
    const double *b;
    double *x;
    double *r, *rh, *p, *v, *s, *t, *y, *z;
    double *red;              // [8][nb] block partials
    double *out;              // [0] iterations, [1] final relative residual, [2] status
    double rtol;
    int max_it;
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block sum of K values -> red[slot_k * gridDim.x + blockIdx.x]
template <int K>
__device__ __forceinline__ void partials(double (&v)[K], double *red, const int (&slot)[K])
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
            double s = lane < kThreads / 32 ? sh[k][lane] : 0.0;
            s = warp_sum(s);
            if (lane == 0) red[slot[k] * gridDim.x + blockIdx.x] = s;
        }
    }
    __syncthreads();
}

// every block: sum of the partials of K slots in a fixed order
template <int K>
__device__ __forceinline__ void totals(const double *red, const int (&slot)[K], double (&out)[K])
{
    __shared__ double sh[K][kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nb = gridDim.x;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nb; i += kThreads) s += red[slot[k] * nb + i];
        s = warp_sum(s);
        if (lane == 0) sh[k][w] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < kThreads / 32; ++i) s += sh[k][i];
        out[k] = s;
    }
    __syncthreads();
}

// out = B^-1 in (node blocks), zero on prescribed dofs
template <int NDOF>
__device__ __forceinline__ void apply_binv(const double *binv, const uint8_t *fixed, int64_t nd, const double *in,
                                           double *out)
{
    double u[NDOF];
#pragma unroll
    for (int i = 0; i < NDOF; ++i) u[i] = in[nd * NDOF + i];
    const double *Bi = binv + nd * NDOF * NDOF;
#pragma unroll
    for (int i = 0; i < NDOF; ++i) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < NDOF; ++k) s += Bi[i * NDOF + k] * u[k];
        out[nd * NDOF + i] = fixed[nd * NDOF + i] ? 0.0 : s;
    }
}

// y = A x on free rows (x is zero on prescribed dofs), y = 0 on prescribed rows;
// group of G lanes per node; accumulates this thread's partials <d, y> and <y, y>.
template <int NDOF, int G, class V>
__device__ __forceinline__ void spmv_phase(const KArgs<V> &A, const double *x, double *yv, const double *d,
                                           double &part, double &part_yy)
{
    const int tid = blockIdx.x * kThreads + threadIdx.x;
    const int sub = threadIdx.x & (G - 1);
    const int64_t g0 = tid / G, ng = ((int64_t)gridDim.x * kThreads) / G;
    part = 0.0;
    part_yy = 0.0;
    // every lane of a warp iterates the same number of times (uniform trip count)
    const int64_t iters = (A.n_nodes + ng - 1) / ng;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t nd = g0 + it * ng;
        const bool ok = nd < A.n_nodes;
        double acc[NDOF];
#pragma unroll
        for (int i = 0; i < NDOF; ++i) acc[i] = 0.0;
        if (ok) {
            const int64_t r0 = nd * NDOF;
            const int32_t base = A.rowptr[r0];
            const int32_t len = A.rowptr[r0 + 1] - base;
            for (int j = sub; j < len; j += G) {
                const double xv = x[A.colidx[base + j]];
#pragma unroll
                for (int i = 0; i < NDOF; ++i) acc[i] += (double)A.vals[base + (int64_t)i * len + j] * xv;
            }
        }
#pragma unroll
        for (int i = 0; i < NDOF; ++i)
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
        if (ok && sub < NDOF) {
            double v = 0.0;
#pragma unroll
            for (int i = 0; i < NDOF; ++i)
                if (i == sub) v = acc[i];
            const int64_t r = nd * NDOF + sub;
            if (A.fixed[r]) v = 0.0;
            yv[r] = v;
            part += d[r] * v;
            part_yy += v * v;
        }
    }
}

template <int NDOF, int G, class V>
__global__ void __launch_bounds__(kThreads) bicgstab_kernel(KArgs<V> A)
{
    cg::grid_group grid = cg::this_grid();
    const int64_t tid = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * kThreads;
    enum { S_RHO = 0, S_RR = 1, S_RHV = 2, S_TS = 3, S_TT = 4 };

    // r = b (free), rh = r, x = p = v = 0
    {
        double rr = 0.0;
        for (int64_t i = tid; i < A.n_nodes * NDOF; i += nth) {
            const double bv = A.fixed[i] ? 0.0 : A.b[i];
            A.r[i] = bv;
            A.rh[i] = bv;
            A.x[i] = 0.0;
            A.p[i] = 0.0;
            A.v[i] = 0.0;
            rr += bv * bv;
        }
        double pv[2] = {rr, rr};
        const int sl[2] = {S_RHO, S_RR};
        partials<2>(pv, A.red, sl);
    }
    grid.sync();
    double tot[2];
    {
        const int sl[2] = {S_RHO, S_RR};
        totals<2>(A.red, sl, tot);
    }
    const double bnorm = sqrt(tot[1]);
    double rho = tot[0], rho_old = 1.0, alpha = 1.0, omega = 1.0;
    double rel = 0.0;
    int it = 0, status = 0;
    if (bnorm == 0.0) {
        rel = 0.0;
    } else {
        for (it = 0; it < A.max_it; ++it) {
            // phase A: p = r + beta (p - omega v), y = B^-1 p
            const double beta = (it == 0 || rho_old == 0.0 || omega == 0.0) ? 0.0 : (rho / rho_old) * (alpha / omega);
            for (int64_t nd = tid; nd < A.n_nodes; nd += nth) {
#pragma unroll
                for (int i = 0; i < NDOF; ++i) {
                    const int64_t k = nd * NDOF + i;
                    A.p[k] = A.r[k] + beta * (A.p[k] - omega * A.v[k]);
                }
                apply_binv<NDOF>(A.binv, A.fixed, nd, A.p, A.y);
            }
            grid.sync();
            // phase B: v = A y, <rh, v>
            {
                double prhv, pvv;
                spmv_phase<NDOF, G>(A, A.y, A.v, A.rh, prhv, pvv);
                double pv[1] = {prhv};
                const int sl[1] = {S_RHV};
                partials<1>(pv, A.red, sl);
            }
            grid.sync();
            double t1[1];
            {
                const int sl[1] = {S_RHV};
                totals<1>(A.red, sl, t1);
            }
            alpha = t1[0] != 0.0 ? rho / t1[0] : 0.0;
            // phase C: s = r - alpha v, z = B^-1 s
            for (int64_t nd = tid; nd < A.n_nodes; nd += nth) {
#pragma unroll
                for (int i = 0; i < NDOF; ++i) {
                    const int64_t k = nd * NDOF + i;
                    A.s[k] = A.r[k] - alpha * A.v[k];
                }
                apply_binv<NDOF>(A.binv, A.fixed, nd, A.s, A.z);
            }
            grid.sync();
            // phase D: t = A z, <t, s>, <t, t>
            {
                double ts, tt;
                spmv_phase<NDOF, G>(A, A.z, A.t, A.s, ts, tt);
                double pv[2] = {ts, tt};
                const int sl[2] = {S_TS, S_TT};
                partials<2>(pv, A.red, sl);
            }
            grid.sync();
            double t2[2];
            {
                const int sl[2] = {S_TS, S_TT};
                totals<2>(A.red, sl, t2);
            }
            omega = t2[1] != 0.0 ? t2[0] / t2[1] : 0.0;
            // phase E: x += alpha y + omega z, r = s - omega t, <rh, r>, <r, r>
            {
                double prhr = 0.0, prr = 0.0;
                for (int64_t i = tid; i < A.n_nodes * NDOF; i += nth) {
                    A.x[i] += alpha * A.y[i] + omega * A.z[i];
                    const double rv = A.s[i] - omega * A.t[i];
                    A.r[i] = rv;
                    prhr += A.rh[i] * rv;
                    prr += rv * rv;
                }
                double pv[2] = {prhr, prr};
                const int sl[2] = {S_RHO, S_RR};
                partials<2>(pv, A.red, sl);
            }
            grid.sync();
            double t3[2];
            {
                const int sl[2] = {S_RHO, S_RR};
                totals<2>(A.red, sl, t3);
            }
            rho_old = rho;
            rho = t3[0];
            rel = sqrt(t3[1]) / bnorm;
            if (!(rel == rel)) {            // NaN
                status = 2;
                ++it;
                break;
            }
            if (rel <= A.rtol) {
                ++it;
                break;
            }
            if (rho == 0.0 || omega == 0.0) {   // breakdown with a non-zero residual
                status = 1;
                ++it;
                break;
            }
        }
        if (it >= A.max_it && rel > A.rtol) status = 3;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.out[0] = it;
        A.out[1] = rel;
        A.out[2] = status;
    }
}

// inverse of the ndof x ndof diagonal node blocks (prescribed rows/cols -> identity)
template <int NDOF, class V>
__global__ void block_inverse_kernel(int64_t n_nodes, const int32_t *rowptr, const int32_t *colidx, const V *vals,
                                     const uint8_t *fixed, double *binv)
{
    for (int64_t nd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; nd < n_nodes;
         nd += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r0 = nd * NDOF;
        const int32_t base = rowptr[r0];
        const int32_t len = rowptr[r0 + 1] - base;
        // locate the own-node column block
        int jd = 0;
        for (int j = 0; j < len; j += NDOF)
            if (colidx[base + j] == (int32_t)r0) {
                jd = j;
                break;
            }
        double M[NDOF][2 * NDOF];
#pragma unroll
        for (int i = 0; i < NDOF; ++i)
#pragma unroll
            for (int k = 0; k < NDOF; ++k) {
                const bool fi = fixed[r0 + i], fk = fixed[r0 + k];
                double a = (double)vals[base + (int64_t)i * len + jd + k];
                M[i][k] = (fi || fk) ? (i == k ? 1.0 : 0.0) : a;
                M[i][NDOF + k] = (i == k) ? 1.0 : 0.0;
            }
        // Gauss-Jordan with partial pivoting; a singular block falls back to the identity
        bool ok = true;
#pragma unroll
        for (int c = 0; c < NDOF; ++c) {
            int piv = c;
            double best = fabs(M[c][c]);
#pragma unroll
            for (int i = c + 1; i < NDOF; ++i)
                if (fabs(M[i][c]) > best) {
                    best = fabs(M[i][c]);
                    piv = i;
                }
            if (!(best > 0.0)) {
                ok = false;
                break;
            }
            if (piv != c)
#pragma unroll
                for (int k = 0; k < 2 * NDOF; ++k) {
                    double tmp = M[c][k];
                    M[c][k] = M[piv][k];
                    M[piv][k] = tmp;
                }
            const double inv = 1.0 / M[c][c];
#pragma unroll
            for (int k = 0; k < 2 * NDOF; ++k) M[c][k] *= inv;
#pragma unroll
            for (int i = 0; i < NDOF; ++i)
                if (i != c) {
                    const double f = M[i][c];
#pragma unroll
                    for (int k = 0; k < 2 * NDOF; ++k) M[i][k] -= f * M[c][k];
                }
        }
        double *Bi = binv + nd * NDOF * NDOF;
#pragma unroll
        for (int i = 0; i < NDOF; ++i)
#pragma unroll
            for (int k = 0; k < NDOF; ++k) Bi[i * NDOF + k] = ok ? M[i][NDOF + k] : (i == k ? 1.0 : 0.0);
    }
}

template <int NDOF, class V>
cudaError_t solve_t(const KrylovCtx &c, const V *vals, const double *b, double *x, double rtol, int max_it)
{
    constexpr int G = NDOF == 3 ? 8 : 32;
    block_inverse_kernel<NDOF, V><<<c.num_sms * 4, 256, 0, c.stream>>>(c.n_nodes, c.rowptr, c.colidx, vals, c.fixed,
                                                                       c.binv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    KArgs<V> A;
    A.n_nodes = c.n_nodes;
    A.rowptr = c.rowptr;
    A.colidx = c.colidx;
    A.vals = vals;
    A.fixed = c.fixed;
    A.binv = c.binv;
    A.b = b;
    A.x = x;
    A.r = c.work[0];
    A.rh = c.work[1];
    A.p = c.work[2];
    A.v = c.work[3];
    A.s = c.work[4];
    A.t = c.work[5];
    A.y = c.work[6];
    A.z = c.work[7];
    A.red = c.red;
    A.out = c.out;
    A.rtol = rtol;
    A.max_it = max_it;
    void *args[] = {&A};
    return cudaLaunchCooperativeKernel((void *)bicgstab_kernel<NDOF, G, V>, dim3(c.blocks), dim3(kThreads), args, 0,
                                       c.stream);
}

template <int NDOF, class V>
int coop_blocks(int num_sms)
{
    constexpr int G = NDOF == 3 ? 8 : 32;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bicgstab_kernel<NDOF, G, V>, kThreads, 0) !=
        cudaSuccess)
        return 0;
    if (per_sm > 2) per_sm = 2;
    return per_sm * num_sms;
}

}  // namespace

int krylov_blocks(int ndof, bool fp32_vals, int num_sms)
{
    if (ndof == 3) return fp32_vals ? coop_blocks<3, float>(num_sms) : coop_blocks<3, double>(num_sms);
    return fp32_vals ? coop_blocks<4, float>(num_sms) : coop_blocks<4, double>(num_sms);
}

cudaError_t krylov_solve(const KrylovCtx &c, const void *vals, bool fp32_vals, const double *b, double *x,
                         double rtol, int max_it)
{
    if (c.ndof == 3)
        return fp32_vals ? solve_t<3, float>(c, (const float *)vals, b, x, rtol, max_it)
                         : solve_t<3, double>(c, (const double *)vals, b, x, rtol, max_it);
    return fp32_vals ? solve_t<4, float>(c, (const float *)vals, b, x, rtol, max_it)
                     : solve_t<4, double>(c, (const double *)vals, b, x, rtol, max_it);
}

}  // namespace gd
