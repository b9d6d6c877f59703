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

#include <type_traits>

#include "gd_internal.cuh"

namespace cg = cooperative_groups;

namespace gd {
namespace {

constexpr int kThreads = 256;

template <class V, class T>
struct KArgs {
    int64_t n_nodes;
    const int32_t *rowptr, *colidx;
    const V *vals;
    const uint8_t *fixed;
    const T *binv;            // [n_nodes][NDOF][NDOF] inverse diagonal node blocks
    const double *b;
    double *x_out;            // solution (FP64)
    T *x;                     // iterate (x_out itself when T is double)
    T *r, *rh, *p, *v, *s, *t, *y, *z;
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

// every block: sum of the partials of K slots in a fixed order (warp 0 reads and
// reduces them, the result is broadcast through shared memory)
template <int K>
__device__ __forceinline__ void totals(const double *red, const int (&slot)[K], double (&out)[K])
{
    __shared__ double sh[K];
    const int nb = gridDim.x;
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int i = threadIdx.x; i < nb; i += 32) s += red[slot[k] * nb + i];
            s = warp_sum(s);
            if (threadIdx.x == 0) sh[k] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = sh[k];
    __syncthreads();
}

// out = B^-1 in (node blocks), zero on prescribed dofs
template <int NDOF, class T>
__device__ __forceinline__ void apply_binv(const T *binv, const uint8_t *fixed, int64_t nd, const T *in, T *out)
{
    T u[NDOF];
#pragma unroll
    for (int i = 0; i < NDOF; ++i) u[i] = in[nd * NDOF + i];
    const T *Bi = binv + nd * NDOF * NDOF;
#pragma unroll
    for (int i = 0; i < NDOF; ++i) {
        T s = T(0);
#pragma unroll
        for (int k = 0; k < NDOF; ++k) s += Bi[i * NDOF + k] * u[k];
        out[nd * NDOF + i] = fixed[nd * NDOF + i] ? T(0) : s;
    }
}

// y = A x on free rows (x is zero on prescribed dofs), y = 0 on prescribed rows;
// group of G lanes per node; accumulates this thread's partials <d, y> and <y, y>.
template <int NDOF, int G, class V, class T>
__device__ __forceinline__ void spmv_phase(const KArgs<V, T> &A, const T *x, T *yv, const T *d, double &part,
                                           double &part_yy)
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
        T acc[NDOF];
#pragma unroll
        for (int i = 0; i < NDOF; ++i) acc[i] = T(0);
        if (ok) {
            const int64_t r0 = nd * NDOF;
            const int32_t base = A.rowptr[r0];
            const int32_t len = A.rowptr[r0 + 1] - base;
            for (int j = sub; j < len; j += G) {
                const T xv = x[A.colidx[base + j]];
#pragma unroll
                for (int i = 0; i < NDOF; ++i) acc[i] += (T)A.vals[base + (int64_t)i * len + j] * xv;
            }
        }
#pragma unroll
        for (int i = 0; i < NDOF; ++i)
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
        if (ok && sub < NDOF) {
            T v = T(0);
#pragma unroll
            for (int i = 0; i < NDOF; ++i)
                if (i == sub) v = acc[i];
            const int64_t r = nd * NDOF + sub;
            if (A.fixed[r]) v = T(0);
            yv[r] = v;
            part += (double)d[r] * (double)v;
            part_yy += (double)v * (double)v;
        }
    }
}

// The same product with one lane per row: a warp takes 32 / NDOF consecutive nodes
// and each lane runs its own row, so no partial sums cross lanes.  On this part
// FP64 arithmetic issues at a small fraction of the FP32 rate, and the cross-lane
// reduction of the grouped form nearly doubles the FP64 instructions of the
// product; the FP64 solve therefore uses this form.  The NDOF lanes of a node
// read the same column index and x value (one broadcast per load).
template <int NDOF, class V, class T>
__device__ __forceinline__ void spmv_rows(const KArgs<V, T> &A, const T *x, T *yv, const T *d, double &part,
                                          double &part_yy)
{
    constexpr int NPW = 32 / NDOF;
    const int lane = threadIdx.x & 31;
    const int slot = lane / NDOF, i = lane - slot * NDOF;
    const int64_t wg = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
    part = 0.0;
    part_yy = 0.0;
    if (slot >= NPW) return;
    for (int64_t nd = wg * NPW + slot; nd < A.n_nodes; nd += nw * NPW) {
        const int64_t r = nd * NDOF + i;
        const int32_t base = A.rowptr[nd * NDOF];
        const int32_t len = A.rowptr[nd * NDOF + 1] - base;
        const V *vr = A.vals + base + (int64_t)i * len;
        const int32_t *cr = A.colidx + base;
        T acc = T(0);
#pragma unroll 4
        for (int j = 0; j < len; ++j) acc += (T)vr[j] * x[cr[j]];
        if (A.fixed[r]) acc = T(0);
        yv[r] = acc;
        part += (double)d[r] * (double)acc;
        part_yy += (double)acc * (double)acc;
    }
}

template <int NDOF, int G, class V, class T>
__device__ __forceinline__ void spmv_any(const KArgs<V, T> &A, const T *x, T *yv, const T *d, double &part,
                                         double &part_yy)
{
    if constexpr (std::is_same<T, double>::value) spmv_rows<NDOF, V, T>(A, x, yv, d, part, part_yy);
    else spmv_phase<NDOF, G, V, T>(A, x, yv, d, part, part_yy);
}

template <int NDOF, int G, class V, class T>
__global__ void __launch_bounds__(kThreads) bicgstab_kernel(KArgs<V, T> A)
{
    cg::grid_group grid = cg::this_grid();
    const int64_t tid = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * kThreads;
    enum { S_RHO = 0, S_RR = 1, S_RHV = 2, S_TS = 3, S_TT = 4 };

    // r = b (free), rh = r, x = p = v = 0
    {
        double rr = 0.0;
        for (int64_t i = tid; i < A.n_nodes * NDOF; i += nth) {
            const T bv = A.fixed[i] ? T(0) : (T)A.b[i];
            A.r[i] = bv;
            A.rh[i] = bv;
            A.x[i] = T(0);
            A.p[i] = T(0);
            A.v[i] = T(0);
            rr += (double)bv * (double)bv;
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
                    A.p[k] = A.r[k] + (T)beta * (A.p[k] - (T)omega * A.v[k]);
                }
                apply_binv<NDOF, T>(A.binv, A.fixed, nd, A.p, A.y);
            }
            grid.sync();
            // phase B: v = A y, <rh, v>
            {
                double prhv, pvv;
                spmv_any<NDOF, G, V, T>(A, A.y, A.v, A.rh, prhv, pvv);
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
                    A.s[k] = A.r[k] - (T)alpha * A.v[k];
                }
                apply_binv<NDOF, T>(A.binv, A.fixed, nd, A.s, A.z);
            }
            grid.sync();
            // phase D: t = A z, <t, s>, <t, t>
            {
                double ts, tt;
                spmv_any<NDOF, G, V, T>(A, A.z, A.t, A.s, ts, tt);
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
                    A.x[i] += (T)alpha * A.y[i] + (T)omega * A.z[i];
                    const T rv = A.s[i] - (T)omega * A.t[i];
                    A.r[i] = rv;
                    prhr += (double)A.rh[i] * (double)rv;
                    prr += (double)rv * (double)rv;
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
    if ((void *)A.x != (void *)A.x_out)
        for (int64_t i = tid; i < A.n_nodes * NDOF; i += nth) A.x_out[i] = (double)A.x[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.out[0] = it;
        A.out[1] = rel;
        A.out[2] = status;
    }
}

// inverse of the ndof x ndof diagonal node blocks (prescribed rows/cols -> identity)
template <int NDOF, class V, class T>
__global__ void block_inverse_kernel(int64_t n_nodes, const int32_t *rowptr, const int32_t *colidx, const V *vals,
                                     const uint8_t *fixed, T *binv)
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
        T *Bi = binv + nd * NDOF * NDOF;
#pragma unroll
        for (int i = 0; i < NDOF; ++i)
#pragma unroll
            for (int k = 0; k < NDOF; ++k) Bi[i * NDOF + k] = (T)(ok ? M[i][NDOF + k] : (i == k ? 1.0 : 0.0));
    }
}

template <int NDOF, class V, class T>
cudaError_t solve_t(const KrylovCtx &c, const V *vals, const double *b, double *x, double rtol, int max_it)
{
    constexpr int G = NDOF == 3 ? 8 : 32;
    T *binv = (T *)c.binv;
    block_inverse_kernel<NDOF, V, T><<<c.num_sms * 4, 256, 0, c.stream>>>(c.n_nodes, c.rowptr, c.colidx, vals,
                                                                          c.fixed, binv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    KArgs<V, T> A;
    A.n_nodes = c.n_nodes;
    A.rowptr = c.rowptr;
    A.colidx = c.colidx;
    A.vals = vals;
    A.fixed = c.fixed;
    A.binv = binv;
    A.b = b;
    A.x_out = x;
    T *w[9];
    for (int k = 0; k < 8; ++k) w[k] = (T *)c.work[k];
    w[8] = (T *)c.work_x;
    A.x = std::is_same<T, double>::value ? (T *)x : w[8];
    A.r = w[0];
    A.rh = w[1];
    A.p = w[2];
    A.v = w[3];
    A.s = w[4];
    A.t = w[5];
    A.y = w[6];
    A.z = w[7];
    A.red = c.red;
    A.out = c.out;
    A.rtol = rtol;
    A.max_it = max_it;
    void *args[] = {&A};
    return cudaLaunchCooperativeKernel((void *)bicgstab_kernel<NDOF, G, V, T>, dim3(c.blocks), dim3(kThreads), args, 0,
                                       c.stream);
}

template <int NDOF, class V, class T>
int coop_blocks(int num_sms)
{
    constexpr int G = NDOF == 3 ? 8 : 32;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bicgstab_kernel<NDOF, G, V, T>, kThreads, 0) !=
        cudaSuccess)
        return 0;
    if (per_sm > 2) per_sm = 2;
    return per_sm * num_sms;
}

__global__ void narrow_kernel(const double *in, float *out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

}  // namespace

int krylov_blocks(int ndof, bool fp32_vals, int num_sms)
{
    // the smallest co-resident grid over the variants, so one size fits every launch
    int a = ndof == 3 ? coop_blocks<3, double, double>(num_sms) : coop_blocks<4, double, double>(num_sms);
    int b = ndof == 3 ? coop_blocks<3, float, float>(num_sms) : coop_blocks<4, float, float>(num_sms);
    (void)fp32_vals;
    return a < b ? a : b;
}

cudaError_t krylov_solve(const KrylovCtx &c, const void *vals, bool fp32_vals, const double *b, double *x,
                         double rtol, int max_it, bool fp32_vectors)
{
    if (fp32_vectors) {
        if (!fp32_vals) return cudaErrorInvalidValue;
        return c.ndof == 3 ? solve_t<3, float, float>(c, (const float *)vals, b, x, rtol, max_it)
                           : solve_t<4, float, float>(c, (const float *)vals, b, x, rtol, max_it);
    }
    if (c.ndof == 3)
        return fp32_vals ? solve_t<3, float, double>(c, (const float *)vals, b, x, rtol, max_it)
                         : solve_t<3, double, double>(c, (const double *)vals, b, x, rtol, max_it);
    return fp32_vals ? solve_t<4, float, double>(c, (const float *)vals, b, x, rtol, max_it)
                     : solve_t<4, double, double>(c, (const double *)vals, b, x, rtol, max_it);
}

cudaError_t narrow_to_float(const double *in, float *out, int64_t n, cudaStream_t s)
{
    narrow_kernel<<<1024, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

}  // namespace gd
