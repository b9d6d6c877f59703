// gd_gmres.cu -- restarted GMRES(m) for the Newton systems (gd_options.krylov =
// GD_GMRES, and the fallback when BiCGStab breaks down or stalls in an FP64 solve).
//
// The paper solves each Newton system with a direct LU factorisation (Sec. 3.2); the
// device solves it iteratively.  BiCGStab's short recurrences can break down on the
// non-symmetric, softening tangent of the monolithic scheme; GMRES minimises the
// residual over the Krylov space and cannot break down before convergence.
//
// Right preconditioning by the node-block Jacobi inverse, K M^-1 u = b, x = M^-1 u;
// Arnoldi with classical Gram-Schmidt applied twice (two multi-dot / multi-axpy
// passes per step: the same orthogonality as modified Gram-Schmidt with two
// reductions instead of j); Givens rotations and the small triangular solve on the
// host.  All vectors are FP64 on the device; one host round trip per Arnoldi step
// reads the Hessenberg column.  The restart residual is the true b - K x.
// Prescribed dofs: every vector is zero there and the operator is the identity.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "gd_internal.cuh"

namespace gd {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out = M^-1 in per node block (binv [n_nodes][ndof][ndof]); 0 on prescribed dofs
__global__ void bjacobi_kernel(int64_t n_nodes, int ndof, const double *binv, const uint8_t *fixed, const double *in,
                               double *out)
{
    const int64_t n = n_nodes * ndof;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t nd = r / ndof;
        const int i = (int)(r - nd * ndof);
        double s = 0.0;
        for (int k = 0; k < ndof; ++k) s += binv[(nd * ndof + i) * ndof + k] * in[nd * ndof + k];
        out[r] = fixed[r] ? 0.0 : s;
    }
}

// partial[b * k + j] = block b's sum of V_j . w over the free dofs, j < k (k <= kMaxM + 1)
constexpr int kMaxM = 64;
__global__ void __launch_bounds__(kT) multidot_kernel(int64_t n, const double *V, int64_t ldv, int k, const double *w,
                                                      const uint8_t *fixed, double *partial)
{
    __shared__ double sh[kMaxM + 1][kT / 32];
    double acc[kMaxM + 1];
    for (int j = 0; j < k; ++j) acc[j] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = fixed[i] ? 0.0 : w[i];
        for (int j = 0; j < k; ++j) acc[j] += V[j * ldv + i] * wi;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = 0; j < k; ++j) {
        const double s = wsum(acc[j]);
        if (lane == 0) sh[j][wid] = s;
    }
    __syncthreads();
    for (int j = wid; j < k; j += kT / 32) {
        double s = lane < kT / 32 ? sh[j][lane] : 0.0;
        s = wsum(s);
        if (lane == 0) partial[(int64_t)blockIdx.x * k + j] = s;
    }
}

// h[j] = sum over blocks of partial[b * k + j] (one warp per j, fixed order)
__global__ void sum_partials_kernel(const double *partial, int nb, int k, double *h, double *h_acc)
{
    const int lane = threadIdx.x & 31, j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (j >= k) return;
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += partial[(int64_t)b * k + j];
    s = wsum(s);
    if (lane == 0) {
        h[j] = s;
        if (h_acc) h_acc[j] += s;
    }
}

// w -= sum_j h[j] V_j (sign = -1), or w += (sign = +1)
__global__ void multiaxpy_kernel(int64_t n, const double *V, int64_t ldv, int k, const double *h, double sign,
                                 double *w)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += h[j] * V[j * ldv + i];
        w[i] += sign * s;
    }
}

// v = w / *nrm (zero when the norm is zero)
__global__ void scale_kernel(int64_t n, const double *w, const double *nrm, double *v)
{
    const double a = *nrm > 0.0 ? 1.0 / *nrm : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = w[i] * a;
}

}  // namespace

// Solves K x = b on the free dofs (K: c.vals with prescribed rows/columns eliminated,
// the operator of launch_spmv with free_only) by right-preconditioned GMRES(m).
// binv: node-block inverses of K (launch_block_inverse); ws: device work space of
// gmres_workspace_doubles(n, m, nb) doubles.  x is overwritten (the solve starts at 0).
// Returns the iterations and the true final relative residual in iters / rel;
// converged is set when rel <= rtol.
cudaError_t gmres_solve(const SolverCtx &c, const double *binv, const double *b, double *x, double rtol, int m,
                        int max_it, double *ws, int &iters, double &rel, bool &converged)
{
    const int64_t n = c.n;
    const int nb = c.blocks;
    if (m < 1) m = 1;
    if (m > kMaxM) m = kMaxM;
    double *V = ws;                             // [m + 1][n]
    double *z = V + (size_t)(m + 1) * n, *w = z + n, *u = w + n;
    double *partial = u + n;                    // [nb][m + 1]
    double *h = partial + (size_t)nb * (m + 1); // [m + 1] this pass
    double *hc = h + (m + 1);                   // [m + 1] accumulated column
    double *nrm = hc + (m + 1);                 // [2]
    const int grid = (int)std::min<int64_t>((n + kT - 1) / kT, (int64_t)nb);
    iters = 0;
    rel = 1.0;
    converged = false;
    cudaError_t e;
    auto sync_read = [&](double *dst, const double *src, size_t cnt) {
        e = cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        return e;
    };
    // ||b|| on the free dofs
    if ((e = launch_norm2_free(c, b, nrm, nullptr)) != cudaSuccess) return e;
    double bn = 0.0;
    if ((e = sync_read(&bn, nrm, 1)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(x, 0, sizeof(double) * n, c.stream)) != cudaSuccess) return e;
    if (!(bn > 0.0)) {
        rel = 0.0;
        converged = true;
        return cudaSuccess;
    }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), col(m + 2);
    // r0 = b (x = 0)
    if ((e = cudaMemcpyAsync(w, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c.stream)) != cudaSuccess) return e;
    double beta = bn;
    while (iters < max_it) {
        // V_0 = r / beta
        if ((e = launch_norm2_free(c, w, nrm, nullptr)) != cudaSuccess) return e;
        scale_kernel<<<grid, kT, 0, c.stream>>>(n, w, nrm, V);
        if ((e = sync_read(&beta, nrm, 1)) != cudaSuccess) return e;
        rel = beta / bn;
        if (rel <= rtol || !(beta > 0.0)) {
            converged = rel <= rtol;
            break;
        }
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        for (; j < m && iters < max_it; ++j, ++iters) {
            // w = K M^-1 V_j
            bjacobi_kernel<<<grid, kT, 0, c.stream>>>(c.n_nodes, c.ndof, binv, c.fixed, V + (size_t)j * n, z);
            if ((e = launch_spmv(c, z, w, 1)) != cudaSuccess) return e;
            // two classical Gram-Schmidt passes against V_0..V_j
            if ((e = cudaMemsetAsync(hc, 0, sizeof(double) * (m + 1), c.stream)) != cudaSuccess) return e;
            for (int pass = 0; pass < 2; ++pass) {
                multidot_kernel<<<nb, kT, 0, c.stream>>>(n, V, n, j + 1, w, c.fixed, partial);
                sum_partials_kernel<<<(j + 1 + 7) / 8, kT, 0, c.stream>>>(partial, nb, j + 1, h, hc);
                multiaxpy_kernel<<<grid, kT, 0, c.stream>>>(n, V, n, j + 1, h, -1.0, w);
            }
            if ((e = launch_norm2_free(c, w, nrm, nullptr)) != cudaSuccess) return e;
            scale_kernel<<<grid, kT, 0, c.stream>>>(n, w, nrm, V + (size_t)(j + 1) * n);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = sync_read(col.data(), hc, (size_t)(j + 1))) != cudaSuccess) return e;
            double hn = 0.0;
            if ((e = sync_read(&hn, nrm, 1)) != cudaSuccess) return e;
            col[j + 1] = hn;
            // previous rotations, then a new one that zeroes col[j + 1]
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = t;
            }
            const double d = std::hypot(col[j], col[j + 1]);
            cs[j] = d > 0.0 ? col[j] / d : 1.0;
            sn[j] = d > 0.0 ? col[j + 1] / d : 0.0;
            col[j] = d;
            col[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = col[i];
            if (std::fabs(g[j + 1]) <= rtol * bn || !(hn > 0.0)) {
                ++j;
                ++iters;
                break;
            }
        }
        // y = H^-1 g (upper triangular, j columns); u = V y; x += M^-1 u
        for (int i = j - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * m + k] * y[k];
            const double hii = H[(size_t)i * m + i];
            y[i] = hii != 0.0 ? s / hii : 0.0;
        }
        if ((e = cudaMemcpyAsync(h, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, c.stream)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(u, 0, sizeof(double) * n, c.stream)) != cudaSuccess) return e;
        multiaxpy_kernel<<<grid, kT, 0, c.stream>>>(n, V, n, j, h, 1.0, u);
        bjacobi_kernel<<<grid, kT, 0, c.stream>>>(c.n_nodes, c.ndof, binv, c.fixed, u, z);
        if ((e = launch_axpy_free(c, x, z, 1.0)) != cudaSuccess) return e;
        // true residual w = b - K x for the restart
        if ((e = launch_spmv(c, x, z, 1)) != cudaSuccess) return e;
        if ((e = launch_residual(c, b, z, w, nrm + 1)) != cudaSuccess) return e;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // the true residual of the returned x
    if ((e = launch_spmv(c, x, z, 1)) != cudaSuccess) return e;
    if ((e = launch_residual(c, b, z, w, nrm + 1)) != cudaSuccess) return e;
    double rn = 0.0;
    if ((e = sync_read(&rn, nrm + 1, 1)) != cudaSuccess) return e;
    rel = rn / bn;
    converged = rel <= rtol;
    return cudaSuccess;
}

size_t gmres_workspace_doubles(int64_t n, int m, int nb)
{
    if (m > kMaxM) m = kMaxM;
    return (size_t)(m + 1) * n + 3 * (size_t)n + (size_t)nb * (m + 1) + 2 * (size_t)(m + 1) + 2;
}

int gmres_max_m() { return kMaxM; }

}  // namespace gd
