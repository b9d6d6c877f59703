// gd_krylov.cu -- the Newton system solve as ONE persistent cooperative kernel:
// node-block-Jacobi preconditioned BiCGStab (van der Vorst, 1992).
//
// The paper solves each Newton system with a direct LU factorisation (Sec. 3.2);
// on the device an iterative solve is used instead.  All blocks of a
// cooperative launch are co-resident, so phases are separated by grid-wide
// barriers instead of kernel launches.  Every grid-wide sum ends in one global
// accumulator that all blocks read after the barrier, so every block holds the
// same scalars and takes the same branch (no host round trip).  The loop ends
// on the device when ||r|| <= rtol ||b||, on breakdown, or after max_it
// iterations.  Single systems may add a second, coarse level to the
// preconditioner (gd_coarse.cu): three more phases per application.
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
    T *r, *rh, *p, *v, *s, *t, *y, *z, *w;
    double *red;              // [8][nb] block partials
    double *out;              // [0] iterations, [1] final relative residual, [2] status
    double rtol;
    int max_it;
    // shared-memory copy of the block's rows for the products (single-system kernel):
    // 0 none, 1 column lists, 2 column lists and values; lmax = longest row
    int cache;
    int lmax;
    // coarse level (single-system kernel with CO): P [n_nodes][NDOF][nm], the coarse
    // unknowns of every node's aggregate, the inverse coarse matrix
    // (FP32 for FP32 vectors, FP64 otherwise), restriction sums [2][nc] and coarse
    // solution [nc] in the vector type, status word of the inversion
    int c_nc;
    const float *c_P;
    const int32_t *c_node;    // 8 x first coarse unknown + count, per node
    const float *c_X32;
    const double *c_X64;
    T *c_rc, *c_cc;
    const int *c_status;
    int c_xs;                 // 1: each CTA keeps its rows of the inverse in shared memory
};

template <int NDOF>
struct CoarseModes {
    static constexpr int NM = NDOF == 3 ? 4 : 7;     // ndof constants + rigid rotations (2D: 1, 3D: 3)
};

template <class T>
__device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// restriction P^T w of the node whose NDOF values sit in lanes base..base+NDOF-1:
// the node's lanes split its nm coarse components and add them to rc (atomics).
// co: the node's packed coarse unknowns (8 x first + count), pP: its basis values
// [NDOF][nm] (shared-memory record or global).  Called by every lane of the warp.
template <int NDOF, int LPN, class T>
__device__ __forceinline__ void coarse_restrict(bool node_ok, int sub, int base, T w, T *rc, int32_t co,
                                                const float *pP)
{
    constexpr int NM = CoarseModes<NDOF>::NM;
    T wk[NDOF];
#pragma unroll
    for (int k = 0; k < NDOF; ++k) wk[k] = __shfl_sync(0xffffffffu, w, base + k);
    if (!node_ok) return;
    const int32_t o = co >> 3, n = co & 7;
    for (int m = sub; m < n; m += LPN) {
        T sum = T(0);
#pragma unroll
        for (int k = 0; k < NDOF; ++k) sum += (T)pP[k * NM + m] * wk[k];
        atomicAdd(rc + o + m, sum);
    }
}

// cc = Ac^-1 rc: the coarse rows go to the CTAs in turn (rows b, b + grid, ...),
// up to eight rows of a CTA at once, its threads along the rows.  Each thread
// first loads all of its rc values (independent loads in flight together) and
// reuses them for every row.  sX: the CTA's rows in shared memory (row q of the
// CTA at sX + q nc), or null to read them from the global inverse.
template <class V, class T>
__device__ __forceinline__ void coarse_solve(const KArgs<V, T> &A, const T *rc, T *cc, const T *sX)
{
    constexpr int JMAX = (kCoarseMax + kThreads - 1) / kThreads;
    __shared__ T part[8][kThreads / 32];
    const int32_t nc = A.c_nc, nb = gridDim.x, b = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const T *Xg;
    if constexpr (std::is_same<T, double>::value) Xg = A.c_X64;
    else Xg = A.c_X32;
    T rv[JMAX];
#pragma unroll
    for (int jj = 0; jj < JMAX; ++jj) {
        const int32_t j = tid + jj * kThreads;
        rv[jj] = j < nc ? rc[j] : T(0);
    }
    for (int32_t q0 = 0; b + q0 * nb < nc; q0 += 8) {
        T acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = T(0);
#pragma unroll
        for (int jj = 0; jj < JMAX; ++jj) {
            const int32_t j = tid + jj * kThreads;
            if (j < nc) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int32_t k = b + (q0 + q) * nb;
                    if (k < nc) acc[q] += (sX ? sX[(q0 + q) * nc + j] : Xg[(int64_t)k * nc + j]) * rv[jj];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const T s = warp_sum_t(acc[q]);
            if (lane == 0) part[q][wib] = s;
        }
        __syncthreads();
        if (tid < 8) {
            const int32_t k = b + (q0 + tid) * nb;
            if (k < nc) {
                T s = T(0);
#pragma unroll
                for (int w = 0; w < kThreads / 32; ++w) s += part[tid][w];
                cc[k] = s;
            }
        }
        __syncthreads();
    }
}

// row sub of P cc for a node with packed coarse unknowns co and basis values pP
template <int NDOF, class T>
__device__ __forceinline__ T coarse_prolong(int sub, const T *cc, int32_t co, const float *pP)
{
    constexpr int NM = CoarseModes<NDOF>::NM;
    const int32_t o = co >> 3, n = co & 7;
    T s = T(0);
#pragma unroll
    for (int m = 0; m < NM; ++m)
        if (m < n) s += (T)pP[sub * NM + m] * cc[o + m];
    return s;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid-wide sums of the single-system kernel.  Each block reduces its threads'
// values and adds the block sum into a global FP64 accumulator with one atomic
// add; after the grid barrier every block reads the finished total, one load per
// slot.  (Summing every block's partial in every block costs a round trip per
// partial line and was measured at 3.6-5.6 us per reduction.)  All blocks read
// the same total, so they take the same decisions; the order of the atomic adds,
// and with it the last bits of a total, can differ from run to run.  Two
// accumulators per slot alternate between iterations: block 0 clears the other
// one when it reads the current one, which is safe because every block read the
// other one two barriers earlier and the next adds into it come two barriers
// later.  acc[2 slot + parity]; the launcher clears all of them before the launch.
template <int K>
__device__ __forceinline__ void acc_add(double (&v)[K], double *acc, const int (&slot)[K], int par)
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
            if (lane == 0) atomicAdd(acc + 2 * slot[k] + par, s);
        }
    }
    __syncthreads();
}

template <int K>
__device__ __forceinline__ void acc_read(double *acc, const int (&slot)[K], int par, double (&out)[K])
{
    __shared__ double sh[K];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            sh[k] = __ldcg(acc + 2 * slot[k] + par);
            if (blockIdx.x == 0) acc[2 * slot[k] + (par ^ 1)] = 0.0;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = sh[k];
    __syncthreads();
}

// Per-thread dot-product accumulator.  FP64 vectors: a plain FP64 sum.  FP32
// vectors: each product is split exactly into its rounded value and rounding
// error (a fused multiply-add gives the error), and both are added with a
// compensated (two-sum) FP32 accumulation; the thread's sum is widened to FP64
// once, and every sum across threads and blocks is FP64.  On this part FP64
// arithmetic and conversions issue at a small fraction of the FP32 rate, and a
// per-row FP64 product with two widenings made the FP32 solve FP64-bound.
template <class T>
struct DotAcc {
    double s = 0.0;
    __device__ __forceinline__ void add(T x, T y) { s += (double)x * (double)y; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x, float y)
    {
        // _rn intrinsics: the compiler must not fuse these into multiply-adds
        const float p = __fmul_rn(x, y);
        const float e = fmaf(x, y, -p);        // x y = p + e exactly
        const float t = __fadd_rn(s, p);       // two-sum of s and p
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// ---------------------------------------------------------------------------
// Single system, three grid barriers per iteration.
//
// Right-preconditioned BiCGStab on B = A M^-1 (M the node-block diagonal; the
// solution is x = M^-1 x~).  The classic iteration multiplies B p and B s, whose
// inputs are only known after a reduction, so it needs five barriers.  Here the
// products kept are u = B r and q = B v: with v_n = B p_n and t_n = B s_n,
//   t_n     = u_n - alpha q_n,
//   v_{n+1} = u_{n+1} + beta (v_n - omega q_n),
// so v and t follow elementwise, and every dot product is still taken directly
// (no expanded inner products).  One iteration:
//   1  p = r + beta (p - omega v), v = u + beta (v - omega q), y = M^-1 v, <rh, v>
//   -- barrier: sigma = <rh, v>, alpha = rho / sigma
//   2  q = A y, s = r - alpha v (stored in r), t = u - alpha q, <t, s>, <t, t>
//   -- barrier: omega
//   3  x~ += alpha p + omega s, r = s - omega t, y = M^-1 r, <rh, r>, <r, r>
//   -- barrier: rho, ||r||, stop test, beta
//   4  u = A y   (phase 1 of the next iteration reads only rows this lane wrote)
// All phases give each row to the same lane (FP64: one lane per row; FP32: G lanes
// per node, the row's lane holding the reduced value), so nothing but the two
// products reads another lane's rows.  A zero <rh, r> or omega with the residual
// still above tolerance restarts the recurrences with rh = r (at most 16 times).
// ---------------------------------------------------------------------------
template <int NDOF, int G, class T>
struct RowMap {
    static constexpr int LPN = std::is_same<T, double>::value ? NDOF : G;   // lanes per node
    static constexpr int NPW = 32 / LPN;                                    // nodes per warp pass
};

// U independent row products per lane (U node groups of the warp at once): the
// loads of the U rows are issued together, so a lane waits for one chain of
// dependent loads (row pointer, column index, x) instead of U of them in turn.
// The product phases are bound by that latency, not by bandwidth or arithmetic.
// cs[u] (may be null): the node's shared-memory record, its row length then its
// column indices; cv[u] (may be null): its values, row i at cv[u] + i lmax.  Without
// them the row is read from the CSR arrays in global memory.
template <int NDOF, int LPN, int U, class V, class T>
__device__ __forceinline__ void row_products(const KArgs<V, T> &A, const int32_t (&nd)[U], const bool (&ok)[U],
                                             int sub, const T *x, T (&out)[U], const int32_t *const (&cs)[U],
                                             const V *const (&cv)[U])
{
    int32_t base[U], len[U];
    int lmax = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (cs[u]) {
            base[u] = (ok[u] && !cv[u]) ? A.rowptr[nd[u] * NDOF] : 0;
            len[u] = ok[u] ? cs[u][0] : 0;
        } else {
            base[u] = ok[u] ? A.rowptr[nd[u] * NDOF] : 0;
            len[u] = ok[u] ? A.rowptr[nd[u] * NDOF + 1] - base[u] : 0;
        }
        lmax = len[u] > lmax ? len[u] : lmax;
    }
    if constexpr (LPN == NDOF) {
#pragma unroll
        for (int u = 0; u < U; ++u) out[u] = T(0);
#pragma unroll 4
        for (int j = 0; j < lmax; ++j) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j < len[u]) {
                    const int32_t col = cs[u] ? cs[u][1 + j] : A.colidx[base[u] + j];
                    const V a = cv[u] ? cv[u][sub * A.lmax + j] : A.vals[base[u] + sub * len[u] + j];
                    out[u] += (T)a * x[col];
                }
        }
    } else {
        T acc[U][NDOF];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int i = 0; i < NDOF; ++i) acc[u][i] = T(0);
#pragma unroll 4
        for (int j = sub; j < lmax; j += LPN) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j < len[u]) {
                    const T xv = x[cs[u] ? cs[u][1 + j] : A.colidx[base[u] + j]];
#pragma unroll
                    for (int i = 0; i < NDOF; ++i)
                        acc[u][i] += (T)(cv[u] ? cv[u][i * A.lmax + j] : A.vals[base[u] + i * len[u] + j]) * xv;
                }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int i = 0; i < NDOF; ++i)
#pragma unroll
                for (int o = LPN / 2; o > 0; o >>= 1) acc[u][i] += __shfl_xor_sync(0xffffffffu, acc[u][i], o);
            T v = T(0);
#pragma unroll
            for (int i = 0; i < NDOF; ++i)
                if (i == sub) v = acc[u][i];
            out[u] = v;
        }
    }
}

// row sub of M^-1 w for the node whose NDOF row values sit in lanes base..base+NDOF-1
template <int NDOF, class T>
__device__ __forceinline__ T node_apply(const T *binv, int64_t nd_wide, bool node_ok, int sub, int base, T w, bool fixed)
{
    T out = T(0);
#pragma unroll
    for (int k = 0; k < NDOF; ++k) {
        const T wk = __shfl_sync(0xffffffffu, w, base + k);
        if (node_ok && sub < NDOF) out += binv[(nd_wide * NDOF + sub) * NDOF + k] * wk;
    }
    return fixed ? T(0) : out;
}

// FP32 vectors: built for four CTAs per SM (64 registers; the two-level variants spill
// up to 80 bytes), FP64 vectors for two
template <int NDOF, int G, int UP, class V, class T, bool CO = false>
__global__ void __launch_bounds__(kThreads, std::is_same<T, float>::value ? 4 : 2) bicgstab3_kernel(KArgs<V, T> A)
{
    using M = RowMap<NDOF, G, T>;
    constexpr int LPN = M::LPN, NPW = M::NPW;
    // UP: node groups per product round (a launch-shape choice of the autotuner)
    cg::grid_group grid = cg::this_grid();
    const int lane = threadIdx.x & 31;
    const int slot = lane / LPN, sub = lane - slot * LPN, nbase = slot * LPN;
    const int32_t gw = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int32_t nw = (gridDim.x * kThreads) >> 5;
    const int32_t n_nodes = (int32_t)A.n_nodes;
    const int32_t passes = (n_nodes + nw * NPW - 1) / (nw * NPW);   // warp-uniform
    // CO: two-level preconditioner M^-1 = D^-1 + P Ac^-1 P^T.  The node-block part is
    // applied where the vector is formed, together with the restriction P^T (atomic
    // sums into rc); after the phase's barrier, Ac^-1 rc (coarse rows spread over the CTAs),
    // a barrier, the prolongation P added to the owned rows, and a barrier before
    // the product reads them.  Skipped when the inversion reported a zero pivot.
    bool co = false;
    if constexpr (CO) co = __ldcg(A.c_status) == 0;
    T *rc0 = nullptr, *rc1 = nullptr, *cc = nullptr;
    if constexpr (CO) {
        rc0 = A.c_rc;
        rc1 = A.c_rc + A.c_nc;
        cc = A.c_cc;
    }
    // vector roles: r (also s), rh, p, v, q, t, y = M^-1 v (read by phase 2's product),
    // w = M^-1 r (read by phase 4's product), u.  y and w must differ: phase 1 of the
    // next iteration writes y with no barrier after phase 4, whose product still reads
    // other lanes' w
    T *r = A.r, *rh = A.rh, *p = A.p, *v = A.v, *q = A.s, *t = A.t, *y = A.y, *wv = A.w, *u = A.z, *xt = A.x;
    // shared-memory rows (A.cache > 0): one record per (pass, warp of the block, node
    // slot): [row length, column indices ...] with stride lmax + 1, then the values,
    // NDOF x lmax per record; the launcher sizes the dynamic shared memory for
    // passes x warps x NPW records
    extern __shared__ __align__(16) unsigned char kdyn[];
    const int wib = threadIdx.x >> 5;
    const int32_t n_rec = passes * (kThreads / 32) * NPW;
    int32_t *scol = reinterpret_cast<int32_t *>(kdyn);
    V *sval = reinterpret_cast<V *>(kdyn + ((((size_t)n_rec * (A.lmax + 1) * sizeof(int32_t)) + 15) & ~(size_t)15));
    auto rec_of = [&](int32_t ps) { return (ps * (kThreads / 32) + wib) * NPW + slot; };
    // coarse data of the same records (CO with a row cache): packed coarse unknowns,
    // then the basis values [NDOF][nm] of every record
    constexpr int NM = CoarseModes<NDOF>::NM;
    const bool cco = co && A.cache > 0;
    int32_t *sco = nullptr;
    float *sP = nullptr;
    if (cco) {
        size_t off = (((size_t)n_rec * (A.lmax + 1) * sizeof(int32_t)) + 15) & ~(size_t)15;
        if (A.cache == 2) off += ((size_t)n_rec * NDOF * A.lmax * sizeof(V) + 15) & ~(size_t)15;
        sco = reinterpret_cast<int32_t *>(kdyn + off);
        sP = reinterpret_cast<float *>(kdyn + off + (((size_t)n_rec * sizeof(int32_t) + 15) & ~(size_t)15));
    }
    // the CTA's rows of the coarse inverse (CO with c_xs): after the coarse records
    T *sX = nullptr;
    if constexpr (CO) {
        if (co && A.c_xs) {
            size_t off = (((size_t)n_rec * (A.lmax + 1) * sizeof(int32_t)) + 15) & ~(size_t)15;
            if (A.cache == 2) off += ((size_t)n_rec * NDOF * A.lmax * sizeof(V) + 15) & ~(size_t)15;
            off += (((size_t)n_rec * sizeof(int32_t) + 15) & ~(size_t)15) +
                   (((size_t)n_rec * NDOF * NM * sizeof(float) + 15) & ~(size_t)15);
            sX = reinterpret_cast<T *>(kdyn + off);
            const T *Xg;
            if constexpr (std::is_same<T, double>::value) Xg = A.c_X64;
            else Xg = A.c_X32;
            const int32_t nc = A.c_nc;
            for (int32_t q = 0; blockIdx.x + q * gridDim.x < nc; ++q)
                for (int32_t j = threadIdx.x; j < nc; j += kThreads)
                    sX[(size_t)q * nc + j] = Xg[(int64_t)(blockIdx.x + q * gridDim.x) * nc + j];
            __syncthreads();
        }
    }
    // a node's coarse data (node_ok lanes only)
    auto cnode = [&](int32_t ps, int32_t nd, int32_t &c, const float *&pp) {
        if (cco) {
            const int32_t rec = rec_of(ps);
            c = sco[rec];
            pp = sP + (size_t)rec * NDOF * NM;
        } else {
            c = A.c_node[nd];
            pp = A.c_P + (size_t)nd * NDOF * NM;
        }
    };
    auto coarse_apply = [&](T *rc, T *dst) {
        coarse_solve<V, T>(A, rc, cc, sX);
        grid.sync();
        for (int32_t ps = 0; ps < passes; ++ps) {
            const int32_t nd = (gw + ps * nw) * NPW + slot;
            if (slot < NPW && nd < n_nodes && sub < NDOF) {
                int32_t c;
                const float *pp;
                cnode(ps, nd, c, pp);
                dst[nd * NDOF + sub] += coarse_prolong<NDOF, T>(sub, cc, c, pp);
            }
        }
        for (int32_t k = blockIdx.x * kThreads + threadIdx.x; k < A.c_nc; k += gridDim.x * kThreads) rc[k] = T(0);
        grid.sync();
    };
    // restriction of a node value held by this lane (every lane calls it)
    auto restrict_node = [&](int32_t ps, int32_t nd, bool node_ok, T val, T *rc) {
        int32_t c = 0;
        const float *pp = nullptr;
        if (node_ok) cnode(ps, nd, c, pp);
        coarse_restrict<NDOF, LPN, T>(node_ok, sub, nbase, val, rc, c, pp);
    };
    if (A.cache > 0) {
        for (int32_t ps = 0; ps < passes; ++ps) {
            const int32_t nd = (gw + ps * nw) * NPW + slot;
            if (slot < NPW && nd < n_nodes) {
                const int32_t rec = rec_of(ps);
                const int32_t base = A.rowptr[nd * NDOF];
                const int32_t len = A.rowptr[nd * NDOF + 1] - base;
                int32_t *cs = scol + (size_t)rec * (A.lmax + 1);
                if (sub == 0) cs[0] = len;
                for (int32_t j = sub; j < len; j += LPN) cs[1 + j] = A.colidx[base + j];
                if (A.cache == 2) {
                    V *cv = sval + (size_t)rec * NDOF * A.lmax;
                    for (int i = 0; i < NDOF; ++i)
                        for (int32_t j = sub; j < len; j += LPN) cv[i * A.lmax + j] = A.vals[base + i * len + j];
                }
                if (cco) {
                    if (sub == 0) sco[rec] = A.c_node[nd];
                    for (int i = sub; i < NDOF * NM; i += LPN) sP[(size_t)rec * NDOF * NM + i] = A.c_P[(size_t)nd * NDOF * NM + i];
                }
            }
        }
        __syncwarp();       // each warp reads only its own records
    }
    // accumulator slots (two parities each, see acc_add); the initial <r, r> uses
    // parity 1 of the slots that iteration 0's phase 3 fills in parity 0
    enum { S_RHO = 0, S_RR = 1, S_SIG = 2, S_TS = 3, S_TT = 4 };

    // init: r = b (free), rh = r, p = r, v = q = x~ = 0, y = M^-1 r; <r, r>
    {
        DotAcc<T> rr;
        for (int32_t ps = 0; ps < passes; ++ps) {
            const int32_t nd = (gw + ps * nw) * NPW + slot;
            const bool node_ok = slot < NPW && nd < n_nodes;
            const bool own = node_ok && sub < NDOF;
            const int32_t row = nd * NDOF + sub;
            const bool fx = own ? A.fixed[row] != 0 : true;
            const T bv = (own && !fx) ? (T)A.b[row] : T(0);
            const T yv = node_apply<NDOF, T>(A.binv, nd, node_ok, sub, nbase, bv, fx);
            if (co) restrict_node(ps, nd, node_ok, bv, rc0);
            if (own) {
                r[row] = bv;
                rh[row] = bv;
                p[row] = bv;
                v[row] = T(0);
                q[row] = T(0);
                xt[row] = T(0);
                wv[row] = yv;
                rr.add(bv, bv);
            }
        }
        double pv[2] = {rr.value(), rr.value()};
        const int sl[2] = {S_RHO, S_RR};
        acc_add<2>(pv, A.red, sl, 1);
    }
    grid.sync();
    double tot[2];
    {
        const int sl[2] = {S_RHO, S_RR};
        acc_read<2>(A.red, sl, 1, tot);
    }
    const double bnorm = sqrt(tot[1]);
    double rho = tot[0], alpha = 0.0, omega = 1.0, beta = 0.0, rel = 0.0;
    int it = 0, status = 0, restarts = 0;
    if (!(bnorm > 0.0)) {
        if (!(bnorm == 0.0)) status = 2;
    } else {
        if (co) coarse_apply(rc0, wv);
        // u = A w
        for (int32_t ps0 = 0; ps0 < passes; ps0 += UP) {
            int32_t ndu[UP];
            bool oku[UP];
            T au[UP];
#pragma unroll
            for (int k = 0; k < UP; ++k) {
                ndu[k] = (gw + (ps0 + k) * nw) * NPW + slot;
                oku[k] = ps0 + k < passes && slot < NPW && ndu[k] < n_nodes;
            }
            const int32_t *csu[UP];
#pragma unroll
            for (int k = 0; k < UP; ++k) csu[k] = A.cache > 0 ? scol + (size_t)rec_of(ps0 + k) * (A.lmax + 1) : nullptr;
            const V *cvu[UP];
#pragma unroll
            for (int k = 0; k < UP; ++k) cvu[k] = A.cache == 2 ? sval + (size_t)rec_of(ps0 + k) * NDOF * A.lmax : nullptr;
            row_products<NDOF, LPN, UP, V, T>(A, ndu, oku, sub, wv, au, csu, cvu);
#pragma unroll
            for (int k = 0; k < UP; ++k)
                if (oku[k] && sub < NDOF) {
                    const int32_t row = ndu[k] * NDOF + sub;
                    u[row] = A.fixed[row] ? T(0) : au[k];
                }
        }
        for (it = 0; it < A.max_it; ++it) {
            // phase 1
            {
                DotAcc<T> s1;
                const T tb = (T)beta, tbo = (T)(beta * omega);
                for (int32_t ps = 0; ps < passes; ++ps) {
                    const int32_t nd = (gw + ps * nw) * NPW + slot;
                    const bool node_ok = slot < NPW && nd < n_nodes;
                    const bool own = node_ok && sub < NDOF;
                    const int32_t row = nd * NDOF + sub;
                    T vn = T(0);
                    bool fx = true;
                    if (own) {
                        fx = A.fixed[row] != 0;
                        const T vo = v[row];
                        p[row] = r[row] + tb * p[row] - tbo * vo;
                        vn = u[row] + tb * vo - tbo * q[row];
                        v[row] = vn;
                        s1.add(rh[row], vn);
                    }
                    const T yv = node_apply<NDOF, T>(A.binv, nd, node_ok, sub, nbase, vn, fx);
                    if (co) restrict_node(ps, nd, node_ok, vn, rc0);
                    if (own) y[row] = yv;
                }
                double pv[1] = {s1.value()};
                const int sl[1] = {S_SIG};
                acc_add<1>(pv, A.red, sl, it & 1);
            }
            grid.sync();
            {
                double t1[1];
                const int sl[1] = {S_SIG};
                acc_read<1>(A.red, sl, it & 1, t1);
                alpha = t1[0] != 0.0 ? rho / t1[0] : 0.0;
            }
            if (co) coarse_apply(rc0, y);
            // phase 2
            {
                DotAcc<T> ts, tt;
                const T ta = (T)alpha;
                for (int32_t ps0 = 0; ps0 < passes; ps0 += UP) {
                    int32_t ndu[UP];
                    bool oku[UP];
                    T au[UP];
#pragma unroll
                    for (int k = 0; k < UP; ++k) {
                        ndu[k] = (gw + (ps0 + k) * nw) * NPW + slot;
                        oku[k] = ps0 + k < passes && slot < NPW && ndu[k] < n_nodes;
                    }
                    const int32_t *csu[UP];
#pragma unroll
            for (int k = 0; k < UP; ++k) csu[k] = A.cache > 0 ? scol + (size_t)rec_of(ps0 + k) * (A.lmax + 1) : nullptr;
            const V *cvu[UP];
#pragma unroll
            for (int k = 0; k < UP; ++k) cvu[k] = A.cache == 2 ? sval + (size_t)rec_of(ps0 + k) * NDOF * A.lmax : nullptr;
            row_products<NDOF, LPN, UP, V, T>(A, ndu, oku, sub, y, au, csu, cvu);
#pragma unroll
                    for (int k = 0; k < UP; ++k)
                        if (oku[k] && sub < NDOF) {
                            const int32_t row = ndu[k] * NDOF + sub;
                            const T qn = A.fixed[row] ? T(0) : au[k];
                            q[row] = qn;
                            const T sv = r[row] - ta * v[row];
                            const T tv = u[row] - ta * qn;
                            r[row] = sv;
                            t[row] = tv;
                            ts.add(tv, sv);
                            tt.add(tv, tv);
                        }
                }
                double pv[2] = {ts.value(), tt.value()};
                const int sl[2] = {S_TS, S_TT};
                acc_add<2>(pv, A.red, sl, it & 1);
            }
            grid.sync();
            {
                double t2[2];
                const int sl[2] = {S_TS, S_TT};
                acc_read<2>(A.red, sl, it & 1, t2);
                omega = t2[1] != 0.0 ? t2[0] / t2[1] : 0.0;
            }
            // phase 3
            {
                DotAcc<T> prr, prhr;
                const T ta = (T)alpha, to = (T)omega;
                for (int32_t ps = 0; ps < passes; ++ps) {
                    const int32_t nd = (gw + ps * nw) * NPW + slot;
                    const bool node_ok = slot < NPW && nd < n_nodes;
                    const bool own = node_ok && sub < NDOF;
                    const int32_t row = nd * NDOF + sub;
                    T rn = T(0);
                    bool fx = true;
                    if (own) {
                        fx = A.fixed[row] != 0;
                        const T sv = r[row];
                        xt[row] += ta * p[row] + to * sv;
                        rn = sv - to * t[row];
                        r[row] = rn;
                        prhr.add(rh[row], rn);
                        prr.add(rn, rn);
                    }
                    const T wn = node_apply<NDOF, T>(A.binv, nd, node_ok, sub, nbase, rn, fx);
                    if (co) restrict_node(ps, nd, node_ok, rn, rc1);
                    if (own) wv[row] = wn;
                }
                double pv[2] = {prhr.value(), prr.value()};
                const int sl[2] = {S_RHO, S_RR};
                acc_add<2>(pv, A.red, sl, it & 1);
            }
            grid.sync();
            double t3[2];
            {
                const int sl[2] = {S_RHO, S_RR};
                acc_read<2>(A.red, sl, it & 1, t3);
            }
            rel = sqrt(t3[1]) / bnorm;
            if (!(rel == rel)) {
                status = 2;
                ++it;
                break;
            }
            if (rel <= A.rtol) {
                ++it;
                break;
            }
            bool restart = false;
            if (t3[0] == 0.0 || omega == 0.0 || rho == 0.0) {
                if (restarts >= 16) {
                    status = 1;
                    ++it;
                    break;
                }
                ++restarts;
                restart = true;
                beta = 0.0;
                rho = t3[1];
            } else {
                beta = (t3[0] / rho) * (alpha / omega);
                rho = t3[0];
            }
            if (co) coarse_apply(rc1, wv);
            // phase 4: u = A w (and rh = r on a restart)
            for (int32_t ps0 = 0; ps0 < passes; ps0 += UP) {
                int32_t ndu[UP];
                bool oku[UP];
                T au[UP];
#pragma unroll
                for (int k = 0; k < UP; ++k) {
                    ndu[k] = (gw + (ps0 + k) * nw) * NPW + slot;
                    oku[k] = ps0 + k < passes && slot < NPW && ndu[k] < n_nodes;
                }
                const int32_t *csu[UP];
#pragma unroll
            for (int k = 0; k < UP; ++k) csu[k] = A.cache > 0 ? scol + (size_t)rec_of(ps0 + k) * (A.lmax + 1) : nullptr;
            const V *cvu[UP];
#pragma unroll
            for (int k = 0; k < UP; ++k) cvu[k] = A.cache == 2 ? sval + (size_t)rec_of(ps0 + k) * NDOF * A.lmax : nullptr;
            row_products<NDOF, LPN, UP, V, T>(A, ndu, oku, sub, wv, au, csu, cvu);
#pragma unroll
                for (int k = 0; k < UP; ++k)
                    if (oku[k] && sub < NDOF) {
                        const int32_t row = ndu[k] * NDOF + sub;
                        u[row] = A.fixed[row] ? T(0) : au[k];
                        if (restart) rh[row] = r[row];
                    }
            }
        }
        if (it >= A.max_it && rel > A.rtol && status == 0) status = 3;
    }
    // x = M^-1 x~ (in place when x~ is the FP64 output)
    for (int32_t ps = 0; ps < passes; ++ps) {
        const int32_t nd = (gw + ps * nw) * NPW + slot;
        const bool node_ok = slot < NPW && nd < n_nodes;
        const bool own = node_ok && sub < NDOF;
        const int32_t row = nd * NDOF + sub;
        const bool fx = own ? A.fixed[row] != 0 : true;
        const T xv = own ? xt[row] : T(0);
        const T xo = node_apply<NDOF, T>(A.binv, nd, node_ok, sub, nbase, xv, fx);
        if (co) restrict_node(ps, nd, node_ok, xv, rc0);
        if (own) A.x_out[row] = (double)xo;
    }
    if (co) {
        grid.sync();
        coarse_solve<V, T>(A, rc0, cc, sX);
        grid.sync();
        for (int32_t ps = 0; ps < passes; ++ps) {
            const int32_t nd = (gw + ps * nw) * NPW + slot;
            if (slot < NPW && nd < n_nodes && sub < NDOF) {
                int32_t c;
                const float *pp;
                cnode(ps, nd, c, pp);
                A.x_out[nd * NDOF + sub] += (double)coarse_prolong<NDOF, T>(sub, cc, c, pp);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.out[0] = it;
        A.out[1] = rel;
        A.out[2] = status;
    }
}

// ---------------------------------------------------------------------------
// Batched specimens: independent BiCGStab recurrences per specimen in one
// cooperative launch.  Block b owns the contiguous nodes [b chunk, (b+1) chunk)
// and so at most a few specimens (the union mesh lays them end to end); each
// specimen has its own alpha, omega, rho, stopping test and breakdown status, so
// a specimen stops when its own residual meets its own tolerance and its nodes
// are skipped from then on.  Dot products are reduced per specimen: a warp keeps
// a running sum while its 32 consecutive nodes belong to one specimen and adds
// it to a per-warp shared-memory row when the specimen changes; the block writes
// one partial per (slot, specimen), and every block that owns a specimen sums
// that specimen's partials over the blocks it spans in the same order, so all
// owners take the same decisions.  The loop ends when no specimen is active:
// the first owner block of every active specimen counts it into a device
// counter that all blocks read after the next grid barrier.
// ---------------------------------------------------------------------------
constexpr int kWarpsPB = kThreads / 32;
constexpr int kBSlots = 2;                 // partial sums per phase
enum { BS_RHO = 0, BS_RR = 1, BS_RHV = 2, BS_TS = 3, BS_TT = 4 };

struct BShared {
    double acc[kWarpsPB][kBSlots][kMaxSpecPerBlock];
    double rho[kMaxSpecPerBlock], rho_old[kMaxSpecPerBlock], alpha[kMaxSpecPerBlock], omega[kMaxSpecPerBlock];
    double bn[kMaxSpecPerBlock], rel[kMaxSpecPerBlock], tot[kBSlots][kMaxSpecPerBlock];
    int act[kMaxSpecPerBlock], its[kMaxSpecPerBlock], st[kMaxSpecPerBlock], rst[kMaxSpecPerBlock],
        keep[kMaxSpecPerBlock];
    int cnt;
};

// running per-specimen sums of one warp (j = block-local specimen, -1 = none);
// the increments of slot k are products x[k] y[k], accumulated as DotAcc<T>
template <class T>
struct WarpAcc {
    DotAcc<T> v[kBSlots];
    int j = -1;
};

template <class T>
__device__ __forceinline__ void wacc_flush(WarpAcc<T> &a, BShared &S, int w, int lane)
{
    if (a.j >= 0) {
#pragma unroll
        for (int k = 0; k < kBSlots; ++k) {
            const double s = warp_sum(a.v[k].value());
            if (lane == 0) S.acc[w][k][a.j] += s;
        }
    }
    a.j = -1;
#pragma unroll
    for (int k = 0; k < kBSlots; ++k) a.v[k] = DotAcc<T>();
}

// every lane of the warp calls this once per group (valid = the lane holds a row)
template <class T>
__device__ __forceinline__ void wacc_add(WarpAcc<T> &a, BShared &S, int w, int lane, bool valid, int j,
                                         const T (&x)[kBSlots], const T (&y)[kBSlots])
{
    const unsigned vm = __ballot_sync(0xffffffffu, valid);
    if (vm == 0u) return;
    const int j0 = __shfl_sync(0xffffffffu, j, __ffs(vm) - 1);
    const bool uniform = __all_sync(0xffffffffu, !valid || j == j0);
    if (uniform && j0 == a.j) {
        if (valid)
#pragma unroll
            for (int k = 0; k < kBSlots; ++k) a.v[k].add(x[k], y[k]);
        return;
    }
    wacc_flush(a, S, w, lane);
    if (uniform) {
        a.j = j0;
        if (valid)
#pragma unroll
            for (int k = 0; k < kBSlots; ++k) a.v[k].add(x[k], y[k]);
        return;
    }
    // the group straddles specimens: reduce each one separately (at most once per
    // specimen boundary)
    int jmin = valid ? j : 1 << 30, jmax = valid ? j : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        jmin = min(jmin, __shfl_xor_sync(0xffffffffu, jmin, o));
        jmax = max(jmax, __shfl_xor_sync(0xffffffffu, jmax, o));
    }
    for (int jj = jmin; jj <= jmax; ++jj) {
#pragma unroll
        for (int k = 0; k < kBSlots; ++k) {
            const double s = warp_sum((valid && j == jj) ? (double)x[k] * (double)y[k] : 0.0);
            if (lane == 0) S.acc[w][k][jj] += s;
        }
    }
}

// block partials of the phase -> red[(slot * nb + b) * J + j]; clears the rows
__device__ __forceinline__ void bpartials(BShared &S, const gd::BatchKrylov &L, int ns, int slot0, int slot1)
{
    __syncthreads();
    const int nb = gridDim.x;
    for (int t = threadIdx.x; t < kBSlots * ns; t += blockDim.x) {
        const int k = t / ns, j = t - k * ns;
        double s = 0.0;
        for (int w = 0; w < kWarpsPB; ++w) s += S.acc[w][k][j];
        const int slot = k == 0 ? slot0 : slot1;
        if (slot >= 0) L.red[((size_t)slot * nb + blockIdx.x) * L.J + j] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kWarpsPB * kBSlots * kMaxSpecPerBlock; t += blockDim.x)
        (&S.acc[0][0][0])[t] = 0.0;
    __syncthreads();
}

// totals of the block's specimens (after a grid barrier) -> S.tot[k][j]: one warp
// per (slot, specimen) pair loads that specimen's block partials in parallel (a
// large specimen spans many blocks) and reduces them in a fixed pattern
__device__ __forceinline__ void btotals(BShared &S, const gd::BatchKrylov &L, int fs, int ns, int slot0, int slot1)
{
    const int nb = gridDim.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = w; t < kBSlots * ns; t += kWarpsPB) {
        const int k = t / ns, j = t - k * ns;
        const int slot = k == 0 ? slot0 : slot1;
        double s = 0.0;
        if (slot >= 0) {
            const int sp = fs + j;
            const int b0 = L.spec_b0[sp], b1 = L.spec_b1[sp];
            for (int bb = b0 + lane; bb <= b1; bb += 32)
                s += __ldcg(L.red + ((size_t)slot * nb + bb) * L.J + (sp - L.blk_fs[bb]));
        }
        s = warp_sum(s);
        if (lane == 0) S.tot[k][j] = s;
    }
    __syncthreads();
}

// The batch kernel: the three-barrier iteration of bicgstab3_kernel with every
// scalar per specimen.  Block b owns nodes [n0, n1) = [b chunk, (b+1) chunk); its
// warps take node groups of that range in the row mapping of RowMap.
template <int NDOF, int G, int UP, class V, class T>
__global__ void __launch_bounds__(kThreads) bicgstab3_batch_kernel(KArgs<V, T> A, gd::BatchKrylov L)
{
    using M = RowMap<NDOF, G, T>;
    constexpr int LPN = M::LPN, NPW = M::NPW;
    // UP: node groups per product round (a launch-shape choice of the autotuner)
    cg::grid_group grid = cg::this_grid();
    __shared__ BShared S;
    const int b = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int slot = lane / LPN, sub = lane - slot * LPN, nbase = slot * LPN;
    const int32_t n0 = b * (int32_t)L.chunk;
    const int32_t n1 = n0 + (int32_t)L.chunk < (int32_t)A.n_nodes ? n0 + (int32_t)L.chunk : (int32_t)A.n_nodes;
    const int fs = n0 < n1 ? L.blk_fs[b] : 0;
    const int ns = n0 < n1 ? L.blk_ns[b] : 0;
    const int32_t passes = ((int32_t)L.chunk + kWarpsPB * NPW - 1) / (kWarpsPB * NPW);   // grid-uniform
    // y = M^-1 v and w = M^-1 r are separate for the reason given at bicgstab3_kernel
    T *r = A.r, *rh = A.rh, *p = A.p, *v = A.v, *q = A.s, *t = A.t, *y = A.y, *wv = A.w, *u = A.z, *xt = A.x;
    for (int i = threadIdx.x; i < kWarpsPB * kBSlots * kMaxSpecPerBlock; i += blockDim.x) (&S.acc[0][0][0])[i] = 0.0;
    for (int j = threadIdx.x; j < kMaxSpecPerBlock; j += blockDim.x) {
        S.act[j] = 1;
        S.its[j] = 0;
        S.st[j] = 0;
        S.rel[j] = 0.0;
        S.alpha[j] = 0.0;
        S.omega[j] = 1.0;
        S.rho_old[j] = 0.0;     // holds beta between phase 3 and the next phase 1
        S.rst[j] = 0;
        S.keep[j] = 0;
    }
    __syncthreads();
    // node of this lane in pass ps, its block-local specimen (-1: none) and row ownership
    auto node_of = [&](int32_t ps, int32_t &nd, bool &node_ok, int &j) {
        nd = n0 + (w + ps * kWarpsPB) * NPW + slot;
        node_ok = slot < NPW && nd < n1;
        j = node_ok ? L.node_spec[nd] - fs : -1;
    };
    // init: r = b (free), rh = p = r, v = q = x~ = 0, y = M^-1 r; per-specimen ||b||^2
    {
        WarpAcc<T> acc;
        for (int32_t ps = 0; ps < passes; ++ps) {
            int32_t nd;
            bool node_ok;
            int j;
            node_of(ps, nd, node_ok, j);
            const bool own = node_ok && sub < NDOF;
            const int32_t row = nd * NDOF + sub;
            const bool fx = own ? A.fixed[row] != 0 : true;
            const T bv = (own && !fx) ? (T)A.b[row] : T(0);
            const T yv = node_apply<NDOF, T>(A.binv, nd, node_ok, sub, nbase, bv, fx);
            const T xa[kBSlots] = {bv, bv};
            if (own) {
                r[row] = bv;
                rh[row] = bv;
                p[row] = bv;
                v[row] = T(0);
                q[row] = T(0);
                // x~ may be the output itself (FP64): a skipped specimen keeps its x
                if (L.rtol[fs + j] >= 0.0) xt[row] = T(0);
                wv[row] = yv;
            }
            wacc_add(acc, S, w, lane, own, j, xa, xa);
        }
        wacc_flush(acc, S, w, lane);
        bpartials(S, L, ns, BS_RHO, BS_RR);
    }
    grid.sync();
    btotals(S, L, fs, ns, BS_RHO, BS_RR);
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
        const int sp = fs + j;
        S.bn[j] = sqrt(S.tot[1][j]);
        S.rho[j] = S.tot[0][j];
        S.act[j] = S.bn[j] > 0.0 ? 1 : 0;             // a zero right-hand side is solved by x = 0
        if (!(S.bn[j] == S.bn[j])) S.st[j] = 2;
        S.keep[j] = L.rtol[sp] < 0.0 ? 1 : 0;         // skipped: x of this specimen is left as it is
        if (S.keep[j]) S.act[j] = 0;
        if (S.act[j] && b == L.spec_b0[sp]) atomicAdd(&L.active_cnt[0], 1);
    }
    __syncthreads();
    // u = A w
    for (int32_t ps0 = 0; ps0 < passes; ps0 += UP) {
        int32_t ndu[UP];
        bool oku[UP];
        T au[UP];
#pragma unroll
        for (int k = 0; k < UP; ++k) {
            int jk;
            bool nok;
            node_of(ps0 + k, ndu[k], nok, jk);
            oku[k] = ps0 + k < passes && nok && S.act[jk];
        }
        {
            const int32_t *csu[UP] = {};
            const V *cvu[UP] = {};
            row_products<NDOF, LPN, UP, V, T>(A, ndu, oku, sub, wv, au, csu, cvu);
        }
#pragma unroll
        for (int k = 0; k < UP; ++k)
            if (oku[k] && sub < NDOF) {
                const int32_t row = ndu[k] * NDOF + sub;
                u[row] = A.fixed[row] ? T(0) : au[k];
            }
    }
    int it = 0;
    for (it = 0; it < A.max_it; ++it) {
        // phase 1: p, v, y = M^-1 v, <rh, v>
        {
            WarpAcc<T> acc;
            for (int32_t ps = 0; ps < passes; ++ps) {
                int32_t nd;
                bool node_ok;
                int j;
                node_of(ps, nd, node_ok, j);
                const bool on = node_ok && S.act[j];
                const bool own = on && sub < NDOF;
                const int32_t row = nd * NDOF + sub;
                T vn = T(0);
                bool fx = true;
                T xa[kBSlots] = {T(0), T(0)}, ya[kBSlots] = {T(0), T(0)};
                if (own) {
                    const T tb = (T)S.rho_old[j], tbo = (T)(S.rho_old[j] * S.omega[j]);
                    fx = A.fixed[row] != 0;
                    const T vo = v[row];
                    p[row] = r[row] + tb * p[row] - tbo * vo;
                    vn = u[row] + tb * vo - tbo * q[row];
                    v[row] = vn;
                    xa[0] = rh[row];
                    ya[0] = vn;
                }
                const T yv = node_apply<NDOF, T>(A.binv, nd, on, sub, nbase, vn, fx);
                if (own) y[row] = yv;
                wacc_add(acc, S, w, lane, own, j, xa, ya);
            }
            wacc_flush(acc, S, w, lane);
            bpartials(S, L, ns, BS_RHV, -1);
        }
        grid.sync();
        if (threadIdx.x == 0) {
            S.cnt = *(volatile int *)&L.active_cnt[it & 1];
            if (b == 0) L.active_cnt[(it + 1) & 1] = 0;
        }
        btotals(S, L, fs, ns, BS_RHV, -1);            // ends with __syncthreads (S.cnt visible)
        if (S.cnt == 0) break;
        for (int j = threadIdx.x; j < ns; j += blockDim.x)
            if (S.act[j]) S.alpha[j] = S.tot[0][j] != 0.0 ? S.rho[j] / S.tot[0][j] : 0.0;
        __syncthreads();
        // phase 2: q = A y, s = r - alpha v, t = u - alpha q, <t, s>, <t, t>
        {
            WarpAcc<T> acc;
            for (int32_t ps0 = 0; ps0 < passes; ps0 += UP) {
                int32_t ndu[UP];
                bool oku[UP];
                int ju[UP];
                T au[UP];
#pragma unroll
                for (int k = 0; k < UP; ++k) {
                    bool nok;
                    node_of(ps0 + k, ndu[k], nok, ju[k]);
                    oku[k] = ps0 + k < passes && nok && S.act[ju[k]];
                }
                {
                    const int32_t *csu[UP] = {};
                    const V *cvu[UP] = {};
                    row_products<NDOF, LPN, UP, V, T>(A, ndu, oku, sub, y, au, csu, cvu);
                }
#pragma unroll
                for (int k = 0; k < UP; ++k) {
                    const bool own = oku[k] && sub < NDOF;
                    const int j = ju[k];
                    T xa[kBSlots] = {T(0), T(0)}, ya[kBSlots] = {T(0), T(0)};
                    if (own) {
                        const int32_t row = ndu[k] * NDOF + sub;
                        const T ta = (T)S.alpha[j];
                        const T qn = A.fixed[row] ? T(0) : au[k];
                        q[row] = qn;
                        const T sv = r[row] - ta * v[row];
                        const T tv = u[row] - ta * qn;
                        r[row] = sv;
                        t[row] = tv;
                        xa[0] = tv;
                        ya[0] = sv;
                        xa[1] = tv;
                        ya[1] = tv;
                    }
                    wacc_add(acc, S, w, lane, own, j, xa, ya);
                }
            }
            wacc_flush(acc, S, w, lane);
            bpartials(S, L, ns, BS_TS, BS_TT);
        }
        grid.sync();
        btotals(S, L, fs, ns, BS_TS, BS_TT);
        for (int j = threadIdx.x; j < ns; j += blockDim.x)
            if (S.act[j]) S.omega[j] = S.tot[1][j] != 0.0 ? S.tot[0][j] / S.tot[1][j] : 0.0;
        __syncthreads();
        // phase 3: x~ += alpha p + omega s, r = s - omega t, y = M^-1 r, <rh, r>, <r, r>
        {
            WarpAcc<T> acc;
            for (int32_t ps = 0; ps < passes; ++ps) {
                int32_t nd;
                bool node_ok;
                int j;
                node_of(ps, nd, node_ok, j);
                const bool on = node_ok && S.act[j];
                const bool own = on && sub < NDOF;
                const int32_t row = nd * NDOF + sub;
                T rn = T(0);
                bool fx = true;
                T xa[kBSlots] = {T(0), T(0)}, ya[kBSlots] = {T(0), T(0)};
                if (own) {
                    const T ta = (T)S.alpha[j], to = (T)S.omega[j];
                    fx = A.fixed[row] != 0;
                    const T sv = r[row];
                    xt[row] += ta * p[row] + to * sv;
                    rn = sv - to * t[row];
                    r[row] = rn;
                    xa[0] = rh[row];
                    ya[0] = rn;
                    xa[1] = rn;
                    ya[1] = rn;
                }
                const T wn = node_apply<NDOF, T>(A.binv, nd, on, sub, nbase, rn, fx);
                if (own) wv[row] = wn;
                wacc_add(acc, S, w, lane, own, j, xa, ya);
            }
            wacc_flush(acc, S, w, lane);
            bpartials(S, L, ns, BS_RHO, BS_RR);
        }
        grid.sync();
        btotals(S, L, fs, ns, BS_RHO, BS_RR);
        // per-specimen decisions (S.st = 4 marks a restart for phase 4)
        for (int j = threadIdx.x; j < ns; j += blockDim.x) {
            if (!S.act[j]) continue;
            const int sp = fs + j;
            const double rel = sqrt(S.tot[1][j]) / S.bn[j];
            S.rel[j] = rel;
            S.its[j] = it + 1;
            if (!(rel == rel)) {
                S.st[j] = 2;
                S.act[j] = 0;
            } else if (rel <= L.rtol[sp]) {
                S.act[j] = 0;
            } else if (S.tot[0][j] == 0.0 || S.omega[j] == 0.0 || S.rho[j] == 0.0) {
                // restart the recurrences with rh = r (at most 16 times)
                if (S.rst[j] >= 16) {
                    S.st[j] = 1;
                    S.act[j] = 0;
                } else {
                    ++S.rst[j];
                    S.st[j] = 4;
                    S.rho_old[j] = 0.0;            // beta = 0
                    S.rho[j] = S.tot[1][j];
                }
            } else {
                S.rho_old[j] = (S.tot[0][j] / S.rho[j]) * (S.alpha[j] / S.omega[j]);   // beta
                S.rho[j] = S.tot[0][j];
            }
            if (S.act[j] && b == L.spec_b0[sp]) atomicAdd(&L.active_cnt[(it + 1) & 1], 1);
        }
        __syncthreads();
        // phase 4: u = A w (and rh = r on a restart)
        for (int32_t ps0 = 0; ps0 < passes; ps0 += UP) {
            int32_t ndu[UP];
            bool oku[UP];
            int ju[UP];
            T au[UP];
#pragma unroll
            for (int k = 0; k < UP; ++k) {
                bool nok;
                node_of(ps0 + k, ndu[k], nok, ju[k]);
                oku[k] = ps0 + k < passes && nok && S.act[ju[k]];
            }
            {
            const int32_t *csu[UP] = {};
            const V *cvu[UP] = {};
            row_products<NDOF, LPN, UP, V, T>(A, ndu, oku, sub, wv, au, csu, cvu);
        }
#pragma unroll
            for (int k = 0; k < UP; ++k)
                if (oku[k] && sub < NDOF) {
                    const int32_t row = ndu[k] * NDOF + sub;
                    u[row] = A.fixed[row] ? T(0) : au[k];
                    if (S.st[ju[k]] == 4) rh[row] = r[row];
                }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < ns; j += blockDim.x)
            if (S.st[j] == 4) S.st[j] = 0;
        __syncthreads();
    }
    // x = M^-1 x~ (not for skipped specimens)
    for (int32_t ps = 0; ps < passes; ++ps) {
        int32_t nd;
        bool node_ok;
        int j;
        node_of(ps, nd, node_ok, j);
        if (node_ok && S.keep[j]) node_ok = false;     // warp-uniform use below only through node_ok
        const bool own = node_ok && sub < NDOF;
        const int32_t row = nd * NDOF + sub;
        const bool fx = own ? A.fixed[row] != 0 : true;
        const T xv = own ? xt[row] : T(0);
        const T xo = node_apply<NDOF, T>(A.binv, nd, node_ok, sub, nbase, xv, fx);
        if (own) A.x_out[row] = (double)xo;
    }
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
        const int sp = fs + j;
        if (b != L.spec_b0[sp] || S.keep[j]) continue;
        L.out[3 * sp + 0] = S.its[j];
        L.out[3 * sp + 1] = S.rel[j];
        L.out[3 * sp + 2] = S.act[j] ? 3 : S.st[j];   // still active: iteration cap
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

// G: lanes per node of the FP32-vector kernels (FP64 vectors use one lane per row)
template <int NDOF, class V, class T, int G = (NDOF == 3 ? 8 : 32)>
cudaError_t solve_t(const KrylovCtx &c, const V *vals, const double *b, double *x, double rtol, int max_it)
{
    T *binv = (T *)c.binv;
    block_inverse_kernel<NDOF, V, T><<<c.num_sms * 4, 256, 0, c.stream>>>(c.n_nodes, c.rowptr, c.colidx, vals,
                                                                          c.fixed, binv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    KArgs<V, T> A{};
    A.n_nodes = c.n_nodes;
    A.rowptr = c.rowptr;
    A.colidx = c.colidx;
    A.vals = vals;
    A.fixed = c.fixed;
    A.binv = binv;
    A.b = b;
    A.x_out = x;
    T *w[10];
    for (int k = 0; k < 9; ++k) w[k] = (T *)c.work[k];
    w[9] = (T *)c.work_x;
    A.x = std::is_same<T, double>::value ? (T *)x : w[9];
    A.w = w[8];
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
    A.cache = 0;
    A.lmax = 0;
    A.c_nc = 0;
    A.c_P = nullptr;
    A.c_node = nullptr;
    A.c_X32 = nullptr;
    A.c_X64 = nullptr;
    A.c_rc = A.c_cc = nullptr;
    A.c_status = nullptr;
    const bool co = c.coarse && c.coarse->nc > 0;
    if (co) {
        const CoarseSpace &cs = *c.coarse;
        if (c.coarse_refresh) {
            e = coarse_setup(cs, NDOF, c.n_nodes, c.rowptr, c.colidx, vals, std::is_same<V, float>::value, true,
                             c.num_sms, c.stream, c.lmax);
            if (e != cudaSuccess) return e;
        }
        e = cudaMemsetAsync(cs.rc, 0, sizeof(T) * 2 * (size_t)cs.nc, c.stream);
        if (e != cudaSuccess) return e;
        A.c_nc = cs.nc;
        A.c_P = cs.P;
        A.c_node = cs.node_co;
        A.c_X32 = cs.X32;
        A.c_X64 = cs.X64;
        A.c_rc = (T *)cs.rc;
        A.c_cc = (T *)cs.cc;
        A.c_status = cs.status;
    }
    // the grid-wide accumulators (2 parities x 5 slots) start at zero
    e = cudaMemsetAsync(c.red, 0, 10 * sizeof(double), c.stream);
    if (e != cudaSuccess) return e;
    void *args[] = {&A};
    const int up = c.up ? c.up : 1;
    // the two-level variant takes one or two node groups per lane and product round
    const void *fn = co        ? (up == 2 ? (const void *)bicgstab3_kernel<NDOF, G, 2, V, T, true>
                                          : (const void *)bicgstab3_kernel<NDOF, G, 1, V, T, true>)
                     : up == 1 ? (const void *)bicgstab3_kernel<NDOF, G, 1, V, T>
                     : up == 4 ? (const void *)bicgstab3_kernel<NDOF, G, 4, V, T>
                               : (const void *)bicgstab3_kernel<NDOF, G, 2, V, T>;
    // Shared-memory copy of each block's rows: column lists and, when they fit,
    // values, for as long as the grid stays co-resident with that shared memory.
    // The products then wait on the gathered x alone instead of the chain
    // row pointer -> column index -> x.
    size_t smem = 0;
    if (c.lmax > 0 && c.row_cache < 2) {
        using M = RowMap<NDOF, G, T>;
        const int64_t nw = (int64_t)c.blocks * (kThreads / 32);
        const int64_t passes = (c.n_nodes + nw * M::NPW - 1) / (nw * M::NPW);
        const int64_t n_rec = passes * (kThreads / 32) * M::NPW;
        const size_t colb = ((size_t)n_rec * (c.lmax + 1) * sizeof(int32_t) + 15) & ~(size_t)15;
        const size_t valb = ((size_t)n_rec * NDOF * c.lmax * sizeof(V) + 15) & ~(size_t)15;
        // the two-level kernel keeps every record's coarse data beside its row
        const size_t cob = co ? (((size_t)n_rec * sizeof(int32_t) + 15) & ~(size_t)15) +
                                    (((size_t)n_rec * NDOF * CoarseModes<NDOF>::NM * sizeof(float) + 15) & ~(size_t)15)
                              : 0;
        // and, for FP32 vectors where it fits, each CTA's rows of the coarse inverse (with
        // FP64 rows the shared memory they take from the L1 cache slows the products more
        // than it speeds the coarse solve: measured 108 against 100 us per iteration)
        const bool want_xs = co && std::is_same<T, float>::value;
        const size_t xsb = want_xs ? (size_t)((c.coarse->nc + c.blocks - 1) / c.blocks) * c.coarse->nc * sizeof(T) : 0;
        const int need = (c.blocks + c.num_sms - 1) / c.num_sms;      // CTAs per SM of this grid
        // preference: values and inverse rows, columns and inverse rows, values, columns
        const int modes[4][2] = {{2, 1}, {1, 1}, {2, 0}, {1, 0}};
        for (int mi = 0; mi < 4 && A.cache == 0; ++mi) {
            const int mode = modes[mi][0], xs = want_xs ? modes[mi][1] : 0;
            if (!want_xs && modes[mi][1]) continue;
            if (mode == 2 && c.row_cache == 1) continue;      // column lists only
            const size_t sm = colb + (mode == 2 ? valb : 0) + cob + (xs ? xsb : 0);
            if (sm > 200 * 1024) continue;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, sm) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (per_sm >= need) {
                A.cache = mode;
                A.lmax = c.lmax;
                A.c_xs = xs;
                smem = sm;
            }
        }
    }
    return cudaLaunchCooperativeKernel(fn, dim3(c.blocks), dim3(kThreads), args, smem, c.stream);
}

template <int NDOF, class V, class T>
cudaError_t solve_batch_t(const KrylovCtx &c, const gd::BatchKrylov &L, const V *vals, const double *b, double *x,
                          int max_it)
{
    constexpr int G = NDOF == 3 ? 8 : 32;
    T *binv = (T *)c.binv;
    block_inverse_kernel<NDOF, V, T><<<c.num_sms * 4, 256, 0, c.stream>>>(c.n_nodes, c.rowptr, c.colidx, vals,
                                                                          c.fixed, binv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(L.active_cnt, 0, 2 * sizeof(int), c.stream);
    if (e != cudaSuccess) return e;
    KArgs<V, T> A{};
    A.n_nodes = c.n_nodes;
    A.rowptr = c.rowptr;
    A.colidx = c.colidx;
    A.vals = vals;
    A.fixed = c.fixed;
    A.binv = binv;
    A.b = b;
    A.x_out = x;
    T *w[10];
    for (int k = 0; k < 9; ++k) w[k] = (T *)c.work[k];
    w[9] = (T *)c.work_x;
    A.x = std::is_same<T, double>::value ? (T *)x : w[9];
    A.w = w[8];
    A.r = w[0];
    A.rh = w[1];
    A.p = w[2];
    A.v = w[3];
    A.s = w[4];
    A.t = w[5];
    A.y = w[6];
    A.z = w[7];
    A.red = nullptr;
    A.out = nullptr;
    A.rtol = 0.0;
    A.max_it = max_it;
    A.cache = 0;
    A.lmax = 0;
    gd::BatchKrylov Lc = L;
    void *args[] = {&A, &Lc};
    const int up = c.up ? c.up : 1;
    const void *fn = up == 1   ? (const void *)bicgstab3_batch_kernel<NDOF, G, 1, V, T>
                     : up == 4 ? (const void *)bicgstab3_batch_kernel<NDOF, G, 4, V, T>
                               : (const void *)bicgstab3_batch_kernel<NDOF, G, 2, V, T>;
    return cudaLaunchCooperativeKernel(fn, dim3(c.blocks), dim3(kThreads),
                                       args, 0, c.stream);
}

// co-resident CTAs per SM of the solve kernels of one variant (every UP)
template <int NDOF, class V, class T>
int coop_per_sm()
{
    constexpr int G = NDOF == 3 ? 8 : 32;
    constexpr int G2 = (NDOF == 4 && std::is_same<T, float>::value) ? 8 : G;   // the other lane counts
    constexpr int G3 = (NDOF == 4 && std::is_same<T, float>::value) ? 4 : G;   // of the 3D FP32 solve
    const void *fns[16] = {(const void *)bicgstab3_kernel<NDOF, G, 1, V, T>, (const void *)bicgstab3_kernel<NDOF, G, 2, V, T>,
                          (const void *)bicgstab3_kernel<NDOF, G, 4, V, T>,
                          (const void *)bicgstab3_kernel<NDOF, G, 1, V, T, true>,
                          (const void *)bicgstab3_batch_kernel<NDOF, G, 1, V, T>,
                          (const void *)bicgstab3_batch_kernel<NDOF, G, 2, V, T>,
                          (const void *)bicgstab3_batch_kernel<NDOF, G, 4, V, T>,
                          (const void *)bicgstab3_kernel<NDOF, G2, 1, V, T>, (const void *)bicgstab3_kernel<NDOF, G2, 2, V, T>,
                          (const void *)bicgstab3_kernel<NDOF, G2, 4, V, T>,
                          (const void *)bicgstab3_kernel<NDOF, G2, 1, V, T, true>,
                          (const void *)bicgstab3_kernel<NDOF, G3, 1, V, T>,
                          (const void *)bicgstab3_kernel<NDOF, G3, 1, V, T, true>,
                          (const void *)bicgstab3_kernel<NDOF, G, 2, V, T, true>,
                          (const void *)bicgstab3_kernel<NDOF, G2, 2, V, T, true>,
                          (const void *)bicgstab3_kernel<NDOF, G3, 2, V, T, true>};
    int best = 1 << 30;
    for (const void *f : fns) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kThreads, 0) != cudaSuccess) return 0;
        if (per_sm < best) best = per_sm;
    }
    return best;
}

__global__ void narrow_kernel(const double *in, float *out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

}  // namespace

template <int NDOF>
int coop_per_sm_fp32()
{
    constexpr int G = NDOF == 3 ? 8 : 32;
    constexpr int G2 = NDOF == 4 ? 8 : G, G3 = NDOF == 4 ? 4 : G;
    const void *fns[] = {
        (const void *)bicgstab3_kernel<NDOF, G, 1, float, float>, (const void *)bicgstab3_kernel<NDOF, G, 2, float, float>,
        (const void *)bicgstab3_kernel<NDOF, G, 4, float, float>,
        (const void *)bicgstab3_kernel<NDOF, G, 1, float, float, true>,
        (const void *)bicgstab3_kernel<NDOF, G, 2, float, float, true>,
        (const void *)bicgstab3_kernel<NDOF, G2, 1, float, float>, (const void *)bicgstab3_kernel<NDOF, G2, 2, float, float>,
        (const void *)bicgstab3_kernel<NDOF, G2, 4, float, float>,
        (const void *)bicgstab3_kernel<NDOF, G2, 1, float, float, true>,
        (const void *)bicgstab3_kernel<NDOF, G2, 2, float, float, true>,
        (const void *)bicgstab3_kernel<NDOF, G3, 1, float, float>, (const void *)bicgstab3_kernel<NDOF, G3, 2, float, float>,
        (const void *)bicgstab3_kernel<NDOF, G3, 4, float, float>,
        (const void *)bicgstab3_kernel<NDOF, G3, 1, float, float, true>,
        (const void *)bicgstab3_kernel<NDOF, G3, 2, float, float, true>};
    int best = 1 << 30;
    for (const void *f : fns) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kThreads, 0) != cudaSuccess) return 0;
        if (per_sm < best) best = per_sm;
    }
    return best;
}

int krylov_blocks_fp32(int ndof, int num_sms, int cap)
{
    int per_sm = ndof == 3 ? coop_per_sm_fp32<3>() : coop_per_sm_fp32<4>();
    if (cap > 0 && per_sm > cap) per_sm = cap;
    return per_sm * num_sms;
}

int krylov_blocks(int ndof, bool fp32_vals, int num_sms, int cap)
{
    // the smallest co-resident grid over the variants, so one size fits every launch
    int a = ndof == 3 ? coop_per_sm<3, double, double>() : coop_per_sm<4, double, double>();
    int b = ndof == 3 ? coop_per_sm<3, float, float>() : coop_per_sm<4, float, float>();
    int c = ndof == 3 ? coop_per_sm<3, float, double>() : coop_per_sm<4, float, double>();
    (void)fp32_vals;
    int per_sm = a < b ? a : b;
    if (c < per_sm) per_sm = c;
    if (cap > 0 && per_sm > cap) per_sm = cap;
    return per_sm * num_sms;
}

cudaError_t krylov_solve(const KrylovCtx &c, const void *vals, bool fp32_vals, const double *b, double *x,
                         double rtol, int max_it, bool fp32_vectors)
{
    if (fp32_vectors) {
        if (!fp32_vals) return cudaErrorInvalidValue;
        if (c.ndof == 3) return solve_t<3, float, float>(c, (const float *)vals, b, x, rtol, max_it);
        if (c.lanes == 4) return solve_t<4, float, float, 4>(c, (const float *)vals, b, x, rtol, max_it);
        if (c.lanes == 8) return solve_t<4, float, float, 8>(c, (const float *)vals, b, x, rtol, max_it);
        return solve_t<4, float, float>(c, (const float *)vals, b, x, rtol, max_it);
    }
    if (c.ndof == 3)
        return fp32_vals ? solve_t<3, float, double>(c, (const float *)vals, b, x, rtol, max_it)
                         : solve_t<3, double, double>(c, (const double *)vals, b, x, rtol, max_it);
    return fp32_vals ? solve_t<4, float, double>(c, (const float *)vals, b, x, rtol, max_it)
                     : solve_t<4, double, double>(c, (const double *)vals, b, x, rtol, max_it);
}

cudaError_t krylov_solve_batch(const KrylovCtx &c, const BatchKrylov &L, const void *vals, bool fp32_vals,
                               const double *b, double *x, int max_it, bool fp32_vectors)
{
    if (fp32_vectors) {
        if (!fp32_vals) return cudaErrorInvalidValue;
        return c.ndof == 3 ? solve_batch_t<3, float, float>(c, L, (const float *)vals, b, x, max_it)
                           : solve_batch_t<4, float, float>(c, L, (const float *)vals, b, x, max_it);
    }
    if (c.ndof == 3)
        return fp32_vals ? solve_batch_t<3, float, double>(c, L, (const float *)vals, b, x, max_it)
                         : solve_batch_t<3, double, double>(c, L, (const double *)vals, b, x, max_it);
    return fp32_vals ? solve_batch_t<4, float, double>(c, L, (const float *)vals, b, x, max_it)
                     : solve_batch_t<4, double, double>(c, L, (const double *)vals, b, x, max_it);
}

cudaError_t launch_block_inverse(int ndof, int64_t n_nodes, const int32_t *rowptr, const int32_t *colidx,
                                 const void *vals, bool fp32_vals, const uint8_t *fixed, double *binv, int num_sms,
                                 cudaStream_t s)
{
    const int grid = num_sms * 4;
    if (ndof == 3) {
        if (fp32_vals)
            block_inverse_kernel<3, float, double><<<grid, 256, 0, s>>>(n_nodes, rowptr, colidx, (const float *)vals, fixed, binv);
        else
            block_inverse_kernel<3, double, double><<<grid, 256, 0, s>>>(n_nodes, rowptr, colidx, (const double *)vals, fixed, binv);
    } else {
        if (fp32_vals)
            block_inverse_kernel<4, float, double><<<grid, 256, 0, s>>>(n_nodes, rowptr, colidx, (const float *)vals, fixed, binv);
        else
            block_inverse_kernel<4, double, double><<<grid, 256, 0, s>>>(n_nodes, rowptr, colidx, (const double *)vals, fixed, binv);
    }
    return cudaGetLastError();
}

cudaError_t narrow_to_float(const double *in, float *out, int64_t n, cudaStream_t s)
{
    narrow_kernel<<<1024, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

}  // namespace gd
