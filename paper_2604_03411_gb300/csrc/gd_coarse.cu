// gd_coarse.cu -- coarse space of the two-level preconditioner of the Newton
// system solve.
//
// The node-block Jacobi preconditioner alone leaves the BiCGStab iteration count
// growing with the mesh (one iteration moves information one element), and the
// solve then dominates every Newton step.  The second level is an aggregation
// coarse space: the nodes are grouped into connected aggregates of a few dozen
// to a few hundred nodes, and on every aggregate the coarse basis holds the
// constant fields of each nodal unknown (displacement components and the
// non-local damage) and the infinitesimal rigid rotations of the displacement,
// zero on prescribed dofs and orthonormalised per aggregate.  With P the matrix of
// these columns, the Galerkin coarse matrix Ac = P^T A P is assembled from the
// current tangent and inverted densely, and the preconditioner becomes
//   M^-1 = D^-1 + P Ac^-1 P^T      (D: node-block diagonal of A),
// the additive two-level Schwarz form.  The paper solves every Newton system by
// a sparse LU factorisation (Sec. 3.2); this preconditioner only changes how
// fast the iterative replacement converges, not what it converges to.
//
// Host: greedy breadth-first aggregation of the node graph and the per-aggregate
// orthonormal basis (once per handle).  Device: Ac by warp-per-node-row products
// with FP64 atomics, and its explicit inverse by a blocked in-place Gauss-Jordan
// elimination in one cooperative kernel (FP32, diagonal pivots; a zero or
// non-finite pivot sets a status word and the Krylov solve then runs without the
// coarse level).  The inverse is a fixed matrix whatever its accuracy, so the
// preconditioner stays a linear operator: the FP64 Krylov solve applies it in FP64.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "gd_internal.cuh"

namespace cg = cooperative_groups;

namespace gd {

int coarse_modes(int dim) { return dim == 2 ? 4 : 7; }

int32_t coarse_aggregate(int64_t n_nodes, int ndof, const std::vector<int32_t> &rowptr,
                         const std::vector<int32_t> &colidx, int target, std::vector<int32_t> &agg)
{
    if (target < 1) target = 1;
    agg.assign((size_t)n_nodes, -1);
    std::vector<int32_t> queue;
    queue.reserve((size_t)n_nodes);
    int32_t na = 0;
    // neighbours of node i: the column nodes of its first dof row (ndof dofs per node)
    auto row_of = [&](int64_t i, int32_t &b, int32_t &e) {
        b = rowptr[(size_t)(i * ndof)];
        e = rowptr[(size_t)(i * ndof + 1)];
    };
    for (int64_t s = 0; s < n_nodes; ++s) {
        if (agg[s] >= 0) continue;
        queue.clear();
        queue.push_back((int32_t)s);
        agg[s] = na;
        int cnt = 1;
        for (size_t head = 0; head < queue.size() && cnt < target; ++head) {
            int32_t b, e;
            row_of(queue[head], b, e);
            for (int32_t k = b; k < e && cnt < target; k += ndof) {
                const int32_t j = colidx[k] / ndof;
                if (agg[j] < 0) {
                    agg[j] = na;
                    ++cnt;
                    queue.push_back(j);
                }
            }
        }
        ++na;
    }
    // aggregates below a quarter of the target join their smallest neighbour
    std::vector<int64_t> size((size_t)na, 0), ptr((size_t)na + 1, 0);
    for (int64_t i = 0; i < n_nodes; ++i) ++size[agg[i]];
    for (int32_t a = 0; a < na; ++a) ptr[a + 1] = ptr[a] + size[a];
    std::vector<int32_t> nodes((size_t)n_nodes);
    {
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t i = 0; i < n_nodes; ++i) nodes[fill[agg[i]]++] = (int32_t)i;
    }
    std::vector<int32_t> label((size_t)na);
    for (int32_t a = 0; a < na; ++a) label[a] = a;
    auto find = [&](int32_t a) {
        while (label[a] != a) a = label[a];
        return a;
    };
    const int64_t small = std::max(1, target / 4);
    for (int32_t a = 0; a < na; ++a) {
        if (size[a] >= small || label[a] != a) continue;
        int32_t best = -1;
        for (int64_t k = ptr[a]; k < ptr[a + 1]; ++k) {
            int32_t b, e;
            row_of(nodes[k], b, e);
            for (int32_t c = b; c < e; c += ndof) {
                const int32_t o = find(agg[colidx[c] / ndof]);
                if (o == a) continue;
                if (best < 0 || size[o] < size[best] || (size[o] == size[best] && o < best)) best = o;
            }
        }
        if (best >= 0) {
            label[a] = best;
            size[best] += size[a];
            size[a] = 0;
        }
    }
    // compact labels in order of first appearance
    std::vector<int32_t> newid((size_t)na, -1);
    int32_t n_out = 0;
    for (int64_t i = 0; i < n_nodes; ++i) {
        const int32_t r = find(agg[i]);
        if (newid[r] < 0) newid[r] = n_out++;
        agg[i] = newid[r];
    }
    return n_out;
}

void coarse_basis(int dim, int64_t n_nodes, const double *coords, const uint8_t *fixed,
                  const std::vector<int32_t> &agg, int32_t n_agg, std::vector<float> &P, std::vector<int32_t> &coff)
{
    const int ndof = dim + 1, nm = coarse_modes(dim);
    std::vector<int64_t> ptr((size_t)n_agg + 1, 0);
    for (int64_t i = 0; i < n_nodes; ++i) ++ptr[agg[i] + 1];
    for (int32_t a = 0; a < n_agg; ++a) ptr[a + 1] += ptr[a];
    std::vector<int32_t> nodes((size_t)n_nodes);
    {
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t i = 0; i < n_nodes; ++i) nodes[fill[agg[i]]++] = (int32_t)i;
    }
    P.assign((size_t)(n_nodes * ndof * nm), 0.0f);
    coff.assign((size_t)n_agg + 1, 0);
    std::vector<double> q, v;
    for (int32_t a = 0; a < n_agg; ++a) {
        const int64_t n0 = ptr[a], cnt = ptr[a + 1] - n0, len = cnt * ndof;
        double c[3] = {0.0, 0.0, 0.0};
        for (int64_t t = 0; t < cnt; ++t)
            for (int J = 0; J < dim; ++J) c[J] += coords[(int64_t)nodes[n0 + t] * dim + J];
        for (int J = 0; J < dim; ++J) c[J] /= (double)cnt;
        q.assign((size_t)(nm * len), 0.0);
        int kept = 0;
        for (int m = 0; m < nm; ++m) {
            // candidate column m on this aggregate's free dofs
            v.assign((size_t)len, 0.0);
            for (int64_t t = 0; t < cnt; ++t) {
                const int64_t i = nodes[n0 + t];
                double x[3] = {0.0, 0.0, 0.0};
                for (int J = 0; J < dim; ++J) x[J] = coords[i * dim + J] - c[J];
                double *f = v.data() + t * ndof;
                if (m < ndof) {
                    f[m] = 1.0;
                } else if (dim == 2) {
                    f[0] = -x[1];
                    f[1] = x[0];
                } else if (m == ndof) {          // rotation about x
                    f[1] = -x[2];
                    f[2] = x[1];
                } else if (m == ndof + 1) {      // about y
                    f[0] = x[2];
                    f[2] = -x[0];
                } else {                         // about z
                    f[0] = -x[1];
                    f[1] = x[0];
                }
                for (int d = 0; d < ndof; ++d)
                    if (fixed[i * ndof + d]) f[d] = 0.0;
            }
            double nrm0 = 0.0;
            for (double e : v) nrm0 += e * e;
            nrm0 = std::sqrt(nrm0);
            if (!(nrm0 > 0.0)) continue;
            // modified Gram-Schmidt against the kept columns, twice
            for (int pass = 0; pass < 2; ++pass)
                for (int k = 0; k < kept; ++k) {
                    const double *qk = q.data() + (size_t)k * len;
                    double dot = 0.0;
                    for (int64_t r = 0; r < len; ++r) dot += qk[r] * v[r];
                    for (int64_t r = 0; r < len; ++r) v[r] -= dot * qk[r];
                }
            double nrm = 0.0;
            for (double e : v) nrm += e * e;
            nrm = std::sqrt(nrm);
            if (!(nrm > 1e-6 * nrm0)) continue;      // (nearly) dependent on the kept ones
            double *qk = q.data() + (size_t)kept * len;
            for (int64_t r = 0; r < len; ++r) qk[r] = v[r] / nrm;
            ++kept;
        }
        for (int64_t t = 0; t < cnt; ++t) {
            const int64_t i = nodes[n0 + t];
            for (int d = 0; d < ndof; ++d)
                for (int k = 0; k < kept; ++k)
                    P[(size_t)((i * ndof + d) * nm + k)] = (float)q[(size_t)k * len + t * ndof + d];
        }
        coff[a + 1] = coff[a] + kept;
    }
}

namespace {

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Ac += P_i^T A_ij P_j over every node block (i, j): one warp per node row, lanes
// over the row's columns; the lanes' outer products are summed per neighbour
// aggregate before the atomic adds.
template <int NDOF, int NM, class V>
__global__ void __launch_bounds__(256) coarse_assemble_kernel(int64_t n_nodes, const int32_t *rowptr,
                                                              const int32_t *colidx, const V *vals,
                                                              const int32_t *agg, const int32_t *coff,
                                                              const float *P, int nc, double *Ac)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < n_nodes; i += nw) {
        const int32_t base = rowptr[i * NDOF], len = rowptr[i * NDOF + 1] - base;
        const int32_t ai = agg[i], oi = coff[ai], ni = coff[ai + 1] - oi;
        float pi[NDOF][NM];
#pragma unroll
        for (int d = 0; d < NDOF; ++d)
#pragma unroll
            for (int m = 0; m < NM; ++m) pi[d][m] = P[(i * NDOF + d) * NM + m];
        for (int32_t j0 = 0; j0 < len; j0 += 32) {
            const int32_t j = j0 + lane;
            const bool ok = j < len;
            double g[NM];
            float pj[NM];
            int32_t aj = -1;
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                g[m] = 0.0;
                pj[m] = 0.0f;
            }
            if (ok) {
                const int32_t col = colidx[base + j];
                const int32_t jn = col / NDOF, e = col - jn * NDOF;
                aj = agg[jn];
#pragma unroll
                for (int d = 0; d < NDOF; ++d) {
                    const double a = (double)vals[base + d * len + j];
#pragma unroll
                    for (int m = 0; m < NM; ++m) g[m] += (double)pi[d][m] * a;
                }
#pragma unroll
                for (int m = 0; m < NM; ++m) pj[m] = P[((int64_t)jn * NDOF + e) * NM + m];
            }
            unsigned pending = __ballot_sync(0xffffffffu, ok);
            while (pending) {
                const int leader = __ffs(pending) - 1;
                const int32_t a2 = __shfl_sync(0xffffffffu, aj, leader);
                const bool mine = ok && aj == a2;
                pending &= ~__ballot_sync(0xffffffffu, mine);
                const int32_t o2 = coff[a2], n2 = coff[a2 + 1] - o2;
#pragma unroll
                for (int m = 0; m < NM; ++m)
#pragma unroll
                    for (int m2 = 0; m2 < NM; ++m2) {
                        const double s = wsum(mine ? g[m] * (double)pj[m2] : 0.0);
                        if (lane == ((m * NM + m2) & 31) && m < ni && m2 < n2)
                            atomicAdd(&Ac[(int64_t)(oi + m) * nc + o2 + m2], s);
                    }
            }
        }
    }
}

// Ac = P^T A P, one warp per node row block, through shared memory (rows of at most
// kCaMaxLen columns): the lanes first form, for every column j of the node's rows, the
// aggregate a_j of its node, g_j[m] = sum_d P_i[d][m] A[(i,d), j] and the column's
// basis values P_j[m2]; lane 0 numbers the distinct aggregates of the row (a few: the
// aggregates are compact); then every lane sums g_j[m] P_j[m2] over the columns of
// each aggregate for its (m, m2) pairs (49 pairs in 3D: two per lane) and adds each
// sum into Ac once.  FP32 products and sums inside a row, FP64 accumulation across
// rows: the coarse matrix is inverted in FP32 and only preconditions.
constexpr int kCaMaxLen = 256;
constexpr int kCaWarps = 8;

template <int NDOF, int NM>
size_t coarse_asm_smem(int lmax)
{
    return (size_t)kCaWarps * ((size_t)lmax * (3 * sizeof(int32_t) + 2 * NM * sizeof(float)));
}

template <int NDOF, int NM, class V>
__global__ void __launch_bounds__(32 * kCaWarps) coarse_assemble_smem_kernel(int64_t n_nodes, const int32_t *rowptr,
                                                                           const int32_t *colidx, const V *vals,
                                                                           const int32_t *agg, const int32_t *coff,
                                                                           const float *P, int nc, int lmax,
                                                                           double *Ac)
{
    extern __shared__ __align__(16) unsigned char ca_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *wbase = ca_smem + (size_t)wib * ((size_t)lmax * (3 * sizeof(int32_t) + 2 * NM * sizeof(float)));
    float *gs = reinterpret_cast<float *>(wbase);                 // [lmax][NM]
    float *ps = gs + (size_t)lmax * NM;                           // [lmax][NM]
    int32_t *aj_s = reinterpret_cast<int32_t *>(ps + (size_t)lmax * NM);   // [lmax] aggregate of column j
    int32_t *slot = aj_s + lmax;                                  // [lmax] its index among the distinct ones
    int32_t *dist = slot + lmax;                                  // [lmax] distinct aggregates
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int NP = NM * NM;
    for (int64_t i = gw; i < n_nodes; i += nw) {
        const int32_t base = rowptr[i * NDOF], len = rowptr[i * NDOF + 1] - base;
        const int32_t ai = agg[i], oi = coff[ai], ni = coff[ai + 1] - oi;
        float pi[NDOF][NM];
#pragma unroll
        for (int d = 0; d < NDOF; ++d)
#pragma unroll
            for (int m = 0; m < NM; ++m) pi[d][m] = P[(i * NDOF + d) * NM + m];
        for (int32_t j = lane; j < len; j += 32) {
            const int32_t col = colidx[base + j];
            const int32_t jn = col / NDOF, e = col - jn * NDOF;
            float g[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) g[m] = 0.0f;
#pragma unroll
            for (int d = 0; d < NDOF; ++d) {
                const float a = (float)vals[base + d * len + j];
#pragma unroll
                for (int m = 0; m < NM; ++m) g[m] += pi[d][m] * a;
            }
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                gs[j * NM + m] = g[m];
                ps[j * NM + m] = P[((int64_t)jn * NDOF + e) * NM + m];
            }
            aj_s[j] = agg[jn];
        }
        __syncwarp();
        int nd = 0;
        if (lane == 0) {
            for (int32_t j = 0; j < len; ++j) {
                const int32_t a = aj_s[j];
                int k = 0;
                while (k < nd && dist[k] != a) ++k;
                if (k == nd) dist[nd++] = a;
                slot[j] = k;
            }
        }
        nd = __shfl_sync(0xffffffffu, nd, 0);
        __syncwarp();
        for (int k = 0; k < nd; ++k) {
            const int32_t a2 = dist[k], o2 = coff[a2], n2 = coff[a2 + 1] - o2;
            for (int pr = lane; pr < NP; pr += 32) {
                const int m = pr / NM, m2 = pr - m * NM;
                float acc = 0.0f;
                for (int32_t j = 0; j < len; ++j)
                    if (slot[j] == k) acc += gs[j * NM + m] * ps[j * NM + m2];
                if (m < ni && m2 < n2 && acc != 0.0f) atomicAdd(&Ac[(int64_t)(oi + m) * nc + o2 + m2], (double)acc);
            }
        }
        __syncwarp();       // the next row rewrites the warp's records
    }
}

constexpr int kGjRows = 16;      // rows per panel
constexpr int kGjThreads = 512;  // threads per CTA; C columns per thread (nc <= C kGjThreads)

// X = Ac^-1 by blocked in-place Gauss-Jordan elimination with diagonal pivots.
// Panels of kGjRows consecutive rows go to the CTAs in turn (panel K to CTA K
// mod grid).  For panel K, its CTA first eliminates the panel's own pivot
// columns among the panel rows: every thread holds the panel rows' values of
// its columns in registers, and for each pivot the thread holding the pivot
// column publishes that column through shared memory (the rows become D^-1
// [panel rows], D the panel's diagonal block, with D^-1 in the pivot columns).
// After a grid barrier every CTA copies the panel to shared memory and updates
// each of its own rows i by x_i -= x_i[panel columns] * panel, the panel columns
// of x_i starting from zero (thread per column, all of the CTA's rows at once,
// so each panel value read from shared memory serves kGjRows rows).  That is the
// unblocked in-place elimination reordered by panels, one grid barrier per panel.
template <int C>
__global__ void __launch_bounds__(kGjThreads) coarse_invert_kernel(const double *Ac, float *X, double *X64, int nc,
                                                                   int *status)
{
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(16) float gsh[];
    float *pp = gsh;                                 // [kGjRows][nc] panel rows
    float *fc = gsh + kGjRows * nc;                  // [kGjRows] pivot column of the panel rows
    float *Fs = fc + kGjRows;                        // [kGjRows][kGjRows] panel columns of the CTA's rows
    const int tid = threadIdx.x;
    const int nb = gridDim.x, b = blockIdx.x;
    const int64_t gtid = (int64_t)b * kGjThreads + tid, nt = (int64_t)nb * kGjThreads;
    const int64_t n2 = (int64_t)nc * nc;
    for (int64_t k = gtid; k < n2; k += nt) X[k] = (float)Ac[k];
    int bad = 0;
    const int np = (nc + kGjRows - 1) / kGjRows;
    grid.sync();
    for (int K = 0; K < np; ++K) {
        const int r0 = K * kGjRows, pr = min(kGjRows, nc - r0);
        if (K % nb == b) {
            float v[C][kGjRows];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int j = tid + c * kGjThreads;
#pragma unroll
                for (int w = 0; w < kGjRows; ++w) v[c][w] = (j < nc && w < pr) ? X[(int64_t)(r0 + w) * nc + j] : 0.0f;
            }
#pragma unroll
            for (int t = 0; t < kGjRows; ++t) {
                if (t >= pr) break;
                const int col = r0 + t;
#pragma unroll
                for (int c = 0; c < C; ++c)
                    if (tid + c * kGjThreads == col)
#pragma unroll
                        for (int w = 0; w < kGjRows; ++w) fc[w] = v[c][w];
                __syncthreads();
                float piv = fc[t];
                if (!(fabsf(piv) > 0.0f) || !isfinite(piv)) {
                    bad = 1;
                    piv = 1.0f;
                }
                const float inv = 1.0f / piv;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int j = tid + c * kGjThreads;
                    if (j == col) {
#pragma unroll
                        for (int w = 0; w < kGjRows; ++w) v[c][w] = w == t ? inv : -fc[w] * inv;
                    } else {
                        const float pt = v[c][t] * inv;
#pragma unroll
                        for (int w = 0; w < kGjRows; ++w) v[c][w] = w == t ? pt : v[c][w] - fc[w] * pt;
                    }
                }
                __syncthreads();                     // fc is rewritten by the next pivot
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int j = tid + c * kGjThreads;
                if (j < nc)
#pragma unroll
                    for (int w = 0; w < kGjRows; ++w)
                        if (w < pr) X[(int64_t)(r0 + w) * nc + j] = v[c][w];
            }
        }
        grid.sync();
        // this CTA's rows: panels K2 = b, b + grid, ... other than K
        const bool any = b < np && !(b == K && b + nb >= np);
        if (any) {
            for (int64_t k = tid; k < (int64_t)pr * nc; k += kGjThreads) pp[k] = X[(int64_t)r0 * nc + k];
            for (int K2 = b; K2 < np; K2 += nb) {
                if (K2 == K) continue;
                const int i0 = K2 * kGjRows, ri = min(kGjRows, nc - i0);
                if (tid < kGjRows * kGjRows) {
                    const int r = tid / kGjRows, t = tid % kGjRows;
                    Fs[tid] = (r < ri && t < pr) ? X[(int64_t)(i0 + r) * nc + r0 + t] : 0.0f;
                }
                __syncthreads();
                for (int c = 0; c < C; ++c) {
                    const int j = tid + c * kGjThreads;
                    if (j >= nc) break;
                    const bool in_panel = j >= r0 && j < r0 + pr;
                    float pt[kGjRows];
#pragma unroll
                    for (int t = 0; t < kGjRows; ++t) pt[t] = t < pr ? pp[t * nc + j] : 0.0f;
#pragma unroll
                    for (int r = 0; r < kGjRows; ++r) {
                        if (r >= ri) break;
                        float x = in_panel ? 0.0f : X[(int64_t)(i0 + r) * nc + j];
                        const float4 *F4 = reinterpret_cast<const float4 *>(Fs + r * kGjRows);
#pragma unroll
                        for (int q = 0; q < kGjRows / 4; ++q) {
                            const float4 f = F4[q];
                            x -= f.x * pt[4 * q] + f.y * pt[4 * q + 1] + f.z * pt[4 * q + 2] + f.w * pt[4 * q + 3];
                        }
                        X[(int64_t)(i0 + r) * nc + j] = x;
                    }
                }
                __syncthreads();                     // Fs (and then pp) are rewritten
            }
        }
    }
    if (bad) atomicOr(status, 1);
    if (X64) {
        grid.sync();
        for (int64_t k = gtid; k < n2; k += nt) X64[k] = (double)X[k];
    }
}

}  // namespace

template <int NDOF, int NM>
cudaError_t launch_coarse_asm_smem(const CoarseSpace &cs, int64_t n_nodes, const int32_t *rowptr,
                                   const int32_t *colidx, const void *vals, bool fp32_vals, int lmax, int num_sms,
                                   cudaStream_t s)
{
    const size_t smem = coarse_asm_smem<NDOF, NM>(lmax);
    const void *fn = fp32_vals ? (const void *)coarse_assemble_smem_kernel<NDOF, NM, float>
                               : (const void *)coarse_assemble_smem_kernel<NDOF, NM, double>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * kCaWarps, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = num_sms * per_sm;
    if (fp32_vals)
        coarse_assemble_smem_kernel<NDOF, NM, float><<<grid, 32 * kCaWarps, smem, s>>>(
            n_nodes, rowptr, colidx, (const float *)vals, cs.agg, cs.coff, cs.P, cs.nc, lmax, cs.Ac);
    else
        coarse_assemble_smem_kernel<NDOF, NM, double><<<grid, 32 * kCaWarps, smem, s>>>(
            n_nodes, rowptr, colidx, (const double *)vals, cs.agg, cs.coff, cs.P, cs.nc, lmax, cs.Ac);
    return cudaGetLastError();
}

cudaError_t coarse_setup(const CoarseSpace &cs, int ndof, int64_t n_nodes, const int32_t *rowptr,
                         const int32_t *colidx, const void *vals, bool fp32_vals, bool want_x64, int num_sms,
                         cudaStream_t s, int lmax)
{
    const int nc = cs.nc;
    cudaError_t e = cudaMemsetAsync(cs.Ac, 0, sizeof(double) * (size_t)nc * nc, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(cs.status, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int grid = num_sms * 8;
    if (lmax > 0 && lmax <= kCaMaxLen) {
        e = ndof == 3 ? launch_coarse_asm_smem<3, 4>(cs, n_nodes, rowptr, colidx, vals, fp32_vals, lmax, num_sms, s)
                      : launch_coarse_asm_smem<4, 7>(cs, n_nodes, rowptr, colidx, vals, fp32_vals, lmax, num_sms, s);
        if (e != cudaSuccess) return e;
    } else if (ndof == 3) {
        if (fp32_vals)
            coarse_assemble_kernel<3, 4, float><<<grid, 256, 0, s>>>(n_nodes, rowptr, colidx, (const float *)vals,
                                                                     cs.agg, cs.coff, cs.P, nc, cs.Ac);
        else
            coarse_assemble_kernel<3, 4, double><<<grid, 256, 0, s>>>(n_nodes, rowptr, colidx, (const double *)vals,
                                                                      cs.agg, cs.coff, cs.P, nc, cs.Ac);
    } else {
        if (fp32_vals)
            coarse_assemble_kernel<4, 7, float><<<grid, 256, 0, s>>>(n_nodes, rowptr, colidx, (const float *)vals,
                                                                     cs.agg, cs.coff, cs.P, nc, cs.Ac);
        else
            coarse_assemble_kernel<4, 7, double><<<grid, 256, 0, s>>>(n_nodes, rowptr, colidx, (const double *)vals,
                                                                      cs.agg, cs.coff, cs.P, nc, cs.Ac);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int C = (nc + kGjThreads - 1) / kGjThreads;
    const void *fn = C <= 1 ? (const void *)coarse_invert_kernel<1>
                     : C == 2 ? (const void *)coarse_invert_kernel<2>
                     : C == 3 ? (const void *)coarse_invert_kernel<3>
                     : C == 4 ? (const void *)coarse_invert_kernel<4>
                     : C == 5 ? (const void *)coarse_invert_kernel<5>
                              : (const void *)coarse_invert_kernel<6>;
    if (C > 6) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * ((size_t)kGjRows * nc + kGjRows + kGjRows * kGjRows);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kGjThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const double *Ac = cs.Ac;
    float *X = cs.X32;
    double *X64 = want_x64 ? cs.X64 : nullptr;
    int ncv = nc;
    int *st = cs.status;
    void *args[] = {(void *)&Ac, (void *)&X, (void *)&X64, (void *)&ncv, (void *)&st};
    return cudaLaunchCooperativeKernel(fn, dim3(num_sms), dim3(kGjThreads), args, smem, s);
}

}  // namespace gd
