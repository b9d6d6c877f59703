// gd_asm_mixed.cu -- FP32 element kernel of the gradient-enhanced damage model
// (GD_MIXED): the same three lane mappings as the FP64 kernel with FP32 element
// math and FP32 networks; FP64 is kept for the loading/unloading decision
// (Phi_d(kappa_n) > 0 evaluated as FP64 G - kappa_n), the history kappa, and the
// residual accumulation (FP32 element rows added into the FP64 global residual).
// Tangent values are FP32.
//
// One warp owns a batch of 32 quadrature points (4 HEX8 or 8 Q4 elements) and
// switches between three lane mappings:
//   qp mode    lane = quadrature point: kinematics, invariants, energy chain,
//              stress and the per-point records of the tangent;
//   unit mode  lane = network unit, one point at a time: both ICNN layers of the
//              energy network (value, gradient by forward tangents, Hessian by
//              one reverse sweep through layer 2) and every yield-network
//              evaluation of the local damage solve, so the per-point iteration
//              counts cost no divergence;
//   row mode   lane = element row (node a, dof i): the row of the consistent
//              tangent and of the residual, accumulated over the points of one
//              element and scattered into CSR through the slot map.
//
// Paper passages: Sec. 3.1f (F, phi_q, grad phi_q, element residual, Table
// kernel_inputs), Sec. 2.1f (P, Y vector, Y), Sec. 2.2f and Sec. 3.2f Eq. (dd_7_no_nn)
// (local update, KKT), Sec. 3.2f (monolithic scheme), Sec. 4.1f (degradation,
// gradient and penalty energies, Eq. (ostwald_potential)), Sec. 4.2f Eqs. (dd_0),
// (dd_1), (Gq_NN), (dd_7).
#include <cuda_runtime.h>

#include "gd_internal.cuh"

namespace gd {
namespace {

constexpr float kGauss = 0.57735026918962576f;   // 1/sqrt(3)
constexpr float kEpsF = 1.1920929e-7f;

struct MatF {
    float mu_e, lambda_e, eta_d, kappa_d, beta_d, c_d, gamma_d, qcoef;
    int energy, local_max;
};
struct NcF {
    float psi_N0, psi_n, y_N0, y_s;
};
__device__ __forceinline__ NcF ncf(const NetConst &n)
{
    NcF r = {(float)n.psi_N0, (float)n.psi_n, (float)n.y_N0, (float)n.y_s};
    return r;
}
template <class Args>
__device__ __forceinline__ int spec_of(const Args &A, int64_t e) { return A.elem_spec ? __ldg(A.elem_spec + e) : 0; }
template <class Args>
__device__ __forceinline__ const DevNet &psi_of(const Args &A, int s) { return A.psi_tab ? A.psi_tab[s] : A.psi; }
template <class Args>
__device__ __forceinline__ const DevNet &yld_of(const Args &A, int s) { return A.yld_tab ? A.yld_tab[s] : A.yld; }

__device__ __forceinline__ MatF to_f(const MatConst &m)
{
    MatF r;
    r.mu_e = (float)m.mu_e; r.lambda_e = (float)m.lambda_e; r.eta_d = (float)m.eta_d; r.kappa_d = (float)m.kappa_d;
    r.beta_d = (float)m.beta_d; r.c_d = (float)m.c_d; r.gamma_d = (float)m.gamma_d; r.qcoef = (float)m.qcoef;
    r.energy = m.energy; r.local_max = m.local_max;
    return r;
}

__device__ __forceinline__ float softplus(float v) { return fmaxf(v, 0.0f) + log1pf(expf(-fabsf(v))); }
__device__ __forceinline__ float sigm(float v)
{
    float e = expf(-fabsf(v));
    float r = 1.0f / (1.0f + e);
    return v >= 0.0f ? r : e * r;
}
// softplus(v) and its derivative sigmoid(v) from one exponential
__device__ __forceinline__ void sp_sig(float v, float &sp, float &sg)
{
    const float e = expf(-fabsf(v));
    sp = fmaxf(v, 0.0f) + log1pf(e);
    const float r = 1.0f / (1.0f + e);
    sg = v >= 0.0f ? r : e * r;
}
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int DIM>
struct Geo {
    static constexpr int NEN = DIM == 2 ? 4 : 8;
    static constexpr int NQ = NEN;
    static constexpr int NDOF = DIM + 1;
    static constexpr int ND = NEN * NDOF;
    static constexpr int EPW = 32 / NQ;         // elements per batch
    static constexpr int EPR = 32 / ND;         // elements per row pass (Q4: 2, HEX8: 1)
};

// sign of node a along reference axis k (HEX8 ordering; Q4 uses the first four)
__device__ __forceinline__ float node_sgn(int a, int k)
{
    int b = (k == 0) ? ((a & 3) == 1 || (a & 3) == 2) : (k == 1 ? ((a & 3) >= 2) : (a >= 4));
    return b ? 1.0f : -1.0f;
}

// N_a and dN_a/dxi at reference point xi
template <int DIM>
__device__ __forceinline__ void ref_shape(int a, const float *xi, float &N, float *dN)
{
    float f[3], s[3];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        s[k] = node_sgn(a, k);
        f[k] = 0.5f * (1.0f + s[k] * xi[k]);
    }
    N = 1.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) N *= f[k];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        float v = 0.5f * s[k];
#pragma unroll
        for (int l = 0; l < DIM; ++l)
            if (l != k) v *= f[l];
        dN[k] = v;
    }
}

// ---- per-point record (row-mode inputs), floats ----
enum : int {
    Q_JW = 0,
    Q_JINV = 1,      // 9: dxi_k/dX_J at [k*3+J]
    Q_F = 10,        // 9
    Q_P = 19,        // 9: total first Piola-Kirchhoff stress
    Q_M = 28,        // 3: C^-1 grad phi
    Q_H = 31,        // 3: F^-T grad phi
    Q_I1 = 34,
    Q_B = 35,        // 9: F F^T
    Q_FINV = 44,     // 9: F^-1
    Q_HS = 53,       // 6: f_d psi_mn (11 12 13 22 23 33)
    Q_G1 = 59,       // f_d psi_1
    Q_G2 = 60,       // f_d psi_2
    Q_G3J = 61,      // f_d psi_3 J
    Q_PS1 = 62,      // psi_1 (undamaged)
    Q_PS2 = 63,
    Q_PS3J = 64,     // psi_3 J
    Q_CK = 65,       // f_d' c_kappa
    Q_BCK = 66,      // beta_d c_kappa
    Q_FDK = 67,      // f_d' dkappa/dphi
    Q_PP = 68,       // beta_d (1 - dkappa/dphi)
    Q_PEN = 69,      // beta_d (phi - kappa)
    Q_J = 70,        // det F
    Q_REC = 71
};
// ---- per (point, node) vector record ----
enum : int { V_N = 0, V_NN = 3, V_F = 4, V_G2 = 7, V_NT = 10, V_PN = 13, V_MN = 16, V_REC = 17 };

__device__ __forceinline__ int sym6(int i, int j)
{
    // (0,0)0 (0,1)1 (0,2)2 (1,1)3 (1,2)4 (2,2)5
    int a = i < j ? i : j, b = i < j ? j : i;
    return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

// Energy network in unit mode for one point: value, gradient and Hessian of
// N(x) (Sec. 4.2f ICNN).  Layer 1 and the gradient columns of layer 2 are
// forward tangents; the second derivative uses the identity
//   d2N/dx2 = sum_k w3_k sp''(h2_k) g_k g_k^T + sum_j v_j sp''(h1_j) W1_j W1_j^T,
//   g_k = dh2_k/dx,  v = W2^T (w3 o sp'(h2)),
// so layer 2 costs 4 forward columns and 1 reverse column per point.
// Every lane returns the full result.
__device__ void psi_net_unit(const DevNet &net, const float *x, float *out10, float *buf, int lane)
{
    const int w = net.width;
    const float *W1 = net.pf, *b1 = W1 + 3 * w, *W2 = b1 + w, *A2 = W2 + w * w, *b2 = A2 + 3 * w, *w3 = b2 + w,
                 *a3 = w3 + w;
    float *sS = buf, *sD0 = buf + w, *sD1 = buf + 2 * w, *sD2 = buf + 3 * w, *sU = buf + 4 * w;
    float e1[2], W1r[2][3];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int j = lane + 32 * t;
        e1[t] = 0.0f;
        W1r[t][0] = W1r[t][1] = W1r[t][2] = 0.0f;
        if (j < w) {
            float a0 = __ldg(W1 + 3 * j), a1 = __ldg(W1 + 3 * j + 1), a2 = __ldg(W1 + 3 * j + 2);
            float h = __ldg(b1 + j) + a0 * x[0] + a1 * x[1] + a2 * x[2];
            float sg, spv;
            sp_sig(h, spv, sg);
            sS[j] = spv;
            sD0[j] = sg * a0;
            sD1[j] = sg * a1;
            sD2[j] = sg * a2;
            e1[t] = sg * (1.0f - sg);
            W1r[t][0] = a0; W1r[t][1] = a1; W1r[t][2] = a2;
        }
    }
    __syncwarp();
    float acc[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) acc[c] = 0.0f;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int k = lane + 32 * t;
        if (k < w) {
            float h = __ldg(b2 + k), g0 = __ldg(A2 + 3 * k), g1 = __ldg(A2 + 3 * k + 1), g2 = __ldg(A2 + 3 * k + 2);
            h += g0 * x[0] + g1 * x[1] + g2 * x[2];
            const float *col = net.W2Tf + k;     // W2[k][j] = W2T[j*w + k]
            for (int j = 0; j < w; ++j) {
                float wkj = __ldg(col + j * w);
                h += wkj * sS[j];
                g0 += wkj * sD0[j];
                g1 += wkj * sD1[j];
                g2 += wkj * sD2[j];
            }
            float sg, spv;
            sp_sig(h, spv, sg);
            const float wk = __ldg(w3 + k);
            float e2 = wk * sg * (1.0f - sg);
            acc[0] += wk * spv;
            acc[1] += wk * sg * g0;
            acc[2] += wk * sg * g1;
            acc[3] += wk * sg * g2;
            acc[4] += e2 * g0 * g0;
            acc[5] += e2 * g0 * g1;
            acc[6] += e2 * g0 * g2;
            acc[7] += e2 * g1 * g1;
            acc[8] += e2 * g1 * g2;
            acc[9] += e2 * g2 * g2;
            sU[k] = wk * sg;
        }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int j = lane + 32 * t;
        if (j < w) {
            float v = 0.0f;
            const float *row = W2 + j;          // W2[k][j] at k*w + j
            for (int k = 0; k < w; ++k) v += __ldg(row + k * w) * sU[k];
            float c = v * e1[t];
            acc[4] += c * W1r[t][0] * W1r[t][0];
            acc[5] += c * W1r[t][0] * W1r[t][1];
            acc[6] += c * W1r[t][0] * W1r[t][2];
            acc[7] += c * W1r[t][1] * W1r[t][1];
            acc[8] += c * W1r[t][1] * W1r[t][2];
            acc[9] += c * W1r[t][2] * W1r[t][2];
        }
    }
#pragma unroll
    for (int c = 0; c < 10; ++c) out10[c] = warp_sum(acc[c]);
    out10[0] += __ldg(a3) * x[0] + __ldg(a3 + 1) * x[1] + __ldg(a3 + 2) * x[2];
    out10[1] += __ldg(a3);
    out10[2] += __ldg(a3 + 1);
    out10[3] += __ldg(a3 + 2);
    __syncwarp();
}

// Yield network value and slope in unit mode: G(q) = s (N_k(q) - N_k(0)),
// G' = s N_k'(q) (Eq. (Gq_NN)); width 0 is the identity G(q) = q.
__device__ void yield_unit(const DevNet &net, const NcF &nc, float q, float &G, float &Gp, float *buf, int lane)
{
    const int w = net.width;
    if (w == 0) {
        G = q;
        Gp = 1.0f;
        return;
    }
    const float *V1 = net.pf, *c1 = V1 + w, *V2 = c1 + w, *B2 = V2 + w * w, *c2 = B2 + w, *v3 = c2 + w,
                 *b3 = v3 + w;
    float *sS = buf, *sT = buf + w;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int j = lane + 32 * t;
        if (j < w) {
            float a = __ldg(V1 + j);
            float h = __ldg(c1 + j) + a * q;
            float spv, sg;
            sp_sig(h, spv, sg);
            sS[j] = spv;
            sT[j] = sg * a;
        }
    }
    __syncwarp();
    float n0 = 0.0f, n1 = 0.0f;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int k = lane + 32 * t;
        if (k < w) {
            float g = __ldg(B2 + k);
            float h = __ldg(c2 + k) + g * q;
            const float *col = net.W2Tf + k;
            for (int j = 0; j < w; ++j) {
                float wkj = __ldg(col + j * w);
                h += wkj * sS[j];
                g += wkj * sT[j];
            }
            float vk = __ldg(v3 + k);
            float spv, sg;
            sp_sig(h, spv, sg);
            n0 += vk * spv;
            n1 += vk * sg * g;
        }
    }
    n0 = warp_sum(n0);
    n1 = warp_sum(n1);
    float b = __ldg(b3);
    G = nc.y_s * (n0 + b * q - nc.y_N0);
    Gp = nc.y_s * (n1 + b);
    __syncwarp();
}

// r(kappa) = G(q(kappa)) - kappa and dr/dkappa (Eq. (potential_function)),
// q = psi_e + qcoef (phi - kappa) / f_d(kappa) (Eq. (ostwald_potential)).
__device__ __forceinline__ void r_slope(const DevNet &yld, const MatF &m, const NcF &nc, float pe, float phi,
                                        float kappa, float &r, float &dr, float &Gp, float *buf, int lane)
{
    bool dmg = kappa > m.kappa_d;
    float f = dmg ? expf(-m.eta_d * (kappa - m.kappa_d)) : 1.0f;
    float q = pe + m.qcoef * (phi - kappa) / f;
    float dq = m.qcoef * (-1.0f / f + (dmg ? (phi - kappa) * m.eta_d / f : 0.0f));
    float G;
    yield_unit(yld, nc, q, G, Gp, buf, lane);
    r = G - kappa;
    dr = Gp * dq - 1.0f;
}

// KW warps per CTA (a tuning choice: warps are independent, so it only sets the
// granularity of residency and of the persistent grid)
template <int DIM, int KW>
__global__ void __launch_bounds__(32 * KW) asm_fp32_kernel(AsmArgs A)
{
    using G_ = Geo<DIM>;
    constexpr int NEN = G_::NEN, NQ = G_::NQ, NDOF = G_::NDOF, ND = G_::ND, EPW = G_::EPW, EPR = G_::EPR;
    extern __shared__ float smem_f[];
    float *smem = smem_f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wmax = A.wmax;
    // per-warp scratch
    const int scratch = EPW * NEN * (DIM + NDOF) + 32 * Q_REC + 32 * 4 + 32 * 10 + 5 * wmax + 2 * NQ * NEN * V_REC;
    float *ws = smem + warp * scratch;
    float *sX = ws;                                  // [EPW][NEN][DIM]
    float *sD = sX + EPW * NEN * DIM;                // [EPW][NEN][NDOF]
    float *sRec = sD + EPW * NEN * NDOF;             // [32][Q_REC]
    float *sIn = sRec + 32 * Q_REC;                  // [32][4]: network input x (3), then kappa out
    float *sOut = sIn + 32 * 4;                      // [32][10]: N, grad, Hess / local-solve results
    float *sBuf = sOut + 32 * 10;                    // unit-mode buffers
    float *sVec = sBuf + 5 * wmax;                   // [EPR*NQ*NEN][V_REC]
    const MatF m = to_f(A.mat);

    const int64_t n_batches = (A.n_elems + EPW - 1) / EPW;
    for (int64_t batch = (int64_t)blockIdx.x * KW + warp; batch < n_batches;
         batch += (int64_t)gridDim.x * KW) {
        const int64_t e0 = batch * EPW;
        // ---- load element nodes (lane = (element, node)) ----
        for (int t = lane; t < EPW * NEN; t += 32) {
            int el = t / NEN, a = t % NEN;
            int64_t e = e0 + el;
            if (e < A.n_elems) {
                int32_t n = __ldg(A.conn + e * NEN + a);
#pragma unroll
                for (int J = 0; J < DIM; ++J) sX[t * DIM + J] = (float)__ldg(A.X + (int64_t)n * DIM + J);
#pragma unroll
                for (int c = 0; c < NDOF; ++c) sD[t * NDOF + c] = (float)__ldg(A.dofs + (int64_t)n * NDOF + c);
            } else {
#pragma unroll
                for (int J = 0; J < DIM; ++J) sX[t * DIM + J] = (a & 1) ? 1.0f : 0.0f;
#pragma unroll
                for (int c = 0; c < NDOF; ++c) sD[t * NDOF + c] = 0.0f;
            }
        }
        __syncwarp();

        // ================= qp mode: kinematics and invariants =================
        const int el = lane / NQ, q = lane % NQ;
        const int64_t e_me = e0 + el;
        const bool valid = e_me < A.n_elems;
        const NcF nc = ncf(A.netc[valid ? spec_of(A, e_me) : 0]);
        float *rec = sRec + lane * Q_REC;
        float F[3][3], H[3][3], phi = 0.0f, g[3] = {0.0f, 0.0f, 0.0f}, x[3], Jdet;
        {
            const float xi[3] = {(q & 1) ? kGauss : -kGauss, (q & 2) ? kGauss : -kGauss,
                                  (q & 4) ? kGauss : -kGauss};
            const float *Xe = sX + el * NEN * DIM;
            const float *De = sD + el * NEN * NDOF;
            float Jm[3][3] = {{0.0f}};
#pragma unroll
            for (int a = 0; a < NEN; ++a) {
                float Na, dN[3];
                ref_shape<DIM>(a, xi, Na, dN);
#pragma unroll
                for (int J = 0; J < DIM; ++J)
#pragma unroll
                    for (int k = 0; k < DIM; ++k) Jm[J][k] += Xe[a * DIM + J] * dN[k];
            }
            float Ji[3][3] = {{0.0f}}, det;
            if (DIM == 2) {
                det = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
                Ji[0][0] = Jm[1][1] / det; Ji[0][1] = -Jm[0][1] / det;
                Ji[1][0] = -Jm[1][0] / det; Ji[1][1] = Jm[0][0] / det;
            } else {
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
                        Ji[i][j] = Jm[i1][j1] * Jm[i2][j2] - Jm[i1][j2] * Jm[i2][j1];
                    }
                det = Jm[0][0] * Ji[0][0] + Jm[0][1] * Ji[1][0] + Jm[0][2] * Ji[2][0];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) Ji[i][j] /= det;
            }
            rec[Q_JW] = det;
#pragma unroll
            for (int k = 0; k < 9; ++k) rec[Q_JINV + k] = Ji[k / 3][k % 3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int J = 0; J < 3; ++J) H[i][J] = 0.0f;
#pragma unroll
            for (int a = 0; a < NEN; ++a) {
                float Na, dN[3], n[3] = {0.0f, 0.0f, 0.0f};
                ref_shape<DIM>(a, xi, Na, dN);
#pragma unroll
                for (int J = 0; J < DIM; ++J)
#pragma unroll
                    for (int k = 0; k < DIM; ++k) n[J] += dN[k] * Ji[k][J];
                const float pa = De[a * NDOF + DIM];
                phi += Na * pa;
#pragma unroll
                for (int J = 0; J < DIM; ++J) {
                    g[J] += pa * n[J];
#pragma unroll
                    for (int i = 0; i < DIM; ++i) H[i][J] += De[a * NDOF + i] * n[J];
                }
            }
            // C - I = H + H^T + H^T H ; invariants without cancellation
            float Am[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float s = H[i][j] + H[j][i];
#pragma unroll
                    for (int k = 0; k < 3; ++k) s += H[k][i] * H[k][j];
                    Am[i][j] = s;
                }
            float tA = Am[0][0] + Am[1][1] + Am[2][2], AA = 0.0f, tH = H[0][0] + H[1][1] + H[2][2], HH = 0.0f;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    AA += Am[i][j] * Am[j][i];
                    HH += H[i][j] * H[j][i];
                }
            float detH = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
                          H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                          H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
            x[0] = tA;
            x[1] = 2.0f * tA + 0.5f * (tA * tA - AA);
            x[2] = tH + 0.5f * (tH * tH - HH) + detH;
            Jdet = 1.0f + x[2];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? 1.0f : 0.0f);
        }
        // network input (raw or isochoric map)
        float Tm[3][3], T2[3][6];   // dy/dx and d2y/dx2 of the iso map (raw: identity)
        {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
                for (int j = 0; j < 3; ++j) Tm[i][j] = (i == j) ? 1.0f : 0.0f;
#pragma unroll
                for (int j = 0; j < 6; ++j) T2[i][j] = 0.0f;
            }
            float y[3] = {x[0], x[1], x[2]};
            if (m.energy == GD_ENERGY_ICNN_ISO) {
                // I1G = J^-2/3 I1, I2G = I2^3 / (9 J^4) (Eq. (dd_0)); derivatives wrt (I1-3, I2-3, J-1)
                float L = log1pf(x[2]), E = expf(-2.0f / 3.0f * L), I1 = 3.0f + x[0], I2 = 3.0f + x[1], J = Jdet;
                y[0] = 3.0f * expm1f(-2.0f / 3.0f * L) + x[0] * E;
                y[1] = 3.0f * expm1f(3.0f * log1pf(x[1] / 3.0f) - 4.0f * L);
                float J4 = J * J * J * J;
                Tm[0][0] = E;
                Tm[0][2] = -2.0f / 3.0f * I1 * E / J;
                Tm[1][1] = I2 * I2 / (3.0f * J4);
                Tm[1][2] = -4.0f * I2 * I2 * I2 / (9.0f * J4 * J);
                T2[0][2] = -2.0f / 3.0f * E / J;                       // d2 y1 / dx1 dx3
                T2[0][5] = 10.0f / 9.0f * I1 * E / (J * J);            // d2 y1 / dx3^2
                T2[1][3] = 2.0f * I2 / (3.0f * J4);                    // d2 y2 / dx2^2
                T2[1][4] = -4.0f * I2 * I2 / (3.0f * J4 * J);          // d2 y2 / dx2 dx3
                T2[1][5] = 20.0f * I2 * I2 * I2 / (9.0f * J4 * J * J); // d2 y2 / dx3^2
            }
            sIn[lane * 4 + 0] = y[0];
            sIn[lane * 4 + 1] = y[1];
            sIn[lane * 4 + 2] = y[2];
        }
        __syncwarp();

        // ================= unit mode: energy network =================
        if (m.energy != GD_ENERGY_NEO_HOOKE) {
            for (int p = 0; p < 32; ++p) {
                if (e0 + p / NQ >= A.n_elems) break;
                float y[3] = {sIn[p * 4], sIn[p * 4 + 1], sIn[p * 4 + 2]}, out[10];
                psi_net_unit(psi_of(A, spec_of(A, e0 + p / NQ)), y, out, sBuf, lane);
                if (lane == 0)
#pragma unroll
                    for (int c = 0; c < 10; ++c) sOut[p * 10 + c] = out[c];
            }
        }
        __syncwarp();

        // ================= qp mode: energy derivatives wrt (I1-3, I2-3, J-1) =================
        float ps[3], ph[6], pe;
        {
            const float J = Jdet, x3 = x[2];
            if (m.energy == GD_ENERGY_NEO_HOOKE) {
                float L = log1pf(x3);
                pe = 0.5f * m.mu_e * x[0] - m.mu_e * L + 0.5f * m.lambda_e * L * L;
                ps[0] = 0.5f * m.mu_e;
                ps[1] = 0.0f;
                ps[2] = (-m.mu_e + m.lambda_e * L) / J;
#pragma unroll
                for (int c = 0; c < 6; ++c) ph[c] = 0.0f;
                ph[5] = (m.lambda_e + m.mu_e - m.lambda_e * L) / (J * J);
            } else {
                const float *o = sOut + lane * 10;
                float gy[3] = {o[1], o[2], o[3]};
                float hy[6] = {o[4], o[5], o[6], o[7], o[8], o[9]};
                // chain through the input map: dN/dx = T^T dN/dy, d2N/dx2 = T^T H T + sum_m dN/dy_m d2y_m/dx2
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float s = 0.0f;
#pragma unroll
                    for (int mm = 0; mm < 3; ++mm) s += Tm[mm][i] * gy[mm];
                    ps[i] = s;
                }
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = i; j < 3; ++j) {
                        float s = 0.0f;
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int b = 0; b < 3; ++b) s += Tm[a][i] * hy[sym6(a, b)] * Tm[b][j];
#pragma unroll
                        for (int mm = 0; mm < 3; ++mm) s += gy[mm] * T2[mm][sym6(i, j)];
                        ph[sym6(i, j)] = s;
                    }
                // psi_e = mu_e (N - N0 - n x3) + lambda_e t^2, t = (J-1)^2 / J
                float t = x3 * x3 / J, dt = 1.0f - 1.0f / (J * J), d2t = 2.0f / (J * J * J);
                pe = m.mu_e * (o[0] - nc.psi_N0 - nc.psi_n * x3) + m.lambda_e * t * t;
#pragma unroll
                for (int i = 0; i < 3; ++i) ps[i] *= m.mu_e;
#pragma unroll
                for (int c = 0; c < 6; ++c) ph[c] *= m.mu_e;
                ps[2] += -m.mu_e * nc.psi_n + m.lambda_e * 2.0f * t * dt;
                ph[5] += m.lambda_e * 2.0f * (dt * dt + t * d2t);
            }
            sIn[lane * 4 + 0] = pe;
            sIn[lane * 4 + 1] = phi;
            sIn[lane * 4 + 2] = valid ? (float)__ldg(A.kappa_n + e_me * NQ + q) : 0.0f;
        }
        __syncwarp();

        // ================= unit mode: local damage update per point =================
        if (A.kappa_fixed) {
            // frozen history (staggered scheme): the point keeps the given kappa
            float *o = sOut + lane * 10;
            o[0] = valid ? (float)__ldg(A.kappa_fixed + e_me * NQ + q) : 0.0f;
            o[1] = 0.0f;
            o[2] = 0.0f;
            o[3] = -1.0f;
            o[4] = 0.0f;
            o[5] = 0.0f;
        } else
        for (int p = 0; p < 32; ++p) {
            if (e0 + p / NQ >= A.n_elems) break;
            const float ppe = sIn[p * 4], pphi = sIn[p * 4 + 1], kn = sIn[p * 4 + 2];
            const int sp = spec_of(A, e0 + p / NQ);
            const DevNet &yn = yld_of(A, sp);
            const NcF ncp = ncf(A.netc[sp]);
            const double kn_d = __ldg(A.kappa_n + e0 * NQ + p);
            float r, dr, Gp;
            int n_eval = 1;
            r_slope(yn, m, ncp, ppe, pphi, kn, r, dr, Gp, sBuf, lane);
            // loading/unloading decided in FP64: Phi_d(kappa_n) = G(q(kappa_n)) - kappa_n > 0
            const double phi_trial = (double)(r + kn) - kn_d;
            float kappa = kn, fail = 0.0f, loading = 0.0f;
            if (phi_trial > 0.0) {
                loading = 1.0f;
                // Newton iteration on r(kappa) = G(q(kappa)) - kappa from kappa_n (r > 0 there)
                // or from the warm-start guess, bracketing lazily: lo keeps the last point with
                // r > 0; once a point with r <= 0 is met it becomes hi and the iteration turns
                // into the safeguarded Newton-bisection on [lo, hi].  Before that, a step that
                // is not a forward Newton step (slope >= 0) probes ahead geometrically.
                const float kg = A.kappa_guess ? (float)__ldg(A.kappa_guess + e0 * NQ + p) : kn;
                if (kg > kn && isfinite(kg)) {
                    kappa = kg;
                    r_slope(yn, m, ncp, ppe, pphi, kappa, r, dr, Gp, sBuf, lane);
                    ++n_eval;
                }
                float lo = kn, hi = kn;
                bool have_hi = false;
                if (r > 0.0f) lo = kappa;
                else {
                    hi = kappa;
                    have_hi = true;
                }
                float dx_prev = have_hi ? hi - lo : 1.0e30f, dx = dx_prev;
                int it;
                for (it = 0; it < m.local_max; ++it) {
                    const float scale = fabsf(kappa) > 1.0f ? fabsf(kappa) : 1.0f;
                    if (fabsf(r) <= 2e-6f * scale || (have_hi && (hi - lo) <= 4.0f * kEpsF * scale)) break;
                    const float newton = kappa - r / dr;
                    bool take;
                    if (have_hi) {
                        take = (newton > lo) && (newton < hi) && (fabsf(2.0f * r) <= fabsf(dx_prev * dr));
                    } else {
                        // forward Newton step, at most a few times the distance covered so far
                        const float cap = 4.0f * ((float)(r > 1e-12f ? r : 1e-12f) + (kappa - kn));
                        take = dr < 0.0f && newton > lo && (newton - kappa) <= cap;
                    }
                    dx_prev = dx;
                    if (take) {
                        dx = kappa - newton;
                        kappa = newton;
                    } else if (have_hi) {
                        dx = 0.5f * (hi - lo);
                        kappa = lo + dx;
                    } else {
                        const float step = 2.0f * ((kappa - kn) > (r > 1e-12f ? r : 1e-12f) ? (kappa - kn) : (r > 1e-12f ? r : 1e-12f));
                        dx = step;
                        kappa = lo + step;
                    }
                    r_slope(yn, m, ncp, ppe, pphi, kappa, r, dr, Gp, sBuf, lane);
                    ++n_eval;
                    if (r > 0.0f) {
                        lo = kappa;
                    } else {
                        hi = kappa;
                        have_hi = true;
                    }
                }
                if (it >= m.local_max) fail = 1.0f;
            }
            if (lane == 0) {
                float *o = sOut + p * 10;
                if (e0 + p / NQ < A.n_elems) atomicAdd(A.counters + 2, n_eval);
                o[0] = kappa;
                o[5] = loading > 0.5f ? 0.0f : 1.0f;   // elastic: keep the FP64 history exactly
                o[1] = loading;
                o[2] = Gp;
                o[3] = dr;
                o[4] = fail;
            }
        }
        __syncwarp();

        // ================= qp mode: stress and records =================
        {
            const float *o = sOut + lane * 10;
            const float kappa = o[0];
            const bool loading = o[1] > 0.5f;
            if (valid) {
                if (A.kappa_new) {
                    const double kn_d = __ldg(A.kappa_n + e_me * NQ + q);
                    A.kappa_new[e_me * NQ + q] = A.kappa_fixed ? __ldg(A.kappa_fixed + e_me * NQ + q)
                                                 : o[5] > 0.5f ? kn_d : fmax(kn_d, (double)kappa);
                }
                if (A.loading) A.loading[e_me * NQ + q] = loading ? 1 : 0;
                if (o[4] > 0.5f) atomicAdd(A.counters, 1);
                if (loading) atomicAdd(A.counters + 1, 1);
            }
            const bool dmg = kappa > m.kappa_d;
            const float fd = dmg ? expf(-m.eta_d * (kappa - m.kappa_d)) : 1.0f;
            const float fdp = dmg ? -m.eta_d * fd : 0.0f;
            const float ck = loading ? -o[2] / o[3] : 0.0f;          // G' / (1 - G' dq/dkappa)
            const float dkdphi = ck * m.qcoef / fd;                  // dq/dphi = qcoef / f_d
            const float J = Jdet;
            // F^-1 = cof(F)^T / J
            float Fi[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
                    Fi[i][j] = (F[i1][j1] * F[i2][j2] - F[i1][j2] * F[i2][j1]) / J;
                }
            float C[3][3], b[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float s = 0.0f, t = 0.0f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        s += F[k][i] * F[k][j];
                        t += F[i][k] * F[j][k];
                    }
                    C[i][j] = s;
                    b[i][j] = t;
                }
            const float I1 = 3.0f + x[0];
            // h = F^-T g, mvec = F^-1 h = C^-1 g
            float hv[3], mv[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) hv[i] = Fi[0][i] * g[0] + Fi[1][i] * g[1] + Fi[2][i] * g[2];
#pragma unroll
            for (int i = 0; i < 3; ++i) mv[i] = Fi[i][0] * hv[0] + Fi[i][1] * hv[1] + Fi[i][2] * hv[2];
            // P = f_d [2 psi_1 F + 2 psi_2 (I1 F - F C) + psi_3 J F^-T] - c_d h (x) m
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int J2 = 0; J2 < 3; ++J2) {
                    float FC = F[i][0] * C[0][J2] + F[i][1] * C[1][J2] + F[i][2] * C[2][J2];
                    float Ph = 2.0f * ps[0] * F[i][J2] + 2.0f * ps[1] * (I1 * F[i][J2] - FC) + ps[2] * J * Fi[J2][i];
                    rec[Q_P + i * 3 + J2] = fd * Ph - m.c_d * hv[i] * mv[J2];
                    rec[Q_F + i * 3 + J2] = F[i][J2];
                    rec[Q_B + i * 3 + J2] = b[i][J2];
                    rec[Q_FINV + i * 3 + J2] = Fi[i][J2];
                }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                rec[Q_M + i] = mv[i];
                rec[Q_H + i] = hv[i];
            }
            rec[Q_I1] = I1;
#pragma unroll
            for (int c = 0; c < 6; ++c) rec[Q_HS + c] = fd * ph[c];
            rec[Q_G1] = fd * ps[0];
            rec[Q_G2] = fd * ps[1];
            rec[Q_G3J] = fd * ps[2] * J;
            rec[Q_PS1] = ps[0];
            rec[Q_PS2] = ps[1];
            rec[Q_PS3J] = ps[2] * J;
            rec[Q_CK] = fdp * ck;
            rec[Q_BCK] = m.beta_d * ck;
            rec[Q_FDK] = fdp * dkdphi;
            rec[Q_PP] = m.beta_d * (1.0f - dkdphi);
            rec[Q_PEN] = m.beta_d * (phi - kappa);
            rec[Q_J] = J;
            if (!valid) rec[Q_JW] = 0.0f;
        }
        __syncwarp();

        // ================= row mode: element residual and tangent =================
        for (int pass = 0; pass < EPW / EPR; ++pass) {
            // per (point, node) vectors of the EPR elements of this pass
            for (int t = lane; t < EPR * NQ * NEN; t += 32) {
                const int ee = t / (NQ * NEN), qq = (t / NEN) % NQ, a = t % NEN;
                const float *R0 = sRec + ((pass * EPR + ee) * NQ + qq) * Q_REC;
                float *V = sVec + t * V_REC;
                const float xi[3] = {(qq & 1) ? kGauss : -kGauss, (qq & 2) ? kGauss : -kGauss,
                                      (qq & 4) ? kGauss : -kGauss};
                float Na, dN[3], n[3] = {0.0f, 0.0f, 0.0f};
                ref_shape<DIM>(a, xi, Na, dN);
#pragma unroll
                for (int J = 0; J < DIM; ++J)
#pragma unroll
                    for (int k = 0; k < DIM; ++k) n[J] += dN[k] * R0[Q_JINV + k * 3 + J];
                float f[3], bf[3], nt[3], G2[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    f[i] = R0[Q_F + i * 3] * n[0] + R0[Q_F + i * 3 + 1] * n[1] + R0[Q_F + i * 3 + 2] * n[2];
                    nt[i] = R0[Q_FINV + i] * n[0] + R0[Q_FINV + 3 + i] * n[1] + R0[Q_FINV + 6 + i] * n[2];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    bf[i] = R0[Q_B + i * 3] * f[0] + R0[Q_B + i * 3 + 1] * f[1] + R0[Q_B + i * 3 + 2] * f[2];
#pragma unroll
                for (int i = 0; i < 3; ++i) G2[i] = 2.0f * (R0[Q_I1] * f[i] - bf[i]);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    V[V_N + i] = n[i];
                    V[V_F + i] = f[i];
                    V[V_G2 + i] = G2[i];
                    V[V_NT + i] = nt[i];
                    V[V_PN + i] = 2.0f * R0[Q_PS1] * f[i] + R0[Q_PS2] * G2[i] + R0[Q_PS3J] * nt[i];
                }
                V[V_NN] = Na;
                V[V_MN] = R0[Q_M] * n[0] + R0[Q_M + 1] * n[1] + R0[Q_M + 2] * n[2];
            }
            __syncwarp();
            const int ee = lane / ND, row = lane % ND;
            const int a = row / NDOF, i = row % NDOF;
            const int el_local = pass * EPR + ee;
            const int64_t e = e0 + el_local;
            const bool active = (lane < EPR * ND) && (e < A.n_elems);
            float Kr[ND];
#pragma unroll
            for (int c = 0; c < ND; ++c) Kr[c] = 0.0f;
            float Rr = 0.0f;
            const float cd = m.c_d;
            if (active) {
                for (int qq = 0; qq < NQ; ++qq) {
                    const float *R0 = sRec + (el_local * NQ + qq) * Q_REC;
                    const float *Vq = sVec + (ee * NQ + qq) * NEN * V_REC;
                    const float *Va = Vq + a * V_REC;
                    const float Jw = R0[Q_JW];
                    if (i < DIM) {
                        // r_u,a = P n_a J w (Sec. 3.1f)
                        Rr += Jw * (R0[Q_P + i * 3] * Va[V_N] + R0[Q_P + i * 3 + 1] * Va[V_N + 1] +
                                    R0[Q_P + i * 3 + 2] * Va[V_N + 2]);
                        // d2 psi_e/dF2 contracted with grad N_a, grad N_b:
                        //   sum_mn psi_mn G^m_a G^n_b + psi_1 D2(I1) + psi_2 D2(I2) + psi_3 D2(J),
                        // G^1 = 2 F n, G^2 = 2 (I1 F n - F F^T F n), G^3 = J F^-T n,
                        // D2(I1)_ik = 2 (n_a.n_b) d_ik,
                        // D2(I2)_ik = 2 [2 f_a,i f_b,k - f_b,i f_a,k + (I1 n_a.n_b - f_a.f_b) d_ik - (n_a.n_b) b_ik],
                        // D2(J)_ik  = J (nt_a,i nt_b,k - nt_a,k nt_b,i),   f = F n, nt = F^-T n.
                        const float Jd = R0[Q_J];
                        const float Gai[3] = {2.0f * Va[V_F + i], Va[V_G2 + i], Jd * Va[V_NT + i]};
                        const float *HS = R0 + Q_HS;
                        float tn[3];
#pragma unroll
                        for (int nI = 0; nI < 3; ++nI)
                            tn[nI] = HS[sym6(0, nI)] * Gai[0] + HS[sym6(1, nI)] * Gai[1] + HS[sym6(2, nI)] * Gai[2];
                        const float g1 = R0[Q_G1], g2 = R0[Q_G2], g3J = R0[Q_G3J], I1 = R0[Q_I1];
                        const float ck = R0[Q_CK], fdk = R0[Q_FDK];
                        const float hi_ = R0[Q_H + i], mna = Va[V_MN], Pna = Va[V_PN + i];
                        const float fai = Va[V_F + i], ntai = Va[V_NT + i];
#pragma unroll
                        for (int bN = 0; bN < NEN; ++bN) {
                            const float *Vb = Vq + bN * V_REC;
                            const float nn = Va[V_N] * Vb[V_N] + Va[V_N + 1] * Vb[V_N + 1] + Va[V_N + 2] * Vb[V_N + 2];
                            const float ff = Va[V_F] * Vb[V_F] + Va[V_F + 1] * Vb[V_F + 1] + Va[V_F + 2] * Vb[V_F + 2];
                            const float tt =
                                Va[V_NT] * Vb[V_NT] + Va[V_NT + 1] * Vb[V_NT + 1] + Va[V_NT + 2] * Vb[V_NT + 2];
                            const float mnb = Vb[V_MN], ntbi = Vb[V_NT + i], fbi = Vb[V_F + i];
#pragma unroll
                            for (int k = 0; k < DIM; ++k) {
                                const float fbk = Vb[V_F + k], ntbk = Vb[V_NT + k];
                                float v = tn[0] * 2.0f * fbk + tn[1] * Vb[V_G2 + k] + tn[2] * Jd * ntbk;
                                if (k == i) v += 2.0f * g1 * nn + 2.0f * g2 * (I1 * nn - ff);
                                v += 2.0f * g2 * (2.0f * fai * fbk - fbi * Va[V_F + k] - nn * R0[Q_B + i * 3 + k]);
                                v += g3J * (ntai * ntbk - Va[V_NT + k] * ntbi);
                                v += ck * Pna * Vb[V_PN + k];
                                v += cd * (mna * ntbi * R0[Q_H + k] + tt * hi_ * R0[Q_H + k] + mnb * hi_ * Va[V_NT + k]);
                                Kr[bN * NDOF + k] += Jw * v;
                            }
                            Kr[bN * NDOF + DIM] += Jw * (-cd * (mna * ntbi + hi_ * tt) + fdk * Pna * Vb[V_NN]);
                        }
                    } else {
                        // R_phi,a = (Y . grad N_a - Y N_a) J w, Y vec = c_d C^-1 grad phi, -Y = beta_d (phi - kappa)
                        const float Na = Va[V_NN];
                        Rr += Jw * (cd * Va[V_MN] + R0[Q_PEN] * Na);
                        const float bck = R0[Q_BCK], pp = R0[Q_PP];
#pragma unroll
                        for (int bN = 0; bN < NEN; ++bN) {
                            const float *Vb = Vq + bN * V_REC;
                            const float tt =
                                Va[V_NT] * Vb[V_NT] + Va[V_NT + 1] * Vb[V_NT + 1] + Va[V_NT + 2] * Vb[V_NT + 2];
                            const float mnb = Vb[V_MN];
#pragma unroll
                            for (int k = 0; k < DIM; ++k)
                                Kr[bN * NDOF + k] += Jw * (-cd * (R0[Q_H + k] * tt + mnb * Va[V_NT + k]) -
                                                           bck * Na * Vb[V_PN + k]);
                            Kr[bN * NDOF + DIM] += Jw * (cd * tt + pp * Na * Vb[V_NN]);
                        }
                    }
                }
                // scatter through the slot map
                const int32_t na = __ldg(A.conn + e * NEN + a);
                const int64_t rdof = (int64_t)na * NDOF + i;
                if (A.R) atomicAdd(A.R + rdof, (double)Rr);
                if (A.tangent) {
                    const int32_t rb = __ldg(A.rowptr + (int64_t)na * NDOF);
                    const int32_t rowlen = __ldg(A.rowptr + (int64_t)na * NDOF + 1) - rb;
                    const int32_t *sl = A.slot + (e * NEN + a) * NEN;
#pragma unroll
                    for (int bN = 0; bN < NEN; ++bN) {
                        const int64_t pos = (int64_t)__ldg(sl + bN) + (int64_t)i * rowlen;
#pragma unroll
                        for (int k = 0; k < NDOF; ++k) {
                            if (A.vals32) atomicAdd(A.vals32 + pos + k, Kr[bN * NDOF + k]);
                            else atomicAdd(A.vals + pos + k, (double)Kr[bN * NDOF + k]);
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
}

template <int DIM>
size_t smem_bytes(int wmax)
{
    using G_ = Geo<DIM>;
    size_t scratch = G_::EPW * G_::NEN * (DIM + G_::NDOF) + 32 * Q_REC + 32 * 4 + 32 * 10 + 5 * wmax +
                     2 * G_::NQ * G_::NEN * V_REC;
    return scratch * sizeof(float);          // per warp
}

template <int DIM, int KW>
cudaError_t launch_kw(const AsmArgs &a, int num_sms, const AsmTune &t, cudaStream_t s)
{
    size_t sm = smem_bytes<DIM>(a.wmax) * KW;
    int dev = 0, optin = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e0 != cudaSuccess) return e0;
    if (sm > (size_t)optin) return cudaErrorInvalidConfiguration;   // this CTA width does not fit
    cudaError_t err = cudaFuncSetAttribute(asm_fp32_kernel<DIM, KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, asm_fp32_kernel<DIM, KW>, 32 * KW, sm);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    if (t.cta_per_sm > 0 && t.cta_per_sm < per_sm) per_sm = t.cta_per_sm;
    using G_ = Geo<DIM>;
    int64_t batches = (a.n_elems + G_::EPW - 1) / G_::EPW;
    int64_t need = (batches + KW - 1) / KW;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > need) grid = need;
    if (t.grid_max > 0 && grid > t.grid_max) grid = t.grid_max;
    if (grid < 1) grid = 1;
    asm_fp32_kernel<DIM, KW><<<(unsigned)grid, 32 * KW, sm, s>>>(a);
    return cudaGetLastError();
}

// the requested CTA width, or the widest narrower one whose shared memory fits (a
// width tuned for one kernel may not fit another: the FP64 kernel needs twice the
// FP32 kernel's scratch)
template <int DIM>
cudaError_t launch_dim(const AsmArgs &a, int num_sms, const AsmTune &t, cudaStream_t s)
{
    if (t.exact) {
        switch (t.warps) {
        case 1: return launch_kw<DIM, 1>(a, num_sms, t, s);
        case 2: return launch_kw<DIM, 2>(a, num_sms, t, s);
        case 8: return launch_kw<DIM, 8>(a, num_sms, t, s);
        default: return launch_kw<DIM, 4>(a, num_sms, t, s);
        }
    }
    cudaError_t e = cudaErrorInvalidConfiguration;
    if (t.warps >= 8) e = launch_kw<DIM, 8>(a, num_sms, t, s);
    if (e == cudaErrorInvalidConfiguration && t.warps >= 4) e = launch_kw<DIM, 4>(a, num_sms, t, s);
    if (e == cudaErrorInvalidConfiguration && t.warps >= 2) e = launch_kw<DIM, 2>(a, num_sms, t, s);
    if (e == cudaErrorInvalidConfiguration) e = launch_kw<DIM, 1>(a, num_sms, t, s);
    return e;
}

}  // namespace

cudaError_t launch_assemble_fp32(int dim, const AsmArgs &a, int num_sms, cudaStream_t s, const AsmTune &t)
{
    if (a.n_elems <= 0) return cudaSuccess;
    return dim == 2 ? launch_dim<2>(a, num_sms, t, s) : launch_dim<3>(a, num_sms, t, s);
}

}  // namespace gd
