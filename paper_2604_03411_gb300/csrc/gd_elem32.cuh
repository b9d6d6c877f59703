// gd_elem32.cuh -- FP32 element math shared by the two mixed-precision element
// kernels (CUDA-core networks in gd_asm_mixed.cu, tensor-core networks in
// gd_asm_tc.cu): per-point kinematics and invariants, the network input map, the
// energy derivatives with respect to (I1-3, I2-3, J-1), stress and the per-point
// records of the tangent (qp mode, lane = quadrature point), and the element
// residual and tangent rows scattered through the slot map (row mode, lane =
// element row).
//
// Paper passages: Sec. 3.1f (F, phi_q, grad phi_q, element residual, Table
// kernel_inputs), Sec. 2.1f (P, Y vector, Y), Sec. 3.2f (monolithic tangent),
// Sec. 4.1f (degradation, gradient and penalty energies, Eq. (ostwald_potential)),
// Sec. 4.2f Eqs. (dd_0), (dd_1).
#pragma once

#include <cuda_runtime.h>

#include "gd_internal.cuh"

namespace gd {
namespace e32 {

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
    Q_PENM = 71,     // beta_d (|phi| + |kappa|): the magnitude that the penalty's FP32 rounding scales with
    Q_REC = 72
};
// ---- per (point, node) vector record ----
enum : int { V_N = 0, V_NN = 3, V_F = 4, V_G2 = 7, V_NT = 10, V_PN = 13, V_MN = 16, V_REC = 17 };

__device__ __forceinline__ int sym6(int i, int j)
{
    // (0,0)0 (0,1)1 (0,2)2 (1,1)3 (1,2)4 (2,2)5
    int a = i < j ? i : j, b = i < j ? j : i;
    return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

// Yield network value and slope in unit mode: G(q) = s (N_k(q) - N_k(0)),
// G' = s N_k'(q) (Eq. (Gq_NN)); width 0 is the identity G(q) = q.
static __device__ void yield_unit(const DevNet &net, const NcF &nc, float q, float &G, float &Gp, float *buf, int lane)
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

// Local damage update in unit mode (Eq. (dd_7_no_nn)): the smallest root above
// kappa_n of r(kappa) = G(q(kappa)) - kappa, entered with kappa = kappa_n and (r, dr,
// Gp) evaluated there (r > 0: the point is loading) and a warm start kg (used when
// above kappa_n).  On return kappa is the root to |r| <= 2e-6 max(1, kappa) (or a
// bracket of 4 FP32 ulps), r, dr and Gp are evaluated there, n_eval counts the
// evaluations; false when local_max iterations did not reach it.  Every lane takes
// the same path (r and dr are warp-reduced).
// step_test: also stop when the next Newton correction |r / r'| is within the tolerance
// and either the root is bracketed within 1e-2 relative or the iteration is converging
// from one side (the last step a Newton step at least twice as long).  For a starting
// point that FP64 refines: near full damage r' grows like 1 / f_d and |r| cannot get
// below its FP32 rounding; far past the root, where f_d underflows, r' is huge, so a
// wide bracket never qualifies.
__device__ __forceinline__ bool bracketed_newton(const DevNet &yn, const MatF &m, const NcF &ncp, float pe, float phi,
                                                 float kn, float kg, float &kappa, float &r, float &dr, float &Gp,
                                                 int &n_eval, float *buf, int lane, bool step_test = false)
{
    // Newton iteration on r(kappa) = G(q(kappa)) - kappa from kappa_n (r > 0 there)
    // or from the warm-start guess, bracketing lazily: lo keeps the last point with
    // r > 0; once a point with r <= 0 is met it becomes hi and the iteration turns
    // into the safeguarded Newton-bisection on [lo, hi].  Before that, a step that
    // is not a forward Newton step (slope >= 0) probes ahead geometrically.
    if (kg > kn && isfinite(kg)) {
        kappa = kg;
        r_slope(yn, m, ncp, pe, phi, kappa, r, dr, Gp, buf, lane);
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
    bool took_newton = false;
    int it;
    for (it = 0; it < m.local_max; ++it) {
        const float scale = fabsf(kappa) > 1.0f ? fabsf(kappa) : 1.0f;
        if (fabsf(r) <= 2e-6f * scale || (have_hi && (hi - lo) <= 4.0f * kEpsF * scale)) break;
        if (step_test && fabsf(r) <= 2e-6f * scale * fabsf(dr) &&
            (have_hi ? (hi - lo) <= 1e-2f * scale : (took_newton && fabsf(2.0f * r) <= fabsf(dx * dr))))
            break;
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
        took_newton = take;
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
        r_slope(yn, m, ncp, pe, phi, kappa, r, dr, Gp, buf, lane);
        ++n_eval;
        if (r > 0.0f) {
            lo = kappa;
        } else {
            hi = kappa;
            have_hi = true;
        }
    }
    return it < m.local_max;
}

// element nodes of a warp's batch into shared memory (lane = (element, node)).
// Coordinates and displacements are taken relative to the element's first node,
// the differences formed in FP64: the FP32 kinematics use only their differences
// (sum_a grad N_a = 0), and on a fine mesh far from the origin the absolute FP32
// values would lose the element-size digits.  phi stays absolute (its value enters
// the penalty).  Elements past the end get placeholder nodes and zero dofs.
template <int DIM, class Args>
__device__ __forceinline__ void load_nodes(const Args &A, int64_t e0, float *sX, float *sD, int lane)
{
    using G_ = Geo<DIM>;
    constexpr int NEN = G_::NEN, NDOF = G_::NDOF, EPW = G_::EPW;
    for (int t = lane; t < EPW * NEN; t += 32) {
        int el = t / NEN, a = t % NEN;
        int64_t e = e0 + el;
        if (e < A.n_elems) {
            int32_t n = __ldg(A.conn + e * NEN + a), n0 = __ldg(A.conn + e * NEN);
#pragma unroll
            for (int J = 0; J < DIM; ++J)
                sX[t * DIM + J] = (float)(__ldg(A.X + (int64_t)n * DIM + J) - __ldg(A.X + (int64_t)n0 * DIM + J));
#pragma unroll
            for (int c = 0; c < DIM; ++c)
                sD[t * NDOF + c] =
                    (float)(__ldg(A.dofs + (int64_t)n * NDOF + c) - __ldg(A.dofs + (int64_t)n0 * NDOF + c));
            sD[t * NDOF + DIM] = (float)__ldg(A.dofs + (int64_t)n * NDOF + DIM);
        } else {
#pragma unroll
            for (int J = 0; J < DIM; ++J) sX[t * DIM + J] = (a & 1) ? 1.0f : 0.0f;
#pragma unroll
            for (int c = 0; c < NDOF; ++c) sD[t * NDOF + c] = 0.0f;
        }
    }
}

// qp mode: shape gradients, Jacobian (rec[Q_JW], rec[Q_JINV]), H = grad u, F, phi_q,
// grad phi_q, and x = (I1-3, I2-3, J-1) from C - I = H + H^T + H^T H without
// cancellation (Sec. 3.1f; Eq. (dd_0) inputs)
template <int DIM>
__device__ __forceinline__ void qp_kinematics(const float *sX, const float *sD, int el, int q, float *rec,
                                              float (&F)[3][3], float (&H)[3][3], float &phi, float (&g)[3],
                                              float (&x)[3], float &Jdet)
{
    using G_ = Geo<DIM>;
    constexpr int NEN = G_::NEN, NDOF = G_::NDOF;
    phi = 0.0f;
    g[0] = g[1] = g[2] = 0.0f;
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

// network input y (raw: y = x; isochoric: (I1G-3, I2G-3, J-1), Eq. (dd_0)) with
// Tm = dy/dx and T2 = d2y/dx2 (symmetric pairs in sym6 order)
__device__ __forceinline__ void input_map(const MatF &m, const float (&x)[3], float Jdet, float (&Tm)[3][3],
                                          float (&T2)[3][6], float (&yo)[3])
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
    yo[0] = y[0];
    yo[1] = y[1];
    yo[2] = y[2];
}

// energy psi_e and its first (ps) and second (ph, sym6) derivatives with respect to
// x = (I1-3, I2-3, J-1), from the network's value, gradient and Hessian o[10] with
// respect to y (or the closed-form Neo-Hookean energy, Sec. 4.1); psi_e = mu_e (N -
// N0 - n x3) + lambda_e ((J-1)^2/J)^2 (Eq. (dd_0))
__device__ __forceinline__ void energy_derivs(const MatF &m, const NcF &nc, const float (&x)[3], float Jdet,
                                              const float *o, const float (&Tm)[3][3], const float (&T2)[3][6],
                                              float (&ps)[3], float (&ph)[6], float &pe)
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
}

// qp mode: degraded stress P = f_d dpsi_e/dF - c_d (F^-T grad phi) (x) (C^-1 grad phi)
// and the per-point records that the row mode reads (Sec. 2.1f, Sec. 4.1f); kappa
// is the updated history, Gp = G'(q) and dr = dPhi_d/dkappa of the local solve
// (loading points), which give the kappa sensitivities of the monolithic tangent
__device__ __forceinline__ void stress_records(const MatF &m, const float (&F)[3][3], const float (&x)[3],
                                               const float (&g)[3], float phi, float Jdet, const float (&ps)[3],
                                               const float (&ph)[6], float kappa, bool loading, float Gp, float dr,
                                               bool valid, float *rec)
{
    const bool dmg = kappa > m.kappa_d;
    const float fd = dmg ? expf(-m.eta_d * (kappa - m.kappa_d)) : 1.0f;
    const float fdp = dmg ? -m.eta_d * fd : 0.0f;
    const float ck = loading ? -Gp / dr : 0.0f;          // G' / (1 - G' dq/dkappa)
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
    rec[Q_PENM] = m.beta_d * (fabsf(phi) + fabsf(kappa));
    rec[Q_J] = J;
    if (!valid) rec[Q_JW] = 0.0f;
}

// row mode: the element residual rows (FP64 atomics into R) and the tangent rows
// (FP32 or FP64 atomics into the CSR values) of the warp's batch, lane = element row
// (node a, dof i), EPR elements per pass (Sec. 3.1f residual; Sec. 3.2f tangent)
template <int DIM, class Args>
__device__ __forceinline__ void row_mode(const Args &A, const MatF &m, const float *sRec, float *sVec, int64_t e0,
                                         int lane)
{
    using G_ = Geo<DIM>;
    constexpr int NEN = G_::NEN, NQ = G_::NQ, NDOF = G_::NDOF, ND = G_::ND, EPW = G_::EPW, EPR = G_::EPR;
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
        float Rr = 0.0f, Mr = 0.0f;      // Mr: sum of the magnitudes of the row's terms (A.Rabs)
        const float cd = m.c_d;
        if (active) {
            for (int qq = 0; qq < NQ; ++qq) {
                const float *R0 = sRec + (el_local * NQ + qq) * Q_REC;
                const float *Vq = sVec + (ee * NQ + qq) * NEN * V_REC;
                const float *Va = Vq + a * V_REC;
                const float Jw = R0[Q_JW];
                if (i < DIM) {
                    // r_u,a = P n_a J w (Sec. 3.1f)
                    const float t0 = R0[Q_P + i * 3] * Va[V_N], t1 = R0[Q_P + i * 3 + 1] * Va[V_N + 1],
                                t2 = R0[Q_P + i * 3 + 2] * Va[V_N + 2];
                    Rr += Jw * (t0 + t1 + t2);
                    if (A.Rabs) Mr += Jw * (fabsf(t0) + fabsf(t1) + fabsf(t2));
                    if (!A.tangent) continue;      // residual-only pass: no tangent rows
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
                    if (A.Rabs) Mr += Jw * (fabsf(cd * Va[V_MN]) + R0[Q_PENM] * fabsf(Na));
                    if (!A.tangent) continue;
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
            if (A.Rabs) atomicAdd(A.Rabs + rdof, (double)Mr);
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

}  // namespace e32
}  // namespace gd
