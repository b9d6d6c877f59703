// gd_device_fp64.cuh -- FP64 device building blocks shared by the element
// kernel and the adjoint kernel: shape functions, the per-point record layout,
// the energy and yield networks in unit mode (lane = network unit) and the
// local-update residual.  Included inside an anonymous namespace of each
// translation unit.
#pragma once

constexpr double kGauss = 0.57735026918962576451;   // 1/sqrt(3)

__device__ __forceinline__ double softplus(double v) { return fmax(v, 0.0) + log1p(exp(-fabs(v))); }
__device__ __forceinline__ double sigm(double v)
{
    double e = exp(-fabs(v));
    double r = 1.0 / (1.0 + e);
    return v >= 0.0 ? r : e * r;
}
// softplus(v) and its derivative sigmoid(v) from one exponential
__device__ __forceinline__ void sp_sig(double v, double &sp, double &sg)
{
    const double e = exp(-fabs(v));
    sp = fmax(v, 0.0) + log1p(e);
    const double r = 1.0 / (1.0 + e);
    sg = v >= 0.0 ? r : e * r;
}
__device__ __forceinline__ double warp_sum(double v)
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
__device__ __forceinline__ double node_sgn(int a, int k)
{
    int b = (k == 0) ? ((a & 3) == 1 || (a & 3) == 2) : (k == 1 ? ((a & 3) >= 2) : (a >= 4));
    return b ? 1.0 : -1.0;
}

// N_a and dN_a/dxi at reference point xi
template <int DIM>
__device__ __forceinline__ void ref_shape(int a, const double *xi, double &N, double *dN)
{
    double f[3], s[3];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        s[k] = node_sgn(a, k);
        f[k] = 0.5 * (1.0 + s[k] * xi[k]);
    }
    N = 1.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) N *= f[k];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        double v = 0.5 * s[k];
#pragma unroll
        for (int l = 0; l < DIM; ++l)
            if (l != k) v *= f[l];
        dN[k] = v;
    }
}

// ---- per-point record (row-mode inputs), doubles ----
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
// N(x) (Sec. 4.2 ICNN).  Layer 1 and the gradient columns of layer 2 are
// forward tangents; the second derivative uses the identity
//   d2N/dx2 = sum_k w3_k sp''(h2_k) g_k g_k^T + sum_j v_j sp''(h1_j) W1_j W1_j^T,
//   g_k = dh2_k/dx,  v = W2^T (w3 o sp'(h2)),
// so layer 2 costs 4 forward columns and 1 reverse column per point.
// Every lane returns the full result.
__device__ void psi_net_unit(const DevNet &net, const double *x, double *out10, double *buf, int lane,
                             bool hess = true)
{
    const int w = net.width;
    const double *W1 = net.p, *b1 = W1 + 3 * w, *W2 = b1 + w, *A2 = W2 + w * w, *b2 = A2 + 3 * w, *w3 = b2 + w,
                 *a3 = w3 + w;
    double *sS = buf, *sD0 = buf + w, *sD1 = buf + 2 * w, *sD2 = buf + 3 * w, *sU = buf + 4 * w;
    double e1[2], W1r[2][3];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int j = lane + 32 * t;
        e1[t] = 0.0;
        W1r[t][0] = W1r[t][1] = W1r[t][2] = 0.0;
        if (j < w) {
            double a0 = __ldg(W1 + 3 * j), a1 = __ldg(W1 + 3 * j + 1), a2 = __ldg(W1 + 3 * j + 2);
            double h = __ldg(b1 + j) + a0 * x[0] + a1 * x[1] + a2 * x[2];
            double sg, spv;
            sp_sig(h, spv, sg);
            sS[j] = spv;
            sD0[j] = sg * a0;
            sD1[j] = sg * a1;
            sD2[j] = sg * a2;
            e1[t] = sg * (1.0 - sg);
            W1r[t][0] = a0; W1r[t][1] = a1; W1r[t][2] = a2;
        }
    }
    __syncwarp();
    double acc[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) acc[c] = 0.0;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int k = lane + 32 * t;
        if (k < w) {
            double h = __ldg(b2 + k), g0 = __ldg(A2 + 3 * k), g1 = __ldg(A2 + 3 * k + 1), g2 = __ldg(A2 + 3 * k + 2);
            h += g0 * x[0] + g1 * x[1] + g2 * x[2];
            const double *col = net.W2T + k;     // W2[k][j] = W2T[j*w + k]
            for (int j = 0; j < w; ++j) {
                double wkj = __ldg(col + j * w);
                h += wkj * sS[j];
                g0 += wkj * sD0[j];
                g1 += wkj * sD1[j];
                g2 += wkj * sD2[j];
            }
            double sg, spv;
            sp_sig(h, spv, sg);
            const double wk = __ldg(w3 + k);
            double e2 = wk * sg * (1.0 - sg);
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
    // the Hessian's layer-1 term (one reverse column through layer 2): only where the
    // caller needs second derivatives (hess = false: out10[4..9] lack it)
#pragma unroll
    for (int t = 0; t < 2 && hess; ++t) {
        int j = lane + 32 * t;
        if (j < w) {
            double v = 0.0;
            const double *row = W2 + j;          // W2[k][j] at k*w + j
            for (int k = 0; k < w; ++k) v += __ldg(row + k * w) * sU[k];
            double c = v * e1[t];
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
__device__ void yield_unit(const DevNet &net, const NetConst &nc, double q, double &G, double &Gp, double *buf,
                           int lane)
{
    const int w = net.width;
    if (w == 0) {
        G = q;
        Gp = 1.0;
        return;
    }
    const double *V1 = net.p, *c1 = V1 + w, *V2 = c1 + w, *B2 = V2 + w * w, *c2 = B2 + w, *v3 = c2 + w,
                 *b3 = v3 + w;
    double *sS = buf, *sT = buf + w;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int j = lane + 32 * t;
        if (j < w) {
            double a = __ldg(V1 + j);
            double h = __ldg(c1 + j) + a * q;
            double spv, sg;
            sp_sig(h, spv, sg);
            sS[j] = spv;
            sT[j] = sg * a;
        }
    }
    __syncwarp();
    double n0 = 0.0, n1 = 0.0;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int k = lane + 32 * t;
        if (k < w) {
            double g = __ldg(B2 + k);
            double h = __ldg(c2 + k) + g * q;
            const double *col = net.W2T + k;
            for (int j = 0; j < w; ++j) {
                double wkj = __ldg(col + j * w);
                h += wkj * sS[j];
                g += wkj * sT[j];
            }
            double vk = __ldg(v3 + k);
            double spv, sg;
            sp_sig(h, spv, sg);
            n0 += vk * spv;
            n1 += vk * sg * g;
        }
    }
    n0 = warp_sum(n0);
    n1 = warp_sum(n1);
    double b = __ldg(b3);
    G = nc.y_s * (n0 + b * q - nc.y_N0);
    Gp = nc.y_s * (n1 + b);
    __syncwarp();
}

// r(kappa) = G(q(kappa)) - kappa and dr/dkappa (Eq. (potential_function)),
// q = psi_e + qcoef (phi - kappa) / f_d(kappa) (Eq. (ostwald_potential)).
__device__ __forceinline__ void r_slope(const MatConst &m, const DevNet &yld, const NetConst &nc, double pe,
                                        double phi, double kappa, double &r, double &dr, double &Gp, double *buf,
                                        int lane)
{
    bool dmg = kappa > m.kappa_d;
    double f = dmg ? exp(-m.eta_d * (kappa - m.kappa_d)) : 1.0;
    double q = pe + m.qcoef * (phi - kappa) / f;
    double dq = m.qcoef * (-1.0 / f + (dmg ? (phi - kappa) * m.eta_d / f : 0.0));
    double G;
    yield_unit(yld, nc, q, G, Gp, buf, lane);
    r = G - kappa;
    dr = Gp * dq - 1.0;
}


// r(kappa) = G(q(kappa)) - kappa alone (no slope column): the value part of yield_unit
// and r_slope, for the Newton step that polishes an FP32 root
__device__ double r_value(const MatConst &m, const DevNet &net, const NetConst &nc, double pe, double phi,
                          double kappa, double *buf, int lane)
{
    const bool dmg = kappa > m.kappa_d;
    const double f = dmg ? exp(-m.eta_d * (kappa - m.kappa_d)) : 1.0;
    const double q = pe + m.qcoef * (phi - kappa) / f;
    const int w = net.width;
    if (w == 0) return q - kappa;
    const double *V1 = net.p, *c1 = V1 + w, *V2 = c1 + w, *B2 = V2 + w * w, *c2 = B2 + w, *v3 = c2 + w,
                 *b3 = v3 + w;
    double *sS = buf;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int j = lane + 32 * t;
        if (j < w) sS[j] = softplus(__ldg(c1 + j) + __ldg(V1 + j) * q);
    }
    __syncwarp();
    double n0 = 0.0;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        int k = lane + 32 * t;
        if (k < w) {
            double h = __ldg(c2 + k) + __ldg(B2 + k) * q;
            const double *col = net.W2T + k;
            for (int j = 0; j < w; ++j) h += __ldg(col + j * w) * sS[j];
            n0 += __ldg(v3 + k) * softplus(h);
        }
    }
    n0 = warp_sum(n0);
    __syncwarp();
    return nc.y_s * (n0 + __ldg(b3) * q - nc.y_N0) - kappa;
}

// specimen of element e and its networks (single-specimen launches use A.psi / A.yld)
template <class Args>
__device__ __forceinline__ int spec_of(const Args &A, int64_t e) { return A.elem_spec ? __ldg(A.elem_spec + e) : 0; }
template <class Args>
__device__ __forceinline__ const DevNet &psi_of(const Args &A, int s) { return A.psi_tab ? A.psi_tab[s] : A.psi; }
template <class Args>
__device__ __forceinline__ const DevNet &yld_of(const Args &A, int s) { return A.yld_tab ? A.yld_tab[s] : A.yld; }
