// gd_adjoint.cu -- element kernels of the discrete adjoint of the load path
// (gradient of a reaction-curve loss with respect to the network weights).
//
// For load step n the forward state satisfies R^f(d_n; kappa_{n-1}, theta) = 0 with
// kappa_n = K(d_n, kappa_{n-1}, theta) the local update (Sec. 3.2, Eq. (dd_7));
// the reaction is F_n = e_r . R(d_n; ...).  Sweeping the steps backwards with
// the history adjoint kbar_n = dL/dkappa_n (kbar_N = 0):
//   source   s_n  = (dK/dd)^T kbar_n                                  (mode 0 here)
//   solve    K_n^T lambda = -(Fbar_n K_n^T e_r + s_n) on the free dofs   (host + Krylov)
//   weights  w = lambda + Fbar_n e_r
//   theta   += w . dR/dtheta|kappa + (w . dR/dkappa + kbar_n) dkappa/dtheta  (mode 1 here)
//   kbar_{n-1} = w . dR/dkappa + kbar_n on elastic points, 0 on loading points
// because a loading point's kappa_n solves G(q(kappa)) = kappa and does not
// depend on kappa_{n-1}, while an elastic point keeps kappa_n = kappa_{n-1}.
// dkappa/dtheta follows from the implicit-function theorem on Phi_d = 0:
//   dkappa/dtheta = (G' dpsi_e/dtheta_psi + dG/dtheta_yield) / (1 - G' dq/dkappa).
// The parameter derivatives of the networks are reverse sweeps through the
// forward pass and its directional tangent, accumulated per warp in shared
// memory and added to the global gradient with FP64 atomics.
#include <cuda_runtime.h>

#include "gd_internal.cuh"

namespace gd {
namespace {

#include "gd_device_fp64.cuh"

// Reverse sweep of  F = alpha * (grad N(x) . d) + beta * N(x)  with respect to
// the packed parameters (W1 b1 W2 A2 b2 w3 a3) of a two-layer softplus network
// with n_in inputs; lane = unit.  acc holds the gradient with W2 padded to rows
// of (w + 1); buf needs 6 w doubles.  All lanes must call it.
__device__ void net_reverse_unit(const double *P, const double *W2T, int n_in, int w, const double *x,
                                 const double *d, double alpha, double beta, double *acc, double *buf, int lane)
{
    // a3 enters F linearly (grad N . d = ... + a3 . d, N = ... + a3 . x): its gradient
    // needs no parameter value
    const double *W1 = P, *b1 = W1 + w * n_in, *W2 = b1 + w, *A2 = W2 + w * w, *b2 = A2 + w * n_in, *w3 = b2 + w;
    double *aW1 = acc, *ab1 = aW1 + w * n_in, *aW2 = ab1 + w, *aA2 = aW2 + w * (w + 1), *ab2 = aA2 + w * n_in,
           *aw3 = ab2 + w, *aa3 = aw3 + w;
    double *sZ = buf, *sZd = buf + w, *sH = buf + 2 * w, *sHd = buf + 3 * w;
    double s1v[2], s1p[2], hd1[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int j = lane + 32 * t;
        s1v[t] = s1p[t] = hd1[t] = 0.0;
        if (j < w) {
            double h = __ldg(b1 + j), hd = 0.0;
            for (int i = 0; i < n_in; ++i) {
                h += __ldg(W1 + j * n_in + i) * x[i];
                hd += __ldg(W1 + j * n_in + i) * d[i];
            }
            const double sg = sigm(h);
            sZ[j] = softplus(h);
            sZd[j] = sg * hd;
            s1v[t] = sg;
            s1p[t] = sg * (1.0 - sg);
            hd1[t] = hd;
        }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int k = lane + 32 * t;
        if (k < w) {
            double h = __ldg(b2 + k), hd = 0.0;
            for (int i = 0; i < n_in; ++i) {
                h += __ldg(A2 + k * n_in + i) * x[i];
                hd += __ldg(A2 + k * n_in + i) * d[i];
            }
            const double *col = W2T + k;
            for (int j = 0; j < w; ++j) {
                const double wkj = __ldg(col + j * w);
                h += wkj * sZ[j];
                hd += wkj * sZd[j];
            }
            const double sg = sigm(h), sp1 = sg * (1.0 - sg), wk = __ldg(w3 + k);
            const double hbar = alpha * wk * sp1 * hd + beta * wk * sg;
            const double hdbar = alpha * wk * sg;
            aw3[k] += alpha * sg * hd + beta * softplus(h);
            ab2[k] += hbar;
            for (int i = 0; i < n_in; ++i) aA2[k * n_in + i] += hbar * x[i] + hdbar * d[i];
            double *row = aW2 + k * (w + 1);
            for (int j = 0; j < w; ++j) row[j] += hbar * sZ[j] + hdbar * sZd[j];
            sH[k] = hbar;
            sHd[k] = hdbar;
        }
    }
    if (lane == 0)
        for (int i = 0; i < n_in; ++i) aa3[i] += alpha * d[i] + beta * x[i];
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int j = lane + 32 * t;
        if (j < w) {
            double zb = 0.0, zdb = 0.0;
            const double *row = W2 + j;          // W2[k][j] at k*w + j
            for (int k = 0; k < w; ++k) {
                const double wkj = __ldg(row + k * w);
                zb += wkj * sH[k];
                zdb += wkj * sHd[k];
            }
            const double h1b = zb * s1v[t] + zdb * s1p[t] * hd1[t];
            const double hd1b = zdb * s1v[t];
            ab1[j] += h1b;
            for (int i = 0; i < n_in; ++i) aW1[j * n_in + i] += h1b * x[i] + hd1b * d[i];
        }
    }
    __syncwarp();
}

// size of a padded accumulator block for a network
__host__ __device__ inline int acc_size(int n_in, int w) { return w > 0 ? w * n_in + w + w * (w + 1) + w * n_in + w + w + n_in : 0; }

// add a padded accumulator block into the packed gradient (atomics)
__device__ void flush_acc(const double *acc, int n_in, int w, double *out, int lane)
{
    if (w <= 0) return;
    const int n_packed = w * n_in + w + w * w + w * n_in + w + w + n_in;
    const int off_W2 = w * n_in + w;
    for (int p = lane; p < n_packed; p += 32) {
        int src;
        if (p < off_W2) src = p;
        else if (p < off_W2 + w * w) {
            const int k = (p - off_W2) / w, j = (p - off_W2) % w;
            src = off_W2 + k * (w + 1) + j;
        } else src = p + w;            // the w padding slots come before the tail
        const double v = acc[src];
        if (v != 0.0) atomicAdd(out + p, v);
    }
}

template <int DIM>
__global__ void __launch_bounds__(32) adjoint_kernel(AdjArgs A)
{
    using G_ = Geo<DIM>;
    constexpr int NEN = G_::NEN, NQ = G_::NQ, NDOF = G_::NDOF, EPW = G_::EPW;
    extern __shared__ double smem[];
    const int lane = threadIdx.x;
    const int wpsi = A.psi.width, wy = A.yld.width;
    const int wmax = wpsi > wy ? wpsi : wy;
    const int accp = acc_size(3, wpsi), accy = acc_size(1, wy);
    double *accP = smem;
    double *accY = accP + accp;
    double *sX = accY + accy;                           // [EPW][NEN][DIM]
    double *sD = sX + EPW * NEN * DIM;                  // [EPW][NEN][NDOF]
    double *sW = sD + EPW * NEN * NDOF;                 // [EPW][NEN][NDOF] adjoint weights
    double *sQ = sW + EPW * NEN * NDOF;                 // [32][16] per-point scalars
    double *sBuf = sQ + 32 * 16;                        // unit-mode buffers (6 wmax)
    double *sOut = sBuf + 6 * wmax;                     // [32][10]
    for (int i = lane; i < accp + accy; i += 32) smem[i] = 0.0;
    __syncwarp();
    const NetConst nc = *A.netc;
    const MatConst &m = A.mat;
    double gN0 = 0.0, gn = 0.0, gY0 = 0.0, gYp0 = 0.0;   // weights of the normalising constants

    const int64_t n_batches = (A.n_elems + EPW - 1) / EPW;
    for (int64_t batch = blockIdx.x; batch < n_batches; batch += gridDim.x) {
        const int64_t e0 = batch * EPW;
        for (int t = lane; t < EPW * NEN; t += 32) {
            const int el = t / NEN, a = t % NEN;
            const int64_t e = e0 + el;
            if (e < A.n_elems) {
                const int32_t n = __ldg(A.conn + e * NEN + a);
#pragma unroll
                for (int J = 0; J < DIM; ++J) sX[t * DIM + J] = __ldg(A.X + (int64_t)n * DIM + J);
#pragma unroll
                for (int c = 0; c < NDOF; ++c) {
                    sD[t * NDOF + c] = __ldg(A.dofs + (int64_t)n * NDOF + c);
                    sW[t * NDOF + c] = A.w ? __ldg(A.w + (int64_t)n * NDOF + c) : 0.0;
                }
            } else {
#pragma unroll
                for (int J = 0; J < DIM; ++J) sX[t * DIM + J] = node_sgn(a, J) > 0.0 ? 1.0 : 0.0;
#pragma unroll
                for (int c = 0; c < NDOF; ++c) sD[t * NDOF + c] = sW[t * NDOF + c] = 0.0;
            }
        }
        __syncwarp();

        // ---- qp mode: kinematics, adjoint gradients, network input ----
        const int el = lane / NQ, q = lane % NQ;
        const int64_t e_me = e0 + el;
        const bool valid = e_me < A.n_elems;
        double F[3][3], H[3][3], phi = 0.0, x[3], Jdet, Jw, Zf[3][3], zphi = 0.0;
        double dNs[8][3], Ns[8];
        {
            const double xi[3] = {(q & 1) ? kGauss : -kGauss, (q & 2) ? kGauss : -kGauss, (q & 4) ? kGauss : -kGauss};
            const double *Xe = sX + el * NEN * DIM;
            const double *De = sD + el * NEN * NDOF;
            const double *We = sW + el * NEN * NDOF;
            double Jm[3][3] = {{0.0}};
#pragma unroll
            for (int a = 0; a < NEN; ++a) {
                double Na, dN[3];
                ref_shape<DIM>(a, xi, Na, dN);
#pragma unroll
                for (int J = 0; J < DIM; ++J)
#pragma unroll
                    for (int k = 0; k < DIM; ++k) Jm[J][k] += Xe[a * DIM + J] * dN[k];
            }
            double Ji[3][3] = {{0.0}}, det;
            if (DIM == 2) {
                det = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
                Ji[0][0] = Jm[1][1] / det; Ji[0][1] = -Jm[0][1] / det;
                Ji[1][0] = -Jm[1][0] / det; Ji[1][1] = Jm[0][0] / det;
            } else {
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
                        Ji[i][j] = Jm[i1][j1] * Jm[i2][j2] - Jm[i1][j2] * Jm[i2][j1];
                    }
                det = Jm[0][0] * Ji[0][0] + Jm[0][1] * Ji[1][0] + Jm[0][2] * Ji[2][0];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) Ji[i][j] /= det;
            }
            Jw = valid ? det : 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int J = 0; J < 3; ++J) H[i][J] = Zf[i][J] = 0.0;
#pragma unroll
            for (int a = 0; a < NEN; ++a) {
                double Na, dN[3], n[3] = {0.0, 0.0, 0.0};
                ref_shape<DIM>(a, xi, Na, dN);
#pragma unroll
                for (int J = 0; J < DIM; ++J)
#pragma unroll
                    for (int k = 0; k < DIM; ++k) n[J] += dN[k] * Ji[k][J];
#pragma unroll
                for (int J = 0; J < 3; ++J) dNs[a][J] = n[J];
                Ns[a] = Na;
                phi += Na * De[a * NDOF + DIM];
                zphi += Na * We[a * NDOF + DIM];
#pragma unroll
                for (int J = 0; J < DIM; ++J)
#pragma unroll
                    for (int i = 0; i < DIM; ++i) {
                        H[i][J] += De[a * NDOF + i] * n[J];
                        Zf[i][J] += We[a * NDOF + i] * n[J];
                    }
            }
            double Am[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    double s = H[i][j] + H[j][i];
#pragma unroll
                    for (int k = 0; k < 3; ++k) s += H[k][i] * H[k][j];
                    Am[i][j] = s;
                }
            double tA = Am[0][0] + Am[1][1] + Am[2][2], AA = 0.0, tH = H[0][0] + H[1][1] + H[2][2], HH = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    AA += Am[i][j] * Am[j][i];
                    HH += H[i][j] * H[j][i];
                }
            const double detH = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
                                H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                                H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
            x[0] = tA;
            x[1] = 2.0 * tA + 0.5 * (tA * tA - AA);
            x[2] = tH + 0.5 * (tH * tH - HH) + detH;
            Jdet = 1.0 + x[2];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? 1.0 : 0.0);
        }
        double Tm[3][3], T2[3][6], y[3] = {x[0], x[1], x[2]};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int j = 0; j < 3; ++j) Tm[i][j] = (i == j) ? 1.0 : 0.0;
#pragma unroll
            for (int j = 0; j < 6; ++j) T2[i][j] = 0.0;
        }
        if (m.energy == GD_ENERGY_ICNN_ISO) {
            const double L = log1p(x[2]), E = exp(-2.0 / 3.0 * L), I1 = 3.0 + x[0], I2 = 3.0 + x[1], J = Jdet;
            y[0] = 3.0 * expm1(-2.0 / 3.0 * L) + x[0] * E;
            y[1] = 3.0 * expm1(3.0 * log1p(x[1] / 3.0) - 4.0 * L);
            const double J4 = J * J * J * J;
            Tm[0][0] = E;
            Tm[0][2] = -2.0 / 3.0 * I1 * E / J;
            Tm[1][1] = I2 * I2 / (3.0 * J4);
            Tm[1][2] = -4.0 * I2 * I2 * I2 / (9.0 * J4 * J);
        }
        double *Q = sQ + lane * 16;
        Q[0] = y[0];
        Q[1] = y[1];
        Q[2] = y[2];
        __syncwarp();
        if (m.energy != GD_ENERGY_NEO_HOOKE) {
            for (int p = 0; p < 32; ++p) {
                if (e0 + p / NQ >= A.n_elems) break;
                double yy[3] = {sQ[p * 16], sQ[p * 16 + 1], sQ[p * 16 + 2]}, out[10];
                psi_net_unit(A.psi, yy, out, sBuf, lane);
                if (lane == 0)
#pragma unroll
                    for (int c = 0; c < 4; ++c) sOut[p * 10 + c] = out[c];
            }
        }
        __syncwarp();
        // energy value and gradient wrt (I1-3, I2-3, J-1)
        double ps[3], pe;
        {
            const double J = Jdet, x3 = x[2];
            if (m.energy == GD_ENERGY_NEO_HOOKE) {
                const double L = log1p(x3);
                pe = 0.5 * m.mu_e * x[0] - m.mu_e * L + 0.5 * m.lambda_e * L * L;
                ps[0] = 0.5 * m.mu_e;
                ps[1] = 0.0;
                ps[2] = (-m.mu_e + m.lambda_e * L) / J;
            } else {
                const double *o = sOut + lane * 10;
#pragma unroll
                for (int i = 0; i < 3; ++i) ps[i] = Tm[0][i] * o[1] + Tm[1][i] * o[2] + Tm[2][i] * o[3];
                const double t = x3 * x3 / J, dt = 1.0 - 1.0 / (J * J);
                pe = m.mu_e * (o[0] - nc.psi_N0 - nc.psi_n * x3) + m.lambda_e * t * t;
#pragma unroll
                for (int i = 0; i < 3; ++i) ps[i] *= m.mu_e;
                ps[2] += -m.mu_e * nc.psi_n + m.lambda_e * 2.0 * t * dt;
            }
        }
        const double kn = valid ? __ldg(A.kappa_prev + e_me * NQ + q) : 0.0;
        const double kc = valid ? __ldg(A.kappa_cur + e_me * NQ + q) : 0.0;
        Q[3] = pe;
        Q[4] = phi;
        Q[5] = kn;
        Q[6] = kc;
        __syncwarp();
        // ---- unit mode: the forward loading decision and G, G' at kappa_n ----
        for (int p = 0; p < 32; ++p) {
            if (e0 + p / NQ >= A.n_elems) break;
            const double ppe = sQ[p * 16 + 3], pphi = sQ[p * 16 + 4], pkn = sQ[p * 16 + 5], pkc = sQ[p * 16 + 6];
            double r, dr, Gp;
            r_slope(A.mat, A.yld, nc, ppe, pphi, pkn, r, dr, Gp, sBuf, lane);
            const double loading = r > 0.0 ? 1.0 : 0.0;
            r_slope(A.mat, A.yld, nc, ppe, pphi, pkc, r, dr, Gp, sBuf, lane);
            if (lane == 0) {
                sOut[p * 10 + 4] = loading;
                sOut[p * 10 + 5] = Gp;
                sOut[p * 10 + 6] = dr;
                sOut[p * 10 + 7] = r + pkc;     // G(q(kappa_n))
            }
        }
        __syncwarp();
        // ---- qp mode: coupling coefficients ----
        const double *o = sOut + lane * 10;
        const bool loading = o[4] > 0.5;
        const double Gp = o[5], rp = o[6], Gn = o[7];
        const bool dmg = kc > m.kappa_d;
        const double fd = dmg ? exp(-m.eta_d * (kc - m.kappa_d)) : 1.0;
        const double fdp = dmg ? -m.eta_d * fd : 0.0;
        const double ck = loading ? -Gp / rp : 0.0;
        double Fi[3][3], C[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
                Fi[i][j] = (F[i1][j1] * F[i2][j2] - F[i1][j2] * F[i2][j1]) / Jdet;
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < 3; ++k) s += F[k][i] * F[k][j];
                C[i][j] = s;
            }
        const double I1 = 3.0 + x[0];
        double Ph[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int J2 = 0; J2 < 3; ++J2) {
                const double FC = F[i][0] * C[0][J2] + F[i][1] * C[1][J2] + F[i][2] * C[2][J2];
                Ph[i][J2] = 2.0 * ps[0] * F[i][J2] + 2.0 * ps[1] * (I1 * F[i][J2] - FC) + ps[2] * Jdet * Fi[J2][i];
            }
        if (A.mode == 0) {
            // source (dK/dd)^T kbar: dkappa/dF = c_k P_hat, dkappa/dphi = c_k qcoef / f_d (loading points)
            const double kb = valid ? __ldg(A.kbar + e_me * NQ + q) : 0.0;
            const double sF = kb * ck, sPhi = kb * ck * m.qcoef / fd;
            // each point adds its own contribution to the element rows (no quadrature
            // weight: kappa is a per-point quantity)
            if (valid && (sF != 0.0 || sPhi != 0.0)) {
#pragma unroll
                for (int a = 0; a < NEN; ++a) {
                    const int32_t na = __ldg(A.conn + e_me * NEN + a);
#pragma unroll
                    for (int i = 0; i < DIM; ++i) {
                        const double v = sF * (Ph[i][0] * dNs[a][0] + Ph[i][1] * dNs[a][1] + Ph[i][2] * dNs[a][2]);
                        atomicAdd(A.rhs + (int64_t)na * NDOF + i, v);
                    }
                    atomicAdd(A.rhs + (int64_t)na * NDOF + DIM, sPhi * Ns[a]);
                }
            }
            __syncwarp();
            continue;
        }
        // ---- mode 1: weights of the reverse sweeps ----
        const double kb = valid ? __ldg(A.kbar + e_me * NQ + q) : 0.0;
        double zP = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int J2 = 0; J2 < 3; ++J2) zP += Zf[i][J2] * Ph[i][J2];
        const double omega = Jw * (fdp * zP - m.beta_d * zphi) + kb;
        if (valid && A.kbar_prev) A.kbar_prev[e_me * NQ + q] = loading ? 0.0 : omega;
        // directional derivatives of the invariants along zeta_F
        double c1 = 0.0, c2 = 0.0, c3 = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int J2 = 0; J2 < 3; ++J2) {
                const double FC = F[i][0] * C[0][J2] + F[i][1] * C[1][J2] + F[i][2] * C[2][J2];
                c1 += 2.0 * F[i][J2] * Zf[i][J2];
                c2 += 2.0 * (I1 * F[i][J2] - FC) * Zf[i][J2];
                c3 += Jdet * Fi[J2][i] * Zf[i][J2];
            }
        const double alpha = valid ? Jw * fd * m.mu_e : 0.0;
        const double beta = (valid && loading) ? omega * ck * m.mu_e : 0.0;
        double dy[3];
#pragma unroll
        for (int mm = 0; mm < 3; ++mm) dy[mm] = Tm[mm][0] * c1 + Tm[mm][1] * c2 + Tm[mm][2] * c3;
        gN0 -= beta;
        gn -= alpha * c3 + beta * x[2];
        const double wyld = (valid && loading && A.yld.width > 0) ? omega * nc.y_s / (-rp) : 0.0;
        gY0 -= wyld;
        gYp0 -= wyld * Gn;
        // q at kappa_n for the yield sweep
        const double qn = pe + m.qcoef * (phi - kc) / fd;
        Q[7] = dy[0];
        Q[8] = dy[1];
        Q[9] = dy[2];
        Q[10] = alpha;
        Q[11] = beta;
        Q[12] = wyld;
        Q[13] = qn;
        __syncwarp();
        for (int p = 0; p < 32; ++p) {
            if (e0 + p / NQ >= A.n_elems) break;
            const double *Qp = sQ + p * 16;
            if (m.energy != GD_ENERGY_NEO_HOOKE && (Qp[10] != 0.0 || Qp[11] != 0.0)) {
                const double yy[3] = {Qp[0], Qp[1], Qp[2]}, dd[3] = {Qp[7], Qp[8], Qp[9]};
                net_reverse_unit(A.psi.p, A.psi.W2T, 3, wpsi, yy, dd, Qp[10], Qp[11], accP, sBuf, lane);
            }
            if (Qp[12] != 0.0) {
                const double qq = Qp[13], d0 = 0.0;
                net_reverse_unit(A.yld.p, A.yld.W2T, 1, wy, &qq, &d0, 0.0, Qp[12], accY, sBuf, lane);
            }
        }
        __syncwarp();
    }
    if (A.mode == 1) {
        flush_acc(accP, 3, wpsi, A.theta_bar, lane);
        flush_acc(accY, 1, wy, A.theta_bar + A.psi.n_params, lane);
        gN0 = warp_sum(gN0);
        gn = warp_sum(gn);
        gY0 = warp_sum(gY0);
        gYp0 = warp_sum(gYp0);
        if (lane == 0) {
            atomicAdd(A.glob + 0, gN0);
            atomicAdd(A.glob + 1, gn);
            atomicAdd(A.glob + 2, gY0);
            atomicAdd(A.glob + 3, gYp0);
        }
    }
}

// normalising constants: psi N(0) with weight glob[0], n = grad N(0) . c_n with
// glob[1]; yield N_k(0) with glob[2], N_k'(0) with glob[3]
__global__ void adjoint_globals_kernel(DevNet psi, DevNet yld, int energy, const double *glob, double *theta_bar)
{
    extern __shared__ double smem[];
    const int lane = threadIdx.x;
    const int accp = acc_size(3, psi.width), accy = acc_size(1, yld.width);
    const int wmax = psi.width > yld.width ? psi.width : yld.width;
    double *accP = smem, *accY = accP + accp, *buf = accY + accy;
    for (int i = lane; i < accp + accy; i += 32) smem[i] = 0.0;
    (void)wmax;
    __syncwarp();
    if (energy != GD_ENERGY_NEO_HOOKE && psi.width > 0) {
        const double x0[3] = {0.0, 0.0, 0.0};
        const double cn[3] = {energy == GD_ENERGY_ICNN_RAW ? 2.0 : 0.0, energy == GD_ENERGY_ICNN_RAW ? 4.0 : 0.0, 1.0};
        net_reverse_unit(psi.p, psi.W2T, 3, psi.width, x0, cn, glob[1], glob[0], accP, buf, lane);
    }
    if (yld.width > 0) {
        const double q0 = 0.0, d1 = 1.0;
        net_reverse_unit(yld.p, yld.W2T, 1, yld.width, &q0, &d1, glob[3], glob[2], accY, buf, lane);
    }
    __syncwarp();
    flush_acc(accP, 3, psi.width, theta_bar, lane);
    flush_acc(accY, 1, yld.width, theta_bar + psi.n_params, lane);
}

template <int DIM>
cudaError_t launch_adj(const AdjArgs &a, int num_sms, cudaStream_t s)
{
    using G_ = Geo<DIM>;
    const int wmax = a.psi.width > a.yld.width ? a.psi.width : a.yld.width;
    const size_t sm = sizeof(double) * (acc_size(3, a.psi.width) + acc_size(1, a.yld.width) +
                                        G_::EPW * G_::NEN * (DIM + 2 * G_::NDOF) + 32 * 16 + 6 * wmax + 32 * 10);
    cudaError_t err = cudaFuncSetAttribute(adjoint_kernel<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjoint_kernel<DIM>, 32, sm);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    const int64_t batches = (a.n_elems + G_::EPW - 1) / G_::EPW;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > batches) grid = batches;
    if (grid < 1) grid = 1;
    adjoint_kernel<DIM><<<(unsigned)grid, 32, sm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint(int dim, const AdjArgs &a, int num_sms, cudaStream_t s)
{
    if (a.n_elems <= 0) return cudaSuccess;
    return dim == 2 ? launch_adj<2>(a, num_sms, s) : launch_adj<3>(a, num_sms, s);
}

cudaError_t launch_adjoint_globals(const DevNet &psi, const DevNet &yld, int energy, const double *glob,
                                   double *theta_bar, cudaStream_t s)
{
    const int wmax = psi.width > yld.width ? psi.width : yld.width;
    const size_t sm = sizeof(double) * (acc_size(3, psi.width) + acc_size(1, yld.width) + 6 * wmax + 8);
    cudaError_t err = cudaFuncSetAttribute(adjoint_globals_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    adjoint_globals_kernel<<<1, 32, sm, s>>>(psi, yld, energy, glob, theta_bar);
    return cudaGetLastError();
}

}  // namespace gd
