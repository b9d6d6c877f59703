// gd_asm_fp64.cu -- FP64 element kernel of the gradient-enhanced damage model.
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
// Paper passages: Sec. 3.1 (F, phi_q, grad phi_q, element residual, Table
// kernel_inputs), Sec. 2.1 (P, Y vector, Y), Sec. 2.2 and Sec. 3.2 Eq. (dd_7_no_nn)
// (local update, KKT), Sec. 3.2 (monolithic scheme), Sec. 4.1 (degradation,
// gradient and penalty energies, Eq. (ostwald_potential)), Sec. 4.2 Eqs. (dd_0),
// (dd_1), (Gq_NN), (dd_7).
#include <cuda_runtime.h>

#include "gd_elem32.cuh"
#include "gd_internal.cuh"

namespace gd {
namespace {

// trial yield values farther than this (relative to max(1, kappa_n)) from zero are
// decided by the FP32 evaluation; closer ones by an FP64 evaluation
constexpr double kTrialMargin = 1e-4;


#include "gd_device_fp64.cuh"

// KW warps per CTA (a tuning choice: warps are independent, so it only sets the
// granularity of residency and of the persistent grid)
template <int DIM, int KW>
__global__ void __launch_bounds__(32 * KW) asm_fp64_kernel(AsmArgs A)
{
    using G_ = Geo<DIM>;
    constexpr int NEN = G_::NEN, NQ = G_::NQ, NDOF = G_::NDOF, ND = G_::ND, EPW = G_::EPW, EPR = G_::EPR;
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wmax = A.wmax;
    // per-warp scratch
    const int scratch = EPW * NEN * (DIM + NDOF) + 32 * Q_REC + 32 * 4 + 32 * 10 + 5 * wmax + 2 * NQ * NEN * V_REC;
    double *ws = smem + warp * scratch;
    double *sX = ws;                                  // [EPW][NEN][DIM]
    double *sD = sX + EPW * NEN * DIM;                // [EPW][NEN][NDOF]
    double *sRec = sD + EPW * NEN * NDOF;             // [32][Q_REC]
    double *sIn = sRec + 32 * Q_REC;                  // [32][4]: network input x (3), then kappa out
    double *sOut = sIn + 32 * 4;                      // [32][10]: N, grad, Hess / local-solve results
    double *sBuf = sOut + 32 * 10;                    // unit-mode buffers
    double *sVec = sBuf + 5 * wmax;                   // [EPR*NQ*NEN][V_REC]
    const MatConst &m = A.mat;

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
                for (int J = 0; J < DIM; ++J) sX[t * DIM + J] = __ldg(A.X + (int64_t)n * DIM + J);
#pragma unroll
                for (int c = 0; c < NDOF; ++c) sD[t * NDOF + c] = __ldg(A.dofs + (int64_t)n * NDOF + c);
            } else {
#pragma unroll
                for (int J = 0; J < DIM; ++J) sX[t * DIM + J] = (a & 1) ? 1.0 : 0.0;
#pragma unroll
                for (int c = 0; c < NDOF; ++c) sD[t * NDOF + c] = 0.0;
            }
        }
        __syncwarp();

        // ================= qp mode: kinematics and invariants =================
        const int el = lane / NQ, q = lane % NQ;
        const int64_t e_me = e0 + el;
        const bool valid = e_me < A.n_elems;
        const NetConst nc = A.netc[valid ? spec_of(A, e_me) : 0];
        double *rec = sRec + lane * Q_REC;
        double F[3][3], H[3][3], phi = 0.0, g[3] = {0.0, 0.0, 0.0}, x[3], Jdet;
        {
            const double xi[3] = {(q & 1) ? kGauss : -kGauss, (q & 2) ? kGauss : -kGauss,
                                  (q & 4) ? kGauss : -kGauss};
            const double *Xe = sX + el * NEN * DIM;
            const double *De = sD + el * NEN * NDOF;
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
                for (int J = 0; J < 3; ++J) H[i][J] = 0.0;
#pragma unroll
            for (int a = 0; a < NEN; ++a) {
                double Na, dN[3], n[3] = {0.0, 0.0, 0.0};
                ref_shape<DIM>(a, xi, Na, dN);
#pragma unroll
                for (int J = 0; J < DIM; ++J)
#pragma unroll
                    for (int k = 0; k < DIM; ++k) n[J] += dN[k] * Ji[k][J];
                const double pa = De[a * NDOF + DIM];
                phi += Na * pa;
#pragma unroll
                for (int J = 0; J < DIM; ++J) {
                    g[J] += pa * n[J];
#pragma unroll
                    for (int i = 0; i < DIM; ++i) H[i][J] += De[a * NDOF + i] * n[J];
                }
            }
            // C - I = H + H^T + H^T H ; invariants without cancellation
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
            double detH = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
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
        // network input (raw or isochoric map)
        double Tm[3][3], T2[3][6];   // dy/dx and d2y/dx2 of the iso map (raw: identity)
        {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
                for (int j = 0; j < 3; ++j) Tm[i][j] = (i == j) ? 1.0 : 0.0;
#pragma unroll
                for (int j = 0; j < 6; ++j) T2[i][j] = 0.0;
            }
            double y[3] = {x[0], x[1], x[2]};
            if (m.energy == GD_ENERGY_ICNN_ISO) {
                // I1G = J^-2/3 I1, I2G = I2^3 / (9 J^4) (Eq. (dd_0)); derivatives wrt (I1-3, I2-3, J-1)
                double L = log1p(x[2]), E = exp(-2.0 / 3.0 * L), I1 = 3.0 + x[0], I2 = 3.0 + x[1], J = Jdet;
                y[0] = 3.0 * expm1(-2.0 / 3.0 * L) + x[0] * E;
                y[1] = 3.0 * expm1(3.0 * log1p(x[1] / 3.0) - 4.0 * L);
                double J4 = J * J * J * J;
                Tm[0][0] = E;
                Tm[0][2] = -2.0 / 3.0 * I1 * E / J;
                Tm[1][1] = I2 * I2 / (3.0 * J4);
                Tm[1][2] = -4.0 * I2 * I2 * I2 / (9.0 * J4 * J);
                T2[0][2] = -2.0 / 3.0 * E / J;                       // d2 y1 / dx1 dx3
                T2[0][5] = 10.0 / 9.0 * I1 * E / (J * J);            // d2 y1 / dx3^2
                T2[1][3] = 2.0 * I2 / (3.0 * J4);                    // d2 y2 / dx2^2
                T2[1][4] = -4.0 * I2 * I2 / (3.0 * J4 * J);          // d2 y2 / dx2 dx3
                T2[1][5] = 20.0 * I2 * I2 * I2 / (9.0 * J4 * J * J); // d2 y2 / dx3^2
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
                double y[3] = {sIn[p * 4], sIn[p * 4 + 1], sIn[p * 4 + 2]}, out[10];
                psi_net_unit(psi_of(A, spec_of(A, e0 + p / NQ)), y, out, sBuf, lane, A.tangent != 0);
                if (lane == 0)
#pragma unroll
                    for (int c = 0; c < 10; ++c) sOut[p * 10 + c] = out[c];
            }
        }
        __syncwarp();

        // ================= qp mode: energy derivatives wrt (I1-3, I2-3, J-1) =================
        double ps[3], ph[6], pe;
        {
            const double J = Jdet, x3 = x[2];
            if (m.energy == GD_ENERGY_NEO_HOOKE) {
                double L = log1p(x3);
                pe = 0.5 * m.mu_e * x[0] - m.mu_e * L + 0.5 * m.lambda_e * L * L;
                ps[0] = 0.5 * m.mu_e;
                ps[1] = 0.0;
                ps[2] = (-m.mu_e + m.lambda_e * L) / J;
#pragma unroll
                for (int c = 0; c < 6; ++c) ph[c] = 0.0;
                ph[5] = (m.lambda_e + m.mu_e - m.lambda_e * L) / (J * J);
            } else {
                const double *o = sOut + lane * 10;
                double gy[3] = {o[1], o[2], o[3]};
                double hy[6] = {o[4], o[5], o[6], o[7], o[8], o[9]};
                // chain through the input map: dN/dx = T^T dN/dy, d2N/dx2 = T^T H T + sum_m dN/dy_m d2y_m/dx2
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    double s = 0.0;
#pragma unroll
                    for (int mm = 0; mm < 3; ++mm) s += Tm[mm][i] * gy[mm];
                    ps[i] = s;
                }
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = i; j < 3; ++j) {
                        double s = 0.0;
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int b = 0; b < 3; ++b) s += Tm[a][i] * hy[sym6(a, b)] * Tm[b][j];
#pragma unroll
                        for (int mm = 0; mm < 3; ++mm) s += gy[mm] * T2[mm][sym6(i, j)];
                        ph[sym6(i, j)] = s;
                    }
                // psi_e = mu_e (N - N0 - n x3) + lambda_e t^2, t = (J-1)^2 / J
                double t = x3 * x3 / J, dt = 1.0 - 1.0 / (J * J), d2t = 2.0 / (J * J * J);
                pe = m.mu_e * (o[0] - nc.psi_N0 - nc.psi_n * x3) + m.lambda_e * t * t;
#pragma unroll
                for (int i = 0; i < 3; ++i) ps[i] *= m.mu_e;
#pragma unroll
                for (int c = 0; c < 6; ++c) ph[c] *= m.mu_e;
                ps[2] += -m.mu_e * nc.psi_n + m.lambda_e * 2.0 * t * dt;
                ph[5] += m.lambda_e * 2.0 * (dt * dt + t * d2t);
            }
            sIn[lane * 4 + 0] = pe;
            sIn[lane * 4 + 1] = phi;
            sIn[lane * 4 + 2] = valid ? __ldg(A.kappa_n + e_me * NQ + q) : 0.0;
        }
        __syncwarp();

        // ================= unit mode: local damage update per point =================
        const e32::MatF mf = e32::to_f(A.mat);
        float *fbuf = reinterpret_cast<float *>(sBuf);   // FP32 network buffers (2 w floats)
        if (A.kappa_fixed) {
            // frozen history (staggered scheme): the point keeps the given kappa
            double *o = sOut + lane * 10;
            o[0] = valid ? __ldg(A.kappa_fixed + e_me * NQ + q) : 0.0;
            o[1] = 0.0;
            o[2] = 0.0;
            o[3] = -1.0;
            o[4] = 0.0;
        } else
        for (int p = 0; p < 32; ++p) {
            if (e0 + p / NQ >= A.n_elems) break;
            const double ppe = sIn[p * 4], pphi = sIn[p * 4 + 1], kn = sIn[p * 4 + 2];
            const int sp = spec_of(A, e0 + p / NQ);
            const DevNet &yn = yld_of(A, sp);
            const NetConst ncp = A.netc[sp];
            double r = 0.0, dr = -1.0, Gp = 0.0;
            int n_eval = 0;
            double kappa = kn, fail = 0.0, loading = 0.0;
            // Trial Phi_d(kappa_n) (Eq. (dd_7_no_nn)): the FP32 network decides points
            // clearly off the yield surface, an FP64 evaluation the others.
            const e32::NcF nf = e32::ncf(ncp);
            float r32, dr32, Gp32;
            e32::r_slope(yn, mf, nf, (float)ppe, (float)pphi, (float)kn, r32, dr32, Gp32, fbuf, lane);
            const double scale_n = fabs(kn) > 1.0 ? fabs(kn) : 1.0;
            bool load;
            if (fabs((double)r32) > kTrialMargin * scale_n) {
                load = r32 > 0.0f;
            } else {
                r_slope(A.mat, yn, ncp, ppe, pphi, kn, r, dr, Gp, sBuf, lane);
                ++n_eval;
                load = r > 0.0;
                r32 = (float)r;
                dr32 = (float)dr;
                Gp32 = (float)Gp;
            }
            if (load) {
                loading = 1.0;
                // The root in FP32 (the lazily bracketed Newton iteration of the mixed
                // kernel, from the warm start), then FP64: one value-only evaluation and
                // a Newton step with the FP32 slope (its relative error, ~1e-7, times a
                // correction of ~1e-6 leaves ~1e-13), then one full evaluation and a last
                // Newton step; the slope and G' of that evaluation feed the tangent (they
                // change by ~1e-12 relative over the last step).  Where the FP32 root is not
                // close enough, the FP64 bracketed iteration takes over from it.  Both
                // iterations also stop on the next Newton correction |r / r'| (the step test
                // of the safeguarded Newton-bisection; FP32: 2e-6 relative, FP64: 4 ulp) once
                // the root is bracketed within 1e-2 relative or the iteration converges from
                // one side: near full damage r' grows like 1 / f_d, and r itself cannot get
                // below its rounding.  (A wide bracket does not qualify: far past the root,
                // where f_d underflows, r' is huge and the correction meaningless.)
                const float kg = A.kappa_guess ? (float)__ldg(A.kappa_guess + e0 * NQ + p) : (float)kn;
                float k32 = (float)kn;
                int n32 = 0;
                const bool ok32 = e32::bracketed_newton(yn, mf, nf, (float)ppe, (float)pphi, (float)kn, kg, k32, r32,
                                                        dr32, Gp32, n32, fbuf, lane, true);
                bool done = false;
                if (ok32 && isfinite(k32) && (double)k32 >= kn && dr32 < 0.0f) {
                    const double sc = fabs((double)k32) > 1.0 ? fabs((double)k32) : 1.0;
                    const double r0 = r_value(A.mat, yn, ncp, ppe, pphi, (double)k32, sBuf, lane);
                    ++n_eval;
                    if (fabs(r0) <= 1e-4 * sc) {
                        const double k1 = (double)k32 - r0 / (double)dr32;
                        r_slope(A.mat, yn, ncp, ppe, pphi, k1, r, dr, Gp, sBuf, lane);
                        ++n_eval;
                        if (k1 >= kn && fabs(r) <= 1e-9 * sc && dr < 0.0) {
                            const double k2 = fabs(r) <= 1e-13 * sc ? k1 : k1 - r / dr;
                            kappa = k2 >= kn ? k2 : kn;
                            done = true;
                        }
                    }
                }
                if (!done) {
                    // FP64 lazily bracketed Newton iteration from the FP32 result (the
                    // iteration of the FP64 reference path)
                    r_slope(A.mat, yn, ncp, ppe, pphi, kn, r, dr, Gp, sBuf, lane);
                    ++n_eval;
                    const double kgd = isfinite(k32) ? (double)k32 : kn;
                    if (kgd > kn) {
                        kappa = kgd;
                        r_slope(A.mat, yn, ncp, ppe, pphi, kappa, r, dr, Gp, sBuf, lane);
                        ++n_eval;
                    }
                    double lo = kn, hi = kn;
                    bool have_hi = false;
                    if (r > 0.0) lo = kappa;
                    else {
                        hi = kappa;
                        have_hi = true;
                    }
                    double dx_prev = have_hi ? hi - lo : 1.0e30, dx = dx_prev;
                    bool took_newton = false;
                    int it;
                    for (it = 0; it < m.local_max; ++it) {
                        const double scale = fabs(kappa) > 1.0 ? fabs(kappa) : 1.0;
                        const double ulp4 = 4.0 * 2.220446049250313e-16 * scale;
                        if (fabs(r) <= 1e-13 * scale || (have_hi && (hi - lo) <= ulp4)) break;
                        if (fabs(r) <= ulp4 * fabs(dr) &&
                            (have_hi ? (hi - lo) <= 1e-2 * scale : (took_newton && fabs(2.0 * r) <= fabs(dx * dr))))
                            break;
                        const double newton = kappa - r / dr;
                        bool take;
                        if (have_hi) {
                            take = (newton > lo) && (newton < hi) && (fabs(2.0 * r) <= fabs(dx_prev * dr));
                        } else {
                            // forward Newton step, at most a few times the distance covered so far
                            const double cap = 4.0 * ((double)(r > 1e-12 ? r : 1e-12) + (kappa - kn));
                            take = dr < 0.0 && newton > lo && (newton - kappa) <= cap;
                        }
                        dx_prev = dx;
                        took_newton = take;
                        if (take) {
                            dx = kappa - newton;
                            kappa = newton;
                        } else if (have_hi) {
                            dx = 0.5 * (hi - lo);
                            kappa = lo + dx;
                        } else {
                            const double step =
                                2.0 * ((kappa - kn) > (r > 1e-12 ? r : 1e-12) ? (kappa - kn) : (r > 1e-12 ? r : 1e-12));
                            dx = step;
                            kappa = lo + step;
                        }
                        r_slope(A.mat, yn, ncp, ppe, pphi, kappa, r, dr, Gp, sBuf, lane);
                        ++n_eval;
                        if (r > 0.0) {
                            lo = kappa;
                        } else {
                            hi = kappa;
                            have_hi = true;
                        }
                    }
                    if (it >= m.local_max) fail = 1.0;
                }
            }
            if (lane == 0) {
                double *o = sOut + p * 10;
                if (e0 + p / NQ < A.n_elems) atomicAdd(A.counters + 2, n_eval);
                o[0] = kappa;
                o[1] = loading;
                o[2] = Gp;
                o[3] = dr;
                o[4] = fail;
            }
        }
        __syncwarp();

        // ================= qp mode: stress and records =================
        {
            const double *o = sOut + lane * 10;
            const double kappa = o[0];
            const bool loading = o[1] > 0.5;
            if (valid) {
                if (A.kappa_new) A.kappa_new[e_me * NQ + q] = kappa;
                if (A.loading) A.loading[e_me * NQ + q] = loading ? 1 : 0;
                if (o[4] > 0.5) atomicAdd(A.counters, 1);
                if (loading) atomicAdd(A.counters + 1, 1);
            }
            const bool dmg = kappa > m.kappa_d;
            const double fd = dmg ? exp(-m.eta_d * (kappa - m.kappa_d)) : 1.0;
            const double fdp = dmg ? -m.eta_d * fd : 0.0;
            const double ck = loading ? -o[2] / o[3] : 0.0;          // G' / (1 - G' dq/dkappa)
            const double dkdphi = ck * m.qcoef / fd;                  // dq/dphi = qcoef / f_d
            const double J = Jdet;
            // F^-1 = cof(F)^T / J
            double Fi[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
                    Fi[i][j] = (F[i1][j1] * F[i2][j2] - F[i1][j2] * F[i2][j1]) / J;
                }
            double C[3][3], b[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    double s = 0.0, t = 0.0;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        s += F[k][i] * F[k][j];
                        t += F[i][k] * F[j][k];
                    }
                    C[i][j] = s;
                    b[i][j] = t;
                }
            const double I1 = 3.0 + x[0];
            // h = F^-T g, mvec = F^-1 h = C^-1 g
            double hv[3], mv[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) hv[i] = Fi[0][i] * g[0] + Fi[1][i] * g[1] + Fi[2][i] * g[2];
#pragma unroll
            for (int i = 0; i < 3; ++i) mv[i] = Fi[i][0] * hv[0] + Fi[i][1] * hv[1] + Fi[i][2] * hv[2];
            // P = f_d [2 psi_1 F + 2 psi_2 (I1 F - F C) + psi_3 J F^-T] - c_d h (x) m
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int J2 = 0; J2 < 3; ++J2) {
                    double FC = F[i][0] * C[0][J2] + F[i][1] * C[1][J2] + F[i][2] * C[2][J2];
                    double Ph = 2.0 * ps[0] * F[i][J2] + 2.0 * ps[1] * (I1 * F[i][J2] - FC) + ps[2] * J * Fi[J2][i];
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
            rec[Q_PP] = m.beta_d * (1.0 - dkdphi);
            rec[Q_PEN] = m.beta_d * (phi - kappa);
            rec[Q_J] = J;
            if (!valid) rec[Q_JW] = 0.0;
        }
        __syncwarp();

        // ================= row mode: element residual and tangent =================
        for (int pass = 0; pass < EPW / EPR; ++pass) {
            // per (point, node) vectors of the EPR elements of this pass
            for (int t = lane; t < EPR * NQ * NEN; t += 32) {
                const int ee = t / (NQ * NEN), qq = (t / NEN) % NQ, a = t % NEN;
                const double *R0 = sRec + ((pass * EPR + ee) * NQ + qq) * Q_REC;
                double *V = sVec + t * V_REC;
                const double xi[3] = {(qq & 1) ? kGauss : -kGauss, (qq & 2) ? kGauss : -kGauss,
                                      (qq & 4) ? kGauss : -kGauss};
                double Na, dN[3], n[3] = {0.0, 0.0, 0.0};
                ref_shape<DIM>(a, xi, Na, dN);
#pragma unroll
                for (int J = 0; J < DIM; ++J)
#pragma unroll
                    for (int k = 0; k < DIM; ++k) n[J] += dN[k] * R0[Q_JINV + k * 3 + J];
                double f[3], bf[3], nt[3], G2[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    f[i] = R0[Q_F + i * 3] * n[0] + R0[Q_F + i * 3 + 1] * n[1] + R0[Q_F + i * 3 + 2] * n[2];
                    nt[i] = R0[Q_FINV + i] * n[0] + R0[Q_FINV + 3 + i] * n[1] + R0[Q_FINV + 6 + i] * n[2];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    bf[i] = R0[Q_B + i * 3] * f[0] + R0[Q_B + i * 3 + 1] * f[1] + R0[Q_B + i * 3 + 2] * f[2];
#pragma unroll
                for (int i = 0; i < 3; ++i) G2[i] = 2.0 * (R0[Q_I1] * f[i] - bf[i]);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    V[V_N + i] = n[i];
                    V[V_F + i] = f[i];
                    V[V_G2 + i] = G2[i];
                    V[V_NT + i] = nt[i];
                    V[V_PN + i] = 2.0 * R0[Q_PS1] * f[i] + R0[Q_PS2] * G2[i] + R0[Q_PS3J] * nt[i];
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
            double Kr[ND];
#pragma unroll
            for (int c = 0; c < ND; ++c) Kr[c] = 0.0;
            double Rr = 0.0;
            const double cd = m.c_d;
            if (active) {
                for (int qq = 0; qq < NQ; ++qq) {
                    const double *R0 = sRec + (el_local * NQ + qq) * Q_REC;
                    const double *Vq = sVec + (ee * NQ + qq) * NEN * V_REC;
                    const double *Va = Vq + a * V_REC;
                    const double Jw = R0[Q_JW];
                    if (i < DIM) {
                        // r_u,a = P n_a J w (Sec. 3.1)
                        Rr += Jw * (R0[Q_P + i * 3] * Va[V_N] + R0[Q_P + i * 3 + 1] * Va[V_N + 1] +
                                    R0[Q_P + i * 3 + 2] * Va[V_N + 2]);
                        if (!A.tangent) continue;      // residual-only pass: no tangent rows
                        // d2 psi_e/dF2 contracted with grad N_a, grad N_b:
                        //   sum_mn psi_mn G^m_a G^n_b + psi_1 D2(I1) + psi_2 D2(I2) + psi_3 D2(J),
                        // G^1 = 2 F n, G^2 = 2 (I1 F n - F F^T F n), G^3 = J F^-T n,
                        // D2(I1)_ik = 2 (n_a.n_b) d_ik,
                        // D2(I2)_ik = 2 [2 f_a,i f_b,k - f_b,i f_a,k + (I1 n_a.n_b - f_a.f_b) d_ik - (n_a.n_b) b_ik],
                        // D2(J)_ik  = J (nt_a,i nt_b,k - nt_a,k nt_b,i),   f = F n, nt = F^-T n.
                        const double Jd = R0[Q_J];
                        const double Gai[3] = {2.0 * Va[V_F + i], Va[V_G2 + i], Jd * Va[V_NT + i]};
                        const double *HS = R0 + Q_HS;
                        double tn[3];
#pragma unroll
                        for (int nI = 0; nI < 3; ++nI)
                            tn[nI] = HS[sym6(0, nI)] * Gai[0] + HS[sym6(1, nI)] * Gai[1] + HS[sym6(2, nI)] * Gai[2];
                        const double g1 = R0[Q_G1], g2 = R0[Q_G2], g3J = R0[Q_G3J], I1 = R0[Q_I1];
                        const double ck = R0[Q_CK], fdk = R0[Q_FDK];
                        const double hi_ = R0[Q_H + i], mna = Va[V_MN], Pna = Va[V_PN + i];
                        const double fai = Va[V_F + i], ntai = Va[V_NT + i];
#pragma unroll
                        for (int bN = 0; bN < NEN; ++bN) {
                            const double *Vb = Vq + bN * V_REC;
                            const double nn = Va[V_N] * Vb[V_N] + Va[V_N + 1] * Vb[V_N + 1] + Va[V_N + 2] * Vb[V_N + 2];
                            const double ff = Va[V_F] * Vb[V_F] + Va[V_F + 1] * Vb[V_F + 1] + Va[V_F + 2] * Vb[V_F + 2];
                            const double tt =
                                Va[V_NT] * Vb[V_NT] + Va[V_NT + 1] * Vb[V_NT + 1] + Va[V_NT + 2] * Vb[V_NT + 2];
                            const double mnb = Vb[V_MN], ntbi = Vb[V_NT + i], fbi = Vb[V_F + i];
#pragma unroll
                            for (int k = 0; k < DIM; ++k) {
                                const double fbk = Vb[V_F + k], ntbk = Vb[V_NT + k];
                                double v = tn[0] * 2.0 * fbk + tn[1] * Vb[V_G2 + k] + tn[2] * Jd * ntbk;
                                if (k == i) v += 2.0 * g1 * nn + 2.0 * g2 * (I1 * nn - ff);
                                v += 2.0 * g2 * (2.0 * fai * fbk - fbi * Va[V_F + k] - nn * R0[Q_B + i * 3 + k]);
                                v += g3J * (ntai * ntbk - Va[V_NT + k] * ntbi);
                                v += ck * Pna * Vb[V_PN + k];
                                v += cd * (mna * ntbi * R0[Q_H + k] + tt * hi_ * R0[Q_H + k] + mnb * hi_ * Va[V_NT + k]);
                                Kr[bN * NDOF + k] += Jw * v;
                            }
                            Kr[bN * NDOF + DIM] += Jw * (-cd * (mna * ntbi + hi_ * tt) + fdk * Pna * Vb[V_NN]);
                        }
                    } else {
                        // R_phi,a = (Y . grad N_a - Y N_a) J w, Y vec = c_d C^-1 grad phi, -Y = beta_d (phi - kappa)
                        const double Na = Va[V_NN];
                        Rr += Jw * (cd * Va[V_MN] + R0[Q_PEN] * Na);
                        if (!A.tangent) continue;
                        const double bck = R0[Q_BCK], pp = R0[Q_PP];
#pragma unroll
                        for (int bN = 0; bN < NEN; ++bN) {
                            const double *Vb = Vq + bN * V_REC;
                            const double tt =
                                Va[V_NT] * Vb[V_NT] + Va[V_NT + 1] * Vb[V_NT + 1] + Va[V_NT + 2] * Vb[V_NT + 2];
                            const double mnb = Vb[V_MN];
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
                if (A.R) atomicAdd(A.R + rdof, Rr);
                if (A.tangent) {
                    const int32_t rb = __ldg(A.rowptr + (int64_t)na * NDOF);
                    const int32_t rowlen = __ldg(A.rowptr + (int64_t)na * NDOF + 1) - rb;
                    const int32_t *sl = A.slot + (e * NEN + a) * NEN;
#pragma unroll
                    for (int bN = 0; bN < NEN; ++bN) {
                        const int64_t pos = (int64_t)__ldg(sl + bN) + (int64_t)i * rowlen;
#pragma unroll
                        for (int k = 0; k < NDOF; ++k) {
                            if (A.vals) atomicAdd(A.vals + pos + k, Kr[bN * NDOF + k]);
                            else atomicAdd(A.vals32 + pos + k, (float)Kr[bN * NDOF + k]);
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
    return scratch * sizeof(double);          // per warp
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
    cudaError_t err = cudaFuncSetAttribute(asm_fp64_kernel<DIM, KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, asm_fp64_kernel<DIM, KW>, 32 * KW, sm);
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
    asm_fp64_kernel<DIM, KW><<<(unsigned)grid, 32 * KW, sm, s>>>(a);
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

cudaError_t launch_assemble_fp64(int dim, const AsmArgs &a, int num_sms, cudaStream_t s, const AsmTune &t)
{
    if (a.n_elems <= 0) return cudaSuccess;
    return dim == 2 ? launch_dim<2>(a, num_sms, t, s) : launch_dim<3>(a, num_sms, t, s);
}

// ---------------------------------------------------------------------------
// network constants: N(0), n (S(C=I) = 0), N_k(0), s = 1/N_k'(0)  (Sec. 4.2)
// ---------------------------------------------------------------------------
namespace {
__global__ void prep_nets_kernel(DevNet psi, DevNet yld, int energy, NetConst *out)
{
    __shared__ double buf[5 * kMaxWidth];
    const int lane = threadIdx.x;
    NetConst nc;
    nc.psi_N0 = 0.0;
    nc.psi_n = 0.0;
    nc.y_N0 = 0.0;
    nc.y_s = 1.0;
    if (energy != GD_ENERGY_NEO_HOOKE && psi.width > 0) {
        double x0[3] = {0.0, 0.0, 0.0}, o[10];
        psi_net_unit(psi, x0, o, buf, lane);
        nc.psi_N0 = o[0];
        // dI1/dC = I, dI2/dC = 2 I, dJ/dC = I/2 at C = I (raw); dI1G/dC = dI2G/dC = 0 (Eq. (dd_1))
        nc.psi_n = (energy == GD_ENERGY_ICNN_RAW) ? 2.0 * o[1] + 4.0 * o[2] + o[3] : o[3];
    }
    if (yld.width > 0) {
        NetConst unit;
        unit.y_N0 = 0.0;
        unit.y_s = 1.0;
        double G, Gp;
        yield_unit(yld, unit, 0.0, G, Gp, buf, lane);   // raw N_k(0), N_k'(0)
        nc.y_N0 = G;
        nc.y_s = 1.0 / Gp;
    }
    if (lane == 0) *out = nc;
}

__global__ void transpose_kernel(const double *W2, double *W2T, int w)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < w * w) {
        int k = t / w, j = t % w;
        W2T[j * w + k] = W2[k * w + j];
    }
}
}  // namespace

cudaError_t launch_prep_nets(const DevNet &psi, const DevNet &yld, int energy, NetConst *out, cudaStream_t s)
{
    prep_nets_kernel<<<1, 32, 0, s>>>(psi, yld, energy, out);
    return cudaGetLastError();
}

namespace {
__global__ void to_float_kernel(const double *in, float *out, int n)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = (float)in[t];
}
}  // namespace

cudaError_t launch_net_to_float(const DevNet &net, cudaStream_t s)
{
    if (net.width <= 0) return cudaSuccess;
    to_float_kernel<<<(net.n_params + 255) / 256, 256, 0, s>>>(net.p, net.pf, net.n_params);
    const int ww = net.width * net.width;
    to_float_kernel<<<(ww + 255) / 256, 256, 0, s>>>(net.W2T, net.W2Tf, ww);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const DevNet &net, cudaStream_t s)
{
    if (net.width <= 0) return cudaSuccess;
    const int w = net.width;
    const double *W2 = net.p + w * net.n_in + w;
    transpose_kernel<<<(w * w + 255) / 256, 256, 0, s>>>(W2, net.W2T, w);
    return cudaGetLastError();
}

}  // namespace gd
