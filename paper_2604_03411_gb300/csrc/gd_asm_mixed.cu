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

#include "gd_elem32.cuh"

namespace gd {
namespace {

using namespace e32;

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

template <int DIM, int KW>
__global__ void __launch_bounds__(32 * KW) asm_fp32_kernel(AsmArgs A)
{
    using G_ = Geo<DIM>;
    constexpr int NEN = G_::NEN, NQ = G_::NQ, NDOF = G_::NDOF, EPW = G_::EPW;
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
        load_nodes<DIM>(A, e0, sX, sD, lane);
        __syncwarp();

        // ================= qp mode: kinematics and invariants =================
        const int el = lane / NQ, q = lane % NQ;
        const int64_t e_me = e0 + el;
        const bool valid = e_me < A.n_elems;
        const NcF nc = ncf(A.netc[valid ? spec_of(A, e_me) : 0]);
        float *rec = sRec + lane * Q_REC;
        float F[3][3], H[3][3], phi, g[3], x[3], Jdet;
        qp_kinematics<DIM>(sX, sD, el, q, rec, F, H, phi, g, x, Jdet);
        // network input (raw or isochoric map)
        float Tm[3][3], T2[3][6];   // dy/dx and d2y/dx2 of the iso map (raw: identity)
        {
            float y[3];
            input_map(m, x, Jdet, Tm, T2, y);
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
        energy_derivs(m, nc, x, Jdet, sOut + lane * 10, Tm, T2, ps, ph, pe);
        sIn[lane * 4 + 0] = pe;
        sIn[lane * 4 + 1] = phi;
        sIn[lane * 4 + 2] = valid ? (float)__ldg(A.kappa_n + e_me * NQ + q) : 0.0f;
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
                const float kg = A.kappa_guess ? (float)__ldg(A.kappa_guess + e0 * NQ + p) : kn;
                if (!bracketed_newton(yn, m, ncp, ppe, pphi, kn, kg, kappa, r, dr, Gp, n_eval, sBuf, lane)) fail = 1.0f;
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
            stress_records(m, F, x, g, phi, Jdet, ps, ph, kappa, loading, o[2], o[3], valid, rec);
        }
        __syncwarp();

        // ================= row mode: element residual and tangent =================
        row_mode<DIM>(A, m, sRec, sVec, e0, lane);
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
