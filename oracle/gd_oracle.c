/*
 * gd_oracle.c -- plain, slow FP64 CPU oracle for the gradient-enhanced damage
 * element computation with ICNN constitutive laws (arxiv 2604.03411).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * Derivatives are taken with hyper-dual numbers (v + a e1 + b e2 + ab e1 e2,
 * e1^2 = e2^2 = 0): the first and second derivatives of the scalar free
 * energy and of the yield residual are exact to rounding and come from the
 * arithmetic itself, never from hand-derived stress or tangent formulas.
 *
 * Paper sections followed (function by function, cited where used):
 *   Sec. 2.1, Eq. (internal_energy)        -- free energy split
 *   Sec. 2.1, conjugates P, Y (vector), Y  -- stress and non-local fluxes
 *   Sec. 2.2, Eqs. (damage_function), (q_q_loc_q_nloc), (potential_function),
 *             (flow_rule), (KKT)           -- local damage evolution
 *   Sec. 3.1, Table (kernel_inputs)        -- element kernel inputs
 *   Sec. 3.1                               -- F, phi_q, grad phi_q, element residual
 *   Sec. 3.2, Eq. (dd_7_no_nn)             -- local update equations
 *   Sec. 3.2 (monolithic scheme)           -- kappa updated inside every global iteration
 *   Sec. 4.1, Eqs. (degradation_function), (ostwald_potential) and the
 *             gradient/penalty energies    -- closed-form pieces
 *   Sec. 4.2, Eqs. (dd_0), (dd_1), (Gq_NN), (dd_3), (dd_7) -- PANN model
 *
 * Readings where the paper is silent or garbled (each also listed in the
 * design notes): the ICNN architecture (two softplus layers with an input
 * skip, nonnegative weights); G(q) = s (N_k(q) - N_k(0)) with s = 1/N_k'(0);
 * q_nloc = gamma_d beta_d (phi - kappa) / (eta_d f_d(kappa)) for every kappa;
 * f_d' = 0 for kappa <= kappa_d; the extra lambda_e in dpsi_vol/dC of Eq.
 * (dd_1) is a typo; the normalising term -n (J - 1) that keeps S(C=I) = 0
 * when J - 1 is an ICNN input.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* hyper-dual numbers                                                  */
/* ------------------------------------------------------------------ */
typedef struct { double v, a, b, ab; } hd;

static hd hc(double v) { hd r = {v, 0.0, 0.0, 0.0}; return r; }
static hd hadd(hd x, hd y) { hd r = {x.v + y.v, x.a + y.a, x.b + y.b, x.ab + y.ab}; return r; }
static hd hsub(hd x, hd y) { hd r = {x.v - y.v, x.a - y.a, x.b - y.b, x.ab - y.ab}; return r; }
static hd hscale(hd x, double s) { hd r = {x.v * s, x.a * s, x.b * s, x.ab * s}; return r; }
static hd hmul(hd x, hd y)
{
    hd r = {x.v * y.v, x.v * y.a + x.a * y.v, x.v * y.b + x.b * y.v,
            x.v * y.ab + x.a * y.b + x.b * y.a + x.ab * y.v};
    return r;
}
/* f(x) given f, f', f'' at x.v */
static hd hfun(hd x, double f0, double f1, double f2)
{
    hd r = {f0, f1 * x.a, f1 * x.b, f1 * x.ab + f2 * x.a * x.b};
    return r;
}
static hd hinv(hd x) { double i = 1.0 / x.v; return hfun(x, i, -i * i, 2.0 * i * i * i); }
static hd hdiv(hd x, hd y) { return hmul(x, hinv(y)); }
static hd hexp(hd x) { double e = exp(x.v); return hfun(x, e, e, e); }
static hd hexpm1(hd x) { double e = exp(x.v); return hfun(x, expm1(x.v), e, e); }
static hd hlog1p(hd x) { double i = 1.0 / (1.0 + x.v); return hfun(x, log1p(x.v), i, -i * i); }
static hd hsq(hd x) { return hmul(x, x); }

static double sigmoid(double v)
{
    if (v >= 0.0) return 1.0 / (1.0 + exp(-v));
    double e = exp(v);
    return e / (1.0 + e);
}
static double softplus(double v) { return (v > 0.0 ? v : 0.0) + log1p(exp(-fabs(v))); }
static hd hsoftplus(hd x)
{
    double s = sigmoid(x.v);
    return hfun(x, softplus(x.v), s, s * (1.0 - s));
}

/* ------------------------------------------------------------------ */
/* material                                                            */
/* ------------------------------------------------------------------ */
enum { OR_ICNN_RAW = 0, OR_ICNN_ISO = 1, OR_NEO_HOOKE = 2 };

typedef struct {
    int dim;          /* 2: plane strain (F33 = 1), 3: solid */
    int energy;       /* OR_ICNN_RAW | OR_ICNN_ISO | OR_NEO_HOOKE */
    double mu_e, lambda_e, eta_d, kappa_d, beta_d, c_d, gamma_d;
    int psi_w, y_w;   /* ICNN widths */
    const double *psi_p, *y_p;
    int local_max;    /* cap on local (kappa) iterations */
    /* filled by or_prepare */
    double psi_N0, psi_n, y_N0, y_s;
    /* derivatives with respect to the network weights (the discrete adjoint's
     * element sensitivities): when seeded != 0 the networks read their parameters
     * from the hyper-dual copies psi_ph / y_ph, one entry of which carries a unit
     * derivative, and the normalising constants from the hyper-dual c_* */
    int seeded;
    const hd *psi_ph, *y_ph;
    hd c_N0, c_n, c_yN0, c_ys;
    /* frozen != 0: the history passed as kappa_n is kappa_{n+1} itself, with no local
     * update and no kappa sensitivity in the tangent (the global solve of the staggered
     * scheme, Sec. 3.2, where the history is advanced apart from the nodal solve) */
    int frozen;
} or_mat;

/* Two-layer input-convex network (Amos et al.), softplus activations, input
 * skip connections into the second layer and the output (Sec. 4.2, the ICNN
 * cited for psi_iso and the increasing N_kappa).  Packed parameters:
 * W1[w][n_in] b1[w] W2[w][w] A2[w][n_in] b2[w] w3[w] a3[n_in]. */
static hd icnn(const double *p, int n_in, int w, const hd *x)
{
    const double *W1 = p, *b1 = W1 + w * n_in, *W2 = b1 + w, *A2 = W2 + w * w,
                 *b2 = A2 + w * n_in, *w3 = b2 + w, *a3 = w3 + w;
    hd z1[256];
    for (int j = 0; j < w; ++j) {
        hd h = hc(b1[j]);
        for (int i = 0; i < n_in; ++i) h = hadd(h, hscale(x[i], W1[j * n_in + i]));
        z1[j] = hsoftplus(h);
    }
    hd out = hc(0.0);
    for (int i = 0; i < n_in; ++i) out = hadd(out, hscale(x[i], a3[i]));
    for (int k = 0; k < w; ++k) {
        hd h = hc(b2[k]);
        for (int j = 0; j < w; ++j) h = hadd(h, hscale(z1[j], W2[k * w + j]));
        for (int i = 0; i < n_in; ++i) h = hadd(h, hscale(x[i], A2[k * n_in + i]));
        out = hadd(out, hscale(hsoftplus(h), w3[k]));
    }
    return out;
}

/* The same network with hyper-dual parameters (weight derivatives). */
static hd icnn_p(const hd *p, int n_in, int w, const hd *x)
{
    const hd *W1 = p, *b1 = W1 + w * n_in, *W2 = b1 + w, *A2 = W2 + w * w, *b2 = A2 + w * n_in, *w3 = b2 + w,
             *a3 = w3 + w;
    hd z1[256];
    for (int j = 0; j < w; ++j) {
        hd h = b1[j];
        for (int i = 0; i < n_in; ++i) h = hadd(h, hmul(x[i], W1[j * n_in + i]));
        z1[j] = hsoftplus(h);
    }
    hd out = hc(0.0);
    for (int i = 0; i < n_in; ++i) out = hadd(out, hmul(x[i], a3[i]));
    for (int k = 0; k < w; ++k) {
        hd h = b2[k];
        for (int j = 0; j < w; ++j) h = hadd(h, hmul(z1[j], W2[k * w + j]));
        for (int i = 0; i < n_in; ++i) h = hadd(h, hmul(x[i], A2[k * n_in + i]));
        out = hadd(out, hmul(hsoftplus(h), w3[k]));
    }
    return out;
}

static hd det3(hd M[3][3])
{
    hd t0 = hsub(hmul(M[1][1], M[2][2]), hmul(M[1][2], M[2][1]));
    hd t1 = hsub(hmul(M[1][0], M[2][2]), hmul(M[1][2], M[2][0]));
    hd t2 = hsub(hmul(M[1][0], M[2][1]), hmul(M[1][1], M[2][0]));
    return hadd(hsub(hmul(M[0][0], t0), hmul(M[0][1], t1)), hmul(M[0][2], t2));
}

/* Strain measures from the displacement gradient H (F = I + H).
 * C - I = H + H^T + H^T H  (no O(1) term, so nothing cancels at small strain)
 * I1 - 3 = tr(C - I)
 * I2 - 3 = 2 tr(C - I) + (tr(C-I)^2 - tr((C-I)^2)) / 2    [I2 = tr cof C]
 * J - 1  = tr H + (tr(H)^2 - tr(H H)) / 2 + det H          [det(I + H) expanded]
 * (Sec. 4.2, Eq. (dd_0): I1 = tr C, I2 = tr cof C, J = det F.) */
static void raw_invariants(hd H[3][3], hd x[3], hd A[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            hd s = hadd(H[i][j], H[j][i]);
            for (int k = 0; k < 3; ++k) s = hadd(s, hmul(H[k][i], H[k][j]));
            A[i][j] = s;
        }
    hd a = hadd(hadd(A[0][0], A[1][1]), A[2][2]);
    hd AA = hc(0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) AA = hadd(AA, hmul(A[i][j], A[j][i]));
    x[0] = a;
    x[1] = hadd(hscale(a, 2.0), hscale(hsub(hsq(a), AA), 0.5));
    hd trH = hadd(hadd(H[0][0], H[1][1]), H[2][2]);
    hd HH = hc(0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) HH = hadd(HH, hmul(H[i][j], H[j][i]));
    x[2] = hadd(hadd(trH, hscale(hsub(hsq(trH), HH), 0.5)), det3(H));
}

/* Undamaged strain energy psi_e(C) (the local driving force q_loc, Sec. 2.2).
 *  ICNN_RAW:  mu_e [N(x) - N(0) - n (J-1)] + lambda_e (J + 1/J - 2)^2, x = (I1-3, I2-3, J-1)
 *  ICNN_ISO:  same with x = (I1G-3, I2G-3, J-1), I1G = J^(-2/3) I1, I2G = I2^3/(9 J^4)
 *             (Eq. (dd_0); with the J-column of the weights zero this is exactly
 *             f_d-free part of Eq. (dd_0), since then n = 0)
 *  NEO_HOOKE: mu/2 (I1-3) - mu ln J + lambda/2 (ln J)^2   (Sec. 4.1)
 * n is chosen so that S = 2 dpsi/dC vanishes at C = I (stress normality). */
static hd psi_e(const or_mat *m, hd H[3][3])
{
    hd x[3], A[3][3];
    raw_invariants(H, x, A);
    if (m->energy == OR_NEO_HOOKE) {
        hd lnJ = hlog1p(x[2]);
        return hadd(hsub(hscale(x[0], 0.5 * m->mu_e), hscale(lnJ, m->mu_e)),
                    hscale(hsq(lnJ), 0.5 * m->lambda_e));
    }
    hd xi[3] = {x[0], x[1], x[2]};
    if (m->energy == OR_ICNN_ISO) {
        hd L = hlog1p(x[2]);                                     /* ln J */
        hd e = hexp(hscale(L, -2.0 / 3.0));                      /* J^(-2/3) */
        /* I1G - 3 = 3 (J^(-2/3) - 1) + (I1 - 3) J^(-2/3) */
        xi[0] = hadd(hscale(hexpm1(hscale(L, -2.0 / 3.0)), 3.0), hmul(x[0], e));
        /* I2G - 3 = 3 ((I2/3)^3 J^(-4) - 1) */
        xi[1] = hscale(hexpm1(hsub(hscale(hlog1p(hscale(x[1], 1.0 / 3.0)), 3.0), hscale(L, 4.0))), 3.0);
    }
    hd N, iso;
    if (m->seeded) {
        N = icnn_p(m->psi_ph, 3, m->psi_w, xi);
        iso = hsub(hsub(N, m->c_N0), hmul(x[2], m->c_n));
    } else {
        N = icnn(m->psi_p, 3, m->psi_w, xi);
        iso = hsub(hsub(N, hc(m->psi_N0)), hscale(x[2], m->psi_n));
    }
    /* psi_vol = (J + 1/J - 2)^2 = ((J-1)^2 / J)^2 */
    hd t = hdiv(hsq(x[2]), hadd(hc(1.0), x[2]));
    return hadd(hscale(iso, m->mu_e), hscale(hsq(t), m->lambda_e));
}

/* f_d(kappa) = exp(-eta_d <kappa - kappa_d>_+) = 1 - d   (Eq. (degradation_function));
 * on kappa <= kappa_d it is the constant 1. */
static hd degradation(const or_mat *m, hd kappa)
{
    if (kappa.v > m->kappa_d) return hexp(hscale(hsub(kappa, hc(m->kappa_d)), -m->eta_d));
    return hc(1.0);
}

/* qp variables z = (H_iJ for i,J < dim row-major, phi, (grad phi)_J for J < dim) */
static int nz_of(int dim) { return dim * dim + 1 + dim; }

static void unpack_z(const or_mat *m, const hd *z, hd H[3][3], hd *phi, hd g[3])
{
    int d = m->dim;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[i][j] = hc(0.0);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) H[i][j] = z[i * d + j];
    *phi = z[d * d];
    for (int j = 0; j < 3; ++j) g[j] = (j < d) ? z[d * d + 1 + j] : hc(0.0);
}

/* Psi_int(F, phi, grad phi, kappa) = f_d(kappa) psi_e(C) + c_d/2 gradphi . C^-1 . gradphi
 *                                   + beta_d/2 (phi - kappa)^2
 * (Eq. (internal_energy) with the gradient and penalty terms of Sec. 4.1, Eq. (dd_3)). */
static hd Psi(const or_mat *m, const hd *z, hd kappa)
{
    hd H[3][3], phi, g[3];
    unpack_z(m, z, H, &phi, g);
    hd pe = psi_e(m, H);
    /* C = F^T F, C^-1 = adj(C) / det(C) */
    hd C[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            hd s = hc(0.0);
            for (int k = 0; k < 3; ++k) {
                hd Fki = hadd(H[k][i], hc(k == i ? 1.0 : 0.0));
                hd Fkj = hadd(H[k][j], hc(k == j ? 1.0 : 0.0));
                s = hadd(s, hmul(Fki, Fkj));
            }
            C[i][j] = s;
        }
    hd detC = det3(C);
    hd adj[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
            adj[i][j] = hsub(hmul(C[i1][j1], C[i2][j2]), hmul(C[i1][j2], C[i2][j1]));
        }
    hd gCg = hc(0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) gCg = hadd(gCg, hmul(hmul(g[i], adj[i][j]), g[j]));
    gCg = hdiv(gCg, detC);
    hd fd = degradation(m, kappa);
    hd dk = hsub(phi, kappa);
    return hadd(hadd(hmul(fd, pe), hscale(gCg, 0.5 * m->c_d)), hscale(hsq(dk), 0.5 * m->beta_d));
}

/* Driving force conjugate to d (Eq. (q_q_loc_q_nloc)):
 *   q = q_loc + q_nloc,  q_loc = psi_e (Sec. 2.2),
 *   q_nloc = gamma_d beta_d (phi - kappa) / (eta_d f_d(kappa))  (Eq. (ostwald_potential)). */
static hd q_force(const or_mat *m, hd pe, hd phi, hd kappa)
{
    hd q = pe;
    if (m->gamma_d != 0.0 && m->beta_d != 0.0) {
        double c = m->gamma_d * m->beta_d / m->eta_d;
        q = hadd(q, hscale(hdiv(hsub(phi, kappa), degradation(m, kappa)), c));
    }
    return q;
}

/* Yield function G(q) = s (N_k(q) - N_k(0)), s = 1/N_k'(0): increasing, G(0)=0, G'(0)=1
 * (Eq. (Gq_NN); the argument of N_k is q).  Width 0 selects G(q) = q, the
 * closed-form loading function of Eq. (ostwald_potential). */
static hd yield_G(const or_mat *m, hd q)
{
    if (m->y_w == 0) return q;      /* closed-form model: Phi_d = q - kappa (Eq. (ostwald_potential)) */
    if (m->seeded) return hmul(hsub(icnn_p(m->y_ph, 1, m->y_w, &q), m->c_yN0), m->c_ys);
    hd N = icnn(m->y_p, 1, m->y_w, &q);
    return hscale(hsub(N, hc(m->y_N0)), m->y_s);
}

/* r(z, kappa) = Phi_d = G(q(z, kappa)) - kappa  (Eq. (potential_function)) */
static hd yield_residual(const or_mat *m, const hd *z, hd kappa)
{
    hd H[3][3], phi, g[3];
    unpack_z(m, z, H, &phi, g);
    hd pe = psi_e(m, H);
    return hsub(yield_G(m, q_force(m, pe, phi, kappa)), kappa);
}

/* ------------------------------------------------------------------ */
/* preparation: N(0), n, N_k(0), s                                     */
/* ------------------------------------------------------------------ */
int or_prepare(or_mat *m)
{
    m->psi_N0 = 0.0; m->psi_n = 0.0; m->y_N0 = 0.0; m->y_s = 1.0;
    if (m->energy != OR_NEO_HOOKE) {
        hd x[3] = {hc(0.0), hc(0.0), hc(0.0)};
        m->psi_N0 = icnn(m->psi_p, 3, m->psi_w, x).v;
        double dN[3];
        for (int i = 0; i < 3; ++i) {
            hd xx[3] = {hc(0.0), hc(0.0), hc(0.0)};
            xx[i].a = 1.0;
            dN[i] = icnn(m->psi_p, 3, m->psi_w, xx).a;
        }
        /* S(C = I) = 0: dI1/dC = I, dI2/dC = 2 I, dJ/dC = I/2 at C = I (raw map);
         * dI1G/dC = dI2G/dC = 0 at C = I (Eq. (dd_1)), so only the J column remains. */
        if (m->energy == OR_ICNN_RAW) m->psi_n = 2.0 * dN[0] + 4.0 * dN[1] + dN[2];
        else m->psi_n = dN[2];
    }
    if (m->y_w == 0) return 0;
    hd q0 = hc(0.0);
    q0.a = 1.0;
    hd N = icnn(m->y_p, 1, m->y_w, &q0);
    m->y_N0 = N.v;
    if (!(N.a > 0.0)) return -1;
    m->y_s = 1.0 / N.a;
    return 0;
}

/* ------------------------------------------------------------------ */
/* local damage update at one qp (Sec. 3.2, Eqs. (dd_7_no_nn), (dd_7), (KKT)) */
/* ------------------------------------------------------------------ */
typedef struct {
    double kappa, dlam, q, Phi_trial, fd;
    int loading, iters, fail;
} or_qp_info;

static double r_at(const or_mat *m, const double *z, double kappa)
{
    hd zz[13];
    int nz = nz_of(m->dim);
    for (int c = 0; c < nz; ++c) zz[c] = hc(z[c]);
    return yield_residual(m, zz, hc(kappa)).v;
}
static double dr_dkappa(const or_mat *m, const double *z, double kappa)
{
    hd zz[13];
    int nz = nz_of(m->dim);
    for (int c = 0; c < nz; ++c) zz[c] = hc(z[c]);
    hd k = hc(kappa);
    k.a = 1.0;
    return yield_residual(m, zz, k).a;
}

/* Trial state: Phi_d(kappa_n) <= 0 is elastic (kappa_{n+1} = kappa_n).  Otherwise
 * kappa_{n+1} solves r(kappa) = Phi_d = G(q(kappa)) - kappa = 0 on kappa > kappa_n
 * (Eq. (dd_7_no_nn) with Delta lambda eliminated):
 *   1. bracket: hi = kappa_n + s with s = max(Phi_trial, 1e-12), doubling s while
 *      r(hi) > 0 (at most 200 times); lo = the last point with r > 0;
 *   2. safeguarded Newton from lo: a Newton step is taken only if it lands inside
 *      (lo, hi) and is at most half as long as the step before it, otherwise the
 *      bracket is bisected (the rule of the "rtsafe" scheme of Numerical Recipes);
 *      the bracket is updated from the sign of r after every step;
 *   3. stop when |r| <= 1e-13 max(1, |kappa|) or the bracket is narrower than
 *      4 eps max(1, |kappa|), at most local_max iterations (the paper caps the
 *      local Newton at 100 iterations, Sec. 5.3).
 * Delta lambda = (kappa_{n+1} - kappa_n) / G'(q) (first line of Eq. (dd_7)). */
static void r_and_slope(const or_mat *m, const double *z, double kappa, double *r, double *dr)
{
    hd zz[13];
    int nz = nz_of(m->dim);
    for (int c = 0; c < nz; ++c) zz[c] = hc(z[c]);
    hd k = hc(kappa);
    k.a = 1.0;
    hd v = yield_residual(m, zz, k);
    *r = v.v;
    *dr = v.a;
}

static void local_update(const or_mat *m, const double *z, double kappa_n, or_qp_info *inf)
{
    memset(inf, 0, sizeof(*inf));
    double r0 = r_at(m, z, kappa_n);
    inf->Phi_trial = r0;
    double kappa = kappa_n;
    if (r0 > 0.0) {
        inf->loading = 1;
        double lo = kappa_n, hi, step = r0 > 1e-12 ? r0 : 1e-12;
        int grow = 0;
        hi = kappa_n + step;
        while (r_at(m, z, hi) > 0.0 && grow < 200) {
            lo = hi;
            step *= 2.0;
            hi = kappa_n + step;
            ++grow;
        }
        if (grow >= 200) inf->fail = 1;
        kappa = lo;
        double r, dr;
        r_and_slope(m, z, kappa, &r, &dr);
        double dx_prev = hi - lo, dx = dx_prev;
        int it;
        for (it = 0; it < m->local_max; ++it) {
            double scale = fabs(kappa) > 1.0 ? fabs(kappa) : 1.0;
            if (fabs(r) <= 1e-13 * scale || (hi - lo) <= 4.0 * 2.220446049250313e-16 * scale) break;
            double newton = kappa - r / dr;
            int take = (newton > lo) && (newton < hi) && (fabs(2.0 * r) <= fabs(dx_prev * dr));
            dx_prev = dx;
            if (take) {
                dx = kappa - newton;
                kappa = newton;
            } else {
                dx = 0.5 * (hi - lo);
                kappa = lo + dx;
            }
            r_and_slope(m, z, kappa, &r, &dr);
            if (r > 0.0) lo = kappa; else hi = kappa;
        }
        inf->iters = it;
        if (it >= m->local_max) inf->fail = 1;
    }
    inf->kappa = kappa;
    /* diagnostics: q, f_d and Delta lambda at the converged kappa */
    hd zz[13];
    int nz = nz_of(m->dim);
    for (int c = 0; c < nz; ++c) zz[c] = hc(z[c]);
    hd H[3][3], phi, g[3];
    unpack_z(m, zz, H, &phi, g);
    hd q = q_force(m, psi_e(m, H), phi, hc(kappa));
    hd qd = q;
    qd.a = 1.0;
    double Gp = yield_G(m, qd).a;
    inf->q = q.v;
    inf->fd = degradation(m, hc(kappa)).v;
    inf->dlam = inf->loading ? (kappa - kappa_n) / Gp : 0.0;
}

/* ------------------------------------------------------------------ */
/* qp: first derivatives (conjugates) and consistent second derivatives */
/* ------------------------------------------------------------------ */
/* dPsi[c] = dPsi/dz_c at fixed kappa_{n+1}: (P_iJ, -Y, Y_vec_J)  (Sec. 2.1 conjugates)
 * D[c][e] = d(dPsi/dz_c)/dz_e including kappa_{n+1}(z) through the implicit
 *           function theorem on Phi_d = 0 when the point is loading
 *           (monolithic scheme, Sec. 3.2).
 * With D == NULL only the first derivatives are formed. */
static void qp_eval(const or_mat *m, const double *z, double kappa_n, double *dPsi, double *D, or_qp_info *inf)
{
    int nz = nz_of(m->dim);
    if (m->frozen) {
        memset(inf, 0, sizeof(*inf));
        inf->kappa = kappa_n;            /* not loading: D gets no implicit-function term */
    } else {
        local_update(m, z, kappa_n, inf);
    }
    hd zz[13];
    for (int c = 0; c < nz; ++c) {
        for (int e = 0; e < nz; ++e) zz[e] = hc(z[e]);
        zz[c].a = 1.0;
        dPsi[c] = Psi(m, zz, hc(inf->kappa)).a;
    }
    if (!D) return;
    for (int c = 0; c < nz; ++c)
        for (int e = c; e < nz; ++e) {
            for (int f = 0; f < nz; ++f) zz[f] = hc(z[f]);
            zz[c].a = 1.0;
            zz[e].b = 1.0;
            double v = Psi(m, zz, hc(inf->kappa)).ab;
            D[c * nz + e] = v;
            D[e * nz + c] = v;
        }
    if (inf->loading) {
        double drk = dr_dkappa(m, z, inf->kappa);
        double mixed[13], dkdz[13];
        for (int c = 0; c < nz; ++c) {
            for (int f = 0; f < nz; ++f) zz[f] = hc(z[f]);
            zz[c].a = 1.0;
            hd k = hc(inf->kappa);
            k.b = 1.0;
            mixed[c] = Psi(m, zz, k).ab;                         /* d2 Psi / dz_c dkappa */
            dkdz[c] = -yield_residual(m, zz, hc(inf->kappa)).a / drk; /* IFT */
        }
        for (int c = 0; c < nz; ++c)
            for (int e = 0; e < nz; ++e) D[c * nz + e] += mixed[c] * dkdz[e];
    }
}

/* ------------------------------------------------------------------ */
/* isoparametric elements: Q4 (2x2 Gauss) and HEX8 (2x2x2 Gauss)       */
/* ------------------------------------------------------------------ */
/* node order: Q4 (-1,-1) (1,-1) (1,1) (-1,1); HEX8 the same on z = -1 then z = +1.
 * qp order: lexicographic with xi fastest, points -1/sqrt3, +1/sqrt3, weights 1. */
static const double NODE_SGN[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                      {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

static int nen_of(int dim) { return dim == 2 ? 4 : 8; }
static int nq_of(int dim) { return dim == 2 ? 4 : 8; }

/* N_a, grad_X N_a and J_q w_q at qp q of an element with node coordinates Xe[a*dim + J] */
static int shape_at(int dim, const double *Xe, int q, double *N, double dN[][3], double *Jw)
{
    int nen = nen_of(dim);
    double gp = 1.0 / sqrt(3.0);
    double xi[3] = {(q & 1) ? gp : -gp, (q & 2) ? gp : -gp, (q & 4) ? gp : -gp};
    double dNr[8][3];
    for (int a = 0; a < nen; ++a) {
        double f[3];
        for (int k = 0; k < dim; ++k) f[k] = 0.5 * (1.0 + NODE_SGN[a][k] * xi[k]);
        double Na = 1.0;
        for (int k = 0; k < dim; ++k) Na *= f[k];
        N[a] = Na;
        for (int k = 0; k < dim; ++k) {
            double v = 0.5 * NODE_SGN[a][k];
            for (int l = 0; l < dim; ++l)
                if (l != k) v *= f[l];
            dNr[a][k] = v;
        }
    }
    double Jm[3][3] = {{0}};                 /* Jm[J][k] = dX_J / dxi_k */
    for (int a = 0; a < nen; ++a)
        for (int J = 0; J < dim; ++J)
            for (int k = 0; k < dim; ++k) Jm[J][k] += Xe[a * dim + J] * dNr[a][k];
    double det, inv[3][3];
    if (dim == 2) {
        det = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
        inv[0][0] = Jm[1][1] / det; inv[0][1] = -Jm[0][1] / det;
        inv[1][0] = -Jm[1][0] / det; inv[1][1] = Jm[0][0] / det;
    } else {
        det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1])
            - Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0])
            + Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
                inv[i][j] = (Jm[i1][j1] * Jm[i2][j2] - Jm[i1][j2] * Jm[i2][j1]) / det;
            }
    }
    if (!(det > 0.0)) return -1;
    /* dN_a/dX_J = sum_k dN_a/dxi_k dxi_k/dX_J, dxi/dX = Jm^-1 */
    for (int a = 0; a < nen; ++a)
        for (int J = 0; J < 3; ++J) {
            double s = 0.0;
            if (J < dim)
                for (int k = 0; k < dim; ++k) s += dNr[a][k] * inv[k][J];
            dN[a][J] = s;
        }
    *Jw = det;
    return 0;
}

/* Element residual and consistent tangent (Sec. 3.1):
 *   r_u,a   = sum_q P_q grad N_a J_q w_q
 *   R_phi,a = sum_q (Y_q . grad N_a - Y_q N_a) J_q w_q
 *   K^e     = dR^e / d(u, phi)  (kappa_{n+1} an implicit function of the dofs)
 * Element dofs de[a*ndof + c]: c < dim displacement, c = dim the non-local phi.
 * Outputs: Re[nd], Ke[nd*nd] (row-major, may be NULL), kappa_new[nq], qinfo[nq*6]
 * (kappa, Delta lambda, q, Phi_trial, f_d, loading) may be NULL. Returns the
 * number of local-solve failures, or -1 for a non-positive Jacobian. */
int or_element(const or_mat *m, const double *Xe, const double *de, const double *kappa_n,
               double *Re, double *Ke, double *kappa_new, double *qinfo)
{
    int dim = m->dim, nen = nen_of(dim), nq = nq_of(dim), ndof = dim + 1, nd = nen * ndof;
    int nz = nz_of(dim), fails = 0;
    memset(Re, 0, sizeof(double) * nd);
    if (Ke) memset(Ke, 0, sizeof(double) * nd * nd);
    for (int q = 0; q < nq; ++q) {
        double N[8], dN[8][3], Jw;
        if (shape_at(dim, Xe, q, N, dN, &Jw)) return -1;
        /* B[c][A] = dz_c / dd_A */
        double B[13][32];
        memset(B, 0, sizeof(B));
        for (int a = 0; a < nen; ++a) {
            for (int i = 0; i < dim; ++i)
                for (int J = 0; J < dim; ++J) B[i * dim + J][a * ndof + i] = dN[a][J];
            B[dim * dim][a * ndof + dim] = N[a];
            for (int J = 0; J < dim; ++J) B[dim * dim + 1 + J][a * ndof + dim] = dN[a][J];
        }
        double z[13];
        for (int c = 0; c < nz; ++c) {
            double s = 0.0;
            for (int A = 0; A < nd; ++A) s += B[c][A] * de[A];
            z[c] = s;
        }
        double dPsi[13], D[169];
        or_qp_info inf;
        qp_eval(m, z, kappa_n[q], dPsi, Ke ? D : NULL, &inf);
        fails += inf.fail;
        if (kappa_new) kappa_new[q] = inf.kappa;
        if (qinfo) {
            double *o = qinfo + 6 * q;
            o[0] = inf.kappa; o[1] = inf.dlam; o[2] = inf.q; o[3] = inf.Phi_trial; o[4] = inf.fd;
            o[5] = inf.loading;
        }
        for (int A = 0; A < nd; ++A) {
            double s = 0.0;
            for (int c = 0; c < nz; ++c) s += B[c][A] * dPsi[c];
            Re[A] += s * Jw;
        }
        if (Ke) {
            double DB[13][32];
            for (int c = 0; c < nz; ++c)
                for (int A = 0; A < nd; ++A) {
                    double s = 0.0;
                    for (int e = 0; e < nz; ++e) s += D[c * nz + e] * B[e][A];
                    DB[c][A] = s;
                }
            for (int A = 0; A < nd; ++A)
                for (int Bi = 0; Bi < nd; ++Bi) {
                    double s = 0.0;
                    for (int c = 0; c < nz; ++c) s += B[c][A] * DB[c][Bi];
                    Ke[A * nd + Bi] += s * Jw;
                }
        }
    }
    return fails;
}

/* Whole-mesh loop of or_element.  R[n_nodes*ndof] is overwritten with the
 * assembled residual; Ke_all[E*nd*nd] receives every element matrix (NULL to
 * skip); kappa_new[E*nq]; qinfo[E*nq*6] optional.  Elements [e0, e1).
 * When built with OpenMP the elements are computed on several threads (each
 * element independently, into its own slots); the element residuals are then
 * added into R one element after another in element order, so R is the same
 * to the last bit for any thread count. */
int64_t or_assemble(const or_mat *m, int64_t n_nodes, int64_t e0, int64_t e1, const int32_t *conn,
                    const double *X, const double *dofs, const double *kappa_n, double *R, double *Ke_all,
                    double *kappa_new, double *qinfo)
{
    int dim = m->dim, nen = nen_of(dim), nq = nq_of(dim), ndof = dim + 1, nd = nen * ndof;
    memset(R, 0, sizeof(double) * (size_t)(n_nodes * ndof));
    if (e1 <= e0) return 0;
    double *Re_all = (double *)malloc(sizeof(double) * (size_t)(e1 - e0) * (size_t)nd);
    if (!Re_all) return -1 - e0;
    int64_t fails = 0, bad = e1;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : fails)
    for (int64_t e = e0; e < e1; ++e) {
        double Xe[24], de[32];
        for (int a = 0; a < nen; ++a) {
            int32_t n = conn[e * nen + a];
            for (int J = 0; J < dim; ++J) Xe[a * dim + J] = X[(int64_t)n * dim + J];
            for (int c = 0; c < ndof; ++c) de[a * ndof + c] = dofs[(int64_t)n * ndof + c];
        }
        int f = or_element(m, Xe, de, kappa_n + e * nq, Re_all + (e - e0) * nd,
                           Ke_all ? Ke_all + (e - e0) * nd * nd : NULL, kappa_new ? kappa_new + e * nq : NULL,
                           qinfo ? qinfo + e * nq * 6 : NULL);
        if (f < 0) {
#pragma omp critical
            if (e < bad) bad = e;
        } else {
            fails += f;
        }
    }
    if (bad < e1) {
        free(Re_all);
        return -1 - bad;
    }
    for (int64_t e = e0; e < e1; ++e) {
        const double *Re = Re_all + (e - e0) * nd;
        for (int a = 0; a < nen; ++a) {
            int32_t n = conn[e * nen + a];
            for (int c = 0; c < ndof; ++c) R[(int64_t)n * ndof + c] += Re[a * ndof + c];
        }
    }
    free(Re_all);
    return fails;
}

/* Number of threads of the element loop (OpenMP builds; 1 otherwise).  n <= 0
 * leaves the setting unchanged.  Returns the number that the loop will use. */
int or_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* element sensitivities for the discrete adjoint of the load path      */
/* ------------------------------------------------------------------ */
static int net_size(int n_in, int w) { return w > 0 ? w * n_in + w + w * w + w * n_in + w + w + n_in : 0; }

/* Seeds weight k of theta = [psi params | yield params] in direction dir (1: the
 * a part, 2: the b part) on m, using the hyper-dual copy ph of theta (set up by the
 * caller, no entry seeded), and forms the normalising constants N(0), n, N_k(0),
 * s = 1/N_k'(0) of or_prepare as hyper-duals carrying their derivative with respect
 * to that weight (n: the weight derivative of 2 dN/dx1 + 4 dN/dx2 + dN/dx3 at 0,
 * raw inputs, or of dN/dx3, isochoric inputs). */
static void seed_weight(or_mat *m, hd *ph, int k, int dir)
{
    const int np = m->energy == OR_NEO_HOOKE ? 0 : net_size(3, m->psi_w);
    if (dir == 1) ph[k].a = 1.0;
    else ph[k].b = 1.0;
    m->seeded = 1;
    m->psi_ph = ph;
    m->y_ph = ph + np;
    m->c_N0 = hc(0.0);
    m->c_n = hc(0.0);
    if (np > 0) {
        hd x0[3] = {hc(0.0), hc(0.0), hc(0.0)};
        m->c_N0 = icnn_p(m->psi_ph, 3, m->psi_w, x0);
        hd dN[3];
        for (int i = 0; i < 3; ++i) {
            hd x[3] = {hc(0.0), hc(0.0), hc(0.0)};
            if (dir == 1) x[i].b = 1.0;                  /* the input derivative in the other part */
            else x[i].a = 1.0;
            hd v = icnn_p(m->psi_ph, 3, m->psi_w, x);
            dN[i] = hc(dir == 1 ? v.b : v.a);
            if (dir == 1) dN[i].a = v.ab;
            else dN[i].b = v.ab;
        }
        if (m->energy == OR_ICNN_RAW) m->c_n = hadd(hadd(hscale(dN[0], 2.0), hscale(dN[1], 4.0)), dN[2]);
        else m->c_n = dN[2];
    }
    m->c_yN0 = hc(0.0);
    m->c_ys = hc(1.0);
    if (m->y_w > 0) {
        hd q0 = hc(0.0);
        m->c_yN0 = icnn_p(m->y_ph, 1, m->y_w, &q0);
        hd q1 = hc(0.0);
        if (dir == 1) q1.b = 1.0;
        else q1.a = 1.0;
        hd v = icnn_p(m->y_ph, 1, m->y_w, &q1);
        hd Np = hc(dir == 1 ? v.b : v.a);
        if (dir == 1) Np.a = v.ab;
        else Np.b = v.ab;
        m->c_ys = hinv(Np);
    }
}
static void unseed_weight(or_mat *m, hd *ph, int k)
{
    ph[k].a = 0.0;
    ph[k].b = 0.0;
    m->seeded = 0;
}

/* Partial derivatives of one element's converged-step outputs, at its dofs de and
 * committed history kappa_n (the local update kappa_{n+1}(z, kappa_n; theta) inside,
 * Sec. 3.2 Eq. (dd_7_no_nn)), with theta = [psi params | yield params]:
 *   dR_dth[nd * nth]  dR^e / dtheta_k: the weights' direct part d2Psi/dz dtheta_k plus,
 *                     on loading points, d2Psi/dz dkappa dkappa_{n+1}/dtheta_k
 *   dk_dth[nq * nth]  dkappa_{n+1} / dtheta_k = -(dr/dtheta_k) / (dr/dkappa) on
 *                     loading points (implicit function theorem on r = G(q) - kappa
 *                     = 0), 0 elsewhere
 *   dR_dkp[nd * nq]   dR^e / dkappa_{n,q}: on unloading points kappa_{n+1} = kappa_n,
 *                     so d2Psi/dz dkappa; 0 on loading points (the root does not
 *                     depend on kappa_n)
 *   dk_dkp[nq]        dkappa_{n+1} / dkappa_n: 1 unloading, 0 loading
 *   dk_dd[nq * nd]    dkappa_{n+1} / dd^e (loading points; 0 elsewhere)
 * Row-major; any output may be NULL.  Returns -1 for a non-positive Jacobian. */
int or_element_sens(const or_mat *m0, const double *Xe, const double *de, const double *kappa_n, double *dR_dth,
                    double *dk_dth, double *dR_dkp, double *dk_dkp, double *dk_dd)
{
    or_mat m = *m0;
    m.seeded = 0;
    const int dim = m.dim, nen = nen_of(dim), nq = nq_of(dim), ndof = dim + 1, nd = nen * ndof;
    const int nz = nz_of(dim);
    const int np = m.energy == OR_NEO_HOOKE ? 0 : net_size(3, m.psi_w), ny = net_size(1, m.y_w), nth = np + ny;
    hd *ph = (hd *)malloc(sizeof(hd) * (size_t)(nth > 0 ? nth : 1));
    if (!ph) return -1;
    for (int i = 0; i < np; ++i) ph[i] = hc(m.psi_p[i]);
    for (int i = 0; i < ny; ++i) ph[np + i] = hc(m.y_p[i]);
    if (dR_dth) memset(dR_dth, 0, sizeof(double) * (size_t)nd * nth);
    if (dk_dth) memset(dk_dth, 0, sizeof(double) * (size_t)nq * nth);
    if (dR_dkp) memset(dR_dkp, 0, sizeof(double) * (size_t)nd * nq);
    if (dk_dd) memset(dk_dd, 0, sizeof(double) * (size_t)nq * nd);
    for (int q = 0; q < nq; ++q) {
        double N[8], dN[8][3], Jw;
        if (shape_at(dim, Xe, q, N, dN, &Jw)) {
            free(ph);
            return -1;
        }
        double B[13][32];
        memset(B, 0, sizeof(B));
        for (int a = 0; a < nen; ++a) {
            for (int i = 0; i < dim; ++i)
                for (int J = 0; J < dim; ++J) B[i * dim + J][a * ndof + i] = dN[a][J];
            B[dim * dim][a * ndof + dim] = N[a];
            for (int J = 0; J < dim; ++J) B[dim * dim + 1 + J][a * ndof + dim] = dN[a][J];
        }
        double z[13];
        for (int c = 0; c < nz; ++c) {
            double s = 0.0;
            for (int A = 0; A < nd; ++A) s += B[c][A] * de[A];
            z[c] = s;
        }
        or_qp_info inf;
        local_update(&m, z, kappa_n[q], &inf);
        const double kap = inf.kappa;
        hd zz[13];
        /* d2Psi / dz_c dkappa at the converged kappa */
        double mixed[13], dkdz[13];
        for (int c = 0; c < nz; ++c) {
            for (int f = 0; f < nz; ++f) zz[f] = hc(z[f]);
            zz[c].a = 1.0;
            hd k = hc(kap);
            k.b = 1.0;
            mixed[c] = Psi(&m, zz, k).ab;
        }
        double drk = 1.0;
        if (inf.loading) {
            drk = dr_dkappa(&m, z, kap);
            for (int c = 0; c < nz; ++c) {
                for (int f = 0; f < nz; ++f) zz[f] = hc(z[f]);
                zz[c].a = 1.0;
                dkdz[c] = -yield_residual(&m, zz, hc(kap)).a / drk;
            }
        }
        if (dk_dkp) dk_dkp[q] = inf.loading ? 0.0 : 1.0;
        for (int A = 0; A < nd; ++A) {
            double sk = 0.0, sr = 0.0;
            for (int c = 0; c < nz; ++c) {
                if (inf.loading) sk += dkdz[c] * B[c][A];
                else sr += B[c][A] * mixed[c];
            }
            if (dk_dd) dk_dd[q * nd + A] = sk;
            if (dR_dkp) dR_dkp[A * nq + q] = sr * Jw;
        }
        if (!dR_dth && !dk_dth) continue;
        for (int k = 0; k < nth; ++k) {
            double dk = 0.0;
            if (inf.loading) {
                for (int f = 0; f < nz; ++f) zz[f] = hc(z[f]);
                seed_weight(&m, ph, k, 1);
                dk = -yield_residual(&m, zz, hc(kap)).a / drk;
                unseed_weight(&m, ph, k);
            }
            if (dk_dth) dk_dth[q * nth + k] = dk;
            if (!dR_dth) continue;
            seed_weight(&m, ph, k, 2);
            double v[13];
            for (int c = 0; c < nz; ++c) {
                for (int f = 0; f < nz; ++f) zz[f] = hc(z[f]);
                zz[c].a = 1.0;
                v[c] = Psi(&m, zz, hc(kap)).ab + mixed[c] * dk;
            }
            unseed_weight(&m, ph, k);
            for (int A = 0; A < nd; ++A) {
                double s = 0.0;
                for (int c = 0; c < nz; ++c) s += B[c][A] * v[c];
                dR_dth[A * nth + k] += s * Jw;
            }
        }
    }
    free(ph);
    return 0;
}

/* ------------------------------------------------------------------ */
/* point-wise access for the pins                                      */
/* ------------------------------------------------------------------ */
/* psi_e and its first/second derivatives with respect to the 9 entries of H
 * (dim = 3 layout, row-major) or the dim*dim in-plane entries (dim = 2). */
void or_psi_e(const or_mat *m, const double *H9, double *val, double *grad, double *hess)
{
    int d = m->dim, n = d * d;
    for (int c = -1; c < n; ++c)
        for (int e = (c < 0 ? -1 : c); e < n; ++e) {
            hd H[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) H[i][j] = hc((i < d && j < d) ? H9[i * 3 + j] : 0.0);
            if (c >= 0) H[c / d][c % d].a = 1.0;
            if (e >= 0) H[e / d][e % d].b += 1.0;
            hd p = psi_e(m, H);
            if (c < 0 && e < 0) *val = p.v;
            else if (c < 0) {
                if (grad) grad[e] = p.b;
            } else if (hess) {
                hess[c * n + e] = p.ab;
                hess[e * n + c] = p.ab;
            }
        }
}

/* raw network value, gradient, Hessian at x (n_in inputs, n_in <= 3) */
void or_icnn(const double *p, int n_in, int w, const double *x, double *val, double *grad, double *hess)
{
    for (int c = -1; c < n_in; ++c)
        for (int e = (c < 0 ? -1 : c); e < n_in; ++e) {
            hd xx[3];
            for (int i = 0; i < n_in; ++i) xx[i] = hc(x[i]);
            if (c >= 0) xx[c].a = 1.0;
            if (e >= 0) xx[e].b += 1.0;
            hd v = icnn(p, n_in, w, xx);
            if (c < 0 && e < 0) *val = v.v;
            else if (c < 0) {
                if (grad) grad[e] = v.b;
            } else if (hess) {
                hess[c * n_in + e] = v.ab;
                hess[e * n_in + c] = v.ab;
            }
        }
}

/* plain double-precision network evaluation (no derivatives), for finite differences */
double or_icnn_value(const double *p, int n_in, int w, const double *x)
{
    hd xx[3];
    for (int i = 0; i < n_in; ++i) xx[i] = hc(x[i]);
    return icnn(p, n_in, w, xx).v;
}

/* invariants as functions of C itself: (I1-3, I2-3, J-1, I1G, I2G) and their
 * derivatives with respect to the 9 entries of C taken as independent, for the
 * pins against the closed forms of Eq. (dd_1). */
void or_invariants_of_C(const double *C9, double *out5, double *dC /* [5][9] */)
{
    for (int c = -1; c < 9; ++c) {
        hd C[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) C[i][j] = hc(C9[i * 3 + j]);
        if (c >= 0) C[c / 3][c % 3].a = 1.0;
        hd A[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) A[i][j] = hsub(C[i][j], hc(i == j ? 1.0 : 0.0));
        hd a = hadd(hadd(A[0][0], A[1][1]), A[2][2]);
        hd AA = hc(0.0);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) AA = hadd(AA, hmul(A[i][j], A[j][i]));
        hd I1m3 = a;
        hd I2m3 = hadd(hscale(a, 2.0), hscale(hsub(hsq(a), AA), 0.5));
        hd I3 = det3(C);
        /* J = sqrt(I3) */
        double sJ = sqrt(I3.v);
        hd J = hfun(I3, sJ, 0.5 / sJ, -0.25 / (sJ * I3.v));
        hd L = hfun(I3, 0.5 * log(I3.v), 0.5 / I3.v, -0.5 / (I3.v * I3.v)); /* ln J */
        hd e = hexp(hscale(L, -2.0 / 3.0));
        hd I1G = hmul(hadd(I1m3, hc(3.0)), e);
        hd I2 = hadd(I2m3, hc(3.0));
        hd I2G = hdiv(hmul(hmul(I2, I2), I2), hscale(hmul(hsq(J), hsq(J)), 9.0));
        hd r[5] = {I1m3, I2m3, hsub(J, hc(1.0)), I1G, I2G};
        for (int k = 0; k < 5; ++k) {
            if (c < 0) out5[k] = r[k].v;
            else dC[k * 9 + c] = r[k].a;
        }
    }
}

/* lambda_e psi_vol(J(C)) with derivative wrt C entries (Eq. (dd_0), (dd_1)) */
void or_psi_vol_of_C(const double *C9, double *val, double *dC)
{
    for (int c = -1; c < 9; ++c) {
        hd C[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) C[i][j] = hc(C9[i * 3 + j]);
        if (c >= 0) C[c / 3][c % 3].a = 1.0;
        hd I3 = det3(C);
        double sJ = sqrt(I3.v);
        hd J = hfun(I3, sJ, 0.5 / sJ, -0.25 / (sJ * I3.v));
        hd t = hsub(hadd(J, hinv(J)), hc(2.0));
        hd p = hsq(t);
        if (c < 0) *val = p.v;
        else dC[c] = p.a;
    }
}

/* material point: Psi derivatives + local update at a given z (for pins and the
 * homogeneous driver).  out: dPsi[nz], D[nz*nz] (may be NULL), info[6]. */
void or_qp(const or_mat *m, const double *z, double kappa_n, double *dPsi, double *D, double *info)
{
    or_qp_info inf;
    qp_eval(m, z, kappa_n, dPsi, D, &inf);
    info[0] = inf.kappa; info[1] = inf.dlam; info[2] = inf.q; info[3] = inf.Phi_trial;
    info[4] = inf.fd; info[5] = inf.loading;
}

/* yield G(q) and G'(q) */
void or_yield(const or_mat *m, double q, double *G, double *Gp)
{
    hd qq = hc(q);
    qq.a = 1.0;
    hd v = yield_G(m, qq);
    *G = v.v;
    *Gp = v.a;
}

/* psi_e value at z (undamaged energy, q_loc) */
double or_psi_value(const or_mat *m, const double *z)
{
    hd zz[13];
    int nz = nz_of(m->dim);
    for (int c = 0; c < nz; ++c) zz[c] = hc(z[c]);
    hd H[3][3], phi, g[3];
    unpack_z(m, zz, H, &phi, g);
    return psi_e(m, H).v;
}

/* Element potential at fixed history: Pi^e = sum_q Psi_int(z_q, kappa_q) J_q w_q
 * (the volume part of Eq. (total_potential_energy)); used by the pins that check
 * the residual against finite differences of the energy. */
double or_element_energy(const or_mat *m, const double *Xe, const double *de, const double *kappa)
{
    int dim = m->dim, nen = nen_of(dim), nq = nq_of(dim), ndof = dim + 1;
    int nz = nz_of(dim);
    double E = 0.0;
    for (int q = 0; q < nq; ++q) {
        double N[8], dN[8][3], Jw;
        if (shape_at(dim, Xe, q, N, dN, &Jw)) return NAN;
        hd z[13];
        for (int c = 0; c < nz; ++c) z[c] = hc(0.0);
        for (int a = 0; a < nen; ++a) {
            for (int i = 0; i < dim; ++i)
                for (int J = 0; J < dim; ++J) z[i * dim + J].v += de[a * ndof + i] * dN[a][J];
            z[dim * dim].v += N[a] * de[a * ndof + dim];
            for (int J = 0; J < dim; ++J) z[dim * dim + 1 + J].v += de[a * ndof + dim] * dN[a][J];
        }
        E += Psi(m, z, hc(kappa[q])).v * Jw;
    }
    return E;
}

int or_sizeof_mat(void) { return (int)sizeof(or_mat); }
