"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: closed forms printed
in the paper (Eq. dd_1), textbook solutions (compressible Neo-Hookean under
homogeneous uniaxial load), invariants (stress-free reference, objectivity,
convexity, KKT, dissipation), special cases (homogeneous fields reduce the
finite-element problem to a material point; phi = kappa makes the local and
non-local models coincide, Sec. 5.1) and brute force (central differences of
the element energy and residual).
"""
import json
import os

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_2604_03411_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_rot3(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def model_for(energy, seed=11, w=16, wy=8, dim=3, **mat_kw):
    psi, yld = I.icnn_pair(seed, w, wy)
    mat = I.Material(energy=energy, **mat_kw)
    return oracle.Model(dim, mat, psi.params, w, yld.params, wy), psi, yld


def nh_model(dim, mu, lam, **kw):
    mat = I.Material(mu_e=mu, lambda_e=lam, energy=I.ENERGY_NEO_HOOKE, **kw)
    return oracle.Model(dim, mat, np.zeros(1), 0, np.zeros(1), 0)


# ---------------------------------------------------------------------------
# ICNN: brute force, convexity, monotonicity (Sec. 4.2, ICNN of Amos et al.)
# ---------------------------------------------------------------------------
def numpy_icnn(p, n_in, w, x):
    W1 = p[: w * n_in].reshape(w, n_in); o = w * n_in
    b1 = p[o:o + w]; o += w
    W2 = p[o:o + w * w].reshape(w, w); o += w * w
    A2 = p[o:o + w * n_in].reshape(w, n_in); o += w * n_in
    b2 = p[o:o + w]; o += w
    w3 = p[o:o + w]; o += w
    a3 = p[o:o + n_in]
    sp = lambda v: np.logaddexp(0.0, v)
    z1 = sp(W1 @ x + b1)
    return w3 @ sp(W2 @ z1 + A2 @ x + b2) + a3 @ x


@pytest.mark.parametrize("w", [8, 16, 64])
def test_icnn_value_and_derivatives_brute_force(w):
    rng = np.random.default_rng(w)
    net = I.icnn_weights(rng, 3, w)
    L = oracle.lib()
    for _ in range(20):
        x = rng.normal(0.0, 1.0, 3)
        v = L.or_icnn_value(oracle._ptr(net.params), 3, w, oracle._ptr(x))
        assert abs(v - numpy_icnn(net.params, 3, w, x)) <= 1e-13 * max(1.0, abs(v))
        val, g, H = _icnn_full(net, x)
        h = 1e-5
        for i in range(3):
            e = np.zeros(3); e[i] = h
            fp = numpy_icnn(net.params, 3, w, x + e)
            fm = numpy_icnn(net.params, 3, w, x - e)
            assert abs((fp - fm) / (2 * h) - g[i]) <= 1e-8 * max(1.0, abs(g[i]))
            gp = _icnn_full(net, x + e)[1]
            gm = _icnn_full(net, x - e)[1]
            np.testing.assert_allclose((gp - gm) / (2 * h), H[:, i], rtol=1e-6, atol=1e-9)


def _icnn_full(net, x):
    val = oracle.ctypes.c_double()
    g = np.zeros(net.n_in)
    H = np.zeros(net.n_in * net.n_in)
    oracle.lib().or_icnn(oracle._ptr(net.params), net.n_in, net.width, oracle._ptr(np.asarray(x, float)),
                         oracle.ctypes.byref(val), oracle._ptr(g), oracle._ptr(H))
    return val.value, g, H.reshape(net.n_in, net.n_in)


def test_icnn_convex_and_nondecreasing():
    rng = np.random.default_rng(5)
    for w in (16, 32):
        net = I.icnn_weights(rng, 3, w)
        for _ in range(2000):
            x = rng.normal(0.0, 2.0, 3)
            _, g, H = _icnn_full(net, x)
            assert np.all(g >= 0.0)
            assert np.linalg.eigvalsh(H).min() >= -1e-12
            y = rng.normal(0.0, 2.0, 3)
            fx = numpy_icnn(net.params, 3, w, x)
            fy = numpy_icnn(net.params, 3, w, y)
            fm = numpy_icnn(net.params, 3, w, 0.5 * (x + y))
            assert fm <= 0.5 * (fx + fy) + 1e-12


def test_yield_function_normalised_and_increasing():
    """G(0) = 0, G'(0) = 1, G increasing (Clausius-Duhem condition of Sec. 4.2)."""
    m, _, _ = model_for(I.ENERGY_ICNN_RAW, seed=3, w=16, wy=16)
    G0, Gp0 = m.yield_G(0.0)
    assert abs(G0) < 1e-15 and abs(Gp0 - 1.0) < 1e-14
    qs = np.linspace(-5, 20, 400)
    Gs = np.array([m.yield_G(q)[0] for q in qs])
    assert np.all(np.diff(Gs) > 0)
    assert all(m.yield_G(q)[1] > 0 for q in qs)


# ---------------------------------------------------------------------------
# energy: stress-free reference, Eq. (dd_1) closed forms, objectivity, NH
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("energy", [I.ENERGY_ICNN_RAW, I.ENERGY_ICNN_ISO, I.ENERGY_NEO_HOOKE])
@pytest.mark.parametrize("dim", [2, 3])
def test_stress_free_reference(energy, dim):
    """psi_e(I) = 0 and S(C = I) = 0 for any weights (stress normality, Sec. 4.2)."""
    for seed in range(5):
        m, _, _ = model_for(energy, seed=seed, w=16, dim=dim)
        val, g, _ = m.psi_e(np.zeros((3, 3)))
        assert abs(val) < 1e-15
        assert np.abs(g).max() < 1e-14


def invariants_closed_form(C):
    I1 = np.trace(C)
    I2 = 0.5 * (I1 ** 2 - np.trace(C @ C))
    I3 = np.linalg.det(C)
    J = np.sqrt(I3)
    Ci = np.linalg.inv(C)
    Id = np.eye(3)
    d = {
        "I1": Id, "I2": I1 * Id - C, "J": 0.5 * J * Ci,
        # Eq. (dd_1), rows 4 and 5
        "I1G": I3 ** (-1.0 / 3.0) * (Id - I1 / 3.0 * Ci),
        "I2G": I2 ** 2 / (9.0 * I3 ** 2) * (3 * I1 * Id - 3 * C - 2 * I2 * Ci),
        # Eq. (dd_1), row 3, without the repeated lambda_e
        "vol": (J + 1.0 / J - 2.0) * (1.0 - J ** -2) * J * Ci,
    }
    v = {"I1": I1, "I2": I2, "J": J, "I1G": I3 ** (-1 / 3) * I1, "I2G": I2 ** 3 / (9 * J ** 4)}
    return v, d


def test_invariant_derivatives_match_eq_dd1():
    rng = np.random.default_rng(7)
    L = oracle.lib()
    for _ in range(50):
        F = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
        if np.linalg.det(F) < 0.2:
            continue
        C = F.T @ F
        out = np.zeros(5)
        dC = np.zeros(45)
        L.or_invariants_of_C(oracle._ptr(C.ravel().copy()), oracle._ptr(out), oracle._ptr(dC))
        dC = dC.reshape(5, 3, 3)
        v, d = invariants_closed_form(C)
        for k, name in enumerate(["I1", "I2", "J", "I1G", "I2G"]):
            np.testing.assert_allclose(dC[k], d[name], rtol=1e-12, atol=1e-12)
        val = oracle.ctypes.c_double()
        dv = np.zeros(9)
        L.or_psi_vol_of_C(oracle._ptr(C.ravel().copy()), oracle.ctypes.byref(val), oracle._ptr(dv))
        np.testing.assert_allclose(dv.reshape(3, 3), d["vol"], rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("energy", [I.ENERGY_ICNN_RAW, I.ENERGY_ICNN_ISO])
def test_stress_matches_closed_form_chain(energy):
    """P_e = F S with S = 2 dpsi/dC assembled from the network gradient and the
    closed-form invariant derivatives of Eq. (dd_1) (iso map) or the textbook
    forms (raw map), plus lambda_e dpsi_vol/dC and the normalising -n dJ/dC."""
    rng = np.random.default_rng(8)
    m, psi, _ = model_for(energy, seed=4, w=16, mu_e=1.3, lambda_e=2.0)
    g0 = _icnn_full(psi, np.zeros(3))[1]
    n = (2 * g0[0] + 4 * g0[1] + g0[2]) if energy == I.ENERGY_ICNN_RAW else g0[2]
    for _ in range(30):
        H = 0.3 * rng.standard_normal((3, 3))
        F = np.eye(3) + H
        if np.linalg.det(F) < 0.3:
            continue
        C = F.T @ F
        v, d = invariants_closed_form(C)
        if energy == I.ENERGY_ICNN_RAW:
            x = np.array([v["I1"] - 3, v["I2"] - 3, v["J"] - 1])
            dx = [d["I1"], d["I2"], d["J"]]
        else:
            x = np.array([v["I1G"] - 3, v["I2G"] - 3, v["J"] - 1])
            dx = [d["I1G"], d["I2G"], d["J"]]
        g = _icnn_full(psi, x)[1]
        S = 2 * (1.3 * (g[0] * dx[0] + g[1] * dx[1] + (g[2] - n) * d["J"]) + 2.0 * d["vol"])
        _, P, _ = m.psi_e(H)
        np.testing.assert_allclose(P.reshape(3, 3), F @ S, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_objectivity(dim):
    """Psi(QF) = Psi(F), P(QF) = Q P(F), fluxes unchanged, for Q in SO(3) (SO(2) in plane strain)."""
    rng = np.random.default_rng(9)
    m, _, _ = model_for(I.ENERGY_ICNN_RAW, seed=2, w=16, dim=dim)
    nz = m.nz
    for _ in range(20):
        if dim == 3:
            Q = rand_rot3(rng)
        else:
            t = rng.uniform(0, 2 * np.pi)
            Q = np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]])
        F = np.eye(dim) + 0.25 * rng.standard_normal((dim, dim))
        if np.linalg.det(F) < 0.3:
            continue
        z = np.zeros(nz)
        z[:dim * dim] = (F - np.eye(dim)).ravel()
        z[dim * dim] = rng.uniform(0, 0.5)
        z[dim * dim + 1:] = 0.3 * rng.standard_normal(dim)
        kn = rng.uniform(0, 0.3)
        dP, _, info = m.qp(z, kn, tangent=False)
        zr = z.copy()
        zr[:dim * dim] = (Q @ F - np.eye(dim)).ravel()
        dPr, _, infor = m.qp(zr, kn, tangent=False)
        P = dP[:dim * dim].reshape(dim, dim)
        Pr = dPr[:dim * dim].reshape(dim, dim)
        np.testing.assert_allclose(Pr, Q @ P, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(dPr[dim * dim:], dP[dim * dim:], rtol=1e-11, atol=1e-12)
        assert abs(infor[0] - info[0]) <= 1e-12 * max(1, info[0])


@pytest.mark.parametrize("dim", [2, 3])
def test_neo_hooke_textbook_stress(dim):
    """The closed-form model of Sec. 4.1: P = mu (F - F^-T) + lambda ln J F^-T."""
    rng = np.random.default_rng(10)
    mu, lam = 14.48, 130.3
    m = nh_model(dim, mu, lam)
    for _ in range(30):
        F = np.eye(3)
        F[:dim, :dim] += 0.3 * rng.standard_normal((dim, dim))
        J = np.linalg.det(F)
        if J < 0.3:
            continue
        Fit = np.linalg.inv(F).T
        P = mu * (F - Fit) + lam * np.log(J) * Fit
        _, g, _ = m.psi_e(F - np.eye(3))
        np.testing.assert_allclose(g.reshape(dim, dim), P[:dim, :dim], rtol=1e-11, atol=1e-11)


def test_small_strain_shear_modulus():
    """Linearising S about C = I with n (J - 1) subtracted: mu_0 = 2 mu_e (dN/dx1 + dN/dx2)(0)."""
    m, psi, _ = model_for(I.ENERGY_ICNN_RAW, seed=6, w=32, mu_e=1.7)
    g0 = _icnn_full(psi, np.zeros(3))[1]
    mu0 = 2 * 1.7 * (g0[0] + g0[1])
    gam = 1e-6
    H = np.zeros((3, 3))
    H[0, 1] = gam
    _, P, _ = m.psi_e(H)
    assert abs(P[1] / gam - mu0) <= 1e-5 * mu0


# ---------------------------------------------------------------------------
# damage: degradation, yield, KKT, dissipation
# ---------------------------------------------------------------------------
def test_degradation_properties():
    """f_d(0) = 1, 0 < f_d <= 1, f_d non-increasing (Sec. 2.1)."""
    m, _, _ = model_for(I.ENERGY_ICNN_RAW, dim=2, eta_d=1.5, kappa_d=0.05)
    ks = np.linspace(0, 6, 200)
    fd = []
    for k in ks:
        _, _, info = m.qp(np.zeros(7), k, tangent=False)   # undeformed, phi = 0 -> elastic
        assert info[5] == 0 and info[0] == k
        fd.append(info[4])
    fd = np.array(fd)
    assert fd[0] == 1.0 and np.all(fd > 0) and np.all(fd <= 1) and np.all(np.diff(fd) <= 0)


# ---------------------------------------------------------------------------
# element: residual = gradient of the energy, tangent = Jacobian of the residual
# ---------------------------------------------------------------------------
def _elem_setup(dim, seed):
    rng = np.random.default_rng(seed)
    mesh = I.structured_q4(1, 1) if dim == 2 else I.structured_hex8(1, 1, 1)
    Xe = mesh.coords[mesh.conn[0]] + 0.08 * rng.standard_normal(mesh.coords[mesh.conn[0]].shape)
    nd = mesh.nen * mesh.ndof
    de = np.zeros((mesh.nen, mesh.ndof))
    de[:, :dim] = 0.15 * rng.standard_normal((mesh.nen, dim))
    de[:, dim] = rng.uniform(0.0, 0.6, mesh.nen)
    kn = rng.uniform(0.0, 0.4, mesh.nq)
    return Xe, de.ravel(), kn, nd


@pytest.mark.parametrize("dim", [2, 3])
def test_residual_is_energy_gradient(dim):
    """R^e = d Pi^e / d(u, phi) at the updated history held fixed (Sec. 3.1 weak forms)."""
    m, _, _ = model_for(I.ENERGY_ICNN_RAW, seed=12, w=16, dim=dim)
    Xe, de, kn, nd = _elem_setup(dim, 1)
    Re, _, k1, _ = m.element(Xe, de, kn, tangent=False)
    h = 1e-6
    for A in range(nd):
        dp = de.copy(); dp[A] += h
        dm = de.copy(); dm[A] -= h
        fd = (m.element_energy(Xe, dp, k1) - m.element_energy(Xe, dm, k1)) / (2 * h)
        assert abs(fd - Re[A]) <= 1e-7 * max(1.0, np.abs(Re).max())


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tangent_is_residual_jacobian(dim, seed):
    """K^e vs central differences of R^e with the monolithic kappa update inside;
    no qp may change its loading state under the perturbation (checked)."""
    m, _, _ = model_for(I.ENERGY_ICNN_RAW, seed=12 + seed, w=16, dim=dim)
    Xe, de, kn, nd = _elem_setup(dim, 10 + seed)
    Re, Ke, k1, qi = m.element(Xe, de, kn)
    assert qi[:, 5].sum() > 0, "the state should have loading points"
    h = 1e-6
    Kfd = np.zeros_like(Ke)
    for A in range(nd):
        dp = de.copy(); dp[A] += h
        dm = de.copy(); dm[A] -= h
        Rp, _, _, qp_ = m.element(Xe, dp, kn, tangent=False)
        Rm, _, _, qm_ = m.element(Xe, dm, kn, tangent=False)
        assert np.array_equal(qp_[:, 5], qi[:, 5]) and np.array_equal(qm_[:, 5], qi[:, 5])
        Kfd[:, A] = (Rp - Rm) / (2 * h)
    assert np.abs(Kfd - Ke).max() <= 1e-7 * np.abs(Ke).max()


def test_tangent_symmetric_when_damaged_and_gamma_one():
    """With gamma_d = 1 and kappa > kappa_d the coupling blocks are symmetric
    (f_d' dkappa/dphi = -beta_d c_kappa), so the whole K^e is symmetric:
    a consequence of q_nloc = beta_d (phi - kappa)/(eta_d f_d) being -dPsi/dd."""
    m, _, _ = model_for(I.ENERGY_ICNN_RAW, seed=21, w=16, dim=2, kappa_d=0.0)
    Xe, de, kn, nd = _elem_setup(2, 5)
    Re, Ke, k1, qi = m.element(Xe, de, kn + 0.05)
    assert np.all(k1 > 0.0)
    assert np.abs(Ke - Ke.T).max() <= 1e-10 * np.abs(Ke).max()


# ---------------------------------------------------------------------------
# global: homogeneous patch = material point, Mullins cycle, KKT along the path
# ---------------------------------------------------------------------------
def test_zero_state_gives_zero_residual():
    p = I.config1()
    m = oracle.Model.from_problem(p)
    n = p.mesh.n_nodes * p.mesh.ndof
    R, _, k1, qi, nf = m.assemble(p.mesh, np.zeros(n), np.zeros((p.mesh.n_elems, 4)), tangent=False)
    assert np.abs(R).max() == 0.0 and np.all(k1 == 0.0) and nf == 0


def test_homogeneous_patch_matches_material_point():
    """Uniaxial plane strain on a structured mesh: the FE solution is homogeneous,
    phi = kappa, and the reaction per unit height equals the material point's
    P11 along a load-unload-reload history (Sec. 5.1, phi = kappa)."""
    p = I.config1(n=4)
    m = oracle.Model.from_problem(p)
    load = I.piecewise_path([0.0, 0.6, 0.2, 0.8], [6, 4, 6])
    res = oracle.run_load_path(m, p.mesh, load, keep_states=True)
    P11, lam2, kap = oracle.material_point_uniaxial(m, 1.0 + load)
    np.testing.assert_allclose(res["reaction"], P11, rtol=1e-9, atol=1e-12)
    for s, (dofs, kappa, qi) in enumerate(res["states"]):
        np.testing.assert_allclose(kappa, kap[s], rtol=1e-9, atol=1e-12)
        d = dofs.reshape(-1, 3)
        np.testing.assert_allclose(d[:, 2], kap[s], rtol=1e-8, atol=1e-11)
        y = p.mesh.coords[:, 1]
        np.testing.assert_allclose(d[:, 1], (lam2[s] - 1.0) * y, rtol=1e-8, atol=1e-11)


def test_biaxial_block_matches_material_point():
    """Biaxial stretch of a HEX8 block with rollers on three faces and a free top
    face (the uniform-deformation block of Sec. 5.2): the FE solution is homogeneous,
    F = diag(lam, lam, lam3) with P33 = 0, phi = kappa, and the x-face reaction of the
    unit cube equals P11 of the 3D material-point driver along a load-unload-reload
    history (Sec. 5.1, phi = kappa)."""
    p = I.config3(n=3, n_steps=10)
    m = oracle.Model.from_problem(p)
    load = I.piecewise_path([0.0, 0.4, 0.2, 0.45], [4, 2, 3])
    res = oracle.run_load_path(m, p.mesh, load, keep_states=True)
    P11, lam3, kap = oracle.material_point_biaxial(m, 1.0 + load)
    assert kap[-1] > kap[3] > 0.5, "the path should damage the block and damage again on reloading"
    np.testing.assert_allclose(res["reaction"], P11, rtol=0, atol=1e-9 * np.abs(P11).max())
    np.testing.assert_array_equal(kap[4:6], kap[3])           # unloading keeps the history
    z = p.mesh.coords[:, 2]
    for s, (dofs, kappa, qi) in enumerate(res["states"]):
        np.testing.assert_allclose(kappa, kap[s], rtol=1e-9, atol=1e-12)
        d = dofs.reshape(-1, 4)
        np.testing.assert_allclose(d[:, 3], kap[s], rtol=1e-8, atol=1e-11)
        np.testing.assert_allclose(d[:, 2], (lam3[s] - 1.0) * z, rtol=1e-8, atol=1e-11)


def test_mullins_load_unload_reload():
    """Sec. 1: unloading and reloading follow the same curve below the previous
    maximum stretch, kappa is frozen there, and damage resumes beyond it."""
    m, _, _ = model_for(I.ENERGY_ICNN_RAW, seed=1, w=16, wy=8, dim=2, c_d=0.1)
    up = np.linspace(1.0, 2.0, 11)[1:]
    down = np.linspace(2.0, 1.0, 11)[1:]
    re = np.linspace(1.0, 2.0, 11)[1:]
    beyond = np.linspace(2.0, 2.2, 5)[1:]
    lam = np.concatenate([up, down, re, beyond])
    P, _, k = oracle.material_point_uniaxial(m, lam)
    kmax = k[9]
    assert np.all(np.diff(k[:10]) > 0)
    np.testing.assert_array_equal(k[10:30], kmax)
    # unload at lam_i == reload at lam_i
    np.testing.assert_allclose(P[10:19][::-1], P[20:29], rtol=1e-12, atol=1e-13)
    assert abs(P[29] - P[9]) <= 1e-10 * abs(P[9])
    assert np.all(np.diff(k[29:]) > 0)
    # below the virgin curve on unloading: P_unload(lam) < P_load(lam)
    assert np.all(P[10:19][::-1] < P[:9])


def test_kkt_and_dissipation_along_cfg1_path():
    """At every qp and step: Delta lambda >= 0, Phi_d <= 0 after the update,
    Delta lambda * Phi_d = 0, kappa non-decreasing, D = q (d_{n+1} - d_n) >= 0 (Sec. 2.2)."""
    p = I.config1()
    m = oracle.Model.from_problem(p)
    res = oracle.run_load_path(m, p.mesh, p.load, keep_states=True)
    kprev = np.zeros((p.mesh.n_elems, 4))
    dprev = np.zeros_like(kprev)
    for dofs, kappa, qi in res["states"]:
        dlam, q, fd, loading = qi[..., 1], qi[..., 2], qi[..., 4], qi[..., 5]
        assert np.all(dlam >= 0.0)
        G = np.vectorize(lambda v: m.yield_G(v)[0])(q)
        Phi = G - kappa
        assert np.all(Phi <= 1e-10 * np.maximum(1.0, kappa))
        assert np.all(np.abs(dlam * Phi) <= 1e-10)
        assert np.all(kappa >= kprev)
        d = 1.0 - fd
        assert np.all(q * (d - dprev) >= -1e-14)
        assert np.all(q[loading > 0] >= 0.0)
        kprev, dprev = kappa, d
    assert res["reaction"].max() > 0


def test_local_equals_nonlocal_when_homogeneous():
    """Sec. 5.1: with phi = kappa the non-local term of Eq. (ostwald_potential)
    vanishes, so gamma_d = 0 (local) and gamma_d = 1 give the same homogeneous response."""
    psi, yld = I.icnn_pair(1, 16, 8)
    lam = 1.0 + np.linspace(0, 0.9, 10)
    out = []
    for gam in (0.0, 1.0):
        mat = I.Material(gamma_d=gam)
        m = oracle.Model(2, mat, psi.params, 16, yld.params, 8)
        out.append(oracle.material_point_uniaxial(m, lam))
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=1e-12)
    np.testing.assert_allclose(out[0][2], out[1][2], rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# Sec. 5.1 single HEX8 element, Neo-Hookean with exponential damage
# ---------------------------------------------------------------------------
def nh_uniaxial_3d(mu, lam, stretch):
    """Textbook homogeneous uniaxial state of the compressible Neo-Hookean solid:
    lateral stretch l from P22 = mu (l - 1/l) + lam ln(J)/l = 0, J = stretch l^2."""
    f = lambda l: mu * (l - 1 / l) + lam * np.log(stretch * l * l) / l
    l = brentq(f, 0.3, 1.5, xtol=1e-15, rtol=1e-15)
    J = stretch * l * l
    P11 = mu * (stretch - 1 / stretch) + lam * np.log(J) / stretch
    I1 = stretch ** 2 + 2 * l * l
    psi = 0.5 * mu * (I1 - 3) - mu * np.log(J) + 0.5 * lam * np.log(J) ** 2
    return P11, psi


def test_single_hex8_element_sec51():
    g = json.load(open(os.path.join(GOLDEN, "single_element_e1.json")))
    E, nu = g["E_MPa"], g["nu"]
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mesh = I.biaxial_bc_3d(I.structured_hex8(1, 1, 1))
    # uniaxial: keep the rollers on the three min faces, drive only the x = max face
    keep = ~((mesh.bc_comp == 1) & (mesh.bc_scale > 0))
    mesh.bc_node, mesh.bc_comp, mesh.bc_scale = mesh.bc_node[keep], mesh.bc_comp[keep], mesh.bc_scale[keep]
    steps = np.linspace(0.0, g["u_end_mm"], 21)[1:]
    for case in g["cases_checked"]:
        m = nh_model(3, mu, lam, eta_d=case["eta_d"], kappa_d=case["kappa_d"], beta_d=10.0, c_d=1.0)
        res = oracle.run_load_path(m, mesh, steps, keep_states=True)
        kmax = 0.0
        for s, u in enumerate(steps):
            P11, psi = nh_uniaxial_3d(mu, lam, 1.0 + u)
            kmax = max(kmax, psi)
            fd = np.exp(-case["eta_d"] * max(kmax - case["kappa_d"], 0.0))
            assert abs(res["reaction"][s] - fd * P11) <= 1e-8 * abs(P11)
            np.testing.assert_allclose(res["states"][s][1], kmax, rtol=1e-9)


# ---------------------------------------------------------------------------
# FE patch test on distorted elements, analytic non-local field
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_patch_test_distorted_mesh(dim):
    """Isoparametric patch test: on a mesh with perturbed interior nodes, a linear
    displacement field u = G X with uniform phi = kappa gives a uniform stress, so
    every displacement row of an interior node has zero residual (the Gauss rules
    integrate grad N_a det J exactly for Q4 and HEX8)."""
    rng = np.random.default_rng(21)
    mesh = I.structured_q4(3, 3) if dim == 2 else I.structured_hex8(2, 2, 2)
    X = mesh.coords.copy()
    inner = np.all((X > 1e-9) & (X < 1 - 1e-9), axis=1)
    X[inner] += 0.12 * rng.uniform(-1, 1, (inner.sum(), dim))
    mesh.coords = X
    m, _, _ = model_for(I.ENERGY_ICNN_RAW, seed=3, w=16, dim=dim, kappa_d=1000.0, gamma_d=0.0)
    G = 0.08 * rng.standard_normal((dim, dim))
    d = np.zeros((mesh.n_nodes, dim + 1))
    d[:, :dim] = X @ G.T
    d[:, dim] = 50.0
    kappa = np.full((mesh.n_elems, mesh.nq), 50.0)
    R, _, k1, qi, _ = m.assemble(mesh, d, kappa, tangent=False)
    assert np.all(qi[..., 5] == 0)
    Rn = R.reshape(-1, dim + 1)
    scale = np.abs(Rn[~inner, :dim]).max()
    assert scale > 1e-3
    assert np.abs(Rn[inner, :dim]).max() <= 1e-12 * scale


@pytest.mark.parametrize("stretch", [1.0, 1.5])
def test_nonlocal_field_matches_analytic_solution(stretch):
    """With the displacement prescribed as a uniform stretch lam along x and an
    elastic history kappa_n(x) = k0 + A cos(pi x / L), the non-local equation of
    Sec. 2.1 (grad-energy c_d/2 gradphi.C^-1.gradphi, penalty beta_d/2 (phi-kappa)^2,
    zero flux on the boundary) reduces to -(c_d/lam^2) phi'' + beta_d (phi - kappa) = 0,
    whose solution is phi = k0 + A cos(pi x/L) / (1 + c_d pi^2 / (beta_d lam^2 L^2))."""
    n = 64
    mesh = I.structured_q4(n, 2, 1.0, 0.05)
    x = mesh.coords[:, 0]
    nodes = np.repeat(np.arange(mesh.n_nodes, dtype=np.int32), 2)
    comps = np.tile(np.array([0, 1], np.int8), mesh.n_nodes)
    scale = np.where(comps == 0, (stretch - 1.0) * x[nodes], 0.0)
    mesh.bc_node, mesh.bc_comp, mesh.bc_scale = nodes, comps, scale
    mesh.react_node = np.zeros(0, np.int32)
    psi, _ = I.icnn_pair(2, 16, 8)
    c_d, beta = 0.05, 10.0
    mat = I.Material(c_d=c_d, beta_d=beta, gamma_d=0.0, kappa_d=1000.0)
    m = oracle.Model(2, mat, psi.params, 16, np.zeros(1), 0)
    k0, A = 100.0, 0.5
    h = 1.0 / n
    gp = 1.0 / np.sqrt(3.0)
    ei = np.arange(mesh.n_elems) % n
    xq = np.stack([ei * h + h * (1 + s) / 2 for s in (-gp, gp, -gp, gp)], axis=1)
    kappa = k0 + A * np.cos(np.pi * xq)
    d0 = np.zeros(mesh.n_nodes * 3)
    d0[2::3] = k0
    dofs, k1, res, R = oracle.newton_step(m, mesh, d0, kappa, 1.0, rtol=1e-13, atol=1e-13)
    assert res.converged and np.array_equal(k1, kappa)
    phi = dofs.reshape(-1, 3)[:, 2]
    exact = k0 + A * np.cos(np.pi * x) / (1.0 + c_d * np.pi ** 2 / (beta * stretch ** 2))
    assert np.abs(phi - exact).max() < 3e-4


def test_adjoint_matches_central_differences():
    """The oracle's discrete adjoint of the load path (every state stored, transposed
    LU solves, element sensitivities by hyper-dual numbers) against central
    differences of the whole path (Sec. 3.2 steps re-solved at perturbed weights),
    along a load-unload-reload path with loading and unloading points, for weights of
    both networks and the normalising constants they feed."""
    mesh = I.uniaxial_bc_2d(I.structured_q4(3, 2))
    psi, yld = I.icnn_pair(11, 8, 8)
    mat = I.Material(beta_d=10.0, c_d=10.0 * 0.1 ** 2)
    load = np.array([0.25, 0.5, 0.35, 0.45, 0.6])
    m = oracle.Model(2, mat, psi.params, 8, yld.params, 8)
    w = np.array([1.0, -0.5, 2.0, 0.7, 1.5])
    g, reac = oracle.adjoint_gradient(m, mesh, load, w)
    st = oracle.run_load_path(m, mesh, load, keep_states=True)["states"]
    loading = np.array([qi[..., 5].sum() for _, _, qi in st])
    # unloading, then reloading below the previous maximum (the history is carried
    # through unloading points), then damage again beyond it
    assert loading[2] == 0 and loading[3] == 0 and loading[4] > 0, loading
    theta0 = np.concatenate([psi.params, yld.params])
    npsi = psi.params.size
    assert g.size == theta0.size

    def loss(th):
        mm = oracle.Model(2, mat, th[:npsi], 8, th[npsi:], 8)
        return float(w @ oracle.run_load_path(mm, mesh, load, rtol=1e-13, atol=1e-15)["reaction"])

    # first-layer, second-layer, skip and output weights and biases of both networks
    idx = [0, 5, 30, 100, 130, 137, npsi + 2, npsi + 9, npsi + 40, npsi + 90, npsi + 100, theta0.size - 1]
    scale = np.abs(g).max()
    for i in idx:
        h = 1e-5 * max(abs(theta0[i]), 1e-2)
        tp = theta0.copy()
        tp[i] += h
        tm = theta0.copy()
        tm[i] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert abs(g[i] - fd) <= 2e-8 * scale, (i, g[i], fd)


# ---------------------------------------------------------------------------
# staggered scheme (Sec. 3.2): the history advanced apart from the nodal solve
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_staggered_frozen_element(dim):
    """The nodal solve of the staggered scheme holds kappa: with the history set to
    the monolithic update's kappa_{n+1}, the frozen residual is the monolithic one
    (the same Psi at the same kappa), the history comes back unchanged, and the
    frozen tangent is the central-difference Jacobian of the frozen residual, which
    lacks the implicit-function term of the monolithic tangent."""
    m, _, _ = model_for(I.ENERGY_ICNN_RAW, seed=13, w=16, dim=dim)
    Xe, de, kn, nd = _elem_setup(dim, 21)
    Re, Ke, k1, qi = m.element(Xe, de, kn)
    assert qi[:, 5].sum() > 0, "the state should have loading points"
    m.m.frozen = 1
    try:
        Rf, Kf, kf, _ = m.element(Xe, de, k1)
        assert np.array_equal(kf, k1)
        assert np.abs(Rf - Re).max() <= 1e-12 * np.abs(Re).max()
        h = 1e-6
        Kfd = np.zeros_like(Kf)
        for A in range(nd):
            dp = de.copy(); dp[A] += h
            dm = de.copy(); dm[A] -= h
            Kfd[:, A] = (m.element(Xe, dp, k1, tangent=False)[0] - m.element(Xe, dm, k1, tangent=False)[0]) / (2 * h)
        assert np.abs(Kfd - Kf).max() <= 1e-7 * np.abs(Kf).max()
    finally:
        m.m.frozen = 0
    assert np.abs(Kf - Ke).max() > 1e-3 * np.abs(Ke).max(), "the monolithic tangent carries dkappa/dz"


def test_staggered_path_lag_is_first_order():
    """Sec. 3.2: the staggered update uses fields that were in equilibrium with the
    previous history, a lag of one load step.  Its reaction curve therefore departs
    from the monolithic one by an error of first order in the step: halving the step
    halves the difference at the end of the path; the lag leaves less damage (the
    penalty holds kappa near the lagged phi); and before any point loads (the first
    quarter of this path) the two schemes agree."""
    mesh = I.uniaxial_bc_2d(I.structured_q4(3, 2))
    psi, yld = I.icnn_pair(11, 8, 8)
    mat = I.Material(beta_d=1.0, c_d=0.1 ** 2)
    m = oracle.Model(2, mat, psi.params, 8, yld.params, 8)
    diffs = []
    for n in (20, 40, 80):
        load = np.linspace(0.0, 0.6, n + 1)[1:]
        mo = oracle.run_load_path(m, mesh, load, rtol=1e-12, atol=1e-14)
        st = oracle.run_load_path(m, mesh, load, rtol=1e-12, atol=1e-14, scheme="staggered")
        q = n // 4
        assert np.abs(st["reaction"][:q] - mo["reaction"][:q]).max() <= 1e-10 * np.abs(mo["reaction"]).max()
        assert st["kappa"].max() < mo["kappa"].max()
        diffs.append(st["reaction"][-1] - mo["reaction"][-1])
    assert abs(diffs[-1]) > 1e-3 * abs(mo["reaction"][-1]), "the lag should be visible"
    for a, b in zip(diffs, diffs[1:]):
        assert 1.8 < a / b < 2.2, diffs
