"""FP64 CPU oracle for the gradient-enhanced damage hot path (arxiv 2604.03411).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library; both receive the same seeded inputs.

Layers:
  * ``gd_oracle.c`` (compiled with gcc on first use): per-qp energy, local
    damage update and element residual/tangent, derivatives by hyper-dual
    numbers (see that file's header for the paper sections it follows).
  * this module: global assembly, Dirichlet elimination, the Newton iteration
    with a direct sparse LU (the paper solves each step with an LU
    factorisation and warm-starts from the last converged step, Sec. 3.2), the
    incremental quasi-static load path (monolithic, or the staggered scheme
    with the history advanced after the nodal solve), reactions, the
    homogeneous material-point drivers, and the discrete adjoint of the load
    path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgdoracle.so")

ENERGY = {"raw": 0, "iso": 1, "nh": 2}


def build(force: bool = False) -> str:
    """Compile gd_oracle.c into oracle/_build/libgdoracle.so (plain -O2, IEEE math),
    with OpenMP over the element loop of or_assemble where the compiler has it
    (results do not depend on the thread count)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def threads(n: int = 0) -> int:
    """Sets the oracle's element-loop thread count (n > 0) and returns the count in use."""
    return int(lib().or_threads(int(n)))


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class _OrMat(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("energy", ctypes.c_int),
                ("mu_e", ctypes.c_double), ("lambda_e", ctypes.c_double), ("eta_d", ctypes.c_double),
                ("kappa_d", ctypes.c_double), ("beta_d", ctypes.c_double), ("c_d", ctypes.c_double),
                ("gamma_d", ctypes.c_double),
                ("psi_w", ctypes.c_int), ("y_w", ctypes.c_int),
                ("psi_p", _dp), ("y_p", _dp),
                ("local_max", ctypes.c_int),
                ("psi_N0", ctypes.c_double), ("psi_n", ctypes.c_double),
                ("y_N0", ctypes.c_double), ("y_s", ctypes.c_double),
                ("seeded", ctypes.c_int), ("psi_ph", ctypes.c_void_p), ("y_ph", ctypes.c_void_p),
                ("c_hd", ctypes.c_double * 16), ("frozen", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        # GD_ORACLE_SO points the pins at another build of this file (the mutation
        # test plants mistakes in a copy and checks that the pins catch them)
        so = os.environ.get("GD_ORACLE_SO") or build()
        L = ctypes.CDLL(so)
        P = ctypes.POINTER(_OrMat)
        L.or_prepare.argtypes = [P]
        L.or_prepare.restype = ctypes.c_int
        L.or_element.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_element.restype = ctypes.c_int
        L.or_assemble.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _ip, _dp, _dp, _dp,
                                  _dp, _dp, _dp, _dp]
        L.or_assemble.restype = ctypes.c_int64
        L.or_psi_e.argtypes = [P, _dp, _dp, _dp, _dp]
        L.or_icnn.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
        L.or_icnn_value.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp]
        L.or_icnn_value.restype = ctypes.c_double
        L.or_invariants_of_C.argtypes = [_dp, _dp, _dp]
        L.or_psi_vol_of_C.argtypes = [_dp, _dp, _dp]
        L.or_qp.argtypes = [P, _dp, ctypes.c_double, _dp, _dp, _dp]
        L.or_yield.argtypes = [P, ctypes.c_double, _dp, _dp]
        L.or_psi_value.argtypes = [P, _dp]
        L.or_psi_value.restype = ctypes.c_double
        L.or_element_energy.argtypes = [P, _dp, _dp, _dp]
        L.or_element_energy.restype = ctypes.c_double
        L.or_sizeof_mat.restype = ctypes.c_int
        L.or_element_sens.argtypes = [P, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_element_sens.restype = ctypes.c_int
        L.or_threads.argtypes = [ctypes.c_int]
        L.or_threads.restype = ctypes.c_int
        assert L.or_sizeof_mat() == ctypes.sizeof(_OrMat), "oracle struct layout mismatch"
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray], typ=_dp):
    if a is None:
        return ctypes.cast(None, typ)
    return a.ctypes.data_as(typ)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Model:
    """Constitutive model for one specimen: dimension, energy kind, constants, weights."""

    def __init__(self, dim: int, mat, psi_params, psi_w: int, y_params, y_w: int,
                 energy: Optional[int] = None, local_max: int = 100):
        self.dim = dim
        self.psi_params = _f64(psi_params if psi_params is not None else np.zeros(1))
        self.y_params = _f64(y_params)
        e = mat.energy if energy is None else energy
        self.m = _OrMat(dim, int(e), mat.mu_e, mat.lambda_e, mat.eta_d, mat.kappa_d, mat.beta_d, mat.c_d,
                        mat.gamma_d, int(psi_w), int(y_w), _ptr(self.psi_params), _ptr(self.y_params),
                        int(local_max), 0.0, 0.0, 0.0, 1.0)
        if lib().or_prepare(ctypes.byref(self.m)) != 0:
            raise ValueError("yield network has N'(0) <= 0")

    @classmethod
    def from_problem(cls, prob, energy=None, local_max=100):
        return cls(prob.mesh.dim, prob.mat, prob.psi.params, prob.psi.width, prob.yld.params,
                   prob.yld.width, energy=energy, local_max=local_max)

    @property
    def nz(self):
        return self.dim * self.dim + 1 + self.dim

    # -- point-wise ----------------------------------------------------
    def qp(self, z, kappa_n, tangent=True):
        """(dPsi/dz, consistent dz-tangent or None, info) at one qp; info =
        (kappa, dlambda, q, Phi_trial, f_d, loading)."""
        z = _f64(z)
        dP = np.zeros(self.nz)
        D = np.zeros(self.nz * self.nz) if tangent else None
        info = np.zeros(6)
        lib().or_qp(ctypes.byref(self.m), _ptr(z), float(kappa_n), _ptr(dP), _ptr(D), _ptr(info))
        return dP, (D.reshape(self.nz, self.nz) if tangent else None), info

    def psi_e(self, H):
        """psi_e, d psi_e / dH, d2 psi_e / dH2 over the dim*dim in-plane entries."""
        H9 = np.zeros(9)
        d = self.dim
        H9.reshape(3, 3)[:d, :d] = np.asarray(H)[:d, :d]
        n = d * d
        val = ctypes.c_double()
        g = np.zeros(n)
        h = np.zeros(n * n)
        lib().or_psi_e(ctypes.byref(self.m), _ptr(H9), ctypes.byref(val), _ptr(g), _ptr(h))
        return val.value, g, h.reshape(n, n)

    def yield_G(self, q):
        G = ctypes.c_double()
        Gp = ctypes.c_double()
        lib().or_yield(ctypes.byref(self.m), float(q), ctypes.byref(G), ctypes.byref(Gp))
        return G.value, Gp.value

    def psi_value(self, z):
        return lib().or_psi_value(ctypes.byref(self.m), _ptr(_f64(z)))

    def element_energy(self, Xe, de, kappa):
        return lib().or_element_energy(ctypes.byref(self.m), _ptr(_f64(Xe).ravel()), _ptr(_f64(de).ravel()),
                                       _ptr(_f64(kappa).ravel()))

    # -- element -------------------------------------------------------
    @property
    def n_theta(self):
        """Number of network weights theta = [psi params | yield params]."""
        def size(n_in, w):
            return w * n_in + w + w * w + w * n_in + w + w + n_in if w > 0 else 0
        npsi = 0 if self.m.energy == ENERGY["nh"] else size(3, self.m.psi_w)
        return npsi + size(1, self.m.y_w)

    def element_sens(self, Xe, de, kappa_n):
        """Partial derivatives of an element's converged-step outputs (see or_element_sens):
        dR/dtheta [nd, nth], dkappa_new/dtheta [nq, nth], dR/dkappa_n [nd, nq],
        dkappa_new/dkappa_n [nq], dkappa_new/dd [nq, nd]."""
        nen = 4 if self.dim == 2 else 8
        nq = nen
        nd = nen * (self.dim + 1)
        nth = self.n_theta
        dR = np.zeros(nd * nth)
        dk = np.zeros(nq * nth)
        dRk = np.zeros(nd * nq)
        dkk = np.zeros(nq)
        dkd = np.zeros(nq * nd)
        f = lib().or_element_sens(ctypes.byref(self.m), _ptr(_f64(Xe).ravel()), _ptr(_f64(de).ravel()),
                                  _ptr(_f64(kappa_n).ravel()), _ptr(dR), _ptr(dk), _ptr(dRk), _ptr(dkk), _ptr(dkd))
        if f < 0:
            raise ValueError("non-positive element Jacobian")
        return dR.reshape(nd, nth), dk.reshape(nq, nth), dRk.reshape(nd, nq), dkk, dkd.reshape(nq, nd)

    def element(self, Xe, de, kappa_n, tangent=True):
        nen = 4 if self.dim == 2 else 8
        nq = nen
        nd = nen * (self.dim + 1)
        Xe = _f64(Xe).ravel()
        de = _f64(de).ravel()
        kn = _f64(kappa_n).ravel()
        Re = np.zeros(nd)
        Ke = np.zeros(nd * nd) if tangent else None
        k1 = np.zeros(nq)
        qi = np.zeros(nq * 6)
        f = lib().or_element(ctypes.byref(self.m), _ptr(Xe), _ptr(de), _ptr(kn), _ptr(Re), _ptr(Ke),
                             _ptr(k1), _ptr(qi))
        if f < 0:
            raise ValueError("non-positive element Jacobian")
        return Re, (Ke.reshape(nd, nd) if tangent else None), k1, qi.reshape(nq, 6)

    def assemble(self, mesh, dofs, kappa_n, tangent=True, e0=0, e1=None):
        """Global residual R[n_nodes*ndof], element matrices [E, nd, nd] (or None),
        kappa_new [E, nq], per-qp info [E, nq, 6], number of local-solve failures."""
        E = mesh.n_elems
        e1 = E if e1 is None else e1
        nq = mesh.nq
        nd = mesh.nen * mesh.ndof
        conn = np.ascontiguousarray(mesh.conn, dtype=np.int32)
        X = _f64(mesh.coords)
        d = _f64(dofs).ravel()
        kn = _f64(kappa_n).reshape(E * nq)
        R = np.zeros(mesh.n_nodes * mesh.ndof)
        Ke = np.zeros((e1 - e0) * nd * nd) if tangent else None
        k1 = kn.copy()
        qi = np.zeros(E * nq * 6)
        f = lib().or_assemble(ctypes.byref(self.m), mesh.n_nodes, e0, e1, _ptr(conn, _ip), _ptr(X), _ptr(d),
                              _ptr(kn), _ptr(R), _ptr(Ke), _ptr(k1), _ptr(qi))
        if f < 0:
            raise ValueError(f"non-positive Jacobian in element {-1 - f}")
        return (R, (Ke.reshape(e1 - e0, nd, nd) if tangent else None), k1.reshape(E, nq),
                qi.reshape(E, nq, 6), int(f))


# ---------------------------------------------------------------------------
# global algebra
# ---------------------------------------------------------------------------
def element_dof_map(mesh) -> np.ndarray:
    """[E, nen*ndof] global dof index of every element dof (node-major, dof-minor)."""
    nd = mesh.ndof
    return (mesh.conn.astype(np.int64)[:, :, None] * nd + np.arange(nd)[None, None, :]).reshape(mesh.n_elems, -1)


def global_matrix(mesh, Ke_all) -> sp.csr_matrix:
    """Sum of the element matrices into the global sparse matrix (duplicates summed)."""
    edm = element_dof_map(mesh)
    nd = edm.shape[1]
    rows = np.repeat(edm, nd, axis=1).ravel()
    cols = np.tile(edm, (1, nd)).ravel()
    n = mesh.n_nodes * mesh.ndof
    return sp.coo_matrix((Ke_all.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def dirichlet(mesh):
    """(global dof indices, scale) of the prescribed displacement components."""
    idx = mesh.bc_node.astype(np.int64) * mesh.ndof + mesh.bc_comp.astype(np.int64)
    return idx, mesh.bc_scale.astype(np.float64)


def reaction(mesh, R) -> float:
    """Sum of internal-force components react_comp over react_node (before elimination)."""
    return float(R[mesh.react_node.astype(np.int64) * mesh.ndof + mesh.react_comp].sum())


@dataclass
class StepResult:
    converged: bool
    iterations: int
    residual: float
    reaction: float
    local_failures: int
    qinfo: Optional[np.ndarray] = None


def newton_step(model: Model, mesh, dofs, kappa_n, load_value, rtol=1e-10, atol=1e-12, max_it=25,
                guess=None, max_ls=12):
    """One quasi-static load step of the monolithic scheme (Sec. 3.2): kappa is
    updated inside every global iteration and its tangent enters the global
    system; each linear system is solved directly by sparse LU (the paper's LU,
    Sec. 3.2).  The prescribed components are set to scale*load; the free dofs
    start from ``guess`` (default: the last converged state, the paper's warm
    start).  Each Newton direction is backtracked (halving, at most max_ls times)
    until ||R_free|| drops by the factor (1 - 1e-4 alpha).  Converged when
    ||R_free|| <= max(rtol * max(||R_free^0||, ||R_fixed||), atol), R_fixed being the
    residual on the prescribed dofs (the reaction-force scale).
    Returns (dofs, kappa_new, StepResult, R)."""
    dofs = _f64(dofs if guess is None else guess).ravel().copy()
    bidx, bscale = dirichlet(mesh)
    dofs[bidx] = bscale * load_value
    n = dofs.size
    free = np.ones(n, bool)
    free[bidx] = False
    fidx = np.nonzero(free)[0]
    R, Ke, k1, qi, nfail = model.assemble(mesh, dofs, kappa_n, tangent=True)
    nrm = float(np.linalg.norm(R[fidx]))
    r0 = max(nrm, float(np.linalg.norm(R[bidx])))
    for it in range(max_it + 1):
        if not np.isfinite(nrm):
            break
        if nrm <= max(rtol * r0, atol):
            return dofs, k1, StepResult(True, it, nrm, reaction(mesh, R), nfail, qi), R
        if it == max_it:
            break
        K = global_matrix(mesh, Ke)
        Kff = K[fidx][:, fidx].tocsc()
        delta = spla.spsolve(Kff, -R[fidx])
        alpha = 1.0
        for ls in range(max_ls + 1):
            trial = dofs.copy()
            trial[fidx] += alpha * delta
            Rt, Kt, kt, qt, ft = model.assemble(mesh, trial, kappa_n, tangent=True)
            nt = float(np.linalg.norm(Rt[fidx]))
            if (np.isfinite(nt) and nt <= (1.0 - 1e-4 * alpha) * nrm) or ls == max_ls:
                break
            alpha *= 0.5
        dofs, R, Ke, k1, qi, nfail, nrm = trial, Rt, Kt, kt, qt, ft, nt
    return dofs, k1, StepResult(False, max_it, nrm, reaction(mesh, R), nfail, qi), R


def predictor(dofs, dofs_prev, load_now, load_prev, load_prevprev):
    """Initial guess for the next step: the last converged state plus the previous
    increment scaled to the new load increment (linear extrapolation)."""
    if dofs_prev is None or load_prev == load_prevprev:
        return dofs.copy()
    return dofs + (dofs - dofs_prev) * ((load_now - load_prev) / (load_prev - load_prevprev))


def staggered_step(model: Model, mesh, dofs, kappa_n, load_value, rtol=1e-10, atol=1e-12, max_it=25,
                   guess=None, max_ls=12):
    """One load step of the staggered scheme (Sec. 3.2): the history is advanced
    apart from the nodal solve.  First the (u, phi) equilibrium is solved by Newton
    with kappa held at kappa_n (no local update, no kappa term in the tangent),
    then the local update runs once at the converged fields, against kappa_n.  The
    step takes no further coupled iteration, so the non-local driving force of the
    update comes from fields that were in equilibrium with the previous history:
    the lag the paper describes.  The reaction is the one of that equilibrium.
    Returns (dofs, kappa_new, StepResult, R)."""
    model.m.frozen = 1
    try:
        d1, _, res, R = newton_step(model, mesh, dofs, kappa_n, load_value, rtol, atol, max_it, guess, max_ls)
    finally:
        model.m.frozen = 0
    _, _, k1, qi, nfail = model.assemble(mesh, d1, kappa_n, tangent=False)
    res.local_failures = nfail
    res.qinfo = qi
    return d1, k1, res, R


def run_load_path(model: Model, mesh, load, dofs0=None, kappa0=None, rtol=1e-10, atol=1e-12, max_it=25,
                  keep_states=False, max_cuts=4, scheme="monolithic"):
    """Incremental quasi-static path (Sec. 3.2): for each load value a Newton
    step started from the extrapolated last converged state, then kappa_n <-
    kappa_{n+1}.  A step that fails is retried as two half steps (at most
    max_cuts nested halvings).  scheme: "monolithic" (newton_step) or "staggered"
    (staggered_step).  Returns dict(reaction[n_steps], iterations, dofs, kappa,
    states, cuts)."""
    step = {"monolithic": newton_step, "staggered": staggered_step}[scheme]
    n = mesh.n_nodes * mesh.ndof
    dofs = np.zeros(n) if dofs0 is None else _f64(dofs0).ravel().copy()
    kappa = np.zeros((mesh.n_elems, mesh.nq)) if kappa0 is None else _f64(kappa0).copy()
    reac, iters, states = [], [], []
    hist = {"prev": None, "l1": 0.0, "l2": 0.0, "cuts": 0}

    def advance(target, depth):
        nonlocal dofs, kappa
        g = predictor(dofs, hist["prev"], target, hist["l1"], hist["l2"])
        d1, k1, res, R = step(model, mesh, dofs, kappa, target, rtol, atol, max_it, guess=g)
        if not res.converged and depth < max_cuts:
            hist["cuts"] += 1
            mid = 0.5 * (hist["l1"] + target)
            r1 = advance(mid, depth + 1)
            r1 = advance(target, depth + 1)
            return r1
        if not res.converged:
            raise RuntimeError(f"oracle Newton did not converge at load {target}: |R| = {res.residual:.3e}")
        hist["prev"], hist["l2"], hist["l1"] = dofs, hist["l1"], target
        dofs, kappa = d1, k1
        return res

    for s, lv in enumerate(load):
        res = advance(float(lv), 0)
        reac.append(res.reaction)
        iters.append(res.iterations)
        if keep_states:
            states.append((dofs.copy(), kappa.copy(), res.qinfo.copy()))
    return {"reaction": np.array(reac), "iterations": np.array(iters), "dofs": dofs, "kappa": kappa,
            "states": states, "cuts": hist["cuts"]}


# ---------------------------------------------------------------------------
# discrete adjoint of the load path
# ---------------------------------------------------------------------------
def adjoint_gradient(model: Model, mesh, load, dL_dF, rtol=1e-12, atol=1e-14):
    """Gradient dL/dtheta of a loss of the reaction curve, L(F_1..F_N) with the
    weights dL_dF[n] = dL/dF_n given, through the whole quasi-static path (Sec. 3.2
    monolithic steps), by the discrete adjoint with every state stored.  Step n has
    the equilibrium R_free(d_n, kappa_{n-1}; theta) = 0 with the local update
    kappa_n = K(d_n, kappa_{n-1}; theta) inside (Eq. (dd_7_no_nn)) and the reaction
    F_n = e_r . R(d_n, kappa_{n-1}; theta).  Backwards from n = N with mu_N = 0
    (mu_n = dL/dkappa_n, one entry per qp):
        K_ff^T lambda_n = w_n dF_n/dd + mu_n dK_n/dd            (free dofs)
        dL/dtheta     += w_n dF_n/dtheta + mu_n dK_n/dtheta - lambda_n . dR_free/dtheta
        mu_{n-1}       = w_n dF_n/dkappa_{n-1} + mu_n dK_n/dkappa_{n-1}
                         - lambda_n . dR_free/dkappa_{n-1}
    The partial derivatives come from the element routine (hyper-dual numbers,
    or_element_sens); the transposed systems are solved by sparse LU (the paper's
    direct solve).  Needs a path that converges without step cuts.  Returns
    (gradient [n_theta], reaction curve [N])."""
    res = run_load_path(model, mesh, load, rtol=rtol, atol=atol, keep_states=True)
    if res["cuts"]:
        raise RuntimeError("the adjoint check needs a path without step cuts")
    N = len(load)
    E, nq, nd_n = mesh.n_elems, mesh.nq, mesh.ndof
    n = mesh.n_nodes * nd_n
    edm = element_dof_map(mesh)                        # [E, nd]
    bidx, _ = dirichlet(mesh)
    free = np.ones(n, bool)
    free[bidx] = False
    fidx = np.nonzero(free)[0]
    er = np.zeros(n)
    er[mesh.react_node.astype(np.int64) * nd_n + mesh.react_comp] = 1.0
    nth = model.n_theta
    grad = np.zeros(nth)
    mu = np.zeros((E, nq))
    X = mesh.coords
    for s in range(N - 1, -1, -1):
        d = res["states"][s][0]
        kprev = res["states"][s - 1][1] if s > 0 else np.zeros((E, nq))
        R, Ke, _, _, _ = model.assemble(mesh, d, kprev)
        K = global_matrix(mesh, Ke)
        dR_th = np.zeros((n, nth))
        dR_kp = sp.lil_matrix((n, E * nq))
        dk_th = np.zeros((E, nq, nth))
        dk_kp = np.zeros((E, nq))
        dk_d = np.zeros(n)                             # mu_n . dK_n/dd, scattered to dofs
        for e in range(E):
            c = mesh.conn[e]
            a, b, cc, dd, ee = model.element_sens(X[c], d.reshape(-1, nd_n)[c], kprev[e])
            np.add.at(dR_th, edm[e], a)
            dk_th[e] = b
            for q in range(nq):
                dR_kp[edm[e], e * nq + q] = cc[:, q:q + 1]
            dk_kp[e] = dd
            np.add.at(dk_d, edm[e], mu[e] @ ee)
        dR_kp = dR_kp.tocsr()
        w = float(dL_dF[s])
        rhs = w * (K.T @ er) + dk_d
        Kff = K[fidx][:, fidx].tocsc()
        lam = np.zeros(n)
        lam[fidx] = spla.spsolve(Kff.T.tocsc(), rhs[fidx])
        grad += w * (er @ dR_th) + np.einsum("eq,eqk->k", mu, dk_th) - lam[fidx] @ dR_th[fidx]
        mu = (w * (dR_kp.T @ er) + (mu * dk_kp).ravel() - dR_kp[fidx].T @ lam[fidx]).reshape(E, nq)
    return grad, res["reaction"]


# ---------------------------------------------------------------------------
# homogeneous material-point driver (plane strain uniaxial)
# ---------------------------------------------------------------------------
def material_point_uniaxial(model: Model, stretches, tol=1e-13):
    """Homogeneous plane-strain uniaxial states F = diag(lam, lam2, 1) with P22 = 0.
    With grad phi = 0 the phi-equation gives phi = kappa, so q_nloc = 0 and on
    loading kappa = G(psi_e) (Sec. 5.1: local and non-local coincide when phi =
    kappa).  lam2 is found by a bracketed secant/bisection on P22.
    Returns arrays (P11, lam2, kappa) along the stretch history."""
    from scipy.optimize import brentq
    assert model.dim == 2
    kappa_n = 0.0
    out_P, out_l2, out_k = [], [], []
    lam2_prev = 1.0

    def state(lam, lam2, kn):
        z = np.zeros(7)
        z[0] = lam - 1.0
        z[3] = lam2 - 1.0
        pe = model.psi_value(z)
        G, _ = model.yield_G(pe)
        k = max(kn, G)
        z[4] = k
        dP, _, info = model.qp(z, kn, tangent=False)
        return dP, info

    for lam in stretches:
        f = lambda l2: state(lam, l2, kappa_n)[0][3]
        a, b = lam2_prev * 0.7, lam2_prev * 1.3
        fa, fb = f(a), f(b)
        k = 0
        while fa * fb > 0 and k < 60:
            a *= 0.9
            b *= 1.1
            fa, fb = f(a), f(b)
            k += 1
        l2 = brentq(f, a, b, xtol=tol, rtol=1e-15, maxiter=500)
        dP, info = state(lam, l2, kappa_n)
        kappa_n = info[0]
        lam2_prev = l2
        out_P.append(dP[0])
        out_l2.append(l2)
        out_k.append(kappa_n)
    return np.array(out_P), np.array(out_l2), np.array(out_k)


# ---------------------------------------------------------------------------
# homogeneous material-point driver (3D biaxial)
# ---------------------------------------------------------------------------
def material_point_biaxial(model: Model, stretches, tol=1e-13):
    """Homogeneous 3D states F = diag(lam, lam, lam3) with P33 = 0: equal stretch of
    the x and y faces, the z face traction free (the uniform-deformation block of
    Sec. 5.2 under biaxial load).  As in the plane-strain driver, grad phi = 0 makes
    the phi-equation give phi = kappa, so q_nloc = 0 and on loading kappa = G(psi_e)
    (Sec. 5.1).  lam3 is found by a bracketed root search on P33.
    Returns arrays (P11, lam3, kappa) along the stretch history; P11 is also the
    reaction of a unit cube's x = 1 face."""
    from scipy.optimize import brentq
    assert model.dim == 3
    kappa_n = 0.0
    out_P, out_l3, out_k = [], [], []
    lam3_prev = 1.0

    def state(lam, lam3, kn):
        z = np.zeros(13)
        z[0] = lam - 1.0
        z[4] = lam - 1.0
        z[8] = lam3 - 1.0
        pe = model.psi_value(z)
        G, _ = model.yield_G(pe)
        z[9] = max(kn, G)
        dP, _, info = model.qp(z, kn, tangent=False)
        return dP, info

    for lam in stretches:
        f = lambda l3: state(lam, l3, kappa_n)[0][8]
        a, b = lam3_prev * 0.7, lam3_prev * 1.3
        fa, fb = f(a), f(b)
        k = 0
        while fa * fb > 0 and k < 60:
            a *= 0.9
            b *= 1.1
            fa, fb = f(a), f(b)
            k += 1
        l3 = brentq(f, a, b, xtol=tol, rtol=1e-15, maxiter=500)
        dP, info = state(lam, l3, kappa_n)
        kappa_n = info[0]
        lam3_prev = l3
        out_P.append(dP[0])
        out_l3.append(l3)
        out_k.append(kappa_n)
    return np.array(out_P), np.array(out_l3), np.array(out_k)


def material_point_uniaxial_3d(model: Model, stretches, tol=1e-13):
    """Homogeneous 3D uniaxial states F = diag(lam, lam_t, lam_t) with P22 = P33 = 0
    (isotropic energies: the two lateral stretches are equal); phi = kappa as in the
    other drivers (Sec. 5.1).  Returns arrays (P11, lam_t, kappa)."""
    from scipy.optimize import brentq
    assert model.dim == 3
    kappa_n = 0.0
    out_P, out_l, out_k = [], [], []
    lt_prev = 1.0

    def state(lam, lt, kn):
        z = np.zeros(13)
        z[0] = lam - 1.0
        z[4] = lt - 1.0
        z[8] = lt - 1.0
        pe = model.psi_value(z)
        G, _ = model.yield_G(pe)
        z[9] = max(kn, G)
        dP, _, info = model.qp(z, kn, tangent=False)
        return dP, info

    for lam in stretches:
        f = lambda lt: state(lam, lt, kappa_n)[0][4]
        a, b = lt_prev * 0.7, lt_prev * 1.3
        fa, fb = f(a), f(b)
        k = 0
        while fa * fb > 0 and k < 60:
            a *= 0.9
            b *= 1.1
            fa, fb = f(a), f(b)
            k += 1
        lt = brentq(f, a, b, xtol=tol, rtol=1e-15, maxiter=500)
        dP, info = state(lam, lt, kappa_n)
        kappa_n = info[0]
        lt_prev = lt
        out_P.append(dP[0])
        out_l.append(lt)
        out_k.append(kappa_n)
    return np.array(out_P), np.array(out_l), np.array(out_k)
