"""Seeded synthetic inputs: meshes, boundary sets, ICNN weights, load paths.

This module holds data generation only -- no part of the method's arithmetic
(no energy, no network evaluation, no residual).  Both the CUDA path and the
CPU oracle consume what it produces, so it imports neither.

Shapes follow the paper's studies (Sec. 5): a single-element / small square in
uniaxial load-unload-reload (Sec. 5.1), a uniformly deformed block (Sec. 5.2),
and a notched plate (Sec. 5.3).  The paper's trained weights and datasets are
not available (Sec. 5.1 cites literature data), so seeded random ICNN weights
stand in: weights |N(0, 0.1)|, biases N(0, 0.1), drawn from
``numpy.random.default_rng(seed)`` in the order W1, b1, W2, A2, b2, w3, a3 for
the energy network and then V1, c1, V2, B2, c2, v3, b3 for the yield network.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# energy kinds (shared integer codes with the C ABI)
ENERGY_ICNN_RAW = 0   # ICNN of (I1-3, I2-3, J-1)
ENERGY_ICNN_ISO = 1   # ICNN of (I1G-3, I2G-3, J-1)  (Sec. 4.2, Eq. dd_0)
ENERGY_NEO_HOOKE = 2  # closed-form compressible Neo-Hookean (Sec. 4.1)


@dataclass
class Mesh:
    dim: int                      # 2 (plane strain Q4) or 3 (HEX8)
    coords: np.ndarray            # [n_nodes, dim] float64, reference positions
    conn: np.ndarray              # [n_elems, nen] int32, counter-clockwise / standard HEX8 order
    bc_node: np.ndarray           # [n_bc] int32
    bc_comp: np.ndarray           # [n_bc] int8, displacement component (< dim)
    bc_scale: np.ndarray          # [n_bc] float64: prescribed value = scale * load(t)
    react_node: np.ndarray        # [n_react] int32
    react_comp: int = 0

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.conn.shape[0])

    @property
    def nen(self) -> int:
        return int(self.conn.shape[1])

    @property
    def ndof(self) -> int:
        return self.dim + 1

    @property
    def nq(self) -> int:
        return 4 if self.dim == 2 else 8


@dataclass
class ICNN:
    n_in: int
    width: int
    params: np.ndarray            # packed W1 b1 W2 A2 b2 w3 a3, float64


@dataclass
class Material:
    mu_e: float = 1.0
    lambda_e: float = 10.0
    eta_d: float = 1.0
    kappa_d: float = 0.05
    beta_d: float = 10.0
    c_d: float = 0.1              # beta_d * ell^2
    gamma_d: float = 1.0
    energy: int = ENERGY_ICNN_RAW


@dataclass
class Problem:
    name: str
    mesh: Mesh
    psi: ICNN
    yld: ICNN
    mat: Material
    load: np.ndarray              # [n_steps] load multiplier per step
    precision: str = "fp64"
    extra: dict = field(default_factory=dict)


def icnn_param_count(n_in: int, w: int) -> int:
    return w * n_in + w + w * w + w * n_in + w + w + n_in


def icnn_weights(rng: np.random.Generator, n_in: int, w: int) -> ICNN:
    """|N(0,0.1)| weights, N(0,0.1) biases, drawn in the packed order."""
    W1 = np.abs(rng.normal(0.0, 0.1, size=(w, n_in)))
    b1 = rng.normal(0.0, 0.1, size=w)
    W2 = np.abs(rng.normal(0.0, 0.1, size=(w, w)))
    A2 = np.abs(rng.normal(0.0, 0.1, size=(w, n_in)))
    b2 = rng.normal(0.0, 0.1, size=w)
    w3 = np.abs(rng.normal(0.0, 0.1, size=w))
    a3 = np.abs(rng.normal(0.0, 0.1, size=n_in))
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), A2.ravel(), b2, w3, a3]).astype(np.float64)
    assert p.size == icnn_param_count(n_in, w)
    return ICNN(n_in, w, p)


def icnn_pair(seed: int, w_psi: int, w_y: int):
    rng = np.random.default_rng(seed)
    psi = icnn_weights(rng, 3, w_psi)
    yld = icnn_weights(rng, 1, w_y)
    return psi, yld


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------
def structured_q4(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0) -> Mesh:
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    X, Y = np.meshgrid(xs, ys)                         # [ny+1, nx+1]
    coords = np.stack([X.ravel(), Y.ravel()], axis=1)
    return _q4_from_grid(coords, nx, ny)


def _q4_from_grid(coords: np.ndarray, nx: int, ny: int) -> Mesh:
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    i = i.ravel(); j = j.ravel()
    n0 = j * (nx + 1) + i
    conn = np.stack([n0, n0 + 1, n0 + nx + 2, n0 + nx + 1], axis=1).astype(np.int32)
    m = Mesh(2, coords.astype(np.float64), conn, np.zeros(0, np.int32), np.zeros(0, np.int8),
             np.zeros(0, np.float64), np.zeros(0, np.int32), 0)
    return m


def structured_hex8(nx: int, ny: int, nz: int, lx: float = 1.0, ly: float = 1.0, lz: float = 1.0) -> Mesh:
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    zs = np.linspace(0.0, lz, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")   # x fastest
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i = i.ravel(); j = j.ravel(); k = k.ravel()
    sx, sy = 1, nx + 1
    sz = (nx + 1) * (ny + 1)
    n0 = k * sz + j * sy + i
    conn = np.stack([n0, n0 + sx, n0 + sx + sy, n0 + sy,
                     n0 + sz, n0 + sz + sx, n0 + sz + sx + sy, n0 + sz + sy], axis=1).astype(np.int32)
    return Mesh(3, coords.astype(np.float64), conn, np.zeros(0, np.int32), np.zeros(0, np.int8),
                np.zeros(0, np.float64), np.zeros(0, np.int32), 0)


def notched_plate_q4(n_long: int, n_wide: int, length: float = 2.0, width: float = 1.0,
                     radius: float = 0.1, refine: float = 8.0, single_notch: bool = False) -> Mesh:
    """Mapped Q4 mesh of a plate [0, length] x [0, width] with semicircular edge
    notches of the given radius centred at mid-length on the bottom edge (and on
    the top edge unless ``single_notch``).  Columns are graded along x so that the
    element length near the notch is ``refine`` times smaller than far away;
    each column spans the notched height uniformly."""
    xc = 0.5 * length
    # target spacing h(x): small near the notch, large far away; nodes by equidistribution of 1/h
    s = np.linspace(0.0, length, 20001)
    h = 1.0 - (1.0 - 1.0 / refine) * np.exp(-((s - xc) / (2.5 * radius)) ** 2)
    dens = 1.0 / h
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(s))])
    cum /= cum[-1]
    xs = np.interp(np.linspace(0.0, 1.0, n_long + 1), cum, s)
    xs[0], xs[-1] = 0.0, length

    def notch_depth(x):
        d2 = radius * radius - (x - xc) ** 2
        return np.sqrt(np.maximum(d2, 0.0))

    ybot = notch_depth(xs)
    ytop = width - (0.0 if single_notch else 1.0) * notch_depth(xs)
    eta = np.linspace(0.0, 1.0, n_wide + 1)
    X = np.broadcast_to(xs[None, :], (n_wide + 1, n_long + 1))
    Y = ybot[None, :] + eta[:, None] * (ytop - ybot)[None, :]
    coords = np.stack([X.ravel(), Y.ravel()], axis=1)
    return _q4_from_grid(coords, n_long, n_wide)


def extrude_hex8(m2: Mesh, n_thick: int, thickness: float) -> Mesh:
    """HEX8 mesh of a Q4 mesh extruded along z through n_thick equal layers:
    node (i, layer k) = k * n_nodes_2d + i; each hexahedron is the quadrilateral on
    layer k followed by the same quadrilateral on layer k + 1 (the node order of
    structured_hex8)."""
    nn = m2.n_nodes
    zs = np.linspace(0.0, thickness, n_thick + 1)
    coords = np.concatenate([np.column_stack([m2.coords, np.full(nn, z)]) for z in zs])
    q = m2.conn.astype(np.int64)
    conn = np.concatenate([np.concatenate([q + k * nn, q + (k + 1) * nn], axis=1) for k in range(n_thick)])
    return Mesh(3, coords.astype(np.float64), conn.astype(np.int32), np.zeros(0, np.int32), np.zeros(0, np.int8),
                np.zeros(0, np.float64), np.zeros(0, np.int32), 0)


def notched_plate_hex8(n_long: int, n_wide: int, n_thick: int = 1, length: float = 1.0, width: float = 1.0,
                       thickness: float = 0.01, radius: float = 0.1) -> Mesh:
    """Thin 3D notched plate (the paper's 100 x 100 x 1 plate, nondimensionalised):
    the graded Q4 notched plate of notched_plate_q4 extruded through the thickness."""
    return extrude_hex8(notched_plate_q4(n_long, n_wide, length, width, radius), n_thick, thickness)


# ---------------------------------------------------------------------------
# boundary sets
# ---------------------------------------------------------------------------
def uniaxial_bc_2d(mesh: Mesh, scale: float = 1.0) -> Mesh:
    """Left edge u_x = 0, the node at the origin u_y = 0, right edge u_x = scale*load."""
    x = mesh.coords[:, 0]
    y = mesh.coords[:, 1]
    tol = 1e-9 * (x.max() - x.min())
    left = np.nonzero(np.abs(x - x.min()) < tol)[0]
    right = np.nonzero(np.abs(x - x.max()) < tol)[0]
    corner = left[np.argmin(y[left])]
    nodes = np.concatenate([left, [corner], right]).astype(np.int32)
    comps = np.concatenate([np.zeros(left.size), [1], np.zeros(right.size)]).astype(np.int8)
    scales = np.concatenate([np.zeros(left.size), [0.0], np.full(right.size, scale)]).astype(np.float64)
    mesh.bc_node, mesh.bc_comp, mesh.bc_scale = nodes, comps, scales
    mesh.react_node = right.astype(np.int32)
    mesh.react_comp = 0
    return mesh


def uniaxial_bc_3d(mesh: Mesh, scale: float = 1.0) -> Mesh:
    """Uniaxial pull of a 3D body along x: u_x = 0 on the x=min face, u_y = 0 on its
    y=min edge, u_z = 0 on the z=min face (a symmetry plane), u_x = scale*load on the
    x=max face; the reaction is the x force on that face."""
    c = mesh.coords
    lo = c.min(axis=0)
    hi = c.max(axis=0)
    tol = 1e-9 * float((hi - lo).max())
    left = np.nonzero(np.abs(c[:, 0] - lo[0]) < tol)[0]
    edge = left[np.abs(c[left, 1] - lo[1]) < tol]
    bottom = np.nonzero(np.abs(c[:, 2] - lo[2]) < tol)[0]
    right = np.nonzero(np.abs(c[:, 0] - hi[0]) < tol)[0]
    mesh.bc_node = np.concatenate([left, edge, bottom, right]).astype(np.int32)
    mesh.bc_comp = np.concatenate([np.zeros(left.size), np.ones(edge.size), np.full(bottom.size, 2),
                                   np.zeros(right.size)]).astype(np.int8)
    mesh.bc_scale = np.concatenate([np.zeros(left.size + edge.size + bottom.size),
                                    np.full(right.size, scale)]).astype(np.float64)
    mesh.react_node = right.astype(np.int32)
    mesh.react_comp = 0
    return mesh


def biaxial_bc_3d(mesh: Mesh) -> Mesh:
    """Rollers on the x=0, y=0, z=0 faces; x=max and y=max faces displaced by load
    (u_x = load * lx on x=max, u_y = load * ly on y=max); the z=max face is free."""
    c = mesh.coords
    lo = c.min(axis=0)
    hi = c.max(axis=0)
    tol = 1e-9 * float((hi - lo).max())
    nodes, comps, scales = [], [], []
    for k in range(3):
        f = np.nonzero(np.abs(c[:, k] - lo[k]) < tol)[0]
        nodes.append(f); comps.append(np.full(f.size, k)); scales.append(np.zeros(f.size))
    for k in range(2):
        f = np.nonzero(np.abs(c[:, k] - hi[k]) < tol)[0]
        nodes.append(f); comps.append(np.full(f.size, k)); scales.append(np.full(f.size, hi[k] - lo[k]))
    mesh.bc_node = np.concatenate(nodes).astype(np.int32)
    mesh.bc_comp = np.concatenate(comps).astype(np.int8)
    mesh.bc_scale = np.concatenate(scales).astype(np.float64)
    mesh.react_node = np.nonzero(np.abs(c[:, 0] - hi[0]) < tol)[0].astype(np.int32)
    mesh.react_comp = 0
    return mesh


# ---------------------------------------------------------------------------
# load paths
# ---------------------------------------------------------------------------
def piecewise_path(points: List[float], steps: List[int]) -> np.ndarray:
    out = []
    for a, b, n in zip(points[:-1], points[1:], steps):
        out.append(np.linspace(a, b, n + 1)[1:])
    return np.concatenate(out).astype(np.float64)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------
def config1(seed: int = 1, n: int = 8) -> Problem:
    """2D plane-strain unit square, n x n Q4, uniaxial stretch 1 -> 2.0 -> 1.0 -> 2.2
    in 13 + 12 + 15 steps; psi-ICNN width 16, yield-ICNN width 8; ell = 0.1; FP64."""
    mesh = uniaxial_bc_2d(structured_q4(n, n))
    psi, yld = icnn_pair(seed, 16, 8)
    ell = 0.1
    mat = Material(beta_d=10.0, c_d=10.0 * ell * ell)
    load = piecewise_path([0.0, 1.0, 0.0, 1.2], [13, 12, 15])      # u_x(right) = lambda - 1
    return Problem("square8_q4_uniaxial_cycle", mesh, psi, yld, mat, load, "fp64")


def config2(seed: int = 2, n_long: int = 312, n_wide: int = 128, ell: float = 0.02, n_steps: int = 50) -> Problem:
    """2D notched plate 2:1, semicircular edge notches radius 0.1 at mid-length,
    graded Q4 mesh (~40k elements for the defaults), 50 steps to 60% nominal strain,
    both ICNNs width 32, ell = 0.02 (or 0.04); FP64."""
    mesh = uniaxial_bc_2d(notched_plate_q4(n_long, n_wide))
    psi, yld = icnn_pair(seed, 32, 32)
    mat = Material(beta_d=10.0, c_d=10.0 * ell * ell)
    load = np.linspace(0.0, 0.6 * 2.0, n_steps + 1)[1:]
    return Problem(f"notched_plate_q4_{mesh.n_elems}", mesh, psi, yld, mat, load, "fp64")


def config3(seed: int = 3, n: int = 64, n_steps: int = 30, precision: str = "mixed") -> Problem:
    """3D unit cube, n^3 HEX8, biaxial stretch to lambda = 1.8 in 30 steps, both ICNNs width 64."""
    mesh = biaxial_bc_3d(structured_hex8(n, n, n))
    psi, yld = icnn_pair(seed, 64, 64)
    ell = 0.1
    mat = Material(beta_d=10.0, c_d=10.0 * ell * ell)
    load = np.linspace(0.0, 0.8, n_steps + 1)[1:]
    return Problem(f"cube_hex8_{n}", mesh, psi, yld, mat, load, precision)


def config4(seed: int = 4, n_long: int = 222, n_wide: int = 90, n_steps: int = 30) -> Problem:
    """Adjoint calibration workload: notched plate ~20k Q4, 30 steps, both ICNNs width 32.
    ``extra['theta_star']`` holds the target weights: a seeded ~5% perturbation (seed 40)."""
    mesh = uniaxial_bc_2d(notched_plate_q4(n_long, n_wide))
    psi, yld = icnn_pair(seed, 32, 32)
    mat = Material(beta_d=10.0, c_d=10.0 * 0.04 ** 2)
    load = np.linspace(0.0, 0.3 * 2.0, n_steps + 1)[1:]
    rng = np.random.default_rng(40)
    theta = np.concatenate([psi.params, yld.params])
    theta_star = theta * (1.0 + 0.05 * rng.standard_normal(theta.size))
    # weights must stay nonnegative (biases may have any sign); the perturbation is multiplicative
    fd_rng = np.random.default_rng(41)
    fd_idx = fd_rng.choice(theta.size, size=20, replace=False)
    return Problem(f"notched_plate_q4_{mesh.n_elems}_adjoint", mesh, psi, yld, mat, load, "fp64",
                   extra={"theta_star": theta_star, "fd_index": fd_idx, "checkpoint_every": 5})


def notched_plate_3d(seed: int = 6, n_long: int = 49, n_wide: int = 48, n_steps: int = 100, ell: float = 0.04,
                     width_psi: int = 32, width_yield: int = 32, precision: str = "fp64") -> Problem:
    """The paper's 3D notched-plate geometry: a thin square plate (thickness 1/100 of
    its side) with semicircular edge notches, one HEX8 layer; 2,352 elements for the
    defaults (the paper's finest mesh has 2,350; 16 x 15 and 26 x 24 give its 241
    and 625), pulled along x to 25% nominal strain in n_steps steps."""
    mesh = uniaxial_bc_3d(notched_plate_hex8(n_long, n_wide))
    psi, yld = icnn_pair(seed, width_psi, width_yield)
    mat = Material(beta_d=10.0, c_d=10.0 * ell * ell)
    load = np.linspace(0.0, 0.25, n_steps + 1)[1:]
    return Problem(f"notched_plate_hex8_{mesh.n_elems}", mesh, psi, yld, mat, load, precision)


def uniform_plate_e3(n: int = 5, n_steps: int = 40, u_max: float = 1.0, gamma_d: float = 1.0) -> Problem:
    """The uniform-deformation study of Sec. 5.2: a 10 x 10 x 1 plate (n x n x 1 HEX8)
    pulled along x with lateral faces free, the closed-form Neo-Hookean energy with
    the Ostwald loading function (G(q) = q) and the constants the paper lists
    (E = 210, nu = 0.3, eta_d = 0.002, kappa_d = 0.1, c_d = 1, beta_d = 1000, read as
    nondimensional), u_x to u_max in n_steps; gamma_d = 0 is the local model."""
    mesh = uniaxial_bc_3d(structured_hex8(n, n, 1, 10.0, 10.0, 1.0), scale=10.0)
    E, nu = 210.0, 0.3
    mat = Material(mu_e=E / (2.0 * (1.0 + nu)), lambda_e=E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), eta_d=0.002,
                   kappa_d=0.1, beta_d=1000.0, c_d=1.0, gamma_d=gamma_d, energy=ENERGY_NEO_HOOKE)
    psi = ICNN(3, 0, np.zeros(1))
    yld = ICNN(1, 0, np.zeros(1))
    load = np.linspace(0.0, u_max / 10.0, n_steps + 1)[1:]        # nominal strain: u_x(x = 10) = 10 load
    return Problem(f"uniform_plate_e3_{n}x{n}", mesh, psi, yld, mat, load, "fp64")


def config5(seed: int = 5, n_specimens: int = 96) -> List[Problem]:
    """96 independent specimens: structured Q4 nx ~ U{16..96} x ny ~ U{16..48}, each with
    its own seeded weight set (width in {16, 24, 32}) and a uniaxial path of U{20..60}
    steps to lambda = 2.0; mixed precision."""
    out = []
    for i in range(n_specimens):
        rng = np.random.default_rng(5000 + i)
        nx = int(rng.integers(16, 97))
        ny = int(rng.integers(16, 49))
        w = int(rng.choice([16, 24, 32]))
        steps = int(rng.integers(20, 61))
        h = 1.0 / ny
        mesh = uniaxial_bc_2d(structured_q4(nx, ny, nx * h, 1.0), scale=1.0)
        psi = icnn_weights(rng, 3, w)
        yld = icnn_weights(rng, 1, w)
        mat = Material(beta_d=10.0, c_d=10.0 * 0.1 ** 2)
        load = np.linspace(0.0, 1.0 * nx * h, steps + 1)[1:]
        out.append(Problem(f"specimen{i}_{nx}x{ny}_w{w}", mesh, psi, yld, mat, load, "mixed"))
    return out


def random_state(mesh: Mesh, rng: np.random.Generator, u_amp: float = 0.05, phi_amp: float = 0.2,
                 kappa_amp: float = 0.2, kappa_nq: Optional[int] = None):
    """Seeded random nodal dofs (node-major [n_nodes, ndof]) and history kappa_n [n_elems, nq]:
    smooth displacement field plus noise, phi in [0, phi_amp], kappa_n in [0, kappa_amp]."""
    x = mesh.coords
    ndof = mesh.dim + 1
    d = np.zeros((mesh.n_nodes, ndof))
    for c in range(mesh.dim):
        A = rng.normal(0.0, u_amp, size=(mesh.dim,))
        d[:, c] = x @ A + 0.2 * u_amp * rng.standard_normal(mesh.n_nodes)
    d[:, mesh.dim] = phi_amp * rng.random(mesh.n_nodes)
    nq = kappa_nq or mesh.nq
    kappa = kappa_amp * rng.random((mesh.n_elems, nq))
    return d, kappa
