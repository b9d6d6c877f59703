"""Synthetic 3D notched plate (thin HEX8 plate extruded from the graded Q4 notched
plate) and its uniaxial boundary set, checked on CPU: every hexahedron has a
positive Jacobian at its Gauss points, the extrusion's volume is the extruded
area times the thickness (a prism over planar quadrilaterals), the boundary set
prescribes each (node, component) once and removes all six rigid-body modes,
and the library accepts the mesh."""
import itertools

import numpy as np
import pytest

from paper_2604_03411_gb300 import inputs as I

G = 1.0 / np.sqrt(3.0)


def quad_areas(m2):
    x = m2.coords[m2.conn]                                  # [E, 4, 2]
    xs, ys = x[..., 0], x[..., 1]
    return 0.5 * np.abs(np.sum(xs * np.roll(ys, -1, 1) - np.roll(xs, -1, 1) * ys, axis=1))


def hex_detJ(m3):
    """det J at the 2x2x2 Gauss points of every trilinear hexahedron [E, 8]."""
    X = m3.coords[m3.conn]                                  # [E, 8, 3]
    corners = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                        [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], float)
    out = []
    for xi in itertools.product((-G, G), repeat=3):
        dN = np.empty((8, 3))
        for a, c in enumerate(corners):
            f = [(1 + c[k] * xi[k]) / 2 for k in range(3)]
            for k in range(3):
                g = c[k] / 2
                dN[a, k] = g * f[(k + 1) % 3] * f[(k + 2) % 3]
        J = np.einsum("eaj,ak->ejk", X, dN)
        out.append(np.linalg.det(J))
    return np.stack(out, axis=1)


@pytest.mark.parametrize("nl,nw,nt", [(16, 15, 1), (26, 24, 1), (12, 6, 3)])
def test_extruded_plate_geometry(nl, nw, nt):
    t = 0.01
    m3 = I.notched_plate_hex8(nl, nw, nt, thickness=t)
    m2 = I.notched_plate_q4(nl, nw, 1.0, 1.0)
    assert m3.n_elems == nl * nw * nt and m3.n_nodes == (nl + 1) * (nw + 1) * (nt + 1)
    dj = hex_detJ(m3)
    assert np.all(dj > 0.0)
    vol = dj.sum() * 1.0                                    # Gauss weights are 1
    assert abs(vol - t * quad_areas(m2).sum()) <= 1e-12 * vol


def test_uniaxial_bc_3d_removes_rigid_modes():
    m = I.uniaxial_bc_3d(I.notched_plate_hex8(10, 8, 2))
    pairs = set(zip(m.bc_node.tolist(), m.bc_comp.tolist()))
    assert len(pairs) == m.bc_node.size                     # each (node, component) once
    # the six rigid modes restricted to the prescribed components are independent
    c = m.coords - m.coords.mean(axis=0)
    modes = []
    for k in range(3):
        u = np.zeros((m.n_nodes, 3)); u[:, k] = 1.0; modes.append(u)
    for a, b in ((0, 1), (1, 2), (2, 0)):
        u = np.zeros((m.n_nodes, 3)); u[:, a] = -c[:, b]; u[:, b] = c[:, a]; modes.append(u)
    R = np.array([[u[n, k] for n, k in zip(m.bc_node, m.bc_comp)] for u in modes])
    assert np.linalg.matrix_rank(R) == 6
    right = np.abs(m.coords[:, 0] - m.coords[:, 0].max()) < 1e-12
    assert set(m.react_node.tolist()) == set(np.nonzero(right)[0].tolist())
    assert np.all(m.bc_scale[m.bc_comp == 0][np.isin(m.bc_node[m.bc_comp == 0], m.react_node)] == 1.0)


def test_library_accepts_the_3d_plate():
    from paper_2604_03411_gb300 import build as build_mod
    build_mod.build()
    import paper_2604_03411_gb300.binding as B
    p = I.notched_plate_3d(n_long=16, n_wide=15, n_steps=4)
    rowptr, colidx, slot = B.gd_build_pattern(p.mesh)
    assert rowptr.size == p.mesh.n_nodes * 4 + 1 and slot.shape == (p.mesh.n_elems, 8, 8)
