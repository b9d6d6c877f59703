"""Host logic of the two-level preconditioner's coarse space (no GPU): the
breadth-first aggregation of the node graph covers every node once, keeps every
aggregate connected, sizes the aggregates near the target, and reduces to the
trivial partitions at the extremes; checked against an independent graph built
from the element connectivity."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

from paper_2604_03411_gb300 import inputs as I


@pytest.fixture(scope="module")
def B():
    from paper_2604_03411_gb300 import build as build_mod
    build_mod.build()
    import paper_2604_03411_gb300.binding as binding
    binding.lib()
    return binding


def node_graph(mesh):
    """Node adjacency (nodes sharing an element), from the connectivity alone."""
    conn = np.asarray(mesh.conn, np.int64)
    e = np.repeat(np.arange(conn.shape[0]), conn.shape[1])
    Ne = sp.csr_matrix((np.ones(conn.size), (e, conn.ravel())), shape=(conn.shape[0], mesh.n_nodes))
    return (Ne.T @ Ne).tocsr()


def check_partition(mesh, agg, n_agg):
    assert agg.shape == (mesh.n_nodes,)
    assert agg.min() == 0 and agg.max() == n_agg - 1
    assert np.unique(agg).size == n_agg
    G = node_graph(mesh)
    for a in range(n_agg):
        idx = np.nonzero(agg == a)[0]
        sub = G[idx][:, idx]
        ncomp, _ = csg.connected_components(sub, directed=False)
        assert ncomp == 1, f"aggregate {a} is not connected"
    return np.bincount(agg)


@pytest.mark.parametrize("target", [9, 25, 80])
def test_notched_plate_aggregates(B, target):
    mesh = I.uniaxial_bc_2d(I.notched_plate_q4(60, 24))
    agg, n_agg = B.gd_coarse_aggregates(mesh, target)
    sizes = check_partition(mesh, agg, n_agg)
    assert sizes.max() <= target + target // 4 * 8      # a full aggregate plus a few merged remnants
    assert sizes.min() >= 1
    # the greedy search fills most aggregates to the target
    assert np.median(sizes) >= 0.5 * target
    again, n2 = B.gd_coarse_aggregates(mesh, target)
    assert n2 == n_agg and np.array_equal(again, agg)


def test_hex8_aggregates(B):
    mesh = I.biaxial_bc_3d(I.structured_hex8(7, 6, 5))
    agg, n_agg = B.gd_coarse_aggregates(mesh, 27)
    sizes = check_partition(mesh, agg, n_agg)
    assert sizes.sum() == mesh.n_nodes
    assert np.median(sizes) >= 13


def test_extremes(B):
    mesh = I.uniaxial_bc_2d(I.structured_q4(5, 4))
    agg, n_agg = B.gd_coarse_aggregates(mesh, 1)
    assert n_agg == mesh.n_nodes and np.array_equal(np.sort(agg), np.arange(mesh.n_nodes))
    agg, n_agg = B.gd_coarse_aggregates(mesh, 10 * mesh.n_nodes)
    assert n_agg == 1 and np.all(agg == 0)


def test_small_remnants_are_merged(B):
    """Brute force on a 1 x n strip of Q4 elements (a path-like node graph): every
    aggregate ends with at least a quarter of the target nodes."""
    mesh = I.uniaxial_bc_2d(I.structured_q4(13, 1))
    for target in (3, 4, 6, 8):
        agg, n_agg = B.gd_coarse_aggregates(mesh, target)
        sizes = check_partition(mesh, agg, n_agg)
        assert sizes.min() >= max(1, target // 4)


def test_bad_arguments(B):
    mesh = I.uniaxial_bc_2d(I.structured_q4(3, 3))
    with pytest.raises(B.GDError):
        B.gd_coarse_aggregates(mesh, 0)


def rigid_and_constant_modes(coords, nodes, ndof):
    """Constant field of every nodal unknown and the rigid rotations of the
    displacement on the given nodes (about their centroid): [len(nodes) * ndof, m]."""
    dim = coords.shape[1]
    x = coords[nodes] - coords[nodes].mean(axis=0)
    cols = []
    for k in range(ndof):
        v = np.zeros((len(nodes), ndof)); v[:, k] = 1.0; cols.append(v.ravel())
    pairs = [(0, 1)] if dim == 2 else [(1, 2), (2, 0), (0, 1)]
    for a, b in pairs:
        v = np.zeros((len(nodes), ndof)); v[:, a] = -x[:, b]; v[:, b] = x[:, a]; cols.append(v.ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("dim,target", [(2, 20), (2, 5), (3, 27)])
def test_coarse_basis_orthonormal_and_spanning(B, dim, target):
    """Per aggregate: the kept columns are orthonormal, vanish on prescribed dofs, and
    span the constant fields and rigid rotations restricted to the free dofs."""
    if dim == 2:
        mesh = I.uniaxial_bc_2d(I.notched_plate_q4(24, 10))
    else:
        mesh = I.biaxial_bc_3d(I.structured_hex8(6, 5, 4))
    ndof = dim + 1
    agg, coff, P = B.gd_coarse_basis(mesh, target)
    n_agg = coff.size - 1
    fixed = np.zeros((mesh.n_nodes, ndof), bool)
    fixed[mesh.bc_node, mesh.bc_comp] = True
    assert np.all(P[fixed] == 0.0)
    full = 0
    for a in range(n_agg):
        nodes = np.nonzero(agg == a)[0]
        k = coff[a + 1] - coff[a]
        assert 1 <= k <= P.shape[2]
        assert np.all(P[nodes][:, :, k:] == 0.0)
        Q = P[nodes][:, :, :k].reshape(len(nodes) * ndof, k).astype(np.float64)
        assert np.abs(Q.T @ Q - np.eye(k)).max() < 1e-5
        M = rigid_and_constant_modes(mesh.coords, nodes, ndof)
        M[fixed[nodes].ravel()] = 0.0
        resid = M - Q @ (Q.T @ M)
        assert np.abs(resid).max() <= 1e-5 * max(np.abs(M).max(), 1.0)
        full += k == P.shape[2]
    assert full >= n_agg // 2                                   # most aggregates keep every mode


def test_degenerate_meshes(B):
    """Nodes no element touches form aggregates of their own (the node graph has only
    self-loops there); an aggregate whose displacements are all prescribed keeps only
    the damage field's constant (the rotation and displacement columns vanish)."""
    m = I.uniaxial_bc_2d(I.structured_q4(3, 2))
    n_used = m.n_nodes
    m.coords = np.concatenate([m.coords, [[5.0, 5.0], [6.0, 5.0]]])     # two isolated nodes
    agg, n_agg = B.gd_coarse_aggregates(m, 4)
    assert agg[n_used] != agg[n_used + 1]
    assert np.sum(agg == agg[n_used]) == 1 and np.sum(agg == agg[n_used + 1]) == 1
    # every dof of one isolated node prescribed: its aggregate keeps no column
    m.bc_node = np.concatenate([m.bc_node, [n_used, n_used]]).astype(np.int32)
    m.bc_comp = np.concatenate([m.bc_comp, [0, 1]]).astype(np.int8)
    m.bc_scale = np.concatenate([m.bc_scale, [0.0, 0.0]])
    agg, coff, P = B.gd_coarse_basis(m, 4)
    a = agg[n_used]
    assert coff[a + 1] - coff[a] == 1                     # only the damage field's constant remains
    assert np.all(P[n_used, :2, :] == 0.0)
