"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np
import scipy.sparse as sp


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max() if b.size else 0.0
    if den == 0.0:
        return float(np.abs(a).max()) if a.size else 0.0
    return float(np.abs(a - b).max() / den)


def gpu_assemble(B, torch, h, dofs, kappa, precision="fp64"):
    """(R, K csr, kappa_new, loading) from one gd_assemble call."""
    dev = torch.device("cuda:0")
    rowptr, colidx = B.gd_csr_pattern(h)
    d = torch.tensor(np.ascontiguousarray(dofs).ravel(), dtype=torch.float64, device=dev)
    k = torch.tensor(np.ascontiguousarray(kappa).ravel(), dtype=torch.float64, device=dev)
    R = torch.zeros(d.numel(), dtype=torch.float64, device=dev)
    vt = torch.float64 if precision == "fp64" else torch.float32
    vals = torch.zeros(colidx.size, dtype=vt, device=dev)
    k1 = torch.zeros_like(k)
    ld = torch.zeros(k.numel(), dtype=torch.int8, device=dev)
    B.gd_assemble(h, d, k, R, vals, k1, ld, B.GD_ASM_TANGENT)
    torch.cuda.synchronize()
    n = d.numel()
    K = sp.csr_matrix((vals.double().cpu().numpy(), colidx, rowptr), shape=(n, n))
    return R.cpu().numpy(), K, k1.cpu().numpy().reshape(kappa.shape), ld.cpu().numpy().reshape(kappa.shape)


def oracle_assemble(oracle, prob, dofs, kappa):
    model = oracle.Model.from_problem(prob)
    R, Ke, k1, qi, nf = model.assemble(prob.mesh, dofs, kappa)
    return R, oracle.global_matrix(prob.mesh, Ke), k1, qi


def compare_assembly(Rg, Kg, kg, lg, Ro, Ko, ko, qi, tol=1e-10):
    """Element-by-element comparison; loading flags bit-exact except at points whose
    trial yield value is within 1e-9 of the switch (both branches valid there)."""
    eR = rel_err(Rg, Ro)
    dK = (Kg - Ko).tocoo()
    eK = float(np.abs(dK.data).max() / np.abs(Ko.data).max()) if dK.nnz else 0.0
    ek = rel_err(kg, ko)
    lo = qi[..., 5] > 0.5
    ambiguous = np.abs(qi[..., 3]) < 1e-9 * np.maximum(1.0, np.abs(ko))
    flags_ok = np.all((lg.astype(bool) == lo) | ambiguous)
    # the library's node-block pattern is exactly the set of element dof pairs
    Kg.sort_indices()
    Ko.sort_indices()
    assert np.array_equal(Kg.indptr, Ko.indptr) and np.array_equal(Kg.indices, Ko.indices), "CSR pattern differs"
    return eR, eK, ek, flags_ok


def node_size(mesh):
    """Shortest edge of the elements around every node (graded meshes vary 8x)."""
    x = mesh.coords
    c = mesh.conn
    nen = c.shape[1]
    edges = [(0, 1), (1, 2), (2, 3), (3, 0)]
    if nen == 8:
        edges = edges + [(a + 4, b + 4) for a, b in edges] + [(a, a + 4) for a in range(4)]
    le = np.min([np.linalg.norm(x[c[:, a]] - x[c[:, b]], axis=1) for a, b in edges], axis=0)
    h = np.full(mesh.n_nodes, np.inf)
    for a in range(nen):
        np.minimum.at(h, c[:, a], le)
    return h


def smooth_state(mesh, rng, u_amp=0.05, noise=0.1, phi_amp=0.3, kappa_amp=0.3):
    """Affine displacement plus nodal noise scaled by the local element size (so that
    fine and graded meshes stay far from inversion), phi in [0, phi_amp], kappa_n in
    [0, kappa_amp]."""
    x = mesh.coords
    h = node_size(mesh)
    d = np.zeros((mesh.n_nodes, mesh.ndof))
    for c in range(mesh.dim):
        A = rng.normal(0.0, u_amp, size=mesh.dim)
        d[:, c] = x @ A + noise * h * rng.uniform(-1.0, 1.0, mesh.n_nodes)
    d[:, mesh.dim] = phi_amp * rng.random(mesh.n_nodes)
    kappa = kappa_amp * rng.random((mesh.n_elems, mesh.nq))
    return d, kappa
