"""CPU-side checks of the C ABI: the library loads, exports every function that
include/gd.h declares, its structs match the ctypes mirrors, and the host
logic (mesh validation, CSR pattern, slot map) matches a brute-force build."""
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2604_03411_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gd.h")


@pytest.fixture(scope="module")
def B():
    from paper_2604_03411_gb300 import build as build_mod
    build_mod.build()
    import paper_2604_03411_gb300.binding as binding
    binding.lib()
    return binding


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gd_[a-z_]+)\s*\(", src)))


def test_header_functions_exported(B):
    names = declared_functions()
    assert "gd_create" in names and "gd_backward" in names and len(names) >= 12
    L = B.lib()
    for n in names:
        assert hasattr(L, n), f"{n} declared in gd.h but not exported"
        assert n in B.PROTOTYPES, f"{n} has no binding prototype"
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gd_[a-z_]+)\b", out))
    assert set(names) <= exported


def test_struct_layout_matches_header(B):
    structs = {"gd_mesh": B.GdMesh, "gd_icnn": B.GdIcnn, "gd_material": B.GdMaterial,
               "gd_load_path": B.GdLoadPath, "gd_options": B.GdOptions, "gd_newton_report": B.GdNewtonReport,
               "gd_path_report": B.GdPathReport, "gd_tune_report": B.GdTuneReport}
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"gd.h\"\nint main(void){\n"
    for n in structs:
        prog += f'printf("{n} %zu\\n", sizeof({n}));\n'
    for f, _ in B.GdOptions._fields_:
        prog += f'printf("gd_options.{f} %zu\\n", offsetof(gd_options, {f}));\n'
    prog += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        lines = subprocess.check_output([exe], text=True).split("\n")
    sizes = dict(l.split() for l in lines if l.strip())
    for n, cls in structs.items():
        assert int(sizes[n]) == __import__("ctypes").sizeof(cls), n
    for f, _ in B.GdOptions._fields_:
        assert int(sizes[f"gd_options.{f}"]) == getattr(B.GdOptions, f).offset, f


def test_default_options(B):
    o = B.gd_default_options()
    assert o.precision == B.GD_FP64 and o.local_max == 100 and o.newton_max > 0 and o.krylov_rtol > 0


def brute_pattern(mesh):
    nd = mesh.ndof
    edm = (mesh.conn.astype(np.int64)[:, :, None] * nd + np.arange(nd)).reshape(mesh.n_elems, -1)
    k = edm.shape[1]
    rows = np.repeat(edm, k, axis=1).ravel()
    cols = np.tile(edm, (1, k)).ravel()
    n = mesh.n_nodes * nd
    A = sp.coo_matrix((np.ones(rows.size), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


@pytest.mark.parametrize("mk", ["q4", "hex8", "notch", "shuffled"])
def test_pattern_and_slot_map_brute_force(B, mk):
    if mk == "q4":
        mesh = I.uniaxial_bc_2d(I.structured_q4(7, 5))
    elif mk == "hex8":
        mesh = I.biaxial_bc_3d(I.structured_hex8(3, 4, 2))
    elif mk == "notch":
        mesh = I.uniaxial_bc_2d(I.notched_plate_q4(30, 12))
    else:
        mesh = I.uniaxial_bc_2d(I.structured_q4(6, 6))
        perm = np.random.default_rng(0).permutation(mesh.n_nodes)
        inv = np.argsort(perm)
        mesh.coords = mesh.coords[perm]
        mesh.conn = inv[mesh.conn].astype(np.int32)
        mesh.bc_node = inv[mesh.bc_node].astype(np.int32)
        mesh.react_node = inv[mesh.react_node].astype(np.int32)
    rowptr, colidx, slot = B.gd_build_pattern(mesh)
    A = brute_pattern(mesh)
    assert np.array_equal(rowptr, A.indptr) and np.array_equal(colidx, A.indices)
    nd = mesh.ndof
    for e in range(mesh.n_elems):
        for a in range(mesh.nen):
            na = mesh.conn[e, a]
            r0 = na * nd
            rowlen = rowptr[r0 + 1] - rowptr[r0]
            for b in range(mesh.nen):
                nb = mesh.conn[e, b]
                for i in range(nd):
                    for k in range(nd):
                        pos = slot[e, a, b] + i * rowlen + k
                        assert rowptr[r0 + i] <= pos < rowptr[r0 + i + 1]
                        assert colidx[pos] == nb * nd + k


def test_pattern_rejects_bad_meshes(B):
    mesh = I.uniaxial_bc_2d(I.structured_q4(3, 3))
    bad = I.uniaxial_bc_2d(I.structured_q4(3, 3))
    bad.conn = bad.conn[:, ::-1].copy()                       # clockwise: negative Jacobian
    with pytest.raises(B.GDError) as ei:
        B.gd_build_pattern(bad)
    assert ei.value.status == 2
    bad = I.uniaxial_bc_2d(I.structured_q4(3, 3))
    bad.conn = bad.conn.copy()
    bad.conn[0, 0] = 999
    with pytest.raises(B.GDError) as ei:
        B.gd_build_pattern(bad)
    assert ei.value.status == 2
    dup = I.uniaxial_bc_2d(I.structured_q4(3, 3))
    dup.bc_node = np.concatenate([dup.bc_node, dup.bc_node[:1]]).astype(np.int32)
    dup.bc_comp = np.concatenate([dup.bc_comp, dup.bc_comp[:1]]).astype(np.int8)
    dup.bc_scale = np.concatenate([dup.bc_scale, dup.bc_scale[:1]])
    with pytest.raises(B.GDError) as ei:
        B.gd_build_pattern(dup)
    assert ei.value.status == 1
    rowptr, colidx, slot = B.gd_build_pattern(mesh)
    assert rowptr[-1] == colidx.size


def test_notched_mesh_geometry():
    """The notched plate: positive Jacobians (checked by the library), the narrowest
    section at mid-length is width - 2 r, and elements near the notch are finer."""
    m = I.notched_plate_q4(120, 40)
    x, y = m.coords[:, 0], m.coords[:, 1]
    mid = np.abs(x - 1.0) < 1e-12
    assert abs((y[mid].max() - y[mid].min()) - 0.8) < 1e-12
    xs = np.unique(np.round(x, 12))
    dx = np.diff(xs)
    assert dx[np.argmin(np.abs(xs[:-1] - 1.0))] < 0.3 * dx.max()


def test_batch_create_rejects_bad_specimens(B):
    """gd_create_batch validates every specimen on the host before touching a
    device, naming the specimen in the message."""
    mat = I.Material()
    good = [I.Problem(f"s{i}", I.uniaxial_bc_2d(I.structured_q4(3 + i, 2)), *I.icnn_pair(i, 4, 4), mat,
                      np.linspace(0, 0.1, 3)[1:]) for i in range(3)]
    hexp = I.Problem("h", I.biaxial_bc_3d(I.structured_hex8(2, 2, 2)), *I.icnn_pair(9, 4, 4), mat,
                     np.linspace(0, 0.1, 3)[1:])
    with pytest.raises(B.GDError) as ei:
        B.gd_create_batch([good[0], hexp])
    assert ei.value.status == 1 and "specimen 1" in B.gd_last_error()
    bad = I.uniaxial_bc_2d(I.structured_q4(4, 2))
    bad.conn = bad.conn.copy()
    bad.conn[1, 2] = bad.n_nodes                    # one past this specimen's nodes
    with pytest.raises(B.GDError) as ei:
        B.gd_create_batch(good[:2] + [I.Problem("b", bad, *I.icnn_pair(5, 4, 4), mat, good[0].load)])
    assert ei.value.status == 2 and "specimen 2" in B.gd_last_error()
    flipped = I.uniaxial_bc_2d(I.structured_q4(3, 2))
    flipped.conn = flipped.conn[:, ::-1].copy()
    with pytest.raises(B.GDError) as ei:
        B.gd_create_batch(good[:1] + [I.Problem("f", flipped, *I.icnn_pair(6, 4, 4), mat, good[0].load)])
    assert ei.value.status == 2


def test_binding_constants_match_header_enums(B):
    """Every GD_* enumerator of include/gd.h has the same value in the binding."""
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gd.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    seen = 0
    for body in re.findall(r"enum\s*(?:gd_status\s*)?\{(.*?)\}", hdr, flags=re.S):
        for name, val in re.findall(r"(GD_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            assert hasattr(B, name), name
            assert getattr(B, name) == int(val), name
            seen += 1
    assert seen >= 30
