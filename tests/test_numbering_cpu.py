"""Host logic of the C0 assembly, on the CPU: the library's global numbering
(nir_c0_numbering, no GPU involved) against the numbering-free conforming
space of ``oracle/conforming.py``.  A global vector mapped to the elements
through the numbering (x_loc[i] = s_i x[g_i]) must be continuous, vanish on
the boundary when only free dofs are set, and the sizes must equal the closed
forms (nP+1)^d and (nP-1)^d; for the modified and the GLL-Lagrange basis
(whose numbering has no signs)."""
import ctypes as C
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import conforming as cf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2606_20917_gb300", "libnir.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import importlib.util
        spec = importlib.util.spec_from_file_location("nb", os.path.join(ROOT, "paper_2606_20917_gb300", "build.py"))
        m = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(m)
        m.build()
    lib = C.CDLL(LIB)
    lib.nir_c0_numbering.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.nir_c0_numbering.restype = C.c_int
    return lib


def numbering(lib, shape, P, vert_blocks, basis="modified"):
    M = oracle.num_modes(shape, max(P, 1))
    nel = np.array([v.shape[0] for v in vert_blocks], dtype=np.int64)
    vs = [np.ascontiguousarray(v, dtype=np.int64) for v in vert_blocks]
    ptrs = (C.c_void_p * len(vs))(*[v.ctypes.data for v in vs])
    out = np.zeros(int(nel.sum()) * M, dtype=np.int64)
    ng, nf = C.c_int64(), C.c_int64()
    rc = lib.nir_c0_numbering({"quad": 0, "hex": 2}[shape], P, {"modified": 0, "nodal": 1}[basis], len(vs),
                              nel.ctypes.data, ptrs, out.ctypes.data, C.byref(ng), C.byref(nf))
    return rc, out, ng.value, nf.value


@pytest.mark.parametrize("basis", ["modified", "nodal"])
@pytest.mark.parametrize("shape,n,P,rotate,split", [("quad", 3, 1, False, 1), ("quad", 3, 4, True, 2),
                                                    ("hex", 2, 1, True, 1), ("hex", 2, 2, False, 1),
                                                    ("hex", 2, 4, True, 3), ("hex", 3, 3, True, 2),
                                                    ("hex", 2, 5, True, 1)])
def test_numbering_is_conforming(lib, shape, n, P, rotate, split, basis):
    d = 2 if shape == "quad" else 3
    nodes = W.quad_grid(n, n) if d == 2 else W.hex_grid(n, 1, amp=0.0)
    verts = W.grid_vertices(n, d)
    if rotate:
        nodes, verts, _ = W.rotate_elements(nodes, verts, 1, seed=n * 10 + P)
    cuts = np.linspace(0, verts.shape[0], split + 1).astype(int)
    rc, mp, ng, nf = numbering(lib, shape, P, [verts[a:b] for a, b in zip(cuts[:-1], cuts[1:])], basis)
    assert rc == 0
    if basis == "nodal":
        assert (mp > 0).all()
    assert ng == (n * P + 1) ** d and nf == (n * P - 1) ** d
    assert np.array_equal(np.unique(np.abs(mp)), np.arange(1, ng + 1))
    Z = cf.conforming_basis(shape, P, verts, dirichlet=False, basis=basis)
    Z0 = cf.conforming_basis(shape, P, verts, dirichlet=True, basis=basis)
    rng = np.random.default_rng(P)
    x = rng.uniform(-1, 1, ng)
    xl = np.sign(mp) * x[np.abs(mp) - 1]
    assert np.linalg.norm(xl - Z @ (Z.T @ xl)) <= 1e-12 * np.linalg.norm(xl)
    x[nf:] = 0.0
    xl0 = np.sign(mp) * x[np.abs(mp) - 1]
    assert np.linalg.norm(xl0 - Z0 @ (Z0.T @ xl0)) <= 1e-12 * np.linalg.norm(xl0)
    # the numbering spans the whole space: the local images of all global dofs
    # have the space's dimension
    A = np.zeros((xl.size, ng))
    A[np.arange(xl.size), np.abs(mp) - 1] = np.sign(mp)
    assert np.linalg.matrix_rank(A) == Z.shape[1]


def test_numbering_rejects_bad_input(lib):
    verts = W.grid_vertices(2, 3)
    bad = verts.copy()
    bad[1] = bad[0]
    bad[2] = bad[0]                      # a face held by three elements
    assert numbering(lib, "hex", 2, [bad])[0] == -1
    assert numbering(lib, "quad", 0, [W.grid_vertices(2, 2)])[0] == -1
    assert numbering(lib, "hex", 2, [verts], basis="nodal")[0] == 0
    nel = np.array([verts.shape[0]], dtype=np.int64)
    ptrs = (C.c_void_p * 1)(verts.ctypes.data)
    assert lib.nir_c0_numbering(2, 2, 7, 1, nel.ctypes.data, ptrs, None, None, None) == -1   # unknown basis
