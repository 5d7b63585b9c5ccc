"""The library's host tables (``csrc/nir_basis.cpp``: quadrature, modified
basis, collocation derivatives and the even/odd form) against the oracle's
independent quadrature and Jacobi code (no GPU involved).

A small program (``tests/host/tables.cpp``) dumps the table blob of every
shape for P = 1..9; each entry is recomputed here from the oracle's points and
weights (``oracle.ref_points``, collapse factors included), its Jacobi
polynomials (``oracle.jacobi``) and its collocation matrices
(``oracle.colloc_1d``), following the basis reading of the modified C0
expansion:
  psiA_0 = (1-z)/2, psiA_1 = (1+z)/2, psiA_p = (1-z)(1+z)/4 P^(1,1)_{p-2}(z);
  psiB_0q = psiA_q, psiB_p0 = ((1-z)/2)^p,
  psiB_pq = ((1-z)/2)^p (1+z)/2 P^(2p-1,1)_{q-1}(z)  (p, q >= 1);
  the tetrahedron's third direction uses psiB_cr with c = p + q, the
  pyramid's with c = max(p, q).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_20917_gb300", "csrc")
SHAPES = {"quad": 0, "tri": 1, "hex": 2, "prism": 3, "tet": 4, "pyr": 5}


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ is not available")
    exe = str(tmp_path_factory.mktemp("tables") / "tables")
    cmd = [gxx, "-O1", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "host", "tables.cpp"),
           os.path.join(CSRC, "nir_basis.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]

    def run(shape, P):
        r = subprocess.run([exe, str(SHAPES[shape]), str(P)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        lines = r.stdout.split("\n")
        L = dict(zip(["Ba", "Bb", "Bc", "D1", "D2", "D3", "wq", "Bs", "total"], map(int, lines[0].split())))
        blob = np.array([float(t) for t in lines[1:] if t])
        assert blob.size == L["total"]
        return L, blob
    return run


def psiA(p, z):
    if p == 0:
        return (1 - z) / 2
    if p == 1:
        return (1 + z) / 2
    return (1 - z) * (1 + z) / 4 * np.array([orc.jacobi(p - 2, 1.0, 1.0, float(t)) for t in z])


def psiB(p, q, z):
    if p == 0:
        return psiA(q, z)
    if q == 0:
        return ((1 - z) / 2) ** p
    return ((1 - z) / 2) ** p * (1 + z) / 2 * np.array([orc.jacobi(q - 1, 2.0 * p - 1, 1.0, float(t)) for t in z])


def direction_points(shape, Q):
    eta, _, w = orc.ref_points(shape, Q)
    zs = [eta[:Q, 0], eta[::Q][:Q, 1]]
    if eta.shape[1] == 3:
        zs.append(eta[::Q * Q][:Q, 2])
    return zs, w


def cls_table(z, N):
    """Ragged classes c = 0..N-1 of Q x (N - c) values psiB_c,r(z_k), r < N - c."""
    out = []
    for c in range(N):
        block = np.stack([psiB(c, r, z) for r in range(N - c)], axis=1)   # [Q][N-c]
        out.append(block.ravel())
    return np.concatenate(out)


@pytest.mark.parametrize("shape", list(SHAPES))
def test_host_tables_match_oracle(dump, shape):
    for P in range(1, 10):
        N, Q = P + 1, P + 2
        L, blob = dump(shape, P)
        zs, w = direction_points(shape, Q)
        seg = lambda name, n: blob[L[name]:L[name] + n]
        # first direction: psiA on the symmetric points
        Ba = np.stack([psiA(r, zs[0]) for r in range(N)], axis=1)
        assert np.allclose(seg("Ba", Q * N), Ba.ravel(), rtol=0, atol=1e-13), (shape, P, "Ba")
        # ragged classes of the collapsed directions
        if shape in ("tri", "tet"):
            assert np.allclose(seg("Bb", L["Bc"] - L["Bb"]), cls_table(zs[1], N), rtol=0, atol=1e-13), (P, "Bb")
        if shape in ("prism", "pyr"):   # eta3 classes: p (prism), max(p, q) (pyramid)
            assert np.allclose(seg("Bb", L["Bc"] - L["Bb"]), cls_table(zs[2], N), rtol=0, atol=1e-13), (P, "Bb")
        if shape == "tet":
            assert np.allclose(seg("Bc", L["D1"] - L["Bc"]), cls_table(zs[2], N), rtol=0, atol=1e-13), (P, "Bc")
        # collocation derivatives per direction (directions sharing a rule share a table)
        for k, name in enumerate(["D1", "D2", "D3"][:len(zs)]):
            D = orc.colloc_1d(zs[k])
            assert np.allclose(seg(name, Q * Q), D.ravel(), rtol=1e-12, atol=1e-11 * np.abs(D).max()), (P, name)
        # reference weights per point, collapse factors included
        assert np.allclose(seg("wq", w.size), w, rtol=1e-13, atol=0), (shape, P, "wq")
        # even/odd form of Ba
        ne, no = 1 + (N - 1) // 2, 1 + (N - 2) // 2
        rows = []
        for i in range((Q + 1) // 2):
            rows += [(Ba[i, 0] + Ba[i, 1]) / 2] + [Ba[i, 2 * k] for k in range(1, ne)]
            rows += [(Ba[i, 0] - Ba[i, 1]) / 2] + [Ba[i, 2 * k + 1] for k in range(1, no)]
        assert np.allclose(seg("Bs", len(rows)), rows, rtol=0, atol=1e-13), (shape, P, "Bs")
