"""The threading-over-elements stage code (``csrc/nir_toe.cuh``), compiled
for the host, against the oracle (no GPU involved).

The per-element Helmholtz function of that kernel is built as plain C++ with
AddressSanitizer (``tests/host/toe_stages.cpp``) and run on one affine element
x = A xi + c of every shape (A a fixed sheared, scaled matrix) for P = 1..9.
Its metric input is written out here from the mathematics of the collapsed
coordinates: with the point weights w (collapse factors included),
J = d eta / d xi and K = J A^-1 = d eta / d x, G = w |det A| K K^T and
W = w |det A|; eta1 = 2(1+xi1)/(1-xi2) - 1 (triangle),
2(1+xi1)/(-xi2-xi3) - 1 and eta2 = 2(1+xi2)/(1-xi3) - 1 (tetrahedron),
2(1+xi1)/(1-xi3) - 1 (prism).  The result must equal the oracle's dense
Helmholtz matrix applied to the same coefficients, and no access may leave the
exactly sized scratch (5 Q^d values) or table arrays."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_20917_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"
SHAPES = {"quad": 0, "tri": 1, "hex": 2, "prism": 3, "tet": 4}
REF = {"quad": [[-1, -1], [1, -1], [-1, 1], [1, 1]],
       "tri": [[-1, -1], [1, -1], [-1, 1]],
       "hex": [[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [1, 1, -1], [-1, -1, 1], [1, -1, 1], [-1, 1, 1], [1, 1, 1]],
       "prism": [[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1], [-1, -1, 1], [-1, 1, 1]],
       "tet": [[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]]}


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are not available")
    exe = str(tmp_path_factory.mktemp("toe") / "toe_stages")
    cmd = [gxx, "-O1", "-g", "-std=c++17", "-w", "-fsanitize=address", "-fno-omit-frame-pointer",
           "-I", CUDA_INC, "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "host", "toe_stages.cpp"), os.path.join(CSRC, "nir_basis.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


AFF = {2: np.array([[1.3, 0.4], [-0.2, 0.9]]), 3: np.array([[1.2, 0.3, -0.1], [0.2, 0.8, 0.25], [-0.15, 0.1, 1.1]])}
SHIFT = {2: np.array([0.3, -0.7]), 3: np.array([0.5, -0.2, 0.4])}


def metric(shape, Q):
    eta, _, w = orc.ref_points(shape, Q)
    A = AFF[len(eta[0])]
    Ai, det = np.linalg.inv(A), abs(np.linalg.det(A))
    rows = []
    for e, wk in zip(eta, w):
        if shape in ("quad", "hex"):
            J = np.eye(len(e))
        elif shape == "tri":
            J = np.array([[2 / (1 - e[1]), (1 + e[0]) / (1 - e[1])], [0, 1]])
        elif shape == "prism":
            J = np.array([[2 / (1 - e[2]), 0, (1 + e[0]) / (1 - e[2])], [0, 1, 0], [0, 0, 1]])
        else:
            a = (1 - e[1]) * (1 - e[2])
            J = np.array([[4 / a, 2 * (1 + e[0]) / a, 2 * (1 + e[0]) / a],
                          [0, 2 / (1 - e[2]), (1 + e[1]) / (1 - e[2])], [0, 0, 1]])
        K = J @ Ai
        G = wk * det * K @ K.T
        if len(e) == 2:
            rows.append([G[0, 0], G[0, 1], G[1, 1], wk * det])
        else:
            rows.append([G[0, 0], G[0, 1], G[0, 2], G[1, 1], G[1, 2], G[2, 2], wk * det])
    return np.array(rows)


@pytest.mark.parametrize("shape", list(SHAPES))
def test_toe_stage_code_matches_oracle(harness, shape):
    for P in range(1, 10):
        Q, lam = P + 2, 1.3
        u = np.random.default_rng(P).uniform(-1, 1, orc.num_modes(shape, P))
        G = metric(shape, Q)
        stdin = f"{SHAPES[shape]} {P} {lam!r}\n" + " ".join(repr(float(v)) for v in G.ravel()) + "\n" + \
            " ".join(repr(float(v)) for v in u) + "\n"
        r = subprocess.run([harness], input=stdin, capture_output=True, text=True,
                           env=dict(os.environ, ASAN_OPTIONS="detect_leaks=0"))
        assert r.returncode == 0, (P, r.stderr[-2000:])
        y = np.array([float(t) for t in r.stdout.split()])
        d = len(REF[shape][0])
        nodes = np.array(REF[shape], float) @ AFF[d].T + SHIFT[d]
        ref = orc.helmholtz(shape, P, Q, 1, nodes[None], lam, u[None])[0]
        assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref), P
