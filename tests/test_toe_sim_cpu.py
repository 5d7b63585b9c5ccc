"""The threading-over-elements Helmholtz kernel (``k_helm_toe`` in
``csrc/nir_toe.cuh``) run on the host by an emulated CTA
(``tests/host/toe_sim.cpp``), against the oracle: no GPU involved.

Its 128 threads take warps of 32 elements in turn (a ragged last warp; warps
that run out of elements leave early), move coefficients and results through
the per-warp shared-memory tiles and keep their stage arrays in the global
scratch.  Shared memory, scratch and every array are exactly sized heap blocks
under AddressSanitizer; forward and reverse thread orders must give the same
bits; the result must match the oracle (per-point factors for every
shape, per-element factors for affine quads and hexes)."""
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as orc
from tests.test_cta_sim_cpu import TOL, device_metric, inputs, mesh

SHAPES = {"quad": 0, "tri": 1, "hex": 2, "prism": 3, "tet": 4}   # no such kernel for pyramids
ORDERS = ("fwd", "rev")


@pytest.fixture(scope="module")
def sims(host_sims):
    """{shape: executable} of the threading-over-elements emulation (session builds)."""
    return {k[1]: v for k, v in host_sims.items() if k[0] == "toe"}


def run(exe, P, prec, E, pp, lam, metric, u, order):
    body = f"{E} {pp} {lam!r}\n" + " ".join(repr(float(v)) for v in metric.ravel()) + "\n" + \
        " ".join(repr(float(v)) for v in u.ravel()) + "\n"
    r = subprocess.run([exe, str(P), {"f64": "0", "f32": "1"}[prec]], input=body, capture_output=True, text=True,
                       env=dict(os.environ, ASAN_OPTIONS="detect_leaks=0", SIM_ORDER=order))
    assert r.returncode == 0, (P, prec, order, r.returncode, r.stderr[-4000:])
    return np.array([float(t) for t in r.stdout.split()])


def check(sims, shape, P, prec, E, deformed=True, seed=0, lam=1.2):
    g, nodes = mesh(shape, E, deformed, seed)
    Q = P + 2
    metric = device_metric(shape, Q, g, nodes, "geo")
    pp = 1
    if deformed is None:    # per element: the kernel scales by the point weight
        _, _, w = orc.ref_points(shape, Q)
        metric, pp = metric[:, 0, :] / w[0], 0
    u = inputs(shape, "helm", P, E, seed + 3)
    ys = [run(sims[shape], P, prec, E, pp, lam, metric, u, o) for o in ORDERS]
    for o, y in zip(ORDERS[1:], ys[1:]):
        assert np.array_equal(y, ys[0]), ("order-dependent result", shape, P, prec, o)
    ref = orc.helmholtz(shape, P, Q, g, nodes, lam, u)
    err = np.linalg.norm(ys[0] - ref.ravel()) / np.linalg.norm(ref)
    assert err <= TOL[prec], (shape, P, prec, err)


@pytest.mark.parametrize("shape", list(SHAPES))
def test_toe_kernel_matches_oracle(sims, shape):
    cases = [(P, prec, 3 * 32 + 5 if P <= 4 else 37) for P in (1, 4, 9) for prec in ("f64", "f32")]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        list(ex.map(lambda c: check(sims, shape, *c), cases))


@pytest.mark.parametrize("shape", ["quad", "hex"])
def test_toe_per_element_factors(sims, shape):
    check(sims, shape, 2, "f64", 70, deformed=None)
    check(sims, shape, 2, "f32", 70, deformed=None)
