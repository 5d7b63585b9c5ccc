"""The library's geometric-factor kernel (``k_geometry`` in
``csrc/nir_geom_kernels.cuh``) run on the host (``tests/host/geom_sim.cpp``),
against the oracle's geometric factors: no GPU involved.

The kernel maps element nodes (lattice nodes of curved quads and hexes,
vertices of straight-sided simplices, prisms and pyramids, the pyramid's
rational map included) to the per-point metric W K K^T and W and the
derivative factors K and W, with K = (d eta / d xi)(d xi / d x) and W = w |J|;
per element (times the reference weight at the points) for affine quads and
hexes; and the FP32 copy packed by ``k_pack_metric`` against the packed layout
restated here.  The same convention is what the kernel emulations of the other host
tests are fed with (``device_metric``), so this ties them to the library's own
geometry.  Outputs exactly sized (64-element padding as allocated by the
library) under AddressSanitizer."""
import os
import subprocess

import numpy as np
import pytest

import oracle as orc
from tests.test_cta_sim_cpu import SHAPES, device_metric, mesh


@pytest.fixture(scope="module")
def sim(host_sims):
    return host_sims[("geom",)]


def run(exe, shape, P, g, pp, nodes):
    body = f"{nodes.shape[0]}\n" + " ".join(repr(float(v)) for v in nodes.ravel()) + "\n"
    r = subprocess.run([exe, str(SHAPES[shape]), str(P), str(g), str(pp)], input=body, capture_output=True,
                       text=True, env=dict(os.environ, ASAN_OPTIONS="detect_leaks=0"))
    assert r.returncode == 0, (shape, P, r.returncode, r.stderr[-3000:])
    return np.array([float(t) for t in r.stdout.split()])


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("P", [1, 4, 8])
def test_metric_matches_oracle_factors(sim, shape, P):
    E = 37                                   # a ragged 64-element chunk
    g, nodes = mesh(shape, E, True, seed=P)
    Q = P + 2
    geo = device_metric(shape, Q, g, nodes, "geo")
    lam = device_metric(shape, Q, g, nodes, "lam")
    out = run(sim, shape, P, g, 1, np.ascontiguousarray(nodes))
    epad, NQ, NG = (E + 63) // 64 * 64, geo.shape[1], geo.shape[2]
    assert out.size == geo.size + lam.size + epad * NQ * NG
    got_g, got_l = out[:geo.size].reshape(geo.shape), out[geo.size:geo.size + lam.size].reshape(lam.shape)
    assert np.abs(got_g - geo).max() <= 1e-12 * np.abs(geo).max(), np.abs(got_g - geo).max()
    assert np.abs(got_l - lam).max() <= 1e-12 * np.abs(lam).max(), np.abs(got_l - lam).max()
    # the packed FP32 copy: per 32-element chunk and point, the elements' (G00 G01 G02 G11)
    # quads, then their (G12 G22) pairs, then their W (2-D: one quad (G00 G01 G11 W))
    packed = out[geo.size + lam.size:]
    for e in range(E):
        for n in range(NQ):
            blk = ((e // 32) * NQ + n) * NG * 32
            l = e % 32
            offs = [l * 4 + c for c in range(4)] if NG == 4 else \
                [l * 4 + c for c in range(4)] + [128 + l * 2, 128 + l * 2 + 1, 192 + l]
            np.testing.assert_array_equal(packed[[blk + o for o in offs]].astype(np.float32),
                                          got_g[e, n].astype(np.float32))


@pytest.mark.parametrize("shape", ["quad", "hex"])
def test_per_element_factors_of_affine_cells(sim, shape):
    P, E = 3, 21
    g, nodes = mesh(shape, E, None, seed=4)
    Q = P + 2
    _, _, w = orc.ref_points(shape, Q)
    geo = device_metric(shape, Q, g, nodes, "geo")[:, 0, :] / w[0]      # |J| K K^T and |J|
    lam = device_metric(shape, Q, g, nodes, "lam")[:, 0, :].copy()
    lam[:, -1] /= w[0]                                                    # K and |J|
    out = run(sim, shape, P, g, 0, np.ascontiguousarray(nodes))
    got_g, got_l = out[:geo.size].reshape(geo.shape), out[geo.size:].reshape(lam.shape)
    assert np.abs(got_g - geo).max() <= 1e-12 * np.abs(geo).max()
    assert np.abs(got_l - lam).max() <= 1e-12 * np.abs(lam).max()
