"""The persistent hybrid-mesh kernel's per-item code (``csrc/nir_mesh_inst.cu``)
run on the host by an emulated CTA (``tests/host/mesh_sim.cpp``), against the
oracle: no GPU involved.

One CTA takes a work list that alternates between blocks of different
(shape, P) variants, so it reloads the tables at almost every item; the
low-order FP32/BF16 variants read their contraction tables from the kernel's
constant array (filled at the offsets the library uploads to), the others from
shared memory.  Built with AddressSanitizer (exactly sized shared memory, global
arrays and constant array), run in forward and reverse thread order (the
results must agree bit for bit), and compared block by block with the oracle:
FP32 in 3-D (one and two groups per item) and BF16 in 2-D.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle as orc
from tests.test_cta_sim_cpu import SHAPES, TOL, device_metric, inputs, mesh

CUDA = "/usr/local/cuda"
# (shape, P): low orders use the constant tables in FP32/BF16, the rest shared memory
BLOCKS = {3: [("hex", 2), ("prism", 3), ("tet", 2), ("pyr", 2), ("tet", 4), ("hex", 5)],
          2: [("quad", 2), ("tri", 3), ("quad", 6), ("tri", 8)]}


@pytest.fixture(scope="module")
def sims(host_sims):
    """{(dim, prec): executable} of the mesh-kernel emulation (session builds)."""
    return {(k[1], k[2]): v for k, v in host_sims.items() if k[0] == "mesh"}


def run(exe, blocks, lam, gran, order):
    body = [f"{len(blocks)} {lam!r} {gran}"]
    for b in blocks:
        body.append(f"{SHAPES[b['shape']]} {b['P']} {b['E']}")
        body.append(" ".join(repr(float(v)) for v in b["metric"].ravel()))
        body.append(" ".join(repr(float(v)) for v in b["u"].ravel()))
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0", SIM_ORDER=order,
               LD_LIBRARY_PATH=os.path.join(CUDA, "lib64") + ":" + os.environ.get("LD_LIBRARY_PATH", ""))
    r = subprocess.run([exe], input="\n".join(body) + "\n", capture_output=True, text=True, env=env)
    assert r.returncode == 0, (order, r.returncode, r.stderr[-4000:])
    return np.array([float(t) for t in r.stdout.split()])


@pytest.mark.parametrize("dim,prec,gran", [(3, "f32", 1), (3, "f32", 2), (2, "bf16", 1)])
def test_mesh_items_match_oracle(sims, dim, prec, gran):
    lam = 1.1
    blocks, refs = [], []
    kinds = BLOCKS[dim] if gran == 1 else [BLOCKS[dim][0], BLOCKS[dim][-2], BLOCKS[dim][-1]]
    for i, (shape, P) in enumerate(kinds):
        E = 70 + 7 * i            # several groups per block and a ragged last one
        g, nodes = mesh(shape, E, True, seed=i)
        Q = P + 2
        u = inputs(shape, "helm", P, E, seed=10 + i)
        blocks.append(dict(shape=shape, P=P, E=E, u=u, metric=device_metric(shape, Q, g, nodes, "geo")))
        refs.append(orc.helmholtz(shape, P, Q, g, nodes, lam, u))
    exe = sims[(dim, prec)]
    y = run(exe, blocks, lam, gran, "fwd")
    assert np.array_equal(y, run(exe, blocks, lam, gran, "rev")), "order-dependent result"
    o = 0
    for b, ref in zip(blocks, refs):
        n = ref.size
        got = y[o:o + n].reshape(ref.shape)
        o += n
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= TOL[prec], (b["shape"], b["P"], prec, err)
    assert o == y.size
