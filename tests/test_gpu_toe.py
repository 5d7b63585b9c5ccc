"""GPU parity of the threading-over-elements Helmholtz kernel (launch tuning
variant 4: one thread per element, intermediate tensors in global scratch;
the second GPU strategy of Sec. 3.3) against the FP64 oracle.

  * every shape x P in {1, 2, 3, 5, 8, 9} x precision: the oracle on all elements
    (on a sample for high-order hexes), plus the whole block against the
    default kernel (in FP64 bit for bit: both strategies run the same
    operations in the same order, so the autotuner may switch between them);
    element counts span several warps and a ragged tail;
  * affine tensor blocks (per-element factors), E = 1, several grid sizes
    (one CTA striding over every element gives the same bits), range
    launches through the host-buffer pipeline, a mesh in the concurrent
    block launch form, kernel_info, and the unsupported nodal basis.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 3e-2}

SHAPES = ["quad", "tri", "hex", "prism", "tet"]
_REF = {}


@pytest.fixture(scope="module")
def nir():
    import paper_2606_20917_gb300 as nir
    return nir


@pytest.fixture(scope="module")
def ctx(nir):
    torch.cuda.set_device(0)
    return nir.Context(0)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make_mesh(shape, E, deformed, seed=0):
    """(gorder, nodes[E]): curved (g = 2) or vertex-perturbed affine hexes,
    perturbed quads, Kuhn tets, split prisms, triangles."""
    if shape == "hex":
        n = int(np.ceil(E ** (1 / 3))) + 1
        if deformed:
            return 2, W.hex_grid(n, 2, amp=0.05)[:E]
        return 1, W.perturb_vertices(W.hex_grid(n, 1, amp=0.0)[:E], 0.15, seed)
    if shape == "quad":
        n = int(np.ceil(E ** 0.5)) + 1
        return 1, W.perturb_vertices(W.quad_grid(n, n)[:E], 0.15, seed)
    if shape == "tri":
        n = int(np.ceil((E / 2) ** 0.5)) + 1
        return 1, W.perturb_vertices(W.tri_grid(n, n)[:E], 0.15, seed)
    if shape == "tet":
        n = int(np.ceil((E / 6) ** (1 / 3))) + 1
        return 1, W.perturb_vertices(W.tet_kuhn(n)[:E], 0.1, seed)
    n = int(np.ceil((E / 2) ** (1 / 3))) + 1
    return 1, W.perturb_vertices(W.prism_split(n, n, n)[:E], 0.1, seed)


def block(nir, ctx, shape, P, E, deformed, seed=0):
    g, nodes = make_mesh(shape, E, deformed, seed)
    blk = nir.Block(ctx, shape, E, P, deformed=deformed)
    blk.set_geometry(g, torch.from_numpy(np.ascontiguousarray(nodes)).cuda())
    return g, nodes, blk


def apply(nir, blk, prec, x, lam=1.3):
    y = blk.helmholtz(torch.from_numpy(np.ascontiguousarray(x)).to("cuda", nir.DTYPE[prec]), lam=lam, prec=prec)
    torch.cuda.synchronize()
    return y


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("P", [1, 2, 3, 5, 8, 9])
def test_toe_matches_oracle(nir, ctx, prec, shape, P):
    deformed = shape in ("quad", "hex")
    E = 300 if shape in ("quad", "tri") else (101 if P <= 3 else 45)
    g, nodes, blk = block(nir, ctx, shape, P, E, deformed)
    x = W.coefficients(E, blk.M, seed=P)
    ids = np.arange(E) if (shape != "hex" or P <= 5) else W.sample_elements(E, 6, seed=P)
    key = (shape, P)
    if key not in _REF:
        _REF[key] = oracle.helmholtz(shape, P, P + 2, g, nodes[ids], 1.3, x[ids])
    blk.set_tuning(prec, 4, 0, 0)
    got = apply(nir, blk, prec, x).double().cpu().numpy()
    assert rel(got[ids], _REF[key]) <= TOL[prec]
    blk.set_tuning(prec, 0, 0, 0)
    y0 = apply(nir, blk, prec, x)
    assert rel(got, y0.double().cpu().numpy()) <= TOL[prec]
    if prec == "f64":   # the FP64 kernels of both strategies do the same operations in the same order
        blk.set_tuning(prec, 4, 0, 0)
        assert torch.equal(apply(nir, blk, prec, x), y0)


@pytest.mark.parametrize("shape", ["quad", "hex"])
def test_toe_affine_tensor_blocks(nir, ctx, shape):
    P, E = 4, 77
    g, nodes, blk = block(nir, ctx, shape, P, E, deformed=False, seed=3)
    x = W.coefficients(E, blk.M, seed=1)
    ref = oracle.helmholtz(shape, P, P + 2, g, nodes, 0.7, x)
    for prec in ("f64", "f32"):
        blk.set_tuning(prec, 4, 0, 0)
        y = apply(nir, blk, prec, x, lam=0.7)
        assert rel(y.double().cpu().numpy(), ref) <= TOL[prec], prec
    blk.set_tuning("f64", 4, 0, 0)
    y4 = apply(nir, blk, "f64", x, lam=0.7)
    blk.set_tuning("f64", 0, 0, 0)
    assert torch.equal(apply(nir, blk, "f64", x, lam=0.7), y4)


@pytest.mark.parametrize("shape", SHAPES)
def test_toe_single_element_and_grids(nir, ctx, shape):
    g, nodes, blk = block(nir, ctx, shape, 3, 1, deformed=shape in ("quad", "hex"))
    x = W.coefficients(1, blk.M, seed=2)
    blk.set_tuning("f64", 4, 0, 0)
    got = apply(nir, blk, "f64", x).cpu().numpy()
    assert rel(got, oracle.helmholtz(shape, 3, 5, g, nodes, 1.3, x)) <= TOL["f64"]
    E = 1000
    g, nodes, blk = block(nir, ctx, shape, 2, E, deformed=shape in ("quad", "hex"))
    x = W.coefficients(E, blk.M, seed=4)
    outs = []
    for grid in (1, 3, 0):                       # one CTA striding over all 1000 elements, ..., one wave
        blk.set_tuning("f32", 4, grid, 0)
        outs.append(apply(nir, blk, "f32", x))
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    assert blk.get_tuning("f32")[0] == 4


def test_toe_host_pipeline_ranges(nir, ctx):
    """Chunked host-buffer applies launch element ranges; bits equal the
    device apply."""
    g, nodes, blk = block(nir, ctx, "hex", 3, 3001, True)
    for prec in ("f64", "f32"):
        blk.set_tuning(prec, 4, 0, 0)
        u = torch.from_numpy(W.coefficients(3001, blk.M, 6)).to(nir.DTYPE[prec]).pin_memory()
        out = torch.empty_like(u).pin_memory()
        blk.helmholtz_host(u, out, lam=1.0, prec=prec)
        ref = blk.helmholtz(u.cuda(), lam=1.0, prec=prec).cpu()
        assert torch.equal(out, ref), prec


def test_toe_in_mesh_block_launch_form(nir, ctx):
    blocks, refs = [], []
    for shape, P, E in (("hex", 3, 40), ("tet", 4, 60), ("prism", 2, 50)):
        g, nodes, blk = block(nir, ctx, shape, P, E, deformed=shape == "hex")
        blocks.append((blk, g, nodes, shape, P))
    m = nir.Mesh(ctx, [b[0] for b in blocks])
    x = np.random.default_rng(0).uniform(-1, 1, m.ndof)
    blocks[1][0].set_tuning("f64", 4, 0, 0)
    m.set_launch("f64", "blocks")
    y = m.helmholtz(torch.from_numpy(x).cuda(), prec="f64").cpu().numpy()
    off = 0
    for blk, g, nodes, shape, P in blocks:
        n = blk.nelem * blk.M
        ref = oracle.helmholtz(shape, P, P + 2, g, nodes, 1.0, x[off:off + n].reshape(blk.nelem, blk.M))
        assert rel(y[off:off + n].reshape(blk.nelem, blk.M), ref) <= TOL["f64"], shape
        off += n


def test_toe_kernel_info_and_unsupported(nir, ctx):
    g, nodes, blk = block(nir, ctx, "tet", 4, 20, False)
    blk.set_tuning("f64", 4, 0, 0)
    info = blk.kernel_info("f64", "helm")
    assert info["threads"] == 128 and info["elems_per_cta"] == 128 and info["registers"] > 0
    nodal = nir.Block(ctx, "hex", 8, 2, deformed=True, basis="nodal")
    with pytest.raises(nir.NirError) as e:
        nodal.set_tuning("f64", 4, 0, 0)
    assert e.value.code == -2
    with pytest.raises(nir.NirError):
        blk.set_tuning("f64", 5, 0, 0)


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_toe_scratch_released_when_no_precision_uses_it(nir, ctx):
    """Leaving variant 4 frees the threading-over-elements scratch once no
    precision of the block uses it; the results stay correct."""
    E, P = 4096, 8
    g, nodes, blk = block(nir, ctx, "hex", P, E, False)
    x = W.coefficients(E, blk.M, seed=2)
    y0 = apply(nir, blk, "f64", x).cpu()
    base = free_bytes()
    blk.set_tuning("f64", 4, 0, 0)
    blk.set_tuning("f32", 4, 0, 0)
    held = base - free_bytes()
    expect = 5 * blk.NQ * E * 8   # 5 arrays of Q^3 FP64 values per thread, one thread per element at most
    assert held >= 0.5 * expect, (held, expect)
    assert torch.equal(apply(nir, blk, "f64", x).cpu(), y0)   # FP64: the same bits
    blk.set_tuning("f64", 0, 0, 0)
    assert base - free_bytes() >= 0.5 * expect               # FP32 still uses it
    blk.set_tuning("f32", 0, 0, 0)
    assert abs(base - free_bytes()) < 0.1 * expect           # released
    assert torch.equal(apply(nir, blk, "f64", x).cpu(), y0)


def test_toe_tuning_refused_inside_capture(nir, ctx):
    """Selecting variant 4 allocates and synchronises: refused (STATE) while
    the context stream is being captured, with nothing left half-done."""
    g, nodes, blk = block(nir, ctx, "tet", 3, 64, False)
    s = torch.cuda.Stream()
    c2 = nir.Context(0, s)
    b2 = nir.Block(c2, "tet", 64, 3)
    b2.set_geometry(g, torch.from_numpy(np.ascontiguousarray(nodes)).cuda())
    graph = torch.cuda.CUDAGraph()
    rc = None
    with torch.cuda.graph(graph, stream=s):
        rc = nir.lib().nir_block_set_tuning(b2.h, 0, 4, 0, 0)
        keep = torch.ones(4, device="cuda") * 2   # the capture holds one node
    del keep
    assert rc == -8
    assert b2.get_tuning("f64")[0] == 0
    b2.set_tuning("f64", 4, 0, 0)   # outside the capture it works
    x = W.coefficients(64, b2.M, seed=1)
    assert torch.equal(apply(nir, b2, "f64", x), apply(nir, blk, "f64", x))
