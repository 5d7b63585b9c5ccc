"""The element-group kernels' stage code (``csrc/nir_kernels.cuh``), run on the
host by an emulated CTA (``tests/host/cta_sim.cpp``), against the oracle: no
GPU involved.  This is the bounds and barrier check of the GPU kernels that a
device-side sanitizer would otherwise give.

Every CUDA thread of one CTA is a host thread; the CTA takes every element
group in turn (a full group and a ragged second).  Shared memory and every
global array are exactly sized heap blocks and the emulation is built with
AddressSanitizer, so any index outside them fails the run.  Between two
barriers the threads run one at a time in an order fixed per barrier phase;
each case runs in forward and reverse order (the launch variants also in a
shuffled one) and must give the same bits (a word that one thread writes and another reads or writes between the
same two barriers makes the result depend on the order), and that result must
match the oracle at the precision's tolerance.  Planted mistakes (a barrier
skipped, shared memory or an input one element short) show both checks fire.

The metric is the one the library computes, written here from the oracle's
geometric factors: with K = (d eta / d xi)(d xi / d x) and the weighted
Jacobian W = w |J|, the Helmholtz/mass metric is the upper triangle of
W K K^T then W, and the derivative operators take K row-major then W."""
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as orc
import workloads as W
from oracle import nodal as nd

SHAPES = {"quad": 0, "tri": 1, "hex": 2, "prism": 3, "tet": 4, "pyr": 5}
OPS = {"bwd": 0, "iprod": 1, "physderiv": 2, "iprod_deriv": 3, "mass": 4, "helm": 5}
PREC = {"f64": 0, "f32": 1, "bf16": 2}
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 3e-2}
ORDERS = ("fwd", "rev")          # every case; the variants also run a shuffled order
SHUFFLED = ("fwd", "rev", "7")


@pytest.fixture(scope="module")
def sims(host_sims):
    """{shape: executable} of the CTA emulation (built with the session's host builds)."""
    return {k[1]: v for k, v in host_sims.items() if k[0] == "cta"}


def collapse_jacobian(shape, e):
    """d eta / d xi at the point with collapsed coordinates e."""
    if shape in ("quad", "hex"):
        return np.eye(len(e))
    if shape == "tri":
        return np.array([[2 / (1 - e[1]), (1 + e[0]) / (1 - e[1])], [0, 1]])
    if shape == "prism":
        return np.array([[2 / (1 - e[2]), 0, (1 + e[0]) / (1 - e[2])], [0, 1, 0], [0, 0, 1]])
    if shape == "pyr":
        return np.array([[2 / (1 - e[2]), 0, (1 + e[0]) / (1 - e[2])],
                         [0, 2 / (1 - e[2]), (1 + e[1]) / (1 - e[2])], [0, 0, 1]])
    a = (1 - e[1]) * (1 - e[2])
    return np.array([[4 / a, 2 * (1 + e[0]) / a, 2 * (1 + e[0]) / a],
                     [0, 2 / (1 - e[2]), (1 + e[1]) / (1 - e[2])], [0, 0, 1]])


def device_metric(shape, Q, gorder, nodes, kind):
    """[E][Nq][NG]: kind "geo" (Helmholtz, mass) or "lam" (derivative operators)."""
    Wq, Lam, _ = orc.geom_factors(shape, Q, gorder, nodes)
    eta, _, _ = orc.ref_points(shape, Q)
    J = np.stack([collapse_jacobian(shape, e) for e in eta])
    K = np.einsum("nij,enjl->enil", J, Lam)
    if kind == "lam":
        return np.concatenate([K.reshape(K.shape[0], K.shape[1], -1), Wq[..., None]], axis=2)
    G = Wq[..., None, None] * np.einsum("enil,enjl->enij", K, K)
    iu = np.triu_indices(K.shape[-1])
    return np.concatenate([G[:, :, iu[0], iu[1]], Wq[..., None]], axis=2)


def mesh(shape, E, deformed, seed):
    """(gorder, nodes): curved quads/hexes when deformed, else perturbed
    straight-sided elements (affine for quad/hex when `deformed` is None)."""
    if shape == "hex":
        n = int(np.ceil(E ** (1 / 3))) + 1
        if deformed:
            return 2, W.hex_grid(n, 2, amp=0.05)[:E]
        if deformed is None:   # affine: each element its own sheared, scaled cube
            return 1, affine_cells(shape, E, seed)
        return 1, W.perturb_vertices(W.hex_grid(n, 1, amp=0.0)[:E], 0.15, seed)
    if shape == "quad":
        n = int(np.ceil(E ** 0.5)) + 1
        if deformed is None:
            return 1, affine_cells(shape, E, seed)
        return 1, W.perturb_vertices(W.quad_grid(n, n)[:E], 0.15, seed)
    if shape == "tri":
        n = int(np.ceil((E / 2) ** 0.5)) + 1
        return 1, W.perturb_vertices(W.tri_grid(n, n)[:E], 0.15, seed)
    if shape == "tet":
        n = int(np.ceil((E / 6) ** (1 / 3))) + 1
        return 1, W.perturb_vertices(W.tet_kuhn(n)[:E], 0.1, seed)
    if shape == "prism":
        n = int(np.ceil((E / 2) ** (1 / 3))) + 1
        return 1, W.perturb_vertices(W.prism_split(n, n, n)[:E], 0.1, seed)
    n = int(np.ceil((E / 6) ** (1 / 3))) + 1
    nodes = W.perturb_vertices(W.pyramid_split(n, n, n)[:E], 0.1, seed).copy()
    rng = np.random.default_rng(seed + 100)   # base vertex off the parallelogram: rational map
    nodes[:, 2, :] += 0.08 / n * rng.uniform(-1, 1, (E, 3))
    return 1, nodes


def affine_cells(shape, E, seed):
    d = 2 if shape == "quad" else 3
    ref = np.array([[-1, -1], [1, -1], [-1, 1], [1, 1]], float) if d == 2 else np.array(
        [[i, j, k] for k in (-1, 1) for j in (-1, 1) for i in (-1, 1)], float)
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(E):
        A = np.eye(d) * rng.uniform(0.5, 1.5) + 0.2 * rng.uniform(-1, 1, (d, d))
        out.append(ref @ A.T + rng.uniform(-1, 1, d))
    return np.array(out)


def inputs(shape, op, P, E, seed):
    Q, d = P + 2, orc.dim(shape)
    M, NQ = orc.num_modes(shape, P), orc.num_points(shape, Q)
    if op in ("bwd", "mass", "helm"):
        return W.coefficients(E, M, seed)
    if op == "iprod_deriv":
        return W.phys_samples(E, NQ, seed + 1, ncomp=d)
    return W.phys_samples(E, NQ, seed + 1)


def oracle_op(shape, P, g, nodes, op, x, lam, nodal=0):
    Q = P + 2
    o = nd if nodal else orc
    if op == "bwd":
        return o.bwd(shape, P, Q, x)
    if op == "iprod":
        return o.iprod(shape, P, Q, g, nodes, x)
    if op == "physderiv":
        return orc.physderiv(shape, Q, g, nodes, x)   # no expansion involved
    if op == "iprod_deriv":
        return o.iprod_deriv(shape, P, Q, g, nodes, x)
    if op == "mass":
        return o.mass(shape, P, Q, g, nodes, x)
    return o.helmholtz(shape, P, Q, g, nodes, lam, x)


def run_sim(exe, shape, P, op, prec, variant, E, pp, lam, nodal, fields, metric, order="fwd", env=None):
    args = [exe, str(SHAPES[shape]), str(P), str(OPS[op]), str(PREC[prec]), str(variant)]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0", SIM_ORDER=order, **(env or {}))
    if E == 0:
        r = subprocess.run(args, input="0 1 0 0 1\n", capture_output=True, text=True, env=env)
        assert r.returncode == 0, r.stderr[-3000:]
        return tuple(int(t) for t in r.stdout.split())
    body = [f"{E} {pp} {lam!r} {nodal} {len(fields) if op == 'helm' else 1}",
            " ".join(repr(float(v)) for v in metric.ravel())]
    body += [" ".join(repr(float(v)) for v in np.asarray(f).ravel()) for f in fields]
    r = subprocess.run(args, input="\n".join(body) + "\n", capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise SimFailed(r.returncode, r.stderr[-4000:])
    return np.array([float(t) for t in r.stdout.split()])


class SimFailed(Exception):
    def __init__(self, rc, err):
        super().__init__(f"emulation exited {rc}: {err}")
        self.rc, self.err = rc, err


def case(shape, P, op, prec, variant=0, deformed=True, nfields=1, lam=1.3, seed=0, epb=None, nodal=0):
    """(E, pp, metric, fields, reference) of one case."""
    E = epb + max(1, epb // 3)              # a full group and a ragged second
    g, nodes = mesh(shape, E, deformed, seed)
    Q = P + 2
    pp = 0 if deformed is None else 1
    metric = device_metric(shape, Q, g, nodes, "lam" if op in ("physderiv", "iprod_deriv") else "geo")
    if not pp:   # per element: the kernel scales the weighted entries by the point weight
        _, _, w = orc.ref_points(shape, Q)
        metric = metric[:, 0, :].copy()
        if op in ("physderiv", "iprod_deriv"):
            metric[:, -1] /= w[0]           # K is unweighted; W = |J|
        else:
            metric /= w[0]                  # |J| K K^T and |J|
    if op == "iprod_deriv":
        x = inputs(shape, op, P, E, seed)
        fields = [x[c] for c in range(x.shape[0])]
        refs = [oracle_op(shape, P, g, nodes, op, x, lam, nodal)]
    elif op == "helm":
        fields = [inputs(shape, op, P, E, seed + f) for f in range(nfields)]
        refs = [oracle_op(shape, P, g, nodes, op, f, lam, nodal) for f in fields]
    else:
        fields = [inputs(shape, op, P, E, seed)]
        refs = [oracle_op(shape, P, g, nodes, op, fields[0], lam, nodal)]
    return E, pp, metric, fields, np.concatenate([np.asarray(r).ravel() for r in refs])


def check(sims, shape, P, op, prec, variant=0, deformed=True, nfields=1, lam=1.3, seed=0, env=None, nodal=0,
          orders=ORDERS):
    """Run one case in every order; returns the relative error against the oracle
    (asserting bit-identical results across orders and the tolerance)."""
    exe = sims[shape]
    epb = run_sim(exe, shape, P, op, prec, variant, 0, 1, lam, 0, [], None)[0]
    E, pp, metric, fields, ref = case(shape, P, op, prec, variant, deformed, nfields, lam, seed, epb, nodal)
    ys = [run_sim(exe, shape, P, op, prec, variant, E, pp, lam, nodal, fields, metric, order=o, env=env)
          for o in orders]
    for o, y in zip(orders[1:], ys[1:]):
        assert np.array_equal(y, ys[0]), ("order-dependent result", shape, P, op, prec, variant, o)
    assert ys[0].shape == ref.shape
    err = np.linalg.norm(ys[0] - ref) / np.linalg.norm(ref)
    assert err <= TOL[prec], (shape, P, op, prec, variant, err)
    return err


def run_cases(sims, cases):
    """Run cases (kwargs of check) on all host cores; every one must pass."""
    def one(kw):
        try:
            check(sims, **kw)
            return None
        except (AssertionError, SimFailed) as e:
            return (kw, str(e)[:3000])
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        bad = [r for r in ex.map(one, cases) if r]
    assert not bad, bad[:3]


@pytest.mark.parametrize("shape", list(SHAPES))
def test_every_operator(sims, shape):
    """Every operator in FP64 and FP32 at P = 1, 2, 4 on the curved or
    perturbed mesh of the shape (per-point factors)."""
    run_cases(sims, [dict(shape=shape, P=P, op=op, prec=prec)
                     for op in OPS for prec in ("f64", "f32") for P in (1, 2, 4)])


@pytest.mark.parametrize("shape", list(SHAPES))
def test_helmholtz_variants_fields_and_bf16(sims, shape):
    """The Helmholtz launch variants (half and double groups, the persistent
    mesh kernel's form, two elements per thread on quads/hexes), three fields
    in one call, and BF16 storage."""
    cases = [dict(shape=shape, P=2, op="helm", prec=prec, variant=v, orders=SHUFFLED)
             for prec in ("f64", "f32") for v in (1, 2, 3)]
    cases += [dict(shape=shape, P=3, op="helm", prec=prec, nfields=3, orders=SHUFFLED)
              for prec in ("f64", "f32", "bf16")]
    cases += [dict(shape=shape, P=P, op=op, prec="bf16") for op in ("bwd", "iprod", "helm") for P in (1, 4)]
    if shape in ("quad", "hex"):   # two elements per thread
        cases += [dict(shape=shape, P=P, op="helm", prec=prec, variant=5, orders=SHUFFLED)
                  for prec in ("f32", "bf16") for P in (1, 2, 3, 4)]
        cases += [dict(shape=shape, P=3, op="helm", prec="f32", variant=5, nfields=3)]
    run_cases(sims, cases)


@pytest.mark.parametrize("shape", list(SHAPES))
def test_high_order_helmholtz(sims, shape):
    """P = 6 and 9: groups of 4 to 16 elements, whose buffer strides are chosen
    for the warp's bank mapping, every launch variant in FP32, the default one
    in BF16 and FP64."""
    variants = (0, 1, 2, 3) + ((5,) if shape in ("quad", "hex") else ())
    cases = [dict(shape=shape, P=P, op="helm", prec="f32", variant=v) for P in (6, 9) for v in variants]
    cases += [dict(shape=shape, P=P, op="helm", prec=prec) for P in (6, 9) for prec in ("bf16", "f64")]
    run_cases(sims, cases)


@pytest.mark.parametrize("shape", ["quad", "hex"])
def test_per_element_factors_and_nodal_basis(sims, shape):
    """Affine quads/hexes with per-element factors, and the GLL-Lagrange basis."""
    cases = [dict(shape=shape, P=3, op=op, prec=prec, deformed=None) for op in OPS for prec in ("f64", "f32")]
    cases += [dict(shape=shape, P=P, op=op, prec=prec, nodal=1) for op in ("bwd", "iprod", "mass", "helm")
              for prec in ("f64", "f32") for P in (2, 4)]
    cases += [dict(shape=shape, P=P, op="helm", prec="f32", variant=5, **kw)
              for P in (2, 4) for kw in (dict(deformed=None), dict(nodal=1))]
    run_cases(sims, cases)


def bank_degree(S, step, units, kw):
    """Most 4-byte addresses u*S + step*s (u < units, s < kw) on one of 32 banks."""
    cnt = [0] * 32
    for u in range(units):
        for s in range(kw):
            cnt[(u * S + step * s) % 32] += 1
    return max(cnt)


@pytest.mark.parametrize("shape", list(SHAPES))
def test_buffer_strides(sims, shape):
    """The per-unit stride of every FP32 Helmholtz group size at P = 1..4, 6, 9:
    odd (one structural index of 32 units covers the banks) for groups of 32 or
    more units; otherwise within 32 of the odd stride and no worse than it over
    the neighbour steps 1, N and Q (recounted here), and never below the
    points per element.  Paired units keep the odd stride."""
    seen = 0
    for P in (1, 2, 3, 4, 6, 9):
        N, Q = P + 1, P + 2
        nq = orc.num_points(shape, Q)
        s0 = nq + 1 if nq % 2 == 0 else nq
        for v in (0, 1, 2) + ((5,) if shape in ("quad", "hex") else ()):
            epb, nt, S, epu = run_sim(sims[shape], shape, P, "helm", "f32", v, 0, 1, 1.0, 0, [], None)
            assert S >= nq and nt % 32 == 0
            if epu >= 32 or v == 5:
                assert S == s0, (P, v, S)
                continue
            kw = 32 // epu
            cost = lambda x: sum(bank_degree(x, st, epu, kw) for st in (1, N, Q))
            assert s0 <= S < s0 + 32 and cost(S) <= cost(s0), (P, v, S, cost(S), cost(s0))
            seen += 1
    assert seen > 0 or orc.dim(shape) == 2   # 2-D groups hold 32 or more elements


@pytest.mark.parametrize("shape,op,prec,variant", [("hex", "helm", "f32", 0), ("hex", "helm", "f32", 3),
                                                    ("tet", "bwd", "f64", 0), ("pyr", "iprod", "f32", 0)])
def test_dropped_barriers_are_caught(sims, shape, op, prec, variant):
    """Every thread skipping its k-th barrier: each dropped barrier either
    leaves the result intact in every order (it guarded nothing in this
    configuration) or makes it order-dependent; none gets past the order check
    to fail only against the oracle, and most are caught."""
    def one(k):
        try:
            check(sims, shape, 2, op, prec, variant=variant, env={"SIM_DROP_BARRIER": str(k)})
            return 0
        except AssertionError as e:
            assert "order-dependent" in str(e), (k, str(e)[:500])
            return 1
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        caught = sum(ex.map(one, range(1, 16)))
    assert caught >= 6, caught


@pytest.mark.parametrize("what", ["smem", "input"])
def test_short_arrays_are_caught(sims, what):
    """Shared memory or an input one element short: AddressSanitizer reports."""
    for shape, op, prec in [("hex", "helm", "f32"), ("tri", "mass", "f64"), ("pyr", "physderiv", "f64")]:
        with pytest.raises(SimFailed) as ei:
            check(sims, shape, 2, op, prec, env={"SIM_SHORT": what})
        assert "AddressSanitizer" in ei.value.err
