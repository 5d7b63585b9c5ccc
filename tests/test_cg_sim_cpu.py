"""The CG solver's vector kernels (``csrc/nir_cg_kernels.cuh``) run on the host
by an emulated grid (``tests/host/cg_sim.cpp``): no GPU involved.

Several CTAs of 256 threads, run one after another, each publish a partial and
the last to take the ticket sums them; warp shuffles are exchanges between
barriers.  Vectors, partials and scalars are exactly sized heap blocks under
AddressSanitizer, and three thread orders must give the same bits.  Checked
against exact arithmetic: FP64 dot products against the correctly rounded sum
of the exact products; the FP32-vector option's compensated dot products
(Dot2) against the same on an ill-conditioned pair whose plain FP32 sum loses
every digit; and one CG iteration (start, alpha, update, direction) against
numpy in FP64 and FP32."""
import math
import os
import subprocess

import numpy as np
import pytest

ORDERS = ("fwd", "rev", "5")


@pytest.fixture(scope="module")
def sim(host_sims):
    return host_sims[("cg",)]


def run(exe, test, prec, grid, body, order):
    r = subprocess.run([exe, test, {"f64": "0", "f32": "1"}[prec], str(grid)], input=body, capture_output=True,
                       text=True, env=dict(os.environ, ASAN_OPTIONS="detect_leaks=0", SIM_ORDER=order,
                                           LD_LIBRARY_PATH="/usr/local/cuda/lib64:" +
                                           os.environ.get("LD_LIBRARY_PATH", "")))
    assert r.returncode == 0, (test, prec, grid, order, r.returncode, r.stderr[-3000:])
    return np.array([float(t) for t in r.stdout.split()])


def run_orders(exe, test, prec, grid, body, orders=ORDERS):
    ys = [run(exe, test, prec, grid, body, o) for o in orders]
    for o, y in zip(orders[1:], ys[1:]):
        assert np.array_equal(y, ys[0]), ("order-dependent result", test, prec, o)
    return ys[0]


def text(n, *vecs):
    return f"{n}\n" + "\n".join(" ".join(repr(float(v)) for v in x) for x in vecs) + "\n"


def exact_dot(a, b):
    """Correctly rounded sum of the exact products (each exact in FP64 for FP32 inputs)."""
    return math.fsum(float(x) * float(y) for x, y in zip(a, b))


@pytest.mark.parametrize("grid", [3])
def test_fp64_dot(sim, grid):
    n = 3 * 256 * 4 * 2 + 123          # several grid-stride steps and a ragged tail
    rng = np.random.default_rng(1)
    a, b = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    got = run_orders(sim, "dot", "f64", grid, text(n, a, b))
    scale = float(np.abs(a * b).sum())
    for v in got:                        # k_dot, then k_alpha (FP64 vectors: plain FP64 sums)
        assert abs(v - exact_dot(a, b)) <= 1e-14 * scale


@pytest.mark.parametrize("grid", [4])
def test_fp32_compensated_dot_is_fp64_accurate(sim, grid):
    """Pairs with sum |a_i b_i| ~ 1e3 and a . b ~ 1e-6: a plain FP32 sum keeps no
    digit of it, FP64 accumulation of the stored values (k_dot) and the
    compensated FP32 accumulation (k_alpha's p . Ap) keep FP64-level accuracy."""
    n = 4 * 256 * 4 + 77
    rng = np.random.default_rng(2)
    a = rng.uniform(-1, 1, n).astype(np.float32)
    b = rng.uniform(-1, 1, n).astype(np.float32)
    # cancel: append the negated products' partners so that the exact dot is tiny
    h = n // 2
    a[h:2 * h] = a[:h]
    b[h:2 * h] = -b[:h]
    b[-1] = np.float32(1e-6)
    a[-1] = np.float32(1.0)
    exact = exact_dot(a, b)
    scale = math.fsum(abs(float(x) * float(y)) for x, y in zip(a, b))
    naive = np.float32(0)
    for x, y in zip(a, b):
        naive = np.float32(naive + np.float32(x * y))
    got = run_orders(sim, "dot", "f32", grid, text(n, a, b))
    assert abs(float(naive) - exact) > 1e-9 * scale          # the plain FP32 sum is off
    for v in got:
        assert abs(v - exact) <= 1e-15 * scale + 1e-12 * abs(exact), (v, exact)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 2e-6)])
def test_cg_iteration(sim, prec, tol):
    n = 256 * 4 * 3 + 45               # one grid-stride step of 3 CTAs and a ragged tail
    rng = np.random.default_rng(3)
    dt = np.float64 if prec == "f64" else np.float32
    r, x = (rng.uniform(-1, 1, n).astype(dt) for _ in range(2))
    dinv = rng.uniform(0.5, 2.0, n).astype(dt)
    # Ap as an SPD operator would give it: p = z = dinv r weighted positively (p . Ap > 0)
    Ap = (dinv.astype(np.float64) * r * rng.uniform(0.5, 1.5, n)).astype(dt)
    out = run_orders(sim, "cg", prec, 3, text(n, r, dinv, Ap, x), orders=ORDERS[:2])
    rz0, rr0, pAp, alpha, rz1, rr1, beta = out[:7]
    xs, rs, zs, ps, pTs = out[7:].reshape(5, n)
    R, D, A, X = (v.astype(np.float64) for v in (r, dinv, Ap, x))
    z = D * R
    assert abs(rz0 - exact_dot(R, z.astype(dt))) <= tol * abs(R * z).sum()
    assert abs(rr0 - exact_dot(R, R)) <= 1e-14 * (R * R).sum()
    P = z.astype(dt).astype(np.float64)                      # p = z, stored in the vector type
    assert abs(pAp - exact_dot(P, A)) <= tol * abs(P * A).sum()
    assert abs(alpha - rz0 / pAp) <= 1e-15 * abs(alpha)
    xn, rn = X + alpha * P, R - alpha * A
    zn = D * rn
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(xs, xn) <= tol and rel(rs, rn) <= tol and rel(zs, zn) <= tol
    assert abs(rz1 - float(np.dot(rn, zn))) <= tol * abs(rn * zn).sum()
    assert abs(beta - rz1 / rz0) <= 1e-14 * abs(beta)
    pn = zn + beta * P
    assert rel(ps, pn) <= tol and rel(pTs, pn) <= tol
