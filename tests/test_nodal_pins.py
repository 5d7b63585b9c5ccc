"""Pins of the nodal (GLL-Lagrange) oracle, ``oracle/nodal.py``:

* the Lagrange family is cardinal at the GLL nodes and a partition of unity,
  its derivatives sum to zero (textbook properties);
* nodal coefficients taken as the values of a polynomial of degree <= P per
  direction reproduce it exactly at the quadrature points;
* the nodal and modified bases span the same space, so every nodal operator
  equals the (separately pinned) modified-basis oracle's after the change of
  basis Phi (modified basis at the nodes): H_nodal = Phi^-T H_mod Phi^-1,
  iprod_nodal = Phi^-T iprod_mod, bwd_nodal = bwd_mod Phi^-1.
"""
import numpy as np
import pytest

import oracle as orc
import workloads as W
from oracle import nodal as nd


def node_points(shape, N):
    z = nd.gll_nodes(N)
    if shape == "quad":
        p, q = np.meshgrid(z, z, indexing="ij")          # mode p N + q: p along xi1, outermost
        return np.stack([p.ravel(), q.ravel()], axis=1)
    p, q, r = np.meshgrid(z, z, z, indexing="ij")
    return np.stack([p.ravel(), q.ravel(), r.ravel()], axis=1)


@pytest.mark.parametrize("N", [2, 3, 5, 9])
def test_cardinal_partition_of_unity(N):
    z = nd.gll_nodes(N)
    L, dL = nd.lagrange_1d(z, z)
    assert np.allclose(L, np.eye(N), atol=1e-13)
    x = np.random.default_rng(N).uniform(-1, 1, 40)
    L, dL = nd.lagrange_1d(z, x)
    assert np.allclose(L.sum(axis=1), 1.0, atol=1e-12)
    assert np.allclose(dL.sum(axis=1), 0.0, atol=1e-10)


@pytest.mark.parametrize("shape,P", [("quad", 3), ("hex", 2), ("hex", 4)])
def test_polynomial_reproduction(shape, P):
    d = 2 if shape == "quad" else 3
    Q = P + 2
    X = node_points(shape, P + 1)
    rng = np.random.default_rng(P)
    a = rng.uniform(-1, 1, size=(P + 1,) * d)            # sum a[i,j,(k)] x^i y^j (z^k)
    def f(pts):
        v = np.zeros(pts.shape[0])
        for idx in np.ndindex(*a.shape):
            v += a[idx] * np.prod([pts[:, c] ** idx[c] for c in range(d)], axis=0)
        return v
    coeff = f(X)[None, :]
    _, xi, _ = orc.ref_points(shape, Q)
    assert np.allclose(nd.bwd(shape, P, Q, coeff)[0], f(xi), atol=1e-11)


@pytest.mark.parametrize("shape,P", [("quad", 4), ("hex", 3)])
def test_change_of_basis_matches_modified_oracle(shape, P):
    Q, lam = P + 2, 1.3
    if shape == "quad":
        g, nodes = 1, W.perturb_vertices(W.quad_grid(2, 2), 0.1, 3)
    else:
        g, nodes = 2, W.hex_grid(2, 2, amp=0.05)
    Phi, _ = orc.eval_basis(shape, P, node_points(shape, P + 1))   # [nodes][modified modes]
    Pi = np.linalg.inv(Phi)
    Hm = orc.helmholtz_matrix(shape, P, Q, g, nodes, lam)
    Hn = nd.helmholtz_matrices(shape, P, Q, g, nodes, lam)
    for e in range(nodes.shape[0]):
        ref = Pi.T @ Hm[e] @ Pi
        assert np.abs(Hn[e] - ref).max() <= 1e-11 * np.abs(ref).max()
    rng = np.random.default_rng(1)
    f = rng.uniform(-1, 1, size=(nodes.shape[0], orc.num_points(shape, Q)))
    assert np.allclose(nd.iprod(shape, P, Q, g, nodes, f), orc.iprod(shape, P, Q, g, nodes, f) @ Pi,
                       rtol=0, atol=1e-12)
    x = rng.uniform(-1, 1, size=(nodes.shape[0], (P + 1) ** orc.dim(shape)))
    assert np.allclose(nd.bwd(shape, P, Q, x), orc.bwd(shape, P, Q, x @ Pi.T), rtol=0, atol=1e-12)
    fs = rng.uniform(-1, 1, size=(orc.dim(shape), nodes.shape[0], orc.num_points(shape, Q)))
    assert np.allclose(nd.iprod_deriv(shape, P, Q, g, nodes, fs), orc.iprod_deriv(shape, P, Q, g, nodes, fs) @ Pi,
                       rtol=0, atol=1e-11)
    Mn = nd.mass_matrices(shape, P, Q, g, nodes)
    Mm = Hm - orc.helmholtz_matrix(shape, P, Q, g, nodes, lam - 1.0)   # lambda-difference isolates M
    assert np.abs(Mn[0] - Pi.T @ Mm[0] @ Pi).max() <= 1e-11 * np.abs(Mn[0]).max()
