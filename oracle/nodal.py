"""Nodal (Lagrange) expansions on quadrilaterals and hexahedra -- the oracle.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).

The paper names Lagrange bases as a further expansion type for its elemental
operators (conclusion); on tensor shapes the operators keep their definition
(Sec. 2.1: B, W, Lambda) with the basis matrix built from Lagrange polynomials.
Here, with N = P + 1 modes per direction, the 1-D basis is the Lagrange
polynomial family through the N Gauss-Lobatto-Legendre points, l_j(z_i) =
delta_ij, evaluated at the Q quadrature points by the product formula; the
d-dimensional modes are tensor products, packed p outermost like the modified
basis (mode (p, q, r) = l_p(xi1) l_q(xi2) l_r(xi3)).  Operators are formed as
dense matrix products from B, its xi-gradient and the oracle's geometric
factors:
    BwdTrans = B u,  IProductWRTBase = B^T W f,
    IProductWRTDerivBase = sum_l (D_xl B)^T W f_l,  D_xl B = sum_i (d xi_i/d x_l) dB_i,
    mass = B^T W B,  Helmholtz = sum_l (D_xl B)^T W (D_xl B) + lambda B^T W B.
"""
from __future__ import annotations

import numpy as np

import oracle as orc


def gll_nodes(N: int) -> np.ndarray:
    return orc.quad_rule("gll", N)[0]


def lagrange_1d(nodes: np.ndarray, x: np.ndarray):
    """(L [len(x)][N], dL [len(x)][N]): l_j(x) and l_j'(x) by the product formula."""
    x = np.asarray(x, dtype=np.float64)
    N = nodes.size
    L = np.ones((x.size, N))
    dL = np.zeros((x.size, N))
    for j in range(N):
        for m in range(N):
            if m == j:
                continue
            L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
        # derivative: sum over the factor left out
        for k in range(N):
            if k == j:
                continue
            term = np.full(x.size, 1.0 / (nodes[j] - nodes[k]))
            for m in range(N):
                if m == j or m == k:
                    continue
                term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            dL[:, j] += term
    return L, dL


def ref_basis(shape: str, P: int, Q: int):
    """(B [Nq][M], dB [d][Nq][M]) of the nodal basis at the shape's quadrature
    points (GLL, first direction fastest)."""
    assert shape in ("quad", "hex")
    d = 2 if shape == "quad" else 3
    N = P + 1
    z = orc.quad_rule("gll", Q)[0]
    L, dL = lagrange_1d(gll_nodes(N), z)
    if d == 2:
        # point n = i + Q j (xi1 fastest), mode m = p N + q (p along xi1)
        B = np.einsum("ip,jq->jipq", L, L).reshape(Q * Q, N * N)
        dB = np.stack([np.einsum("ip,jq->jipq", dL, L).reshape(Q * Q, N * N),
                       np.einsum("ip,jq->jipq", L, dL).reshape(Q * Q, N * N)])
        return B, dB
    B = np.einsum("ip,jq,kr->kjipqr", L, L, L).reshape(Q ** 3, N ** 3)
    dB = np.stack([np.einsum("ip,jq,kr->kjipqr", dL, L, L).reshape(Q ** 3, N ** 3),
                   np.einsum("ip,jq,kr->kjipqr", L, dL, L).reshape(Q ** 3, N ** 3),
                   np.einsum("ip,jq,kr->kjipqr", L, L, dL).reshape(Q ** 3, N ** 3)])
    return B, dB


def _geo(shape, Q, gorder, nodes):
    W, Lam, _ = orc.geom_factors(shape, Q, gorder, nodes)   # Lam[e][n][i][l] = d xi_i / d x_l
    return W, Lam


def _dx(dB, Lam):
    """D_xl B per element: [E][d][Nq][M]."""
    return np.einsum("enil,inm->elnm", Lam, dB)


def eval_basis(shape: str, P: int, xi):
    """Nodal basis at arbitrary reference points xi [n][d] -> [n][M]."""
    xi = np.asarray(xi, dtype=np.float64)
    z = gll_nodes(P + 1)
    L = [lagrange_1d(z, xi[:, c])[0] for c in range(xi.shape[1])]
    if xi.shape[1] == 2:
        return np.einsum("np,nq->npq", L[0], L[1]).reshape(xi.shape[0], -1)
    return np.einsum("np,nq,nr->npqr", L[0], L[1], L[2]).reshape(xi.shape[0], -1)


def bwd(shape, P, Q, coeff):
    B, _ = ref_basis(shape, P, Q)
    return np.asarray(coeff) @ B.T


def iprod(shape, P, Q, gorder, nodes, phys):
    B, _ = ref_basis(shape, P, Q)
    W, _ = _geo(shape, Q, gorder, nodes)
    return (W * np.asarray(phys)) @ B


def iprod_deriv(shape, P, Q, gorder, nodes, f):
    """f: [d][E][Nq] -> [E][M]."""
    B, dB = ref_basis(shape, P, Q)
    W, Lam = _geo(shape, Q, gorder, nodes)
    DX = _dx(dB, Lam)
    return np.einsum("elnm,en,len->em", DX, W, np.asarray(f))


def mass_matrices(shape, P, Q, gorder, nodes):
    B, _ = ref_basis(shape, P, Q)
    W, _ = _geo(shape, Q, gorder, nodes)
    return np.einsum("nm,en,nk->emk", B, W, B)


def helmholtz_matrices(shape, P, Q, gorder, nodes, lam):
    B, dB = ref_basis(shape, P, Q)
    W, Lam = _geo(shape, Q, gorder, nodes)
    DX = _dx(dB, Lam)
    L = np.einsum("elnm,en,elnk->emk", DX, W, DX)
    return L + lam * mass_matrices(shape, P, Q, gorder, nodes)


def mass(shape, P, Q, gorder, nodes, coeff):
    return np.einsum("emk,ek->em", mass_matrices(shape, P, Q, gorder, nodes), np.asarray(coeff))


def helmholtz(shape, P, Q, gorder, nodes, lam, coeff):
    return np.einsum("emk,ek->em", helmholtz_matrices(shape, P, Q, gorder, nodes, lam), np.asarray(coeff))
