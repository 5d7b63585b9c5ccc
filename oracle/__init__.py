"""FP64 CPU oracle for the spectral/hp elemental operators (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package.  The product library never imports it.  The arithmetic
lives in ``oracle.c`` (plain C, dense elemental matrices built from the basis
definitions); this module compiles it with gcc on first use and wraps it with
numpy arrays.

Shapes are named "quad", "tri", "hex", "prism", "tet", "pyr".  Layouts: coefficients
[E][M] (modes packed p outermost), physical values [E][Nq] with point index
i + Q*(j + Q*k) (first direction fastest), derivative fields [d][E][Nq].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_SHAPE = {"quad": 0, "tri": 1, "hex": 2, "prism": 3, "tet": 4, "pyr": 5}
_DIM = {"quad": 2, "tri": 2, "hex": 3, "prism": 3, "tet": 3, "pyr": 3}
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, -O2, OpenMP) if missing or stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            i, d = C.c_int, C.c_double
            sig = {
                "orc_num_modes": (i, [i, i]),
                "orc_num_points": (i, [i, i]),
                "orc_threads": (i, []),
                "orc_jacobi": (d, [i, d, d, d]),
                "orc_jacobi_deriv": (d, [i, d, d, d]),
                "orc_quad_rule": (i, [i, i, _dp, _dp]),
                "orc_ref_points": (i, [i, i, _dp, _dp, _dp]),
                "orc_ref_basis": (i, [i, i, i, _dp, _dp]),
                "orc_eval_basis": (i, [i, i, i, _dp, _dp, _dp]),
                "orc_colloc_1d": (i, [i, _dp, _dp]),
                "orc_colloc_deriv": (i, [i, i, _dp]),
                "orc_geom_factors": (i, [i, i, i, i, _dp, _dp, _dp, C.c_void_p]),
                "orc_bwd": (i, [i, i, i, i, _dp, _dp]),
                "orc_iprod": (i, [i, i, i, i, i, _dp, _dp, _dp]),
                "orc_physderiv": (i, [i, i, i, i, _dp, _dp, _dp]),
                "orc_iprod_deriv": (i, [i, i, i, i, i, _dp, _dp, _dp]),
                "orc_mass": (i, [i, i, i, i, i, _dp, _dp, _dp]),
                "orc_helmholtz": (i, [i, i, i, i, i, _dp, d, _dp, _dp]),
                "orc_helmholtz_matrix": (i, [i, i, i, i, i, _dp, d, _dp]),
                "orc_helmholtz_solve": (i, [i, i, i, i, i, _dp, d, _dp, _dp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _chk(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def dim(shape: str) -> int:
    return _DIM[shape]


def num_modes(shape: str, P: int) -> int:
    m = lib().orc_num_modes(_SHAPE[shape], P)
    _chk(0 if m > 0 else m, "num_modes")
    return m


def num_points(shape: str, Q: int) -> int:
    n = lib().orc_num_points(_SHAPE[shape], Q)
    _chk(0 if n > 0 else n, "num_points")
    return n


def threads() -> int:
    return lib().orc_threads()


def jacobi(n: int, a: float, b: float, x: float) -> float:
    return lib().orc_jacobi(n, a, b, x)


def quad_rule(kind: str, Q: int):
    """kind: 'gll', 'gj0', 'gj1', 'gj2' (Gauss-Jacobi(alpha, 0))."""
    k = {"gll": 0, "gj0": 1, "gj1": 2, "gj2": 3}[kind]
    z = np.zeros(Q)
    w = np.zeros(Q)
    _chk(lib().orc_quad_rule(k, Q, z, w), "quad_rule")
    return z, w


def ref_points(shape: str, Q: int):
    """(eta [Nq][d], xi [Nq][d], w [Nq]) of the shape's quadrature points."""
    nq, d = num_points(shape, Q), dim(shape)
    eta, xi, w = np.zeros((nq, d)), np.zeros((nq, d)), np.zeros(nq)
    _chk(lib().orc_ref_points(_SHAPE[shape], Q, eta, xi, w), "ref_points")
    return eta, xi, w


def ref_basis(shape: str, P: int, Q: int):
    """(B [Nq][M], dB [d][Nq][M]) at the quadrature points (xi-gradient)."""
    nq, d, M = num_points(shape, Q), dim(shape), num_modes(shape, P)
    B, dB = np.zeros((nq, M)), np.zeros((d, nq, M))
    _chk(lib().orc_ref_basis(_SHAPE[shape], P, Q, B, dB), "ref_basis")
    return B, dB


def eval_basis(shape: str, P: int, xi):
    """(B [n][M], dB [d][n][M]) at arbitrary points xi [n][d] (off the collapse)."""
    xi = _f64(xi)
    n, d, M = xi.shape[0], dim(shape), num_modes(shape, P)
    B, dB = np.zeros((n, M)), np.zeros((d, n, M))
    _chk(lib().orc_eval_basis(_SHAPE[shape], P, n, xi.ravel(), B, dB), "eval_basis")
    return B, dB


def colloc_1d(z):
    z = _f64(z)
    D = np.zeros((z.size, z.size))
    _chk(lib().orc_colloc_1d(z.size, z, D), "colloc_1d")
    return D


def colloc_deriv(shape: str, Q: int):
    nq, d = num_points(shape, Q), dim(shape)
    D = np.zeros((d, nq, nq))
    _chk(lib().orc_colloc_deriv(_SHAPE[shape], Q, D), "colloc_deriv")
    return D


def geom_factors(shape: str, Q: int, gorder: int, nodes, with_x: bool = False):
    """(W [E][Nq], dxi_dx [E][Nq][d][d], x [E][Nq][d] or None)."""
    nodes = _f64(nodes)
    E, nq, d = nodes.shape[0], num_points(shape, Q), dim(shape)
    W, L = np.zeros((E, nq)), np.zeros((E, nq, d, d))
    X = np.zeros((E, nq, d)) if with_x else None
    xp = X.ctypes.data_as(C.c_void_p) if with_x else None
    _chk(lib().orc_geom_factors(_SHAPE[shape], Q, E, gorder, nodes.ravel(), W, L, xp), "geom_factors")
    return W, L, X


def bwd(shape, P, Q, coeff):
    coeff = _f64(coeff)
    E = coeff.shape[0]
    out = np.zeros((E, num_points(shape, Q)))
    _chk(lib().orc_bwd(_SHAPE[shape], P, Q, E, coeff.ravel(), out), "bwd")
    return out


def iprod(shape, P, Q, gorder, nodes, phys):
    phys, nodes = _f64(phys), _f64(nodes)
    E = phys.shape[0]
    out = np.zeros((E, num_modes(shape, P)))
    _chk(lib().orc_iprod(_SHAPE[shape], P, Q, E, gorder, nodes.ravel(), phys.ravel(), out), "iprod")
    return out


def physderiv(shape, Q, gorder, nodes, phys):
    phys, nodes = _f64(phys), _f64(nodes)
    E = phys.shape[0]
    out = np.zeros((dim(shape), E, num_points(shape, Q)))
    _chk(lib().orc_physderiv(_SHAPE[shape], Q, E, gorder, nodes.ravel(), phys.ravel(), out), "physderiv")
    return out


def iprod_deriv(shape, P, Q, gorder, nodes, f):
    """f: [d][E][Nq] -> sum_l (D_xl B)^T W f_l, [E][M]."""
    f, nodes = _f64(f), _f64(nodes)
    E = f.shape[1]
    out = np.zeros((E, num_modes(shape, P)))
    _chk(lib().orc_iprod_deriv(_SHAPE[shape], P, Q, E, gorder, nodes.ravel(), f.ravel(), out), "iprod_deriv")
    return out


def mass(shape, P, Q, gorder, nodes, coeff):
    coeff, nodes = _f64(coeff), _f64(nodes)
    out = np.zeros_like(coeff)
    _chk(lib().orc_mass(_SHAPE[shape], P, Q, coeff.shape[0], gorder, nodes.ravel(), coeff.ravel(), out), "mass")
    return out


def helmholtz(shape, P, Q, gorder, nodes, lam, coeff):
    coeff, nodes = _f64(coeff), _f64(nodes)
    out = np.zeros_like(coeff)
    _chk(lib().orc_helmholtz(_SHAPE[shape], P, Q, coeff.shape[0], gorder, nodes.ravel(), float(lam),
                             coeff.ravel(), out), "helmholtz")
    return out


def helmholtz_matrix(shape, P, Q, gorder, nodes, lam):
    """Dense elemental matrices H^e [E][M][M]."""
    nodes = _f64(nodes)
    E, M = nodes.shape[0], num_modes(shape, P)
    out = np.zeros((E, M, M))
    _chk(lib().orc_helmholtz_matrix(_SHAPE[shape], P, Q, E, gorder, nodes.ravel(), float(lam), out),
         "helmholtz_matrix")
    return out


def helmholtz_solve(shape, P, Q, gorder, nodes, lam, b):
    """Per-element dense Cholesky solve H^e x = b."""
    b, nodes = _f64(b), _f64(nodes)
    out = np.zeros_like(b)
    _chk(lib().orc_helmholtz_solve(_SHAPE[shape], P, Q, b.shape[0], gorder, nodes.ravel(), float(lam),
                                   b.ravel(), out), "helmholtz_solve")
    return out
