"""Exact multivariate polynomials for pinning the oracle (test helper).

A polynomial is a dict {exponent tuple: coefficient}.  Integrals over the unit
cube, unit simplex and unit prism use the closed forms
  cube:    prod 1/(a_i+1)
  simplex: a! b! (c!) / (a+b(+c)+d)!            (Dirichlet integral)
  prism:   {x,z >= 0, x+z <= 1} x [0,1]:  a! c! / (a+c+2)! * 1/(b+1)
evaluated in exact rational arithmetic.
"""
from __future__ import annotations

import itertools
from fractions import Fraction
from math import factorial

import numpy as np


def mono(exps, c=1.0):
    return {tuple(exps): c}


def add(p, q, s=1.0):
    r = dict(p)
    for k, v in q.items():
        r[k] = r.get(k, 0.0) + s * v
    return {k: v for k, v in r.items() if v != 0.0}


def scale(p, s):
    return {k: s * v for k, v in p.items()}


def mul(p, q):
    r = {}
    for k1, v1 in p.items():
        for k2, v2 in q.items():
            k = tuple(a + b for a, b in zip(k1, k2))
            r[k] = r.get(k, 0.0) + v1 * v2
    return r


def deriv(p, i):
    r = {}
    for k, v in p.items():
        if k[i] == 0:
            continue
        kk = list(k)
        kk[i] -= 1
        r[tuple(kk)] = r.get(tuple(kk), 0.0) + v * k[i]
    return r


def evaluate(p, X):
    X = np.asarray(X, dtype=np.float64)
    out = np.zeros(X.shape[:-1])
    for k, v in p.items():
        t = np.full(X.shape[:-1], v)
        for i, a in enumerate(k):
            if a:
                t = t * X[..., i] ** a
        out = out + t
    return out


def compose_affine(p, A, b):
    """q(y) = p(A y + b) for A [d][d], b [d]."""
    d = len(b)
    lin = []
    for i in range(d):
        li = {tuple([0] * d): float(b[i])}
        for j in range(d):
            e = [0] * d
            e[j] = 1
            li = add(li, mono(e, float(A[i][j])))
        lin.append(li)
    r = {}
    for k, v in p.items():
        t = {tuple([0] * d): v}
        for i, a in enumerate(k):
            for _ in range(a):
                t = mul(t, lin[i])
        r = add(r, t)
    return r


def _int_mono(kind, k):
    if kind == "cube":
        v = Fraction(1)
        for a in k:
            v /= (a + 1)
        return v
    if kind == "simplex":
        num = 1
        for a in k:
            num *= factorial(a)
        return Fraction(num, factorial(sum(k) + len(k)))
    if kind == "prism":  # variables (x, y, z); triangle in (x, z)
        a, b, c = k
        return Fraction(factorial(a) * factorial(c), factorial(a + c + 2)) / (b + 1)
    raise KeyError(kind)


def integrate(p, kind):
    return float(sum(Fraction(v) * _int_mono(kind, k) for k, v in p.items()))


def random_poly(d, deg, rng, total=True):
    """Random polynomial with total degree <= deg (or degree <= deg per variable)."""
    p = {}
    for k in itertools.product(range(deg + 1), repeat=d):
        if total and sum(k) > deg:
            continue
        p[k] = float(rng.uniform(-1, 1))
    return p


def monomials(d, deg, total=True):
    out = []
    for k in itertools.product(range(deg + 1), repeat=d):
        if total and sum(k) > deg:
            continue
        out.append(k)
    return out
