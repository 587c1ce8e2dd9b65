"""Exact right-hand side -div(f^e - f^v) of the compressible Navier-Stokes equations (Sec. 2.1)
for smooth periodic fields, derived symbolically with sympy from the primitive fields (rho, v, p).
Used to pin the oracle's physics and metric terms by grid convergence.

The viscous flux uses the stress tensor of Sec. 2.1 and the heat flux mu c_p/Pr grad T with
T = p/(rho R) (reading G1), i.e. mu gamma/((gamma-1) Pr) grad(p/rho). Nothing here reuses the
oracle's formulas in terms of conserved-variable gradients.

Two fields: "tgv", the Taylor-Green initial condition (div v = 0), and "wave", a compressible
periodic field with div v != 0 and non-uniform density (test data only).
"""
from __future__ import annotations

import functools

import numpy as np
import sympy as sp

_x, _y, _z = sp.symbols("x y z", real=True)


def _fields(name, gamma, mach):
    x, y, z = _x, _y, _z
    g = sp.nsimplify(gamma)
    p0 = 1 / (g * sp.nsimplify(mach) ** 2)
    if name == "tgv":
        rho = sp.Integer(1) + 0 * x
        v = [sp.sin(x) * sp.cos(y) * sp.cos(z), -sp.cos(x) * sp.sin(y) * sp.cos(z), 0 * x]
        p = p0 + sp.Rational(1, 16) * (sp.cos(2 * x) + sp.cos(2 * y)) * (sp.cos(2 * z) + 2)
    elif name == "wave":
        rho = 1 + sp.Rational(1, 5) * sp.sin(x + y) * sp.cos(z)
        v = [sp.sin(x) * sp.cos(y) * sp.cos(z) + sp.Rational(3, 10) * sp.cos(z),
             -sp.cos(x) * sp.sin(y) * sp.cos(z) + sp.Rational(1, 5) * sp.sin(x),
             sp.Rational(2, 5) * sp.sin(x) * sp.cos(y) * sp.sin(z)]
        p = p0 + sp.Rational(1, 2) * sp.cos(2 * x) * sp.cos(y) + sp.Rational(3, 10) * sp.sin(z)
    else:
        raise ValueError(name)
    return rho, v, p, g


@functools.lru_cache(maxsize=16)
def state_function(name: str, gamma: float, mach: float):
    """Conserved variables at points xyz [n,3] -> [5, n]."""
    rho, v, p, g = _fields(name, gamma, mach)
    E = p / (g - 1) + rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) / 2
    fns = [sp.lambdify((_x, _y, _z), e, "numpy") for e in (rho, rho * v[0], rho * v[1], rho * v[2], E)]

    def f(xyz):
        return np.stack([np.broadcast_to(fn(xyz[:, 0], xyz[:, 1], xyz[:, 2]), (xyz.shape[0],)) for fn in fns])

    return f


@functools.lru_cache(maxsize=16)
def rhs_function(name: str, gamma: float, mach: float, mu: float, Pr: float):
    """Exact -div(f^e - f^v) at points xyz [n,3] -> [5, n]."""
    X = (_x, _y, _z)
    rho, v, p, g = _fields(name, gamma, mach)
    E = p / (g - 1) + rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) / 2
    muv, Prv = sp.nsimplify(mu), sp.nsimplify(Pr)
    divv = sum(sp.diff(v[i], X[i]) for i in range(3))
    tau = [[muv * (sp.diff(v[j], X[i]) + sp.diff(v[i], X[j])) - (sp.Rational(2, 3) * muv * divv if i == j else 0)
            for j in range(3)] for i in range(3)]
    heat = [muv * g / ((g - 1) * Prv) * sp.diff(p / rho, X[d]) for d in range(3)]
    flux = []
    for d in range(3):
        fe = [rho * v[d], rho * v[d] * v[0] + (p if d == 0 else 0), rho * v[d] * v[1] + (p if d == 1 else 0),
              rho * v[d] * v[2] + (p if d == 2 else 0), v[d] * (E + p)]
        fv = [0, tau[0][d], tau[1][d], tau[2][d], sum(v[i] * tau[i][d] for i in range(3)) + heat[d]]
        flux.append([fe[a] - fv[a] for a in range(5)])
    rhs = [-sum(sp.diff(flux[d][a], X[d]) for d in range(3)) for a in range(5)]
    fns = [sp.lambdify((_x, _y, _z), r, "numpy") for r in rhs]

    def f(xyz):
        return np.stack([np.broadcast_to(fn(xyz[:, 0], xyz[:, 1], xyz[:, 2]), (xyz.shape[0],)) for fn in fns])

    return f


def tgv_rhs_function(gamma, mach, mu, Pr):
    return rhs_function("tgv", gamma, mach, mu, Pr)
