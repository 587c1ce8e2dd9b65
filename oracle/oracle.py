"""ctypes wrapper of the FP64 oracle (oracle/fr_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only users. The GPU library never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fr_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE arithmetic: no FMA contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=gnu99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", SRC, "-o", LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = C.CDLL(LIB)
        dp = C.POINTER(C.c_double)
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, dp, C.POINTER(C.c_int),
                                C.POINTER(C.c_int), dp, C.POINTER(C.c_int)]
        L.or_create4.restype = C.c_void_p
        L.or_create4.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, dp,
                                 C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), dp,
                                 C.POINTER(C.c_int)]
        L.or_pyr_rule.argtypes = [C.c_int, dp, dp]
        L.or_pyr_solution_points.argtypes = [C.c_int, dp]
        L.or_create3.restype = C.c_void_p
        L.or_create3.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, dp, C.POINTER(C.c_int),
                                 C.POINTER(C.c_int), C.POINTER(C.c_int), dp, C.POINTER(C.c_int)]
        L.or_gauss_jacobi.argtypes = [C.c_int, C.c_int, dp, dp]
        L.or_tet_rule.argtypes = [C.c_int, dp, dp]
        L.or_tet_solution_points.argtypes = [C.c_int, dp]
        L.or_create2.restype = C.c_void_p
        L.or_create2.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, dp, C.POINTER(C.c_int),
                                 C.POINTER(C.c_int), dp, C.POINTER(C.c_int)]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_set_threads.argtypes = [C.c_void_p, C.c_int]
        for fn in ("or_num_values", "or_num_fvalues", "or_num_pairs"):
            getattr(L, fn).restype = C.c_long
            getattr(L, fn).argtypes = [C.c_void_p]
        L.or_sol_coords.argtypes = [C.c_void_p, dp]
        L.or_flux_coords.argtypes = [C.c_void_p, dp]
        L.or_pairs.argtypes = [C.c_void_p, C.POINTER(C.c_long), C.POINTER(C.c_long)]
        L.or_rhs.argtypes = [C.c_void_p, dp, dp]
        L.or_rhs_stages.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp, dp, dp]
        L.or_rk4.argtypes = [C.c_void_p, dp, C.c_double, C.c_int]
        L.or_diagnostics.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_etype_dims.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int)]
        L.or_get_operator.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
        L.or_element_geometry.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
        L.or_gauss_legendre.argtypes = [C.c_int, dp, dp]
        L.or_tri_rule.argtypes = [C.c_int, dp, dp]
        L.or_tri_solution_points.argtypes = [C.c_int, dp]
        L.or_tri_basis_values.argtypes = [C.c_int, C.c_int, dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def gauss_legendre(n):
    x = np.zeros(n); w = np.zeros(n)
    lib().or_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def tri_rule(k):
    xy = np.zeros((k * k, 2)); w = np.zeros(k * k)
    lib().or_tri_rule(k, _dp(xy), _dp(w))
    return xy, w


def gauss_jacobi(n, alpha):
    """n-point Gauss rule for the weight (1-x)^alpha on [-1, 1]."""
    x = np.zeros(n); w = np.zeros(n)
    if lib().or_gauss_jacobi(n, alpha, _dp(x), _dp(w)) != 0:
        raise ValueError("Gauss rule construction failed")
    return x, w


def tet_rule(k):
    xyz = np.zeros((k ** 3, 3)); w = np.zeros(k ** 3)
    if lib().or_tet_rule(k, _dp(xyz), _dp(w)) != 0:
        raise ValueError("tetrahedron rule construction failed")
    return xyz, w


def tet_solution_points(p):
    xyz = np.zeros(((p + 1) * (p + 2) * (p + 3) // 6, 3))
    lib().or_tet_solution_points(p, _dp(xyz))
    return xyz


def pyr_rule(k):
    xyz = np.zeros((k ** 3, 3)); w = np.zeros(k ** 3)
    if lib().or_pyr_rule(k, _dp(xyz), _dp(w)) != 0:
        raise ValueError("pyramid rule construction failed")
    return xyz, w


def pyr_solution_points(p):
    xyz = np.zeros(((p + 1) * (p + 2) * (2 * p + 3) // 6, 3))
    lib().or_pyr_solution_points(p, _dp(xyz))
    return xyz


def tri_solution_points(p):
    xy = np.zeros((64, 2))
    n = lib().or_tri_solution_points(p, _dp(xy))
    if n < 0:
        raise ValueError(f"no printed triangle points for p={p}")
    return xy[:n].copy()


def tri_basis_values(p, xy):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    nt = (p + 1) * (p + 2) // 2
    out = np.zeros((xy.shape[0], nt))
    lib().or_tri_basis_values(p, xy.shape[0], _dp(xy), _dp(out))
    return out


OPS = {"xu": 0, "xf": 1, "nref": 2, "xq": 3, "wq": 4, "M0": 5, "D": 6, "lift": 7, "M7": 8, "M8": 9,
       "Wu": 10, "Agrad": 11, "Adiv": 12, "fpt_face": 13}


class Oracle:
    """One mesh instance with its physical parameters (FP64)."""

    def __init__(self, mesh, p, m, gamma=1.4, Pr=0.71, mu=1.0 / 1600, beta=0.5, tau=0.1, tri_k=5,
                 threads=None, p_ref=0.0, surf=False):
        L = lib()
        verts = np.ascontiguousarray(mesh["verts"], dtype=np.float64)
        hex_v = np.ascontiguousarray(mesh.get("hex_v", np.zeros((0, 8))), dtype=np.int32)
        pri_v = np.ascontiguousarray(mesh.get("pri_v", np.zeros((0, 6))), dtype=np.int32)
        tet_v = np.ascontiguousarray(mesh.get("tet_v", np.zeros((0, 4))), dtype=np.int32)
        pyr_v = np.ascontiguousarray(mesh.get("pyr_v", np.zeros((0, 5))), dtype=np.int32)
        period = np.ascontiguousarray(mesh.get("period", (0.0, 0.0, 0.0)), dtype=np.float64)
        err = C.c_int(0)
        ip = C.POINTER(C.c_int)
        self.h = L.or_create4(p, m, tri_k, int(bool(surf)), gamma, Pr, mu, beta, tau, p_ref, hex_v.shape[0],
                              pri_v.shape[0], tet_v.shape[0], pyr_v.shape[0], verts.shape[0], _dp(verts),
                              hex_v.ctypes.data_as(ip), pri_v.ctypes.data_as(ip), tet_v.ctypes.data_as(ip),
                              pyr_v.ctypes.data_as(ip), _dp(period), C.byref(err))
        if not self.h:
            raise RuntimeError(f"oracle mesh creation failed with status {err.value}")
        self.n_hex, self.n_pri, self.n_tet, self.n_pyr = hex_v.shape[0], pri_v.shape[0], tet_v.shape[0], pyr_v.shape[0]
        self.p, self.m = p, m
        self.nU = L.or_num_values(self.h)
        self.nF = L.or_num_fvalues(self.h)
        self.set_threads(threads if threads else 1)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_destroy(self.h)
            self.h = None

    def set_threads(self, n):
        lib().or_set_threads(self.h, int(n))

    def dims(self, t):
        d = (C.c_int * 4)()
        if lib().or_etype_dims(self.h, t, d) != 0:
            return None
        return tuple(d)

    def op(self, t, name):
        nu, nf, nq, _ = self.dims(t)
        shapes = {"xu": (nu, 3), "xf": (nf, 3), "nref": (nf, 3), "xq": (nq, 3), "wq": (nq,),
                  "M0": (nf, nu), "D": (3, nu, nu), "lift": (nu, nf), "M7": (nq, nu), "M8": (nu, nq),
                  "Wu": (nu,), "Agrad": (3, nu, nu), "Adiv": (nu, 3, nu), "fpt_face": (nf,)}
        out = np.zeros(shapes[name])
        lib().or_get_operator(self.h, t, OPS[name], _dp(out))
        return out

    def geometry(self, e):
        J = np.zeros((3, 3)); Ji = np.zeros((3, 3)); d = np.zeros(1)
        lib().or_element_geometry(self.h, e, _dp(J), _dp(Ji), _dp(d))
        return J, Ji, d[0]

    def sol_coords(self):
        """Solution-point coordinates as a flat [sum_pts, 3] array in element order."""
        out = np.zeros((self.nU // 5, 3))
        lib().or_sol_coords(self.h, _dp(out))
        return out

    def flux_coords(self):
        out = np.zeros((self.nF // 5, 3))
        lib().or_flux_coords(self.h, _dp(out))
        return out

    def pairs(self):
        n = lib().or_num_pairs(self.h)
        L = np.zeros(n, dtype=np.int64); R = np.zeros(n, dtype=np.int64)
        lib().or_pairs(self.h, L.ctypes.data_as(C.POINTER(C.c_long)), R.ctypes.data_as(C.POINTER(C.c_long)))
        return L, R

    def rhs(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
        assert U.size == self.nU
        R = np.zeros_like(U)
        st = lib().or_rhs(self.h, _dp(U), _dp(R))
        if st != 0:
            raise RuntimeError(f"oracle rhs status {st}")
        return R

    def rhs_stages(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
        R = np.zeros_like(U)
        uf = np.zeros(self.nF); cf = np.zeros(self.nF); df = np.zeros(self.nF)
        qu = np.zeros(3 * self.nU); qf = np.zeros(3 * self.nF); fu = np.zeros(3 * self.nU)
        lib().or_rhs_stages(self.h, _dp(U), _dp(R), _dp(uf), _dp(cf), _dp(qu), _dp(qf), _dp(fu), _dp(df))
        return dict(R=R, uf=uf, cf=cf, qu=qu, qf=qf, fu=fu, df=df)

    def rk4(self, U, dt, nsteps):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1).copy()
        lib().or_rk4(self.h, _dp(U), dt, nsteps)
        return U

    def diagnostics(self, U, R=None):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
        out = np.zeros(13)
        Rp = _dp(np.ascontiguousarray(R, dtype=np.float64).reshape(-1)) if R is not None else None
        lib().or_diagnostics(self.h, _dp(U), Rp, _dp(out))
        return dict(volume=out[0], Ek=out[1], eps=out[2], sums=out[3:8].copy(), abs_sums=out[8:13].copy())
