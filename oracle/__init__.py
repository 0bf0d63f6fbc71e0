"""FastVPINNs CPU FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Loaded by the tests, by ``__graft_entry__.smoke()`` and by the benchmark's
CPU-baseline leg; never by the library.  The arithmetic lives in
``fv_oracle.cpp`` (plain per-element loops, FP64); this module only builds it
with g++ and marshals numpy arrays through ctypes.

Every function follows arXiv 2404.12063 (see the header of fv_oracle.cpp for
the section / equation each part restates and the readings taken where the
paper is silent or garbled).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fv_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libfv_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle (-O2, no fast-math, OpenMP over elements)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class OracleProblem(C.Structure):
    _fields_ = [("n_vertices", C.c_int), ("vertices", _dp), ("n_elements", C.c_int), ("cells", _ip),
                ("Q", C.c_int), ("T", C.c_int), ("f_quad", _dp),
                ("n_layers", C.c_int), ("widths", _ip),
                ("n_bd", C.c_int), ("bd_xy", _dp), ("bd_g", _dp), ("tau", C.c_double),
                ("n_s", C.c_int), ("s_xy", _dp), ("s_u", _dp), ("gamma", C.c_double),
                ("bx", C.c_double), ("by", C.c_double), ("norm", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.oracle_loss_grad.restype = C.c_int
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: Optional[np.ndarray], t=_dp):
    return None if a is None else a.ctypes.data_as(t)


# --------------------------------------------------------------- primitives
def gll(Q: int):
    x, w = np.zeros(Q), np.zeros(Q)
    if lib().oracle_gll(Q, _ptr(x), _ptr(w)) != 0:
        raise ValueError("GLL order out of range")
    return x, w


def legendre(n: int, s):
    s = _d(np.atleast_1d(s))
    P, dP = np.zeros_like(s), np.zeros_like(s)
    lib().oracle_legendre(n, s.size, _ptr(s), _ptr(P), _ptr(dP))
    return P, dP


def test_fn(n: int, s):
    s = _d(np.atleast_1d(s))
    v, dv = np.zeros_like(s), np.zeros_like(s)
    lib().oracle_test_fn(n, s.size, _ptr(s), _ptr(v), _ptr(dv))
    return v, dv


def geometry(mesh, Q: int) -> np.ndarray:
    """[n_e, Q*Q, 7]: (x, y, x_xi, x_eta, y_xi, y_eta, D) at the GLL nodes."""
    v, c = _d(mesh.vertices), np.ascontiguousarray(mesh.cells, dtype=np.int32)
    out = np.zeros((c.shape[0], Q * Q, 7))
    lib().oracle_geometry(v.shape[0], _ptr(v), c.shape[0], _ptr(c, _ip), Q, _ptr(out))
    return out


def map_points(vx, vy, xi, eta) -> np.ndarray:
    vx, vy, xi, eta = _d(vx), _d(vy), _d(np.atleast_1d(xi)), _d(np.atleast_1d(eta))
    out = np.zeros((xi.size, 7))
    lib().oracle_map_points(_ptr(vx), _ptr(vy), xi.size, _ptr(xi), _ptr(eta), _ptr(out))
    return out


def quad_points(mesh, Q: int) -> np.ndarray:
    v, c = _d(mesh.vertices), np.ascontiguousarray(mesh.cells, dtype=np.int32)
    out = np.zeros((c.shape[0], Q * Q, 2))
    if lib().oracle_quad_points(v.shape[0], _ptr(v), c.shape[0], _ptr(c, _ip), Q, _ptr(out)) != 0:
        raise ValueError("bad quadrature order")
    return out


def mlp(widths, params, xy):
    w = np.ascontiguousarray(widths, dtype=np.int32)
    p, xy = _d(params), _d(xy).reshape(-1, 2)
    n = xy.shape[0]
    u, ux, uy = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().oracle_mlp(len(widths) - 1, _ptr(w, _ip), _ptr(p), n, _ptr(xy), _ptr(u), _ptr(ux), _ptr(uy))
    return u, ux, uy


def mlp_eps(widths, params, xy):
    """Second output eps(x, y) of a two-output network."""
    w = np.ascontiguousarray(widths, dtype=np.int32)
    p, xy = _d(params), _d(xy).reshape(-1, 2)
    e = np.zeros(xy.shape[0])
    lib().oracle_mlp_eps(len(widths) - 1, _ptr(w, _ip), _ptr(p), xy.shape[0], _ptr(xy), _ptr(e))
    return e


def mlp_cstep_x(widths, params, xy, h=1e-30):
    w = np.ascontiguousarray(widths, dtype=np.int32)
    p, xy = _d(params), _d(xy).reshape(-1, 2)
    n = xy.shape[0]
    dx, dy = np.zeros(n), np.zeros(n)
    lib().oracle_mlp_cstep_x(len(widths) - 1, _ptr(w, _ip), _ptr(p), n, _ptr(xy), C.c_double(h),
                             _ptr(dx), _ptr(dy))
    return dx, dy


# --------------------------------------------------------------- problems
class Bound:
    """A problem bound to the C struct; keeps every array alive."""

    def __init__(self, prob, f_quad: Optional[np.ndarray] = None, norm: int = 0,
                 with_boundary: bool = True, with_sensors: bool = True):
        self.prob = prob
        mesh = prob.mesh
        Q, T = prob.quad_order, prob.test_order
        self.vertices = _d(mesh.vertices)
        self.cells = np.ascontiguousarray(mesh.cells, dtype=np.int32)
        if f_quad is None:
            X = quad_points(mesh, Q)
            f_quad = prob.f(X[..., 0], X[..., 1])
        self.f_quad = _d(f_quad).reshape(self.cells.shape[0], Q * Q)
        self.widths = np.ascontiguousarray(prob.widths, dtype=np.int32)
        nb = prob.bd_xy.shape[0] if with_boundary else 0
        ns = prob.sensor_xy.shape[0] if with_sensors else 0
        self.bd_xy = _d(prob.bd_xy if nb else np.zeros((1, 2)))
        self.bd_g = _d(prob.bd_g if nb else np.zeros(1))
        self.s_xy = _d(prob.sensor_xy if ns else np.zeros((1, 2)))
        self.s_u = _d(prob.sensor_u if ns else np.zeros(1))
        self.s = OracleProblem(self.vertices.shape[0], _ptr(self.vertices), self.cells.shape[0],
                               _ptr(self.cells, _ip), Q, T, _ptr(self.f_quad), len(prob.widths) - 1,
                               _ptr(self.widths, _ip), nb, _ptr(self.bd_xy), _ptr(self.bd_g), prob.tau,
                               ns, _ptr(self.s_xy), _ptr(self.s_u), prob.gamma, prob.b[0], prob.b[1], norm)
        self.n_params = int(sum(prob.widths[i + 1] * (prob.widths[i] + 1) for i in range(len(prob.widths) - 1)))

    def loss_grad(self, params, eps: Optional[float] = None, want_grad=True, want_R=False, want_ubar=False,
                  want_upts=False, n_threads: int = 1, want_eps_field=False):
        p = _d(params)
        eps = self.prob.eps if eps is None else eps
        n_e, Nt, Nq = self.cells.shape[0], self.prob.test_order ** 2, self.prob.quad_order ** 2
        loss4 = np.zeros(4)
        g = np.zeros(self.n_params) if want_grad else None
        de = np.zeros(1)
        R = np.zeros((n_e, Nt)) if want_R else None
        ub = np.zeros((n_e, Nq, 2)) if want_ubar else None
        up = np.zeros((n_e, Nq, 3)) if want_upts else None
        eb = np.zeros((n_e, Nq)) if want_eps_field else None
        ep = np.zeros((n_e, Nq)) if want_eps_field else None
        rc = lib().oracle_loss_grad(C.byref(self.s), _ptr(p), C.c_double(eps), _ptr(loss4), _ptr(g), _ptr(de),
                                    _ptr(R), _ptr(ub), _ptr(up), n_threads, _ptr(eb), _ptr(ep))
        if rc != 0:
            raise ValueError("oracle_loss_grad failed (%d)" % rc)
        out = {"loss": loss4[0], "Lv": loss4[1], "Lb": loss4[2], "Ls": loss4[3], "dL_deps": de[0]}
        if want_grad:
            out["grad"] = g
        if want_R:
            out["R"] = R
        if want_ubar:
            out["ubar"] = ub
        if want_upts:
            out["upts"] = up
        if want_eps_field:
            out["ebar"] = eb          # dL/deps(x_q) of a two-output network
            out["epts"] = ep          # eps(x_q)
        return out

    def loss_value(self, params, eps: Optional[float] = None, want_R=False):
        p = _d(params)
        eps = self.prob.eps if eps is None else eps
        loss4 = np.zeros(4)
        R = np.zeros((self.cells.shape[0], self.prob.test_order ** 2)) if want_R else None
        lib().oracle_loss_value(C.byref(self.s), _ptr(p), C.c_double(eps), _ptr(loss4), _ptr(R))
        return (loss4, R) if want_R else loss4

    def cstep(self, params, idx, eps: Optional[float] = None, h=1e-30, n_threads: int = 1):
        p = _d(params)
        eps = self.prob.eps if eps is None else eps
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        out = np.zeros(idx.size)
        lib().oracle_loss_cstep(C.byref(self.s), _ptr(p), C.c_double(eps), idx.size, _ptr(idx, _ip),
                                C.c_double(h), _ptr(out), n_threads)
        return out

    def residuals_given_grad(self, ux, uy, eps=None):
        eps = self.prob.eps if eps is None else eps
        ux, uy = _d(ux), _d(uy)
        R = np.zeros((self.cells.shape[0], self.prob.test_order ** 2))
        if lib().oracle_residuals_given_grad(C.byref(self.s), _ptr(ux), _ptr(uy), C.c_double(eps), _ptr(R)) != 0:
            raise ValueError("bad orders")
        return R

    def tensors(self):
        n_e, Nt, Nq = self.cells.shape[0], self.prob.test_order ** 2, self.prob.quad_order ** 2
        Gx, Gy, Gv = (np.zeros((n_e, Nt, Nq)) for _ in range(3))
        F = np.zeros((n_e, Nt))
        lib().oracle_build_tensors(C.byref(self.s), _ptr(Gx), _ptr(Gy), _ptr(Gv), _ptr(F))
        return Gx, Gy, Gv, F


def contract(Gx, Gy, Gv, F, ux, uy, eps, bx, by):
    n_e, Nt, Nq = Gx.shape
    R = np.zeros((n_e, Nt))
    lib().oracle_contract(n_e, Nt, Nq, _ptr(_d(Gx)), _ptr(_d(Gy)), _ptr(_d(Gv)), _ptr(_d(F)), _ptr(_d(ux)),
                          _ptr(_d(uy)), C.c_double(eps), C.c_double(bx), C.c_double(by), _ptr(R))
    return R
