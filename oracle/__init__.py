"""Serial FP64 CPU oracle for the N-shaped partition Crank-Nicolson method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2205_00856_b300``) and never imports it.

The arithmetic lives in ``cn_oracle.c`` (plain C99, IEEE double, no fast-math);
this module only builds it with gcc and marshals numpy arrays through ctypes.

Paper: Lutsyshyn, Navarrete, Bauer, "The N-shaped partition method: A novel
parallel implementation of the Crank Nicolson algorithm".
  - ``thomas``            Sec. 2, the serial Thomas algorithm.
  - ``cn_matrix``          Sec. 2, T = 1 + i dt/2 H(t + dt/2) and T^dagger.
  - ``cn_run``             Sec. 2, Eq. (ForwardStep) + Eq. (BackwardStep).
  - ``nshape_reduce``      Sec. 4, Table 1 stages RD, RU, JU, JD.
  - ``nshape_rs``          Sec. 4, Table 1 stage RS.
  - ``nshape_substitute``  Sec. 4, Table 1 stage SS.
  - ``nshape_solve``       Sec. 4.2, Eq. (iteration) (nested application).
  - ``adjoint_run``        discrete adjoint of the CN recursion (the paper
                           has no adjoint; derived from Eq. Cn_both_steps).
  - ``slab``               (module) the CN step over block-owning ranks with
                           the joint-line exchange, Sec. "MPI Implementation"
                           and "Communication and masking of the JD and JU
                           stages"; checked against ``cn_run`` on CPU thread
                           ranks and gloo processes.

Parity status: every function is pinned by ``-m "not gpu"`` tests in
``tests/test_oracle_*.py``; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cn_oracle.c")
_HDR = os.path.join(_HERE, "cn_oracle.h")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

POT_NONE, POT_ARRAY, POT_SOFTCOULOMB, POT_COSSERIES = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile ``cn_oracle.c`` into ``liboracle.so`` (gcc, -O2, no fast-math)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-Wall",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("dx", C.c_double), ("dt", C.c_double), ("x_min", C.c_double),
                ("pot", C.c_int32), ("V0", C.c_void_p), ("soft_s", C.c_double),
                ("cos_a", C.c_void_p), ("n_cos", C.c_int32), ("L", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
            sig = {
                "or_thomas": [i64, vp, vp, vp, vp, vp],
                "or_tridiag_apply": [i64, vp, vp, vp, vp, vp],
                "or_cn_matrix": [vp, dbl, C.c_int, vp, vp, vp],
                "or_cn_run": [vp, vp, vp, i64, vp],
                "or_nshape_reduce": [i64, vp, vp, vp, vp, i64, vp, C.c_int],
                "or_nshape_substitute": [i64, vp, vp, vp, vp, i64, vp, vp, vp],
                "or_nshape_rs": [vp, vp, vp, vp, i64, vp, vp],
                "or_nshape_solve": [i64, vp, vp, vp, vp, i64, vp, i64, vp, C.c_int, vp],
                "or_default_joints": [i64, i64, vp],
                "or_adjoint_run": [vp, vp, vp, i64, vp, vp, vp, vp],
            }
            for name, argt in sig.items():
                f = getattr(lib, name)
                f.argtypes = argt
                f.restype = C.c_int
            _lib = lib
    return _lib


def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.complex128)


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


class Problem:
    """A 1D TDSE grid problem: x_j = x_min + j dx, V(x, t) = Vs(x) + x E(t)."""

    def __init__(self, n, dx, dt, x_min, pot=POT_NONE, V0=None, soft_s=2.0, cos_a=None, L=1.0):
        self.n, self.dx, self.dt, self.x_min = int(n), float(dx), float(dt), float(x_min)
        self.pot, self.soft_s, self.L = int(pot), float(soft_s), float(L)
        self.V0 = None if V0 is None else _f64(V0)
        self.cos_a = None if cos_a is None else _f64(cos_a)
        if self.pot == POT_ARRAY and (self.V0 is None or self.V0.shape != (self.n,)):
            raise ValueError("POT_ARRAY needs V0 of length n")

    def _c(self) -> _Problem:
        return _Problem(self.n, self.dx, self.dt, self.x_min, self.pot,
                        None if self.V0 is None else self.V0.ctypes.data,
                        self.soft_s, None if self.cos_a is None else self.cos_a.ctypes.data,
                        0 if self.cos_a is None else len(self.cos_a), self.L)

    @staticmethod
    def from_dict(cfg: dict) -> "Problem":
        return Problem(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], cfg.get("pot", POT_NONE),
                       cfg.get("V0"), cfg.get("soft_s", 2.0), cfg.get("cos_a"), cfg.get("L", 1.0))


def thomas(b, a, c, d) -> np.ndarray:
    b, a, c, d = map(_c128, (b, a, c, d))
    x = np.empty_like(d)
    _check(_load().or_thomas(len(a), _p(b), _p(a), _p(c), _p(d), _p(x)), "thomas")
    return x


def tridiag_apply(b, a, c, x) -> np.ndarray:
    b, a, c, x = map(_c128, (b, a, c, x))
    y = np.empty_like(x)
    _check(_load().or_tridiag_apply(len(a), _p(b), _p(a), _p(c), _p(x), _p(y)), "tridiag_apply")
    return y


def cn_matrix(prob: Problem, E: float = 0.0, dt_sign: int = 1):
    """Diagonals (b, a, c) of T (dt_sign=+1) or T^dagger (dt_sign=-1)."""
    b = np.empty(prob.n, np.complex128)
    a = np.empty_like(b)
    c = np.empty_like(b)
    pc = prob._c()
    _check(_load().or_cn_matrix(C.byref(pc), float(E), int(dt_sign), _p(b), _p(a), _p(c)), "cn_matrix")
    return b, a, c


def cn_run(prob: Problem, psi0, nsteps: int, E_mid=None) -> np.ndarray:
    psi0 = _c128(psi0)
    out = np.empty_like(psi0)
    E = None if E_mid is None else _f64(E_mid)
    if E is not None and len(E) < nsteps:
        raise ValueError("E_mid shorter than nsteps")
    pc = prob._c()
    _check(_load().or_cn_run(C.byref(pc), _p(psi0), None if E is None else _p(E), int(nsteps), _p(out)),
           "cn_run")
    return out


def default_joints(n: int, P: int) -> np.ndarray:
    J = np.empty(P + 1, np.int64)
    _check(_load().or_default_joints(int(n), int(P), _p(J)), "default_joints")
    return J


def nshape_reduce(b, a, c, d, J, order: int = 1):
    """Table 1 RD/RU/JU/JD; returns the modified (b, a, c, d)."""
    bw, aw, cw, dw = (np.array(v, dtype=np.complex128, copy=True) for v in (b, a, c, d))
    J = np.ascontiguousarray(J, dtype=np.int64)
    _check(_load().or_nshape_reduce(len(aw), _p(bw), _p(aw), _p(cw), _p(dw), len(J) - 1, _p(J), int(order)),
           "nshape_reduce")
    return bw, aw, cw, dw


def nshape_rs(bw, aw, cw, dw, J) -> np.ndarray:
    """Table 1 RS on the joint lines of reduced vectors (copies its inputs)."""
    bw, aw, cw, dw = (np.array(v, dtype=np.complex128, copy=True) for v in (bw, aw, cw, dw))
    J = np.ascontiguousarray(J, dtype=np.int64)
    psi = np.empty(len(J), np.complex128)
    _check(_load().or_nshape_rs(_p(bw), _p(aw), _p(cw), _p(dw), len(J) - 1, _p(J), _p(psi)), "nshape_rs")
    return psi


def nshape_substitute(bw, aw, cw, dw, J, psi_J) -> np.ndarray:
    bw, aw, cw, dw, psi_J = map(_c128, (bw, aw, cw, dw, psi_J))
    J = np.ascontiguousarray(J, dtype=np.int64)
    x = np.empty_like(aw)
    _check(_load().or_nshape_substitute(len(aw), _p(bw), _p(aw), _p(cw), _p(dw), len(J) - 1, _p(J),
                                        _p(psi_J), _p(x)), "nshape_substitute")
    return x


def nshape_solve(b, a, c, d, J, nested_P=(), order: int = 1) -> np.ndarray:
    b, a, c, d = map(_c128, (b, a, c, d))
    J = np.ascontiguousarray(J, dtype=np.int64)
    nP = np.ascontiguousarray(nested_P if len(nested_P) else [0], dtype=np.int64)
    x = np.empty_like(d)
    _check(_load().or_nshape_solve(len(a), _p(b), _p(a), _p(c), _p(d), len(J) - 1, _p(J),
                                   len(nested_P), _p(nP), int(order), _p(x)), "nshape_solve")
    return x


def adjoint_run(prob: Problem, psi0, nsteps: int, wgt, E_mid=None, want_lam0: bool = False):
    """Returns (L, dL/dE_mid[nsteps], lambda_0 or None)."""
    psi0 = _c128(psi0)
    wgt = _f64(wgt)
    E = None if E_mid is None else _f64(E_mid)
    loss = np.zeros(1)
    g = np.zeros(max(nsteps, 1))
    lam0 = np.empty_like(psi0) if want_lam0 else None
    pc = prob._c()
    _check(_load().or_adjoint_run(C.byref(pc), _p(psi0), None if E is None else _p(E), int(nsteps), _p(wgt),
                                  _p(loss), _p(g), None if lam0 is None else _p(lam0)), "adjoint_run")
    return float(loss[0]), g[:nsteps], lam0
