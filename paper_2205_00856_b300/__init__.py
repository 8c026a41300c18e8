"""Python binding of libcn_b300.so: the B300-native N-shaped partition
Crank-Nicolson library (C ABI in include/cn.h).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  Tensors must be contiguous CUDA tensors (complex128 states,
float64 fields) on the plan's device.  There is no CPU fallback: if the shared
library cannot be loaded, every call raises.

Paper: Lutsyshyn, Navarrete, Bauer, "The N-shaped partition method: A novel
parallel implementation of the Crank Nicolson algorithm" (Sec. 2: the CN step;
Sec. 4: the N-shaped partition solve; Eq. iteration: its nesting).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

POT_NONE, POT_ARRAY, POT_SOFTCOULOMB, POT_COSSERIES = 0, 1, 2, 3
ARITH_F64, ARITH_DF64 = 0, 1
FLAG_COEFF_TABLE = 1
FLAG_RECOMPUTE = 2
FLAG_LEVEL_LAUNCHES = 4
FLAG_PERSISTENT_LEVELS = 8
FLAG_SERIAL_BLOCKS = 16

_STATUS = {0: "CN_OK", 1: "CN_ERR_INVALID_ARG", 2: "CN_ERR_UNSUPPORTED", 3: "CN_ERR_OOM", 4: "CN_ERR_CUDA",
           5: "CN_ERR_TIMEOUT", 6: "CN_ERR_NONFINITE", 7: "CN_ERR_BOUNDS"}

# every symbol declared in include/cn.h
EXPORTS = ("cn_plan_create", "cn_plan_destroy", "cn_step", "cn_step_host", "cn_solve_tridiag",
           "cn_plan_query", "cn_plan_profile", "cn_plan_profile_read", "cn_plan_status", "cn_status_string",
           "cn_version", "cn_solve_tridiag_noalloc", "cn_adjoint_step", "cn_field_from_controls",
           "cn_field_grad_to_controls", "cn_batch_create", "cn_batch_destroy", "cn_batch_offsets",
           "cn_batch_step", "cn_batch_status", "cn_plan_create_levels", "cn_step_states", "cn_plan_fill_workspace",
           "cn_batch_fill_workspace", "cn_slab_create", "cn_slab_range", "cn_slab_reduce", "cn_slab_finish",
           "cn_cuda_error_string", "cn_debug_report", "cn_debug_selftest", "cn_plan_set_wait_limit",
           "cn_measure_fp64_rate")
SLAB_MAX = 65536
SLAB_SHARE = 6  # complex values one slab contributes to the joint-line system per step
NOALLOC_MAX_N = 1048576
# (level-0 block, level block) pairs autotune_plan tries by default
PLAN_TUNE_CANDIDATES = tuple((m0, ml) for m0 in (8, 10, 12, 13, 16) for ml in (8, 12, 16, 24))
MAX_LEVELS = 24
# Launch configuration for large single systems (N ~ 2^24, coefficient table on),
# from block-size sweeps of the soft-Coulomb step on B300: (level-0 block, level-1
# block, block of the deeper levels) per arithmetic.
LARGE_GRID_BLOCKS = {ARITH_F64: (32, 16, 8), ARITH_DF64: (13, 10, 8)}
PROFILE_CLASSES = ("reduce_level0", "substitute_level0", "reduce_levels_ge1", "substitute_levels_ge1", "rs_stage",
                   "fused_level0", "levels_persistent")


class CNError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {_STATUS.get(code, code)}"
        if code in (3, 4) and _lib is not None:
            msg += f" ({_lib.cn_cuda_error_string().decode()})"
        super().__init__(msg)


class _Desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("dx", C.c_double), ("dt", C.c_double), ("x_min", C.c_double),
                ("pot", C.c_int32), ("n_cos", C.c_int32), ("V0", C.c_void_p), ("soft_s", C.c_double),
                ("cos_a", C.c_void_p), ("L", C.c_double), ("block", C.c_int32), ("arith", C.c_int32),
                ("flags", C.c_int32), ("level_block", C.c_int32), ("level1_block", C.c_int32)]


class _Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("levels", C.c_int32), ("launches_per_step", C.c_int32),
                ("level_rows", C.c_int64 * MAX_LEVELS), ("level_block", C.c_int32 * MAX_LEVELS),
                ("workspace_bytes", C.c_int64), ("level0_lanes", C.c_int32)]


_lib = None
_lock = threading.Lock()
_use_debug = False


def use_debug_library() -> None:
    """Load the CN_DEBUG build (bounds-checked kernels; include/cn.h) instead of
    the default library.  Must be called before the first call that loads it."""
    global _use_debug
    with _lock:
        if _lib is not None and not _use_debug:
            raise RuntimeError("the default library is already loaded in this process")
        _use_debug = True


def library_path() -> str:
    return _build.DEBUG_LIB if _use_debug else _build.LIB


def load(build_if_missing: bool = True):
    """Load libcn_b300.so (building it in-tree first if allowed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.DEBUG_LIB if _use_debug else _build.LIB
            if build_if_missing and _build.needs_build(path):
                _build.build(debug=_use_debug)
            if not os.path.exists(path):
                raise OSError(f"{os.path.basename(path)} not built ({path})")
            lib = C.CDLL(path)
            vp, i64 = C.c_void_p, C.c_int64
            lib.cn_plan_create.argtypes = [C.POINTER(_Desc), C.POINTER(vp)]
            lib.cn_plan_destroy.argtypes = [vp]
            lib.cn_step.argtypes = [vp, vp, vp, vp, i64, vp]
            lib.cn_step_states.argtypes = [vp, vp, vp, vp, i64, vp]
            lib.cn_step_states.restype = C.c_int
            lib.cn_step_host.argtypes = [vp, vp, vp, vp, i64, vp]
            lib.cn_solve_tridiag.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp]
            lib.cn_plan_status.argtypes = [vp]
            lib.cn_plan_query.argtypes = [vp, C.POINTER(_Info)]
            lib.cn_plan_profile.argtypes = [vp, C.c_int]
            lib.cn_plan_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]
            lib.cn_solve_tridiag_noalloc.argtypes = [vp, vp, vp, vp, vp, i64, C.c_int32, vp]
            lib.cn_adjoint_step.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
            lib.cn_adjoint_step.restype = C.c_int
            dbl = C.c_double
            lib.cn_field_from_controls.argtypes = [vp, i64, dbl, dbl, dbl, i64, vp, vp]
            lib.cn_field_from_controls.restype = C.c_int
            lib.cn_field_grad_to_controls.argtypes = [vp, i64, dbl, dbl, dbl, i64, vp, vp]
            lib.cn_field_grad_to_controls.restype = C.c_int
            lib.cn_solve_tridiag_noalloc.restype = C.c_int
            lib.cn_status_string.argtypes = [C.c_int]
            lib.cn_status_string.restype = C.c_char_p
            lib.cn_version.argtypes = []
            lib.cn_version.restype = C.c_char_p
            lib.cn_cuda_error_string.argtypes = []
            lib.cn_cuda_error_string.restype = C.c_char_p
            lib.cn_debug_report.argtypes = [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
            lib.cn_debug_report.restype = C.c_int
            lib.cn_debug_selftest.argtypes = []
            lib.cn_debug_selftest.restype = C.c_int
            lib.cn_measure_fp64_rate.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double)]
            lib.cn_measure_fp64_rate.restype = C.c_int
            lib.cn_plan_create_levels.argtypes = [C.POINTER(_Desc), C.c_int32, vp, C.POINTER(vp)]
            lib.cn_plan_create_levels.restype = C.c_int
            lib.cn_batch_create.argtypes = [C.POINTER(_Desc), i64, vp, vp, vp, C.POINTER(vp)]
            lib.cn_batch_destroy.argtypes = [vp]
            lib.cn_batch_offsets.argtypes = [vp, vp]
            lib.cn_batch_step.argtypes = [vp, vp, vp, vp, i64, vp]
            lib.cn_batch_status.argtypes = [vp]
            lib.cn_plan_fill_workspace.argtypes = [vp, C.c_int32]
            lib.cn_plan_set_wait_limit.argtypes = [vp, i64, C.c_int32]
            lib.cn_slab_create.argtypes = [C.POINTER(_Desc), C.c_int32, C.c_int32, vp, C.POINTER(vp)]
            lib.cn_slab_range.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
            lib.cn_slab_reduce.argtypes = [vp, vp, vp, vp, vp]
            lib.cn_slab_finish.argtypes = [vp, vp, vp, vp]
            lib.cn_batch_fill_workspace.argtypes = [vp, C.c_int32]
            for f in ("cn_batch_create", "cn_batch_destroy", "cn_batch_offsets", "cn_batch_step", "cn_batch_status",
                      "cn_plan_fill_workspace", "cn_batch_fill_workspace", "cn_slab_create", "cn_slab_range",
                      "cn_slab_reduce", "cn_slab_finish", "cn_plan_set_wait_limit"):
                getattr(lib, f).restype = C.c_int
            for f in ("cn_plan_create", "cn_plan_destroy", "cn_step", "cn_step_host", "cn_solve_tridiag",
                      "cn_plan_status", "cn_plan_query", "cn_plan_profile", "cn_plan_profile_read"):
                getattr(lib, f).restype = C.c_int
            _lib = lib
    return _lib


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise CNError(rc, what)


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev_ptr(t, dtype, n: int, name: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return t.data_ptr()


class Plan:
    """A cn_plan: workspace for systems of n unknowns on the current CUDA device.

    pot / V0 / soft_s / cos_a / L describe the static potential Vs(x) of
    H = -1/2 d^2/dx^2 + Vs(x) + x E(t) on x_j = x_min + j dx.
    levels: explicit nesting (cn_plan_create_levels): the block size of each
    reduced level, the last level solved serially whatever its size; None
    nests with block (level 0) / level1_block (level 1; 0: level_block) /
    level_block until the reduced system has <= 1024 rows, which is solved by
    cyclic reduction.
    """

    def _desc(self, n, dx, dt, x_min, pot, V0, soft_s, cos_a, L, block, arith, flags, level_block, level1_block):
        import torch
        self._lib = load()
        self.dt = float(dt)
        self.arith = int(arith)
        self._V0 = None
        v0p = None
        if pot == POT_ARRAY:
            self._V0 = V0
            v0p = _dev_ptr(V0, torch.float64, int(n), "V0")
        self._cos = None if cos_a is None else np.ascontiguousarray(cos_a, dtype=np.float64)
        return _Desc(int(n), float(dx), float(dt), float(x_min), int(pot),
                     0 if self._cos is None else len(self._cos), v0p, float(soft_s),
                     None if self._cos is None else self._cos.ctypes.data, float(L), int(block), self.arith,
                     int(flags), int(level_block), int(level1_block))

    def __init__(self, n, dx, dt, x_min, pot=POT_NONE, V0=None, soft_s=2.0, cos_a=None, L=1.0,
                 block=0, arith=ARITH_F64, flags=0, level_block=0, levels=None, level1_block=0):
        self.n = int(n)
        d = self._desc(n, dx, dt, x_min, pot, V0, soft_s, cos_a, L, block, arith, flags, level_block, level1_block)
        h = C.c_void_p()
        if levels is None:
            _check(self._lib.cn_plan_create(C.byref(d), C.byref(h)), "cn_plan_create")
        else:
            lv = np.ascontiguousarray(levels, dtype=np.int32)
            _check(self._lib.cn_plan_create_levels(C.byref(d), int(lv.size), lv.ctypes.data, C.byref(h)),
                   "cn_plan_create_levels")
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.cn_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, psi_in, nsteps: int, E_mid=None, psi_out=None, stream=None):
        """nsteps CN steps on device tensors; returns psi_out (allocated if None)."""
        import torch
        pin = _dev_ptr(psi_in, torch.complex128, self.n, "psi_in")
        if psi_out is None:
            psi_out = torch.empty_like(psi_in)
        pout = _dev_ptr(psi_out, torch.complex128, self.n, "psi_out")
        pe = None
        if E_mid is not None:
            if E_mid.numel() < nsteps:
                raise ValueError("E_mid shorter than nsteps")
            pe = _dev_ptr(E_mid, torch.float64, E_mid.numel(), "E_mid")
        _check(self._lib.cn_step(self._h, pin, pout, pe, int(nsteps), _stream_handle(stream)), "cn_step")
        return psi_out

    def step_states(self, psi_in, nsteps: int, E_mid=None, states_out=None, stream=None):
        """nsteps CN steps keeping every result: states_out[k] = psi after step k
        ((nsteps, n) complex128, allocated if None; must not overlap psi_in)."""
        import torch
        pin = _dev_ptr(psi_in, torch.complex128, self.n, "psi_in")
        if states_out is None:
            states_out = torch.empty((int(nsteps), self.n), dtype=torch.complex128, device=psi_in.device)
        pst = _dev_ptr(states_out, torch.complex128, int(nsteps) * self.n, "states_out")
        pe = None
        if E_mid is not None:
            if E_mid.numel() < nsteps:
                raise ValueError("E_mid shorter than nsteps")
            pe = _dev_ptr(E_mid, torch.float64, E_mid.numel(), "E_mid")
        _check(self._lib.cn_step_states(self._h, pin, pst, pe, int(nsteps), _stream_handle(stream)),
               "cn_step_states")
        return states_out

    def step_host(self, psi_in, nsteps: int, E_mid=None, psi_out=None, stream=None):
        """nsteps CN steps on host arrays (numpy or CPU tensors, pinned or not)."""
        pin = np.ascontiguousarray(psi_in, dtype=np.complex128) if not hasattr(psi_in, "data_ptr") else psi_in
        if psi_out is None:
            psi_out = np.empty(self.n, np.complex128)

        def hptr(a, dt, name, n):
            if hasattr(a, "data_ptr"):
                if a.is_cuda or not a.is_contiguous() or a.numel() < n:
                    raise ValueError(f"{name} must be a contiguous host tensor")
                return a.data_ptr()
            if a.dtype != dt or not a.flags.c_contiguous or a.size < n:
                raise ValueError(f"{name} must be contiguous {dt}")
            return a.ctypes.data

        E = None
        if E_mid is not None:
            E = E_mid if hasattr(E_mid, "data_ptr") else np.ascontiguousarray(E_mid, dtype=np.float64)
        _check(self._lib.cn_step_host(self._h, hptr(pin, np.complex128, "psi_in", self.n),
                                      hptr(psi_out, np.complex128, "psi_out", self.n),
                                      None if E is None else hptr(E, np.float64, "E_mid", nsteps),
                                      int(nsteps), _stream_handle(stream)), "cn_step_host")
        return psi_out

    def solve_tridiag(self, b, a, c, d, x=None, stream=None):
        """Solve T x = d (b lower, a diagonal, c upper; complex128 device tensors)."""
        import torch
        ptrs = [_dev_ptr(v, torch.complex128, self.n, nm) for v, nm in ((b, "b"), (a, "a"), (c, "c"), (d, "d"))]
        if x is None:
            x = torch.empty_like(d)
        px = _dev_ptr(x, torch.complex128, self.n, "x")
        _check(self._lib.cn_solve_tridiag(self._h, *ptrs, px, self.n, _stream_handle(stream)), "cn_solve_tridiag")
        return x

    def adjoint_step(self, psi_n, psi_np1, lam_np1, dLdE, E_mid=None, lam_n=None, stream=None):
        """One adjoint step (cn_adjoint_step): lam_n = T_n (T_n^dagger)^{-1} lam_np1 and
        dLdE[0] += dL/dE_n.  dLdE and E_mid are float64 device tensors (E_mid[0] is used)."""
        import torch
        ptrs = [_dev_ptr(v, torch.complex128, self.n, nm)
                for v, nm in ((psi_n, "psi_n"), (psi_np1, "psi_np1"), (lam_np1, "lam_np1"))]
        if lam_n is None:
            lam_n = torch.empty_like(lam_np1)
        pl = _dev_ptr(lam_n, torch.complex128, self.n, "lam_n")
        pg = _dev_ptr(dLdE, torch.float64, dLdE.numel(), "dLdE")
        pe = None if E_mid is None else _dev_ptr(E_mid, torch.float64, E_mid.numel(), "E_mid")
        _check(self._lib.cn_adjoint_step(self._h, *ptrs, pl, pe, pg, _stream_handle(stream)), "cn_adjoint_step")
        return lam_n

    def info(self) -> dict:
        """Nesting levels, kernels per step and workspace of the plan."""
        inf = _Info()
        _check(self._lib.cn_plan_query(self._h, C.byref(inf)), "cn_plan_query")
        L = inf.levels
        return dict(n=inf.n, levels=L, launches_per_step=inf.launches_per_step,
                    level_rows=list(inf.level_rows[:L + 1]), level_block=list(inf.level_block[:L]),
                    workspace_bytes=inf.workspace_bytes, level0_lanes=inf.level0_lanes)

    def profile(self, enable: bool = True) -> None:
        """Bracket every kernel launch with CUDA events (see profile_read)."""
        _check(self._lib.cn_plan_profile(self._h, 1 if enable else 0), "cn_plan_profile")

    def profile_read(self) -> dict:
        """{class: (total ms, launches)} since the previous read (synchronises)."""
        k = len(PROFILE_CLASSES)
        ms = (C.c_double * k)()
        nl = (C.c_int64 * k)()
        _check(self._lib.cn_plan_profile_read(self._h, ms, nl, k), "cn_plan_profile_read")
        return {PROFILE_CLASSES[i]: (float(ms[i]), int(nl[i])) for i in range(k)}

    def status(self) -> int:
        """Synchronise and return (then clear) the device-side status code."""
        return int(self._lib.cn_plan_status(self._h))

    def set_wait_limit(self, timeout_ns: int, missing_ctas: int = 0) -> None:
        """Time limit of the persistent launch's grid barriers; missing_ctas > 0 is a
        test hook that makes every barrier run out (cn_plan_set_wait_limit)."""
        _check(self._lib.cn_plan_set_wait_limit(self._h, int(timeout_ns), int(missing_ctas)),
               "cn_plan_set_wait_limit")

    def fill_workspace(self, byte: int = 0xFF) -> None:
        """Fill every scratch buffer of the plan with `byte` (cn_plan_fill_workspace)."""
        _check(self._lib.cn_plan_fill_workspace(self._h, int(byte)), "cn_plan_fill_workspace")

    def check(self) -> None:
        _check(self.status(), "device status")


class Slab(Plan):
    """Slab `rank` of a grid of n points sharded over `nslabs` ranks (cn_slab_create):
    the rows lo..hi of the grid between two joint lines (both included).  One CN
    step of the whole grid is reduce() on every slab, an all-gather of the
    6-value shares in rank order, and finish() on every slab (the driver is
    paper_2205_00856_b300.sharded).  joints: nslabs + 1 joint lines (None: the
    library's even split)."""

    def __init__(self, n, dx, dt, x_min, nslabs, rank, joints=None, pot=POT_NONE, V0=None, soft_s=2.0, cos_a=None,
                 L=1.0, block=0, arith=ARITH_F64, flags=0, level_block=0, level1_block=0):
        d = self._desc(n, dx, dt, x_min, pot, V0, soft_s, cos_a, L, block, arith, flags, level_block, level1_block)
        self.global_n, self.nslabs, self.rank = int(n), int(nslabs), int(rank)
        jp = None
        if joints is not None:
            self._joints = np.ascontiguousarray(joints, dtype=np.int64)
            if self._joints.size != self.nslabs + 1:
                raise ValueError("joints needs nslabs + 1 entries")
            jp = self._joints.ctypes.data
        h = C.c_void_p()
        _check(self._lib.cn_slab_create(C.byref(d), self.nslabs, self.rank, jp, C.byref(h)), "cn_slab_create")
        self._h = h
        lo, hi = C.c_int64(), C.c_int64()
        _check(self._lib.cn_slab_range(self._h, C.byref(lo), C.byref(hi)), "cn_slab_range")
        self.lo, self.hi = int(lo.value), int(hi.value)
        self.n = self.hi - self.lo + 1  # rows of the slab's local arrays

    def reduce(self, psi_local, E_mid=None, share_out=None, stream=None):
        """Step part 1: the slab's share of the joint-line system (6 complex128 on the device)."""
        import torch
        pin = _dev_ptr(psi_local, torch.complex128, self.n, "psi_local")
        if share_out is None:
            share_out = torch.empty(SLAB_SHARE, dtype=torch.complex128, device=psi_local.device)
        ps = _dev_ptr(share_out, torch.complex128, SLAB_SHARE, "share_out")
        pe = None if E_mid is None else _dev_ptr(E_mid, torch.float64, E_mid.numel(), "E_mid")
        _check(self._lib.cn_slab_reduce(self._h, pin, pe, ps, _stream_handle(stream)), "cn_slab_reduce")
        return share_out

    def finish(self, shares, psi_out, stream=None):
        """Step part 2: every slab's share in rank order (6 nslabs complex128) -> the slab's rows."""
        import torch
        pa = _dev_ptr(shares, torch.complex128, SLAB_SHARE * self.nslabs, "shares")
        po = _dev_ptr(psi_out, torch.complex128, self.n, "psi_out")
        _check(self._lib.cn_slab_finish(self._h, pa, po, _stream_handle(stream)), "cn_slab_finish")
        return psi_out


class Batch:
    """A cn_batch: nsys independent CN systems of uneven sizes stepped together,
    one launch per stage and nesting level for all of them.

    sizes: rows per system; the batch state is one complex128 tensor of
    `total` rows with system s at rows offsets[s]:offsets[s+1].  x_min: per
    system (None: -floor(n_s/2) dx).  cos_a: (nsys, n_cos) coefficients for
    POT_COSSERIES, period L (<= 0: each system's own length n_s dx).  V0
    (POT_ARRAY): float64 tensor of `total` values, read at creation only.
    """

    def __init__(self, sizes, dx, dt, x_min=None, pot=POT_NONE, V0=None, soft_s=2.0, cos_a=None, L=0.0,
                 block=0, arith=ARITH_F64, flags=0, level_block=0, level1_block=0):
        import torch
        self._lib = load()
        self.sizes = np.ascontiguousarray(sizes, dtype=np.int64)
        self.nsys = int(self.sizes.size)
        self.dt = float(dt)
        self.arith = int(arith)
        self.block, self.level_block = int(block), int(level_block)
        xm = None if x_min is None else np.ascontiguousarray(x_min, dtype=np.float64)
        if xm is not None and xm.size != self.nsys:
            raise ValueError("x_min needs one value per system")
        cos = None if cos_a is None else np.ascontiguousarray(cos_a, dtype=np.float64)
        n_cos = 0
        if cos is not None:
            if cos.ndim != 2 or cos.shape[0] != self.nsys:
                raise ValueError("cos_a must have shape (nsys, n_cos)")
            n_cos = cos.shape[1]
        v0p = None
        if pot == POT_ARRAY:
            v0p = _dev_ptr(V0, torch.float64, int(self.sizes.sum()), "V0")
        d = _Desc(0, float(dx), float(dt), 0.0, int(pot), n_cos, v0p, float(soft_s), None, float(L), int(block),
                  self.arith, int(flags), int(level_block), int(level1_block))
        h = C.c_void_p()
        _check(self._lib.cn_batch_create(C.byref(d), self.nsys, self.sizes.ctypes.data,
                                         None if xm is None else xm.ctypes.data,
                                         None if cos is None else cos.ctypes.data, C.byref(h)), "cn_batch_create")
        self._h = h
        self.offsets = np.empty(self.nsys + 1, np.int64)
        _check(self._lib.cn_batch_offsets(self._h, self.offsets.ctypes.data), "cn_batch_offsets")
        self.total = int(self.offsets[-1])

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.cn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, psi_in, nsteps: int, E_mid=None, psi_out=None, stream=None):
        """nsteps CN steps of every system; returns psi_out (allocated if None)."""
        import torch
        pin = _dev_ptr(psi_in, torch.complex128, self.total, "psi_in")
        if psi_out is None:
            psi_out = torch.empty_like(psi_in)
        pout = _dev_ptr(psi_out, torch.complex128, self.total, "psi_out")
        pe = None
        if E_mid is not None:
            if E_mid.numel() < nsteps:
                raise ValueError("E_mid shorter than nsteps")
            pe = _dev_ptr(E_mid, torch.float64, E_mid.numel(), "E_mid")
        _check(self._lib.cn_batch_step(self._h, pin, pout, pe, int(nsteps), _stream_handle(stream)), "cn_batch_step")
        return psi_out

    def capture(self, psi, nsteps: int, E_mid=None):
        """Record nsteps in-place steps of the batch state psi into a CUDA graph;
        graph.replay() then runs them with one host call."""
        import torch
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                self.step(psi, nsteps, E_mid=E_mid, psi_out=psi)
        torch.cuda.current_stream().wait_stream(side)
        return g

    def status(self) -> int:
        return int(self._lib.cn_batch_status(self._h))

    def fill_workspace(self, byte: int = 0xFF) -> None:
        """Fill every scratch buffer of the batch with `byte` (cn_batch_fill_workspace)."""
        _check(self._lib.cn_batch_fill_workspace(self._h, int(byte)), "cn_batch_fill_workspace")

    def check(self) -> None:
        _check(self.status(), "device status")


def autotune_batch(sizes, dx, dt, candidates=None, steps: int = 3, repeats: int = 2, **kw):
    """Pick (block, level_block) for a batch by timing `steps` CN steps of each
    candidate on a synthetic state (the CN step costs the same for any state).
    Returns (best_block, best_level_block, {candidate: ms per step})."""
    import torch
    if candidates is None:
        candidates = [(m0, ml) for m0 in (6, 8, 10, 12, 16) for ml in (8, 16)]
    times = {}
    for m0, ml in candidates:
        b = Batch(sizes, dx, dt, block=m0, level_block=ml, **kw)
        psi = torch.zeros(b.total, dtype=torch.complex128, device="cuda")
        b.step(psi, 1, psi_out=psi)  # warm-up
        best = float("inf")
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.step(psi, steps, psi_out=psi)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / steps)
        b.check()
        times[(m0, ml)] = best
        del psi
        b.close()
    m0, ml = min(times, key=times.get)
    return m0, ml, times


def autotune_plan(n, dx, dt, x_min, candidates=None, steps: int = 10, repeats: int = 2, **kw):
    """Pick (block, level_block) for a single-system plan by timing `steps` CN steps
    of each candidate in place (same cost for any state; a zero state here).
    Returns (best_block, best_level_block, {candidate: ms per step})."""
    import torch
    if candidates is None:
        candidates = list(PLAN_TUNE_CANDIDATES)
    times = {}
    psi = torch.zeros(int(n), dtype=torch.complex128, device="cuda")
    for m0, ml in candidates:
        p = Plan(n, dx, dt, x_min, block=m0, level_block=ml, **kw)
        p.step(psi, 1, psi_out=psi)  # warm-up
        best = float("inf")
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            p.step(psi, steps, psi_out=psi)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / steps)
        p.check()
        p.close()
        times[(m0, ml)] = best
    del psi
    m0, ml = min(times, key=times.get)
    return m0, ml, times


def solve_tridiag_noalloc(b, a, c, d, x=None, arith=ARITH_F64, stream=None):
    """Solve T x = d without a plan and without allocating device memory inside
    the library (cn_solve_tridiag_noalloc), for callers that cannot allocate on
    their solve path.  n <= NOALLOC_MAX_N; calls that overlap on the GPU race."""
    import torch
    lib = load()
    n = a.numel()
    ptrs = [_dev_ptr(v, torch.complex128, n, nm) for v, nm in ((b, "b"), (a, "a"), (c, "c"), (d, "d"))]
    if x is None:
        x = torch.empty_like(d)
    px = _dev_ptr(x, torch.complex128, n, "x")
    _check(lib.cn_solve_tridiag_noalloc(*ptrs, px, n, int(arith), _stream_handle(stream)),
           "cn_solve_tridiag_noalloc")
    return x


def field_from_controls(u, t_final: float, t0: float, dt: float, nsteps: int, out=None, stream=None):
    """E_mid[k] = piecewise-linear field of the control samples u at t0 + (k + 1/2) dt."""
    import torch
    lib = load()
    pu = _dev_ptr(u, torch.float64, u.numel(), "u")
    if out is None:
        out = torch.empty(nsteps, dtype=torch.float64, device=u.device)
    po = _dev_ptr(out, torch.float64, nsteps, "E_mid")
    _check(lib.cn_field_from_controls(pu, u.numel(), float(t_final), float(t0), float(dt), int(nsteps), po,
                                      _stream_handle(stream)), "cn_field_from_controls")
    return out


def field_grad_to_controls(dLdE, t_final: float, t0: float, dt: float, n_controls: int, out=None, stream=None):
    """Transpose of field_from_controls: gradient with respect to the control samples."""
    import torch
    lib = load()
    pg = _dev_ptr(dLdE, torch.float64, dLdE.numel(), "dLdE")
    if out is None:
        out = torch.empty(n_controls, dtype=torch.float64, device=dLdE.device)
    po = _dev_ptr(out, torch.float64, n_controls, "grad_u")
    _check(lib.cn_field_grad_to_controls(pg, dLdE.numel(), float(t_final), float(t0), float(dt), int(n_controls), po,
                                         _stream_handle(stream)), "cn_field_grad_to_controls")
    return out


def version() -> str:
    return load().cn_version().decode()


def fp64_rate():
    """Measured throughput of the device's FP64 pipe: (binary64 FMAs per second,
    binary64 additions per second) of the whole device (cn_measure_fp64_rate)."""
    f, a = C.c_double(), C.c_double()
    _check(load().cn_measure_fp64_rate(C.byref(f), C.byref(a)), "cn_measure_fp64_rate")
    return float(f.value), float(a.value)


def debug_report():
    """CN_DEBUG build: (status, address, bytes) of the first out-of-bounds access
    caught since the previous report (status 0: none; 7: CN_ERR_BOUNDS); the
    default build returns status 2 (CN_ERR_UNSUPPORTED)."""
    a, b = C.c_uint64(), C.c_uint64()
    rc = load().cn_debug_report(C.byref(a), C.byref(b))
    return int(rc), int(a.value), int(b.value)
