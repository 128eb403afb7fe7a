"""Thin Python binding of the C ABI in include/pf.h (argument marshalling only).

Every function has the name of the C entry point it wraps.  Arrays are numpy
float64 / int32 in the caller's bus numbering; device pointers may be given as
integers or as objects with ``data_ptr()`` (e.g. torch CUDA tensors).  All
numeric work runs in the CUDA library ``_lib/libpf.so``; importing this
module fails loudly if that library has not been built.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import cases as _cases

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpf.so")

PF_OK, PF_PENDING = 0, 1
PF_ERR_INVALID, PF_ERR_NOMEM, PF_ERR_MAXITER, PF_ERR_DIVERGED = -1, -2, -3, -4
PF_ERR_SINGULAR, PF_ERR_TIMEOUT, PF_ERR_BUSY, PF_ERR_CUDA = -5, -6, -7, -8
PF_ERR_UNSUPPORTED = -9
PF_SLACK, PF_PV, PF_PQ = 0, 1, 2
PF_NR, PF_NK = 0, 1
PF_FP64, PF_MIXED = 0, 1
PF_SINGLE_PHASE, PF_THREE_PHASE = 1, 3

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_u8p = C.POINTER(C.c_uint8)


class pf_case_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_bus", C.c_int), ("n_branch", C.c_int),
                ("bus_type", _ip), ("v_set", _dp), ("p_gen", _dp), ("q_gen", _dp),
                ("p_load", _dp), ("q_load", _dp), ("zip", _dp),
                ("br_from", _ip), ("br_to", _ip), ("br_r", _dp), ("br_x", _dp),
                ("br_b", _dp), ("phases", _u8p), ("source", C.c_int),
                ("v_source", C.c_double), ("br_phases", _u8p), ("br_z", _dp),
                ("q_min", _dp), ("q_max", _dp)]


class pf_opts(C.Structure):
    _fields_ = [("method", C.c_int), ("precision", C.c_int), ("tol", C.c_double),
                ("max_iter", C.c_int), ("refine_steps", C.c_int),
                ("refine_below", C.c_double),
                ("gmres_restart", C.c_int), ("gmres_max_iter", C.c_int),
                ("gmres_rtol", C.c_double), ("warm_start", C.c_int),
                ("cluster_size", C.c_int), ("block_threads", C.c_int),
                ("scen_per_cta", C.c_int), ("nk_fallback", C.c_int),
                ("kernel_by_kernel", C.c_int), ("krylov", C.c_int), ("q_limits", C.c_int),
                ("refine_stall", C.c_double)]


class pf_info(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int),
                ("linear_iterations", C.c_int), ("fallback", C.c_int),
                ("mismatch", C.c_double), ("max_step", C.c_double),
                ("solve_us", C.c_double), ("q_switched", C.c_int), ("q_rounds", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pf_case_stats(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_bus", C.c_int), ("block_size", C.c_int),
                ("n_unknowns", C.c_int), ("nnz_y", C.c_longlong), ("nnz_lu", C.c_longlong),
                ("n_updates", C.c_longlong), ("levels_factor", C.c_int),
                ("levels_backward", C.c_int), ("levels_ilu", C.c_int),
                ("levels_ilu_backward", C.c_int), ("device_bytes", C.c_longlong),
                ("bytes_per_scenario", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pf_serve_stats(C.Structure):
    _fields_ = [("requests", C.c_uint64), ("group_launches", C.c_uint64),
                ("max_group", C.c_int), ("peak_running", C.c_int),
                ("batch_launches", C.c_uint64), ("max_batch", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


INFO_DTYPE = np.dtype([("status", np.int32), ("iterations", np.int32),
                       ("linear_iterations", np.int32), ("fallback", np.int32),
                       ("mismatch", np.float64), ("max_step", np.float64),
                       ("solve_us", np.float64), ("q_switched", np.int32),
                       ("q_rounds", np.int32)])
assert INFO_DTYPE.itemsize == C.sizeof(pf_info)

_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        sig = {
            "pf_opts_default": (None, [C.POINTER(pf_opts)]),
            "pf_last_error": (C.c_char_p, []),
            "pf_status_str": (C.c_char_p, [C.c_int]),
            "pf_analyze": (C.c_int, [C.POINTER(pf_case_desc), C.POINTER(pf_case_stats)]),
            "pf_ybus": (C.c_int, [C.POINTER(pf_case_desc), C.POINTER(C.c_int64), _ip, _ip, _dp]),
            "pf_symbolic": (C.c_int, [C.POINTER(pf_case_desc), C.c_int, _ip, _ip, _ip, _ip, _ip]),
            "pf_schedule": (C.c_int, [C.POINTER(pf_case_desc), C.c_int, C.POINTER(C.c_int64),
                                      _ip, _ip, _ip, _ip, _ip, _ip, _ip, _ip, _ip]),
            "pf_ctx_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(vp)]),
            "pf_ctx_destroy": (C.c_int, [vp]),
            "pf_create_case": (C.c_int, [vp, C.POINTER(pf_case_desc), C.POINTER(vp)]),
            "pf_destroy_case": (C.c_int, [vp]),
            "pf_case_get_stats": (C.c_int, [vp, C.POINTER(pf_case_stats)]),
            "pf_solve": (C.c_int, [vp, C.POINTER(pf_opts), _dp, _dp, C.POINTER(pf_info)]),
            "pf_solve_batch": (C.c_int, [vp, C.c_int, _dp, _dp, _dp, C.POINTER(pf_opts), _dp,
                                         _dp, C.POINTER(pf_info)]),
            "pf_solve_batch_device": (C.c_int, [vp, C.c_int, vp, vp, vp, C.POINTER(pf_opts), vp,
                                                vp, vp, vp]),
            "pf_submit": (C.c_int, [vp, vp, _dp, _dp, _dp, C.POINTER(pf_opts),
                                    C.POINTER(C.c_uint64)]),
            "pf_submit_batch": (C.c_int, [vp, vp, C.c_int, _dp, _dp, _dp, C.POINTER(pf_opts),
                                          C.POINTER(C.c_uint64)]),
            "pf_poll": (C.c_int, [vp, C.c_uint64, _dp, _dp, C.POINTER(pf_info)]),
            "pf_drain": (C.c_int, [vp, C.c_int]),
            "pf_serve_get_stats": (C.c_int, [vp, C.POINTER(pf_serve_stats)]),
            "pf_case_pattern": (C.c_int, [vp, _ip, _ip]),
            "pf_eval_mismatch": (C.c_int, [vp, _dp, _dp, _dp]),
            "pf_eval_jacobian": (C.c_int, [vp, _dp, _dp, _dp]),
            "pf_newton_step": (C.c_int, [vp, C.POINTER(pf_opts), _dp, _dp, _dp,
                                         C.POINTER(pf_info)]),
            "pf_profile_solve": (C.c_int, [vp, C.c_int, C.POINTER(pf_opts), _dp, vp]),
            "pf_launch_config": (C.c_int, [vp, C.POINTER(pf_opts), C.c_int, _ip, _ip, _ip, _ip]),
            "pf_solve_noalloc": (C.c_int, [vp, C.POINTER(pf_opts), vp, vp, vp, vp, vp, vp, vp]),
            "pf_autotune": (C.c_int, [vp, C.c_int, C.POINTER(pf_opts)]),
            "pf_branch_flows": (C.c_int, [vp, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{lib().pf_status_str(code).decode()}: {msg}")
        self.code = code


def _check(rc):
    if rc < 0:
        raise PfError(rc, lib().pf_last_error().decode())
    return rc


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


def _devptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return C.c_void_p(x)
    return C.c_void_p(x.data_ptr())


# ----------------------------------------------------------------------------
# case descriptions
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class _Desc:
    """A pf_case_desc plus the numpy arrays it points into (kept alive)."""
    desc: pf_case_desc
    keep: list


def make_desc(case) -> _Desc:
    """pf_case_desc for a SinglePhaseCase or ThreePhaseCase."""
    keep = []

    def f64(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return _ptr(a, C.c_double)

    def i32(a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        keep.append(a)
        return _ptr(a, C.c_int32)

    def u8(a):
        a = np.ascontiguousarray(a, dtype=np.uint8)
        keep.append(a)
        return _ptr(a, C.c_uint8)

    d = pf_case_desc()
    if isinstance(case, _cases.SinglePhaseCase):
        d.kind, d.n_bus, d.n_branch = PF_SINGLE_PHASE, case.n_bus, case.n_branch
        d.bus_type = i32(case.bus_type)
        d.v_set, d.p_gen, d.q_gen = f64(case.v_set), f64(case.p_gen), f64(case.q_gen)
        d.p_load, d.q_load, d.zip = f64(case.p_load), f64(case.q_load), f64(case.zip)
        d.br_from, d.br_to = i32(case.br_from), i32(case.br_to)
        d.br_r, d.br_x, d.br_b = f64(case.br_r), f64(case.br_x), f64(case.br_b)
        if case.q_max is not None:  # reactive limits of PV buses
            d.q_min, d.q_max = f64(case.q_min), f64(case.q_max)
    elif isinstance(case, _cases.ThreePhaseCase):
        d.kind, d.n_bus, d.n_branch = PF_THREE_PHASE, case.n_node, case.n_branch
        d.phases = u8(case.phases)
        d.source, d.v_source = case.source, case.v_source
        d.p_load, d.q_load = f64(case.p_load.reshape(-1)), f64(case.q_load.reshape(-1))
        d.zip = f64(case.zip)
        d.br_from, d.br_to = i32(case.br_from), i32(case.br_to)
        d.br_phases = u8(case.br_phases)
        z = np.ascontiguousarray(case.br_z, dtype=np.complex128)
        d.br_z = f64(np.stack([z.real, z.imag], axis=-1).reshape(-1))
        if case.node_type is not None:  # PV nodes
            d.bus_type = i32(case.node_type)
            d.v_set = f64(case.v_set)
            d.p_gen = f64(np.asarray(case.p_gen).reshape(-1))
        if case.q_max is not None:  # reactive limits per node and phase
            d.q_min = f64(np.asarray(case.q_min).reshape(-1))
            d.q_max = f64(np.asarray(case.q_max).reshape(-1))
    else:
        raise TypeError("expected a SinglePhaseCase or ThreePhaseCase")
    return _Desc(d, keep)


def _slots(case_or_kind, n):
    return n if case_or_kind == PF_SINGLE_PHASE else 3 * n


def make_opts(**kw) -> pf_opts:
    """pf_opts with library defaults, overridden by keyword arguments."""
    o = pf_opts()
    lib().pf_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# ----------------------------------------------------------------------------
# host-only calls
# ----------------------------------------------------------------------------

def pf_analyze(case) -> dict:
    d = make_desc(case)
    st = pf_case_stats()
    _check(lib().pf_analyze(C.byref(d.desc), C.byref(st)))
    return st.as_dict()


def pf_ybus(case):
    """(rowptr, col, val) of Ybus; val complex [nnz] or [nnz, 3, 3]."""
    d = make_desc(case)
    nnz = C.c_int64()
    _check(lib().pf_ybus(C.byref(d.desc), C.byref(nnz), None, None, None))
    n = d.desc.n_bus
    ybs = 1 if d.desc.kind == PF_SINGLE_PHASE else 3
    rowptr = np.zeros(n + 1, np.int32)
    col = np.zeros(nnz.value, np.int32)
    val = np.zeros(nnz.value * 2 * ybs * ybs)
    _check(lib().pf_ybus(C.byref(d.desc), C.byref(nnz), _ptr(rowptr, C.c_int32),
                         _ptr(col, C.c_int32), _ptr(val, C.c_double)))
    v = val[0::2] + 1j * val[1::2]
    return rowptr, col, (v if ybs == 1 else v.reshape(-1, 3, 3))


def pf_symbolic(case, method=PF_NR):
    """(perm, rowptr, col, flevel, blevel) of a method's factor pattern."""
    st = pf_analyze(case)
    n = st["n_bus"]
    nnz = st["nnz_lu"] if method == PF_NR else st["nnz_y"]
    d = make_desc(case)
    perm = np.zeros(n, np.int32)
    rowptr = np.zeros(n + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    fl = np.zeros(n, np.int32)
    bl = np.zeros(n, np.int32)
    _check(lib().pf_symbolic(C.byref(d.desc), method, *[_ptr(a, C.c_int32)
                                                        for a in (perm, rowptr, col, fl, bl)]))
    return perm, rowptr, col, fl, bl


def pf_schedule(case, method=PF_NR) -> dict:
    """The packed factor and sweep records the kernels run (pf.h)."""
    d = make_desc(case)
    sz = (C.c_int64 * 6)()
    _check(lib().pf_schedule(C.byref(d.desc), method, sz, *([None] * 9)))
    n, L, Lb, F, T, Cn = list(sz)
    out = {"fac_ptr": np.zeros(L + 1, np.int32), "fac_rec": np.zeros((F, 4), np.int32),
           "tgt_ptr": np.zeros(L + 1, np.int32), "tgt_rec": np.zeros((T, 4), np.int32),
           "con": np.zeros((Cn, 2), np.int32), "flev_ptr": np.zeros(L + 1, np.int32),
           "fwd_rec": np.zeros((n, 4), np.int32), "blev_ptr": np.zeros(Lb + 1, np.int32),
           "bwd_rec": np.zeros((n, 4), np.int32)}
    keys = ("fac_ptr", "fac_rec", "tgt_ptr", "tgt_rec", "con", "flev_ptr", "fwd_rec",
            "blev_ptr", "bwd_rec")
    _check(lib().pf_schedule(C.byref(d.desc), method, sz, *[_ptr(out[k], C.c_int32) for k in keys]))
    return out


# ----------------------------------------------------------------------------
# contexts, cases and solves
# ----------------------------------------------------------------------------

def pf_ctx_create(device=0, budget=0):
    h = C.c_void_p()
    _check(lib().pf_ctx_create(device, budget, C.byref(h)))
    return h


def pf_ctx_destroy(ctx):
    _check(lib().pf_ctx_destroy(ctx))


class CaseHandle:
    """A created pf_case with the facts the binding needs to size arrays."""

    def __init__(self, handle, kind, n):
        self.handle, self.kind, self.n = handle, kind, n

    @property
    def slots(self):
        return _slots(self.kind, self.n)

    @property
    def _as_parameter_(self):
        return self.handle


def pf_create_case(ctx, case) -> CaseHandle:
    d = make_desc(case)
    h = C.c_void_p()
    _check(lib().pf_create_case(ctx, C.byref(d.desc), C.byref(h)))
    return CaseHandle(h, d.desc.kind, d.desc.n_bus)


def pf_destroy_case(c: CaseHandle):
    _check(lib().pf_destroy_case(c.handle))


def pf_case_get_stats(c: CaseHandle) -> dict:
    st = pf_case_stats()
    _check(lib().pf_case_get_stats(c.handle, C.byref(st)))
    return st.as_dict()


def pf_solve(c: CaseHandle, opts: pf_opts | None = None):
    """(vmag, vang, info) of one solve; arrays per bus or per slot."""
    vm = np.zeros(c.slots)
    va = np.zeros(c.slots)
    info = pf_info()
    _check(lib().pf_solve(c.handle, C.byref(opts) if opts else None, _ptr(vm, C.c_double),
                          _ptr(va, C.c_double), C.byref(info)))
    return vm, va, info.as_dict()


def pf_solve_batch(c: CaseHandle, p_load, q_load, p_gen=None, opts: pf_opts | None = None,
                   out=None):
    """Batch of B scenarios: loads [B, slots]; returns vmag, vang [B, slots], info[B].

    ``out`` = (vmag, vang, info) writes into caller buffers (e.g. pinned host
    memory) instead of new arrays."""
    p_load = np.ascontiguousarray(p_load, dtype=np.float64)
    q_load = np.ascontiguousarray(q_load, dtype=np.float64)
    B = p_load.shape[0]
    p_load = p_load.reshape(B, -1)
    q_load = q_load.reshape(B, -1)
    pg = None if p_gen is None else np.ascontiguousarray(p_gen, dtype=np.float64).reshape(B, -1)
    if out is None:
        vm = np.zeros((B, c.slots))
        va = np.zeros((B, c.slots))
        info = np.zeros(B, INFO_DTYPE)
    else:
        vm, va, info = out
        assert vm.flags.c_contiguous and va.flags.c_contiguous and info.dtype == INFO_DTYPE
        assert vm.size == B * c.slots and va.size == B * c.slots and info.size == B
    _check(lib().pf_solve_batch(c.handle, B, _ptr(p_load, C.c_double), _ptr(q_load, C.c_double),
                                _ptr(pg, C.c_double), C.byref(opts) if opts else None,
                                _ptr(vm, C.c_double), _ptr(va, C.c_double),
                                info.ctypes.data_as(C.POINTER(pf_info))))
    return vm, va, info


def pf_branch_flows(c: CaseHandle, vmag, vang, n_branch: int):
    """Branch flows of voltages [B, slots] (or [slots]): dict of p_from,
    q_from, p_to, q_to [B, n_branch * ph] and loss [B, 2] (P, Q)."""
    vm = np.ascontiguousarray(vmag, dtype=np.float64)
    va = np.ascontiguousarray(vang, dtype=np.float64)
    B = vm.shape[0] if vm.ndim == 2 else 1
    vm = vm.reshape(B, -1)
    va = va.reshape(B, -1)
    ph = 1 if c.kind == PF_SINGLE_PHASE else 3
    out = {k: np.zeros((B, n_branch * ph)) for k in ("p_from", "q_from", "p_to", "q_to")}
    loss = np.zeros((B, 2))
    _check(lib().pf_branch_flows(c.handle, B, _ptr(vm, C.c_double), _ptr(va, C.c_double),
                                 *[_ptr(out[k], C.c_double)
                                   for k in ("p_from", "q_from", "p_to", "q_to")],
                                 _ptr(loss, C.c_double)))
    out["loss"] = loss
    return out


def pf_solve_batch_device(c: CaseHandle, B, d_p_load, d_q_load, d_p_gen, opts, d_vmag, d_vang,
                          d_info, stream=0):
    """Device-pointer batch solve, asynchronous on ``stream`` (an int handle)."""
    _check(lib().pf_solve_batch_device(
        c.handle, B, _devptr(d_p_load), _devptr(d_q_load), _devptr(d_p_gen),
        C.byref(opts) if opts else None, _devptr(d_vmag), _devptr(d_vang), _devptr(d_info),
        C.c_void_p(stream)))


def pf_submit(ctx, c: CaseHandle, p_load=None, q_load=None, p_gen=None,
              opts: pf_opts | None = None) -> int:
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
            for a in (p_load, q_load, p_gen)]
    t = C.c_uint64()
    _check(lib().pf_submit(ctx, c.handle, *[_ptr(a, C.c_double) for a in arrs],
                           C.byref(opts) if opts else None, C.byref(t)))
    return t.value


def pf_submit_batch(ctx, c: CaseHandle, p_load=None, q_load=None, p_gen=None,
                    opts: pf_opts | None = None) -> list:
    """B requests queued at once (arrays [B][...]); their tickets."""
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in
            (p_load, q_load, p_gen)]
    B = next(a.shape[0] for a in arrs if a is not None)
    arrs = [None if a is None else a.reshape(B, -1) for a in arrs]
    t = (C.c_uint64 * B)()
    _check(lib().pf_submit_batch(ctx, c.handle, B, *[_ptr(a, C.c_double) for a in arrs],
                                 C.byref(opts) if opts else None, t))
    return list(t)


def pf_poll(ctx, ticket: int, slots: int, values: bool = True):
    """None while pending, else (vmag, vang, info); with values False only
    info is copied out (vmag, vang are None)."""
    vm = np.zeros(slots) if values else None
    va = np.zeros(slots) if values else None
    info = pf_info()
    rc = _check(lib().pf_poll(ctx, ticket, _ptr(vm, C.c_double), _ptr(va, C.c_double),
                              C.byref(info)))
    if rc == PF_PENDING:
        return None
    return vm, va, info.as_dict()


def pf_drain(ctx, timeout_ms=60_000):
    _check(lib().pf_drain(ctx, timeout_ms))


def pf_serve_get_stats(ctx) -> dict:
    """Counters of the context's serving runtime (requests, group launches,
    largest group, most requests on the GPU at once)."""
    st = pf_serve_stats()
    _check(lib().pf_serve_get_stats(ctx, C.byref(st)))
    return st.as_dict()


def pf_case_pattern(c: CaseHandle, nnz: int):
    rowptr = np.zeros(c.n + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    _check(lib().pf_case_pattern(c.handle, _ptr(rowptr, C.c_int32), _ptr(col, C.c_int32)))
    return rowptr, col


def _bs(c):
    return 2 if c.kind == PF_SINGLE_PHASE else 6


def pf_eval_mismatch(c: CaseHandle, vmag, vang):
    vm = np.ascontiguousarray(vmag, dtype=np.float64).reshape(-1)
    va = np.ascontiguousarray(vang, dtype=np.float64).reshape(-1)
    out = np.zeros((c.n, _bs(c)))
    _check(lib().pf_eval_mismatch(c.handle, _ptr(vm, C.c_double), _ptr(va, C.c_double),
                                  _ptr(out, C.c_double)))
    return out


def pf_eval_jacobian(c: CaseHandle, vmag, vang, nnz: int):
    vm = np.ascontiguousarray(vmag, dtype=np.float64).reshape(-1)
    va = np.ascontiguousarray(vang, dtype=np.float64).reshape(-1)
    bs = _bs(c)
    out = np.zeros((nnz, bs, bs))
    _check(lib().pf_eval_jacobian(c.handle, _ptr(vm, C.c_double), _ptr(va, C.c_double),
                                  _ptr(out, C.c_double)))
    return out


def pf_newton_step(c: CaseHandle, vmag, vang, opts: pf_opts | None = None):
    vm = np.ascontiguousarray(vmag, dtype=np.float64).reshape(-1)
    va = np.ascontiguousarray(vang, dtype=np.float64).reshape(-1)
    out = np.zeros((c.n, _bs(c)))
    info = pf_info()
    _check(lib().pf_newton_step(c.handle, C.byref(opts) if opts else None, _ptr(vm, C.c_double),
                                _ptr(va, C.c_double), _ptr(out, C.c_double), C.byref(info)))
    return out, info.as_dict()


PROFILE_PHASES = ("setup", "mismatch_jacobian", "stop_test", "factor", "triangular_solves",
                  "rhs_refinement", "update", "output")


def pf_profile_solve(c: CaseHandle, opts: pf_opts | None = None, B: int = 1):
    """(phase microseconds dict, info records) of one timed solve of B copies
    of the case's own scenario (info: dict for B = 1, structured array else)."""
    ph = np.zeros(len(PROFILE_PHASES))
    info = np.zeros(B, INFO_DTYPE)
    _check(lib().pf_profile_solve(c.handle, B, C.byref(opts) if opts else None,
                                  _ptr(ph, C.c_double), info.ctypes.data_as(C.c_void_p)))
    prof = dict(zip(PROFILE_PHASES, ph.tolist()))
    if B == 1:
        return prof, {k: (info[k][0].item()) for k in info.dtype.names}
    return prof, info


def pf_launch_config(c: CaseHandle, opts: pf_opts | None = None, B: int = 1) -> dict:
    """Launch shape of a solve: grid, cluster, threads, scenarios per cluster."""
    v = [C.c_int32() for _ in range(4)]
    _check(lib().pf_launch_config(c.handle, C.byref(opts) if opts else None, B,
                                  *[C.byref(x) for x in v]))
    return dict(zip(("grid", "cluster", "threads", "scen_per_cluster"), [x.value for x in v]))


def pf_solve_noalloc(c: CaseHandle, opts, d_p_load, d_q_load, d_p_gen, d_vmag, d_vang, d_info,
                     stream=0):
    """Single Newton-Raphson solve whose workspace is the library's fixed
    device array (no allocation); device pointers, asynchronous on stream."""
    _check(lib().pf_solve_noalloc(
        c.handle, C.byref(opts) if opts else None, _devptr(d_p_load), _devptr(d_q_load),
        _devptr(d_p_gen), _devptr(d_vmag), _devptr(d_vang), _devptr(d_info),
        C.c_void_p(stream)))


def pf_autotune(c: CaseHandle, B: int, opts: pf_opts | None = None) -> pf_opts:
    """Time candidate batch launch shapes; the case keeps the fastest for B."""
    o = opts if opts is not None else make_opts()
    _check(lib().pf_autotune(c.handle, B, C.byref(o)))
    return o
