"""ctypes binding of the C ABI declared in ``include/lbm.h``.

Argument marshalling only: every function here forwards to the function of
the same name in ``liblbm_gb300.so`` and turns a negative status into
:class:`LbmError`.  There is no fallback: if the library is missing or does
not load, :func:`load` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_EOVERFLOW, LBM_ECUDA = 0, -1, -2, -3
LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ENOMEM, LBM_EFLAGS = -4, -5, -6, -7
LBM_ORDER_LEX, LBM_ORDER_BLOCKED, LBM_ORDER_MORTON1, LBM_ORDER_MORTON2 = 0, 1, 2, 3
LBM_ORDER_HILBERT = 4
LBM_F64, LBM_F32, LBM_F32S, LBM_F16S, LBM_BF16S, LBM_F64X = 0, 1, 2, 3, 4, 5

# Every exported entry point with (restype, argtypes); the symbol test checks
# this list against the declarations in include/lbm.h.
_vp, _i32, _i64, _u32, _d = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                             ctypes.c_double)


# Allocator callbacks of lbm_set_allocator: alloc(bytes, stream, ctx) -> ptr,
# release(ptr, stream, ctx).
LBM_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
LBM_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class lbm_ordering(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("block", ctypes.c_int32 * 3),
                ("periodic", ctypes.c_uint32)]


SIGNATURES = {
    "lbm_ordering_keys": (ctypes.c_int, [_vp, lbm_ordering, _vp, _vp]),
    "lbm_build_sparse": (ctypes.c_int, [_vp, _vp, lbm_ordering, _vp, _vp]),
    "lbm_sparse_info": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lbm_state_create": (ctypes.c_int, [_vp, _i32, _i32, _vp]),
    "lbm_state_set_pdfs": (ctypes.c_int, [_vp, _vp]),
    "lbm_state_get_pdfs": (ctypes.c_int, [_vp, _vp]),
    "lbm_state_get_raw": (ctypes.c_int, [_vp, _vp]),
    "lbm_state_set_raw": (ctypes.c_int, [_vp, _vp]),
    "lbm_state_reset": (ctypes.c_int, [_vp]),
    "lbm_set_damping": (ctypes.c_int, [_vp, _vp]),
    "lbm_step": (ctypes.c_int, [_vp, _i32, _d, _d, _vp]),
    "lbm_step_timed": (ctypes.c_int, [_vp, _i32, _d, _d, _vp, _vp]),
    "lbm_reduce_flux": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
    "lbm_moments": (ctypes.c_int, [_vp, _vp, _vp]),
    "lbm_state_steps": (ctypes.c_int, [_vp, _vp]),
    "lbm_synchronize": (ctypes.c_int, [_vp, _d]),
    "lbm_set_timeout": (None, [_d]),
    "lbm_step_f64_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _i64, _d, _d, _vp, _vp, _vp, _vp]),
    "lbm_state_create_batched": (ctypes.c_int, [_vp, _i32, _i32, _i32, _vp]),
    "lbm_batch_layout": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lbm_batch_config": (ctypes.c_int, [_vp, _i32, _i32, _i32]),
    "lbm_batch_groups": (ctypes.c_int, [_vp, _i64, _vp]),
    "lbm_batch_resident": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
    "lbm_set_allocator": (ctypes.c_int, [LBM_ALLOC_FN, LBM_FREE_FN, _vp]),
    "lbm_batch_tune": (ctypes.c_int, [_vp, _i32, _d, _d, _vp, _vp, _vp, _vp]),
    "lbm_halo_gather": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i32, _vp]),
    "lbm_adjoint_create": (ctypes.c_int, [_vp, _i32, _i32, _vp]),
    "lbm_adjoint_forward": (ctypes.c_int, [_vp, _d, _d, _vp, _i32, _vp]),
    "lbm_adjoint_backward": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_adjoint_step": (ctypes.c_int, [_vp, _vp, _i32, _d, _d, _vp, _i32, _vp, _vp, _vp]),
    "lbm_free": (None, [_vp]),
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_abi_version": (ctypes.c_int32, []),
}

_lock = threading.Lock()
_lib = None


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"lbm status {status}: {message}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load ``liblbm_gb300.so``; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing: build it first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int) -> None:
    if status != LBM_OK:
        raise LbmError(status, load().lbm_last_error().decode(errors="replace"))


def _dims(dims):
    return (ctypes.c_int32 * 3)(*[int(d) for d in dims])


def make_ordering(kind: int, block=(1, 1, 1), periodic: int = 0) -> lbm_ordering:
    return lbm_ordering(int(kind), (ctypes.c_int32 * 3)(*[int(b) for b in block]),
                        int(periodic))


def lbm_ordering_keys(dims, ordering: lbm_ordering, keys_dev: int, stream: int) -> None:
    _check(load().lbm_ordering_keys(_dims(dims), ordering, keys_dev, stream))


def lbm_build_sparse(flags: int, dims, ordering: lbm_ordering, stream: int) -> int:
    out = ctypes.c_void_p()
    _check(load().lbm_build_sparse(flags, _dims(dims), ordering, stream, ctypes.byref(out)))
    return out.value


def lbm_sparse_info(sparse: int, want_adj: bool = True):
    """(n_fluid, cells_dev, adj_dev, inv_dev) as Python ints; adj_dev is 0
    unless want_adj (asking for it may build the public links)."""
    n = ctypes.c_int64()
    cells, adj, inv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().lbm_sparse_info(sparse, ctypes.byref(n), ctypes.byref(cells),
                                  ctypes.byref(adj) if want_adj else None, ctypes.byref(inv)))
    return n.value, cells.value or 0, adj.value or 0, inv.value or 0


def lbm_state_create(sparse: int, precision: int, scale_exp: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(load().lbm_state_create(sparse, int(precision), int(scale_exp), ctypes.byref(out)))
    return out.value


def lbm_state_set_pdfs(state: int, f_dev: int) -> None:
    _check(load().lbm_state_set_pdfs(state, f_dev))


def lbm_state_get_pdfs(state: int, f_dev: int) -> None:
    _check(load().lbm_state_get_pdfs(state, f_dev))


def lbm_state_get_raw(state: int, raw: int) -> None:
    _check(load().lbm_state_get_raw(state, raw))


def lbm_state_set_raw(state: int, raw: int) -> None:
    _check(load().lbm_state_set_raw(state, raw))


def lbm_state_reset(state: int) -> None:
    _check(load().lbm_state_reset(state))


def lbm_set_damping(state: int, alpha_dev) -> None:
    _check(load().lbm_set_damping(state, alpha_dev))


def lbm_step(state: int, n_steps: int, omega_plus: float, omega_minus: float, force) -> None:
    f = (ctypes.c_double * 3)(*[float(v) for v in force])
    _check(load().lbm_step(state, int(n_steps), float(omega_plus), float(omega_minus), f))


def lbm_step_timed(state: int, n_steps: int, omega_plus: float, omega_minus: float,
                   force) -> float:
    """lbm_step, returning the device time of the steps in milliseconds."""
    f = (ctypes.c_double * 3)(*[float(v) for v in force])
    ms = ctypes.c_double(0.0)
    _check(load().lbm_step_timed(state, int(n_steps), float(omega_plus), float(omega_minus), f,
                                 ctypes.byref(ms)))
    return ms.value


def lbm_reduce_flux(state: int, axis: int):
    """(mass, flux) of the most recent step."""
    m, q = ctypes.c_double(), ctypes.c_double()
    _check(load().lbm_reduce_flux(state, int(axis), ctypes.byref(m), ctypes.byref(q)))
    return m.value, q.value


def lbm_moments(state: int, rho_dev: int, u_dev: int) -> None:
    _check(load().lbm_moments(state, rho_dev, u_dev))


def lbm_state_steps(state: int) -> int:
    s = ctypes.c_int64()
    _check(load().lbm_state_steps(state, ctypes.byref(s)))
    return s.value


def lbm_synchronize(state: int, timeout_s: float = 0.0) -> None:
    _check(load().lbm_synchronize(state, float(timeout_s)))


def lbm_set_timeout(timeout_s: float) -> None:
    load().lbm_set_timeout(float(timeout_s))


def lbm_state_create_batched(sparses, precision: int, scale_exp: int = 0) -> int:
    arr = (ctypes.c_void_p * len(sparses))(*sparses)
    out = ctypes.c_void_p()
    _check(load().lbm_state_create_batched(arr, len(sparses), int(precision), int(scale_exp),
                                           ctypes.byref(out)))
    return out.value


def lbm_batch_layout(state: int):
    """(begin [n_beds], count [n_beds], n_padded) as Python lists/int."""
    nb = ctypes.c_int32()
    _check(load().lbm_batch_layout(state, ctypes.byref(nb), None, None, None))
    begin = (ctypes.c_int64 * nb.value)()
    count = (ctypes.c_int64 * nb.value)()
    npad = ctypes.c_int64()
    _check(load().lbm_batch_layout(state, None, begin, count, ctypes.byref(npad)))
    return list(begin), list(count), npad.value


def lbm_batch_config(state: int, block: int, cells_per_thread: int, use_graph: bool) -> None:
    _check(load().lbm_batch_config(state, int(block), int(cells_per_thread), int(bool(use_graph))))


_allocator = None   # the callbacks in use, kept alive while the library holds them


def lbm_set_allocator(alloc, release) -> None:
    """Route the library's device memory through alloc(nbytes, stream) -> ptr
    and release(ptr, stream) (Python callables; stream is a cudaStream_t as
    int or None), or back to cudaMalloc with (None, None)."""
    global _allocator
    if alloc is None and release is None:
        _check(load().lbm_set_allocator(LBM_ALLOC_FN(), LBM_FREE_FN(), None))
        _allocator = None
        return

    def _alloc(nbytes, stream, ctx):
        try:
            return alloc(int(nbytes), stream)
        except Exception:   # becomes LBM_ENOMEM in the calling function
            return None

    def _release(ptr, stream, ctx):
        release(ptr, stream)

    cbs = (LBM_ALLOC_FN(_alloc), LBM_FREE_FN(_release))
    _check(load().lbm_set_allocator(cbs[0], cbs[1], None))
    _allocator = cbs


def lbm_batch_groups(state: int, nbytes: int) -> int:
    """Set the L2 group budget in bytes (0: one group; < 0: the default);
    returns the number of groups."""
    g = ctypes.c_int32(0)
    _check(load().lbm_batch_groups(state, int(nbytes), ctypes.byref(g)))
    return g.value


def lbm_batch_resident(state: int, mode: int):
    """Resident steps on (1) or off (0), or the barrier time-limit check
    (-1); returns (number of groups, resident capacity in cells)."""
    g, c = ctypes.c_int32(0), ctypes.c_int64(0)
    _check(load().lbm_batch_resident(state, int(mode), ctypes.byref(g), ctypes.byref(c)))
    return g.value, c.value


def _forces(forces):
    flat = [float(v) for row in forces for v in row]
    return (ctypes.c_double * len(flat))(*flat)


def lbm_step_batched(state: int, n_steps: int, omega_plus: float, omega_minus: float,
                     forces) -> None:
    """lbm_step on a batched state; forces is a sequence of (Fx, Fy, Fz)."""
    _check(load().lbm_step(state, int(n_steps), float(omega_plus), float(omega_minus),
                           _forces(forces)))


def lbm_reduce_flux_batched(state: int, axis: int, n_beds: int):
    m = (ctypes.c_double * n_beds)()
    q = (ctypes.c_double * n_beds)()
    _check(load().lbm_reduce_flux(state, int(axis), m, q))
    return list(m), list(q)


def lbm_batch_tune(state: int, steps_per_candidate: int, omega_plus: float, omega_minus: float,
                   forces):
    """(block, cells_per_thread, [9 candidate times in ms])."""
    b, c = ctypes.c_int32(), ctypes.c_int32()
    ms = (ctypes.c_float * 9)()
    _check(load().lbm_batch_tune(state, int(steps_per_candidate), float(omega_plus),
                                 float(omega_minus), _forces(forces), ctypes.byref(b),
                                 ctypes.byref(c), ms))
    return b.value, c.value, list(ms)


def lbm_halo_gather(src_dev: int, slots_dev: int, count: int, dst_dev: int, elem_bytes: int,
                    stream: int) -> None:
    _check(load().lbm_halo_gather(src_dev, slots_dev, int(count), dst_dev, int(elem_bytes),
                                  stream))


def lbm_adjoint_create(state: int, n_steps: int, stride: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(load().lbm_adjoint_create(state, int(n_steps), int(stride), ctypes.byref(out)))
    return out.value


def lbm_adjoint_forward(adjoint: int, omega_plus: float, omega_minus: float, force,
                        axis: int) -> float:
    f = (ctypes.c_double * 3)(*[float(v) for v in force])
    J = ctypes.c_double()
    _check(load().lbm_adjoint_forward(adjoint, float(omega_plus), float(omega_minus), f,
                                      int(axis), ctypes.byref(J)))
    return J.value


def lbm_adjoint_backward(adjoint: int, dJdalpha_dev=None, dJdf0_dev=None):
    """dJ/dF as a tuple; fills the optional device outputs."""
    dF = (ctypes.c_double * 3)()
    _check(load().lbm_adjoint_backward(adjoint, dF, dJdalpha_dev, dJdf0_dev))
    return tuple(dF)


def lbm_adjoint_step(state: int, adjoint: int, n_steps: int, omega_plus: float,
                     omega_minus: float, force, axis: int, dJdalpha_dev=None):
    """(J, dJ/dF) of one forward + reverse pass."""
    f = (ctypes.c_double * 3)(*[float(v) for v in force])
    J = ctypes.c_double()
    dF = (ctypes.c_double * 3)()
    _check(load().lbm_adjoint_step(state, adjoint, int(n_steps), float(omega_plus),
                                   float(omega_minus), f, int(axis), ctypes.byref(J), dF,
                                   dJdalpha_dev))
    return J.value, tuple(dF)


def lbm_free(handle) -> None:
    if handle:
        load().lbm_free(handle)


def lbm_last_error() -> str:
    return load().lbm_last_error().decode(errors="replace")


def lbm_abi_version() -> int:
    return int(load().lbm_abi_version())


def lbm_step_f64_noalloc(f_src_dev: int, f_dst_dev: int, adj_dev: int, n_fluid: int,
                         omega_plus: float, omega_minus: float, force, alpha_dev,
                         sums_dev: int, stream: int) -> None:
    """One FP64 step on caller-owned arrays with no device allocation (for
    callers that cannot allocate); see include/lbm.h."""
    f = (ctypes.c_double * 3)(*[float(v) for v in force])
    _check(load().lbm_step_f64_noalloc(f_src_dev, f_dst_dev, adj_dev, int(n_fluid),
                                       float(omega_plus), float(omega_minus), f, alpha_dev,
                                       sums_dev, stream))
