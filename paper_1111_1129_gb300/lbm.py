"""PyTorch-facing wrapper of the C ABI: sparse lattices and solver states.

PyTorch supplies device memory for inputs and outputs and the CUDA stream;
every step of the path runs in the library's kernels.  Names follow the C
functions (``lbm_build_sparse`` -> :class:`SparseLattice`, ``lbm_step`` ->
:meth:`LBMState.step`, ...).
"""
from __future__ import annotations

import math

import torch

from . import capi

ORDERINGS = {"lex": capi.LBM_ORDER_LEX, "blocked": capi.LBM_ORDER_BLOCKED,
             "morton1": capi.LBM_ORDER_MORTON1, "morton2": capi.LBM_ORDER_MORTON2,
             "hilbert": capi.LBM_ORDER_HILBERT}
PRECISIONS = {"f64": capi.LBM_F64, "f32": capi.LBM_F32, "f32s": capi.LBM_F32S,
              "f16s": capi.LBM_F16S, "bf16s": capi.LBM_BF16S, "f64x": capi.LBM_F64X}
STORAGE_BYTES = {"f64": 8, "f32": 4, "f32s": 4, "f16s": 2, "bf16s": 2, "f64x": 8}


def omega_minus(omega_plus: float, magic: float = 3.0 / 16.0) -> float:
    """Odd relaxation rate from the even one and the TRT magic parameter
    Lambda = (1/w+ - 1/2)(1/w- - 1/2); Lambda = 3/16 puts bounce-back walls
    exactly half-way between nodes."""
    return 1.0 / (0.5 + magic / (1.0 / omega_plus - 0.5))


def deviation_bound(force: float, tube_radius: float, omega_plus: float) -> float:
    """Upper estimate of |f_q - w_q| for a body-force-driven flow in a tube.

    The fastest flow the force can drive through a tube of this radius is
    the empty tube's Hagen-Poiseuille centreline speed u = F R^2 / (4 nu);
    packing only slows it.  The largest equilibrium deviation is then about
    w_q 3 |c.u| <= u / 6 (axis and diagonal links alike); a factor 2 covers
    density and non-equilibrium parts."""
    nu = (1.0 / omega_plus - 0.5) / 3.0
    u = abs(force) * tube_radius * tube_radius / (4.0 * nu)
    return 2.0 * u / 6.0


def shifted_scale_exp(dev_bound: float, target_log2: int = 14) -> int:
    """Scale exponent k of the 16-bit shifted forms: the largest expected
    deviation times 2^k lands at 2^target_log2, below FP16's largest finite
    value (65504 ~ 2^16) with 4x headroom.  Because FP16 and BF16 are
    floating point, a k that is a few powers of two too small costs no
    precision; only overflow (k far too large) would."""
    if dev_bound <= 0:
        return 0
    return int(max(0, min(40, math.floor(target_log2 - math.log2(dev_bound)))))


def use_torch_allocator(enabled: bool = True) -> None:
    """Take the library's device memory from PyTorch's caching allocator
    (enabled), so that it shows in torch.cuda.memory_allocated() and is
    reused with PyTorch's own blocks, or from cudaMalloc (disabled).  Only
    while no library handle is alive."""
    if not enabled:
        capi.lbm_set_allocator(None, None)
        return

    def alloc(nbytes: int, stream) -> int:
        return torch.cuda.caching_allocator_alloc(max(nbytes, 1), torch.cuda.current_device(),
                                                  int(stream or 0))

    def release(ptr: int, stream) -> None:
        torch.cuda.caching_allocator_delete(ptr)

    capi.lbm_set_allocator(alloc, release)


class _DeviceView:
    """Borrowed device buffer exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def _borrow(ptr: int, shape, typestr: str, dtype) -> torch.Tensor:
    if ptr == 0 or math.prod(shape) == 0:
        return torch.empty(shape, dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceView(ptr, shape, typestr), device="cuda")


def _stream_handle(stream) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def ordering_keys(dims, ordering: str = "lex", block=(8, 8, 8), stream=None) -> torch.Tensor:
    """Numbering-scheme key of every box cell, shape [nz, ny, nx], uint64
    values stored in an int64 tensor."""
    nx, ny, nz = (int(d) for d in dims)
    keys = torch.empty((nz, ny, nx), dtype=torch.int64, device="cuda")
    capi.lbm_ordering_keys((nx, ny, nz), capi.make_ordering(ORDERINGS[ordering], block),
                           keys.data_ptr(), _stream_handle(stream))
    return keys


class SparseLattice:
    """Sparse representation of a voxelised domain (``lbm_build_sparse``).

    flags: uint8 tensor [nz, ny, nx] (0 fluid, 1 solid), on the GPU or the
    host (host flags are copied to the device first)."""

    def __init__(self, flags: torch.Tensor, ordering: str = "lex", block=(8, 8, 8),
                 periodic: int = 0, stream=None):
        if flags.dtype != torch.uint8 or flags.dim() != 3:
            raise ValueError("flags must be a uint8 tensor [nz, ny, nx]")
        self.stream = torch.cuda.current_stream() if stream is None else stream
        flags = flags.to("cuda", non_blocking=True).contiguous()
        nz, ny, nx = flags.shape
        self.dims = (nx, ny, nz)
        self.ordering = ordering
        self.block = tuple(block)
        self.periodic = int(periodic)
        self._handle = None
        self._handle = capi.lbm_build_sparse(
            flags.data_ptr(), self.dims,
            capi.make_ordering(ORDERINGS[ordering], block, periodic),
            int(self.stream.cuda_stream))
        # the public links are built on first request (adjacency())
        self.n, self._cells, _, self._inv = capi.lbm_sparse_info(self._handle, want_adj=False)
        self._adj = 0

    @property
    def handle(self) -> int:
        return self._handle

    def cells(self) -> torch.Tensor:
        """Copy of cells[N] (box index of each fluid cell, in order)."""
        return _borrow(self._cells, (self.n,), "<i4", torch.int32).clone()

    def adjacency(self) -> torch.Tensor:
        """Copy of adj[18, N] (slot q N + m)."""
        if not self._adj:
            self._adj = capi.lbm_sparse_info(self._handle)[2]
        return _borrow(self._adj, (18, self.n), "<i4", torch.int32).clone()

    def inverse(self) -> torch.Tensor:
        """Copy of inv[nz, ny, nx] (fluid index or -1)."""
        nx, ny, nz = self.dims
        return _borrow(self._inv, (nz, ny, nx), "<i4", torch.int32).clone()

    def gather(self, dense: torch.Tensor) -> torch.Tensor:
        """Box-layout field [..., nz, ny, nx] -> fluid order [..., N]."""
        idx = self.cells().long()
        return dense.reshape(dense.shape[:-3] + (-1,))[..., idx]

    def close(self):
        if self._handle:
            capi.lbm_free(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LBMState:
    """Solver state: PDFs in one of the storage forms (``lbm_state_create``)."""

    def __init__(self, lattice: SparseLattice, precision: str = "f64", scale_exp: int = 0):
        self.lattice = lattice
        self.precision = precision
        self.scale_exp = int(scale_exp)
        self._handle = None
        self._handle = capi.lbm_state_create(lattice.handle, PRECISIONS[precision],
                                             self.scale_exp)

    @property
    def handle(self) -> int:
        return self._handle

    @property
    def n(self) -> int:
        return self.lattice.n

    def step(self, n_steps: int, omega_plus: float, omega_minus: float, force) -> None:
        capi.lbm_step(self._handle, n_steps, omega_plus, omega_minus, force)

    def step_timed(self, n_steps: int, omega_plus: float, omega_minus: float, force) -> float:
        """``step``, returning the device time of the steps in milliseconds
        (CUDA events on the state's stream; synchronises)."""
        return capi.lbm_step_timed(self._handle, n_steps, omega_plus, omega_minus, force)

    def reduce_flux(self, axis: int):
        """(mass, mean axial velocity) of the most recent step, FP64."""
        return capi.lbm_reduce_flux(self._handle, axis)

    def moments(self):
        """(rho [N], u [3, N]) of the most recent step's collision, FP64."""
        rho = torch.empty(self.n, dtype=torch.float64, device="cuda")
        u = torch.empty((3, self.n), dtype=torch.float64, device="cuda")
        capi.lbm_moments(self._handle, rho.data_ptr(), u.data_ptr())
        return rho, u

    def get_pdfs(self) -> torch.Tensor:
        f = torch.empty((19, self.n), dtype=torch.float64, device="cuda")
        capi.lbm_state_get_pdfs(self._handle, f.data_ptr())
        return f

    def set_pdfs(self, f: torch.Tensor) -> None:
        f = f.to(device="cuda", dtype=torch.float64).contiguous()
        if f.shape != (19, self.n):
            raise ValueError(f"expected PDFs of shape (19, {self.n})")
        capi.lbm_state_set_pdfs(self._handle, f.data_ptr())
        self._keep = f

    def get_raw(self) -> torch.Tensor:
        """The current PDFs as stored ([19, N] words of the storage form,
        as an integer tensor of the storage width): exact for every form."""
        dtype = {8: torch.int64, 4: torch.int32, 2: torch.int16}[STORAGE_BYTES[self.precision]]
        raw = torch.empty((19, self.n), dtype=dtype, device="cuda")
        capi.lbm_state_get_raw(self._handle, raw.data_ptr())
        return raw

    def set_raw(self, raw: torch.Tensor) -> None:
        """Overwrite the current PDFs with words from :meth:`get_raw` of a
        state of the same form and scale."""
        width = STORAGE_BYTES[self.precision]
        raw = raw.to(device="cuda").contiguous()
        if raw.shape != (19, self.n) or raw.element_size() != width:
            raise ValueError(f"expected ({19}, {self.n}) words of {width} bytes")
        capi.lbm_state_set_raw(self._handle, raw.data_ptr())
        self._keep = raw

    def set_damping(self, alpha) -> None:
        if alpha is None:
            capi.lbm_set_damping(self._handle, None)
            return
        a = alpha.to(device="cuda", dtype=torch.float64).contiguous()
        if a.shape != (self.n,):
            raise ValueError(f"expected damping of shape ({self.n},)")
        capi.lbm_set_damping(self._handle, a.data_ptr())
        self._keep_alpha = a

    @property
    def steps(self) -> int:
        return capi.lbm_state_steps(self._handle)

    def reset(self) -> None:
        """Back to rest (f_q = w_q); clears the step count."""
        capi.lbm_state_reset(self._handle)

    def save(self, path: str, **meta) -> None:
        """Checkpoint: the PDFs as stored (exact) and decoded to FP64, with
        the lattice's identity, to ``path`` (.npz).  Extra keyword values
        are stored alongside."""
        import numpy as np
        lat = self.lattice
        np.savez(path, raw=self.get_raw().cpu().numpy(), pdfs=self.get_pdfs().cpu().numpy(),
                 dims=np.array(lat.dims),
                 ordering=np.array(lat.ordering), block=np.array(lat.block),
                 periodic=np.array(lat.periodic), n=np.array(lat.n),
                 cells=lat.cells().cpu().numpy(), precision=np.array(self.precision),
                 scale_exp=np.array(self.scale_exp), steps=np.array(self.steps),
                 **{k: np.asarray(v) for k, v in meta.items()})

    def load(self, path: str) -> dict:
        """Restore PDFs written by :meth:`save` into this state; the lattice
        must be the same list (same cells in the same order).  A checkpoint
        of the same storage form and scale is restored word for word (a run
        resumed from it continues bit for bit); another form is converted
        from the FP64 PDFs.  Returns the stored metadata."""
        import numpy as np
        with np.load(path) as z:
            data = {k: z[k] for k in z.files}
        if int(data["n"]) != self.n or not np.array_equal(data["cells"],
                                                          self.lattice.cells().cpu().numpy()):
            raise ValueError("checkpoint was written for a different cell list")
        same_scale = (self.precision not in ("f16s", "bf16s")
                      or int(data["scale_exp"]) == self.scale_exp)
        if "raw" in data and str(data["precision"]) == self.precision and same_scale:
            self.set_raw(torch.from_numpy(data["raw"]))
        else:
            self.set_pdfs(torch.from_numpy(data["pdfs"]))
        return data

    def synchronize(self, timeout_s: float = 0.0) -> None:
        capi.lbm_synchronize(self._handle, timeout_s)

    def close(self):
        if self._handle:
            capi.lbm_free(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Adjoint:
    """Checkpointed reverse pass for K steps of a state (``lbm_adjoint_*``)."""

    def __init__(self, state: LBMState, n_steps: int, stride: int = 0):
        self.state = state
        self.n_steps = int(n_steps)
        self._handle = None
        self._handle = capi.lbm_adjoint_create(state.handle, self.n_steps, int(stride))

    @property
    def handle(self) -> int:
        return self._handle

    def forward(self, omega_plus: float, omega_minus: float, force, axis: int) -> float:
        """J = mean u_axis of the collision of step K, from the state's
        current PDFs (the state is not advanced)."""
        return capi.lbm_adjoint_forward(self._handle, omega_plus, omega_minus, force, axis)

    def backward(self, want_alpha: bool = True, want_f0: bool = False):
        """(dJ/dF [3] tuple, dJ/dalpha [N] or None, dJ/df0 [19, N] or None)."""
        n = self.state.n
        da = torch.empty(n, dtype=torch.float64, device="cuda") if want_alpha else None
        df0 = torch.empty((19, n), dtype=torch.float64, device="cuda") if want_f0 else None
        dF = capi.lbm_adjoint_backward(self._handle, None if da is None else da.data_ptr(),
                                       None if df0 is None else df0.data_ptr())
        return dF, da, df0

    def close(self):
        if self._handle:
            capi.lbm_free(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LBMFlux(torch.autograd.Function):
    """Differentiable mean axial velocity after K steps.

    ``LBMFlux.apply(force, alpha, adjoint, omega_plus, omega_minus, axis)``
    with force a float64 tensor [3] and alpha a float64 tensor [N] (fluid
    order) or None returns J as a 0-d float64 tensor; backward runs the
    checkpointed adjoint and returns dJ/dF and dJ/dalpha."""

    @staticmethod
    def forward(ctx, force, alpha, adjoint: Adjoint, omega_plus, omega_minus, axis):
        st = adjoint.state
        if alpha is not None:
            st.set_damping(alpha.detach())
        J = adjoint.forward(omega_plus, omega_minus, force.detach().cpu().tolist(), axis)
        ctx.adjoint = adjoint
        ctx.has_alpha = alpha is not None
        ctx.force_device = force.device
        return torch.tensor(J, dtype=torch.float64, device=force.device)

    @staticmethod
    def backward(ctx, gJ):
        dF, da, _ = ctx.adjoint.backward(want_alpha=ctx.has_alpha)
        grad_force = gJ * torch.tensor(dF, dtype=torch.float64, device=ctx.force_device)
        grad_alpha = gJ.to(da.device) * da if ctx.has_alpha else None
        return grad_force, grad_alpha, None, None, None, None


class BatchedState:
    """Many independent beds stepped together (``lbm_state_create_batched``).

    Each bed keeps its own force; per-bed results are bit-identical to
    stepping the bed alone."""

    def __init__(self, lattices, precision: str = "f32s", scale_exp: int = 0):
        self.lattices = list(lattices)
        self.precision = precision
        self._handle = None
        self._handle = capi.lbm_state_create_batched([l.handle for l in self.lattices],
                                                     PRECISIONS[precision], scale_exp)
        self.begin, self.count, self.n_padded = capi.lbm_batch_layout(self._handle)

    @property
    def handle(self) -> int:
        return self._handle

    @property
    def n_beds(self) -> int:
        return len(self.lattices)

    @property
    def n_fluid(self) -> int:
        return int(sum(self.count))

    def configure(self, block: int = 256, cells_per_thread: int = 1, use_graph: bool = True):
        capi.lbm_batch_config(self._handle, block, cells_per_thread, use_graph)

    def groups(self, nbytes: int = -1) -> int:
        """Step the beds in L2-sized groups of at most `nbytes` working set
        (0: all beds in every launch; < 0: the default, 0.6 of the L2);
        returns the number of groups.  Results do not depend on it."""
        return capi.lbm_batch_groups(self._handle, nbytes)

    def resident(self, mode: int = 1):
        """Resident steps: each group that fits takes all but its reducing
        step in one cooperative launch that keeps the links in shared
        memory (1), per-step launches (0), or the barrier time-limit check
        (-1).  Returns (number of groups, resident capacity in cells).
        Results do not depend on it."""
        return capi.lbm_batch_resident(self._handle, mode)

    def tune(self, steps_per_candidate: int, omega_plus: float, omega_minus: float, forces):
        """Pick the fastest launch shape (advances the state)."""
        return capi.lbm_batch_tune(self._handle, steps_per_candidate, omega_plus, omega_minus,
                                   forces)

    def step(self, n_steps: int, omega_plus: float, omega_minus: float, forces) -> None:
        capi.lbm_step_batched(self._handle, n_steps, omega_plus, omega_minus, forces)

    def reduce_flux(self, axis: int):
        """(mass [n_beds], flux [n_beds]) of the most recent step."""
        return capi.lbm_reduce_flux_batched(self._handle, axis, self.n_beds)

    def reset(self) -> None:
        """Back to rest, keeping the captured graph valid."""
        capi.lbm_state_reset(self._handle)

    def get_pdfs(self, bed: int = None) -> torch.Tensor:
        f = torch.empty((19, self.n_padded), dtype=torch.float64, device="cuda")
        capi.lbm_state_get_pdfs(self._handle, f.data_ptr())
        if bed is None:
            return f
        b, c = self.begin[bed], self.count[bed]
        return f[:, b:b + c]

    def close(self):
        if self._handle:
            capi.lbm_free(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
