"""Ghost exchange between ranks that each own one chunk of the fluid-cell
list (Sec. 2 and Fig. 1c: the 1-D list cut into equal chunks; every rank
receives the PDFs its remote links pull before each step).

One :class:`ChunkRunner` per process.  It holds the rank's local PDF arrays
(own cells in SoA rows, then the ghost run, as laid out by
:func:`~paper_1111_1129_gb300.partition.plan`) and its local adjacency on
the GPU.  Before every step it

1. packs, for each peer, the values that peer's ghosts mirror with
   ``lbm_halo_gather`` (one device gather per peer, slots from the plan),
2. moves them with ``torch.distributed`` point-to-point messages: device
   buffers directly with the NCCL backend, through pinned host buffers with
   gloo (which has no GPU transport),
3. writes what it receives into the ghost run, one contiguous slice per peer,

then steps its chunk with ``lbm_step_f64_noalloc`` on the local adjacency.
The per-cell arithmetic is that of an unsplit ``lbm_step`` on an FP64 state,
so the chunks' PDFs equal the unsplit run's bit for bit; the mass and flux
are one all-reduce of the ranks' four FP64 sums.

Every step of the computation runs in the library's kernels; this module
only plans buffers and calls the transport.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from . import capi
from .partition import RankPlan

_W = [1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12


class ChunkRunner:
    """A rank's chunk of a sparse list in FP64, stepped with ghost exchange.

    plan: this rank's :class:`RankPlan`; send: ``{peer: owner-local slots}``
    this rank sends (``plan()``'s ``send[rank]``).  ``group`` is the process
    group of the ranks that share the list (default: the world)."""

    def __init__(self, plan: RankPlan, send: dict, group=None, device=None):
        self.plan = plan
        self.group = group
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        backend = dist.get_backend(group)
        self.host_staged = backend != "nccl"
        n, size = plan.count, plan.local_size
        w = torch.tensor(_W, dtype=torch.float64, device=self.device)
        self.f = [torch.zeros(max(size, 1), dtype=torch.float64, device=self.device)
                  for _ in range(2)]
        if n > 0:
            self.f[0][:19 * n] = w.repeat_interleave(n)
        self.cur = 0
        self.adj = torch.from_numpy(np.ascontiguousarray(plan.adj, np.int32)).to(self.device)
        self.sums = torch.zeros(4, dtype=torch.float64, device=self.device)
        self.peers_out = sorted(int(j) for j in send)
        self.peers_in = sorted(int(j) for j in plan.recv_from)
        self.slots = {j: torch.from_numpy(np.ascontiguousarray(send[j], np.int64)).to(self.device)
                      for j in self.peers_out}
        self.sendbuf = {j: torch.empty(int(send[j].size), dtype=torch.float64, device=self.device)
                        for j in self.peers_out}
        if self.host_staged:
            self.send_host = {j: torch.empty(b.numel(), dtype=torch.float64).pin_memory()
                              for j, b in self.sendbuf.items()}
            self.recv_host = {j: torch.empty(plan.recv_from[j][1], dtype=torch.float64)
                              .pin_memory() for j in self.peers_in}
        self.steps = 0

    @property
    def n(self) -> int:
        return self.plan.count

    def set_pdfs(self, f_own: torch.Tensor) -> None:
        """Own PDFs [19, count] (FP64)."""
        f_own = f_own.to(device=self.device, dtype=torch.float64).contiguous()
        if f_own.shape != (19, self.n):
            raise ValueError(f"expected PDFs of shape (19, {self.n})")
        self.f[self.cur][:19 * self.n] = f_own.reshape(-1)

    def pdfs(self) -> torch.Tensor:
        """Own PDFs [19, count] after the last step (a view)."""
        return self.f[self.cur][:19 * self.n].view(19, self.n)

    def _rank(self, j: int) -> int:
        """Global rank of group member j."""
        return j if self.group is None else dist.get_global_rank(self.group, j)

    def exchange(self) -> None:
        """Fill the ghost run of the current PDFs from the owning ranks."""
        stream = torch.cuda.current_stream(self.device)
        src = self.f[self.cur]
        for j in self.peers_out:
            buf = self.sendbuf[j]
            capi.lbm_halo_gather(src.data_ptr(), self.slots[j].data_ptr(), buf.numel(),
                                 buf.data_ptr(), 8, int(stream.cuda_stream))
        base = 19 * self.n
        if self.host_staged:
            for j in self.peers_out:
                self.send_host[j].copy_(self.sendbuf[j], non_blocking=True)
            stream.synchronize()
            reqs = [dist.isend(self.send_host[j], dst=self._rank(j), group=self.group)
                    for j in self.peers_out]
            reqs += [dist.irecv(self.recv_host[j], src=self._rank(j), group=self.group)
                     for j in self.peers_in]
            for r in reqs:
                r.wait()
            for j in self.peers_in:
                off, length = self.plan.recv_from[j]
                src[base + off:base + off + length].copy_(self.recv_host[j], non_blocking=True)
        else:
            ops = [dist.P2POp(dist.isend, self.sendbuf[j], self._rank(j), self.group)
                   for j in self.peers_out]
            ops += [dist.P2POp(dist.irecv,
                               src[base + self.plan.recv_from[j][0]:
                                   base + self.plan.recv_from[j][0] + self.plan.recv_from[j][1]],
                               self._rank(j), self.group) for j in self.peers_in]
            if ops:
                for r in dist.batch_isend_irecv(ops):
                    r.wait()

    def step(self, n_steps: int, omega_plus: float, omega_minus: float, force,
             alpha: torch.Tensor | None = None) -> None:
        """n_steps steps, each after a ghost exchange; alpha: FP64 damping
        of the own cells [count] or None."""
        stream = int(torch.cuda.current_stream(self.device).cuda_stream)
        a_ptr = None if alpha is None else alpha.data_ptr()
        for _ in range(int(n_steps)):
            self.exchange()
            capi.lbm_step_f64_noalloc(self.f[self.cur].data_ptr(), self.f[self.cur ^ 1].data_ptr(),
                                      self.adj.data_ptr(), self.n, omega_plus, omega_minus, force,
                                      a_ptr, self.sums.data_ptr(), stream)
            self.cur ^= 1
            self.steps += 1

    def reduce_flux(self, axis: int, n_total: int):
        """(mass, mean axial velocity) of the last step over all ranks:
        one all-reduce of the ranks' (sum rho, sum u) in FP64."""
        if self.steps < 1:
            raise RuntimeError("no step taken yet")
        s = self.sums.clone()
        if self.host_staged:
            s = s.cpu()
        dist.all_reduce(s, group=self.group)
        s = s.cpu().tolist()
        return s[0], s[1 + int(axis)] / max(int(n_total), 1)
