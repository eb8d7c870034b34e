"""GB300-native sparse D3Q19 TRT lattice Boltzmann solver.

The hot path (sparse assembly, stream-collide sweep, reductions) runs in
hand-written sm_103a CUDA kernels behind the C ABI of ``include/lbm.h``
(``liblbm_gb300.so``, built by :mod:`paper_1111_1129_gb300.build`).  This
package holds the ctypes binding (:mod:`.capi`), the PyTorch-facing wrapper
(:mod:`.lbm`) and the seeded input generator (:mod:`.inputs`).  Importing it
loads nothing; the library is loaded on first use and its absence is an
error, never a fallback.
"""

__all__ = ["SparseLattice", "LBMState", "Adjoint", "LBMFlux", "BatchedState", "omega_minus", "ordering_keys",
           "deviation_bound", "shifted_scale_exp", "use_torch_allocator"]


def __getattr__(name):
    if name in __all__:
        from . import lbm
        return getattr(lbm, name)
    raise AttributeError(name)
