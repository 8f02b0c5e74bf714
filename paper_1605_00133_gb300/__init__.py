"""GB300-native compressed-sensing photoacoustic tomography operators (arXiv:1605.00133).

The forward operator A (k-space pseudospectral wave propagation to a planar detector), its exact
adjoint A^T and the sub-sampling operator C (random single points or scrambled Hadamard patterns)
are hand-written CUDA kernels for sm_103a in libpat.so, behind the C ABI of include/pat.h.
"""
from . import presets, synth  # noqa: F401

__all__ = ["presets", "synth", "PatOperator"]


def __getattr__(name):
    if name == "PatOperator":
        from .operators import PatOperator
        return PatOperator
    raise AttributeError(name)
