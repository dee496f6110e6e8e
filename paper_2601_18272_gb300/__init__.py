"""GB300 (sm_103a) library for the coupled lattice-kinetic-scheme / rigid-body forward march and its
discrete adjoint, the hot path of "Topology optimization of passively moving rigid bodies in
unsteady flows" (arXiv 2601.18272).

The compute runs in ``lib/liblks_gb300.so`` (hand-written CUDA behind the C ABI of include/lks.h);
``lks`` is the ctypes binding and ``autograd`` wraps it as a torch.autograd.Function.
"""
from .lks import Solver, load  # noqa: F401
