"""Oracle: plain FP64 CPU statement of the coupled LKS / rigid-body step and its exact adjoint.

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may use it. The CUDA library never imports it and shares no code with it.
"""
