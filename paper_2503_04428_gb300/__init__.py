"""GB300 (sm_103a) Godunov cell update of HERACLES++ (arXiv:2503.04428).

``libhydro.so`` (built from ``csrc/`` by :mod:`.build`) holds the CUDA kernels
behind the C ABI of ``include/hydro.h``; :mod:`.hydro` is its ctypes binding
and :mod:`.workloads` the seeded synthetic inputs.
"""
