"""GB300-native constraint-penalization lattice Boltzmann method (arXiv 2511.01629).

The compute path is the C-ABI library ``liblbmpen.so`` built from ``csrc/``;
``lbm`` is its thin ctypes binding.  Import the binding lazily so that the
workload generator can be used without a GPU.
"""

__all__ = ["workloads", "lbm"]
