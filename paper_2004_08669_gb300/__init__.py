"""GB300-native CTMRG for the polyhedron vector-spin models of arXiv:2004.08669.

The compute path is the CUDA library ``libctm_gb300.so`` behind the C-ABI of
``include/ctm.h``; ``paper_2004_08669_gb300.ctm`` is its thin ctypes binding
(handles, the temperature scan, the correlation length, the autotuner).
``scan`` splits a temperature scan across ranks, ``thermo`` takes central
differences of the observables through one scan, ``autograd`` makes the
converged free energy a torch.autograd function of beta (its backward is the
library's implicit differentiation), ``workloads`` holds the spin tables and
synthetic inputs.  Importing the package does not load the
CUDA library; ``ctm`` loads it on first use and raises if it is missing.
"""
__all__ = ["workloads", "ctm", "scan", "thermo", "autograd"]
