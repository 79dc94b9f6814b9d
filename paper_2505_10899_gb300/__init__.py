"""GB300 (sm_103a) library for the coupled, locally volume-conserving lattice
Boltzmann step of Xiong, Wang & Liu (arXiv 2505.10899).

The compute path is the CUDA library ``_lib/liblbm_gb300.so`` behind the C ABI
of ``include/lbm_api.h``; ``paper_2505_10899_gb300.lbm`` is its ctypes binding.
Import the binding explicitly (``from paper_2505_10899_gb300 import lbm``); it
raises ImportError when the library has not been built.
"""
