"""GB300 (sm_103a) tensor-network-states amplitudes of random quantum circuits
on arbitrary qubit graphs, after Guo, Zhao and Huang, arXiv:2011.02621.

The compute path is libtn.so (C ABI in include/tn.h, CUDA kernels in csrc/);
``paper_2011_02621_gb300.tn`` is its Python binding. Build with
``paper_2011_02621_gb300.build.build()``.
"""
