"""GB300-native colloidal two-component Shan-Chen lattice Boltzmann (LBsoft method).

The compute path is the C-ABI library ``liblbgb.so`` (hand-written sm_103a CUDA);
``paper_2004_04080_gb300.lbgb`` is its thin ctypes binding.
"""
__all__ = ["lbgb", "workloads"]
