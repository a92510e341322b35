"""GB300-native (sm_103a) time step of the BGK/MRT lattice Boltzmann scheme for the
space-fractional advection-diffusion equation (Cartalade, Younsi & Neel, arXiv:1706.09161).

``paper_1706_09161_gb300.lbm`` is the ctypes binding of the C-ABI library
(``include/lbm_fade.h``); ``paper_1706_09161_gb300.workloads`` generates seeded
synthetic inputs.  Importing the package does not load the CUDA library.
"""
