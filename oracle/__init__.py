"""FP64 CPU oracle of the fractional-ADE lattice Boltzmann scheme (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  It shares no code with the CUDA path.
"""
