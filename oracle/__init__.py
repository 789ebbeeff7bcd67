"""FP64 CPU oracle for the 2D radix-2 DIT FFT (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The library never does.
"""
