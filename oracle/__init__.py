"""FP64 CPU oracle of the hierarchical solver -- TEST INFRASTRUCTURE ONLY.

Plain statements of what arXiv 1611.03189 computes, used to check the CUDA
library.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
may import this package; the library never does.

  hsolver.py         block-sparse factorization (Algorithm 1, Sec. 3.2, Sec. 6),
                     solve (Algorithm 2), PCG / GMRES / stationary iteration.
  dense_emulator.py  brute-force dense extended-system emulator (eq. extended,
                     eq. eliminated) used to pin hsolver.py on tiny grids.
"""
