"""CPU oracle for the quasi-periodic HBS solver.

TEST INFRASTRUCTURE ONLY: a plain, slow FP64 restatement of the discrete
problem (dense fill + LAPACK solve) used to check the CUDA library.  Only the
tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may
import it; the library never does, and it shares no code with the library.
"""
