"""CPU oracle for the M-RA hot path.  TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy implementation written from the paper (Katzfuss, "A
multi-resolution approximation for massive spatial datasets", JASA 2017).
Only the test suite, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import it; the CUDA library never does.
"""
