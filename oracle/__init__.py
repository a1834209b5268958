"""CPU FP64 oracle for the AMG-Krylov solve (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The CUDA library never calls it and it never calls the library.
"""
