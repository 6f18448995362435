"""FP64 CPU oracle for the freeform-lens trace (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline and
reference legs may import this package. The product path never does.
"""
