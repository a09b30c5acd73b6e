"""CPU FP64 oracle (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import anything here.  The CUDA library never calls it and shares no code
with it.
"""
