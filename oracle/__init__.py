"""FP64 CPU oracle for the sLLG hysteresis-loop path.  Test infrastructure only (see oracle.py)."""
