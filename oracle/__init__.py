"""FP64 CPU oracle for the omega-FQ solve.  Test infrastructure only (see oracle.py)."""
