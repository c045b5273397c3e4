"""FP64 CPU oracle of the GRNND build.  Test infrastructure only (see oracle.py)."""
