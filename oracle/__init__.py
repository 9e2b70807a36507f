"""FP64 CPU oracle of the detection path (test infrastructure only; see oracle.py)."""
