"""FP64 CPU oracle of the batched physics step (test infrastructure, see oracle.py)."""
