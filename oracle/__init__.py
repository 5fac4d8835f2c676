"""FP64 CPU oracle (test infrastructure only; see gf_oracle.py)."""
