"""FP64 CPU oracle (test infrastructure only; see acom_oracle.py)."""
