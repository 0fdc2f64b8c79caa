"""CPU oracle (test infrastructure only; see lo_oracle.py)."""
