"""CPU oracle (test infrastructure only; see ppl_oracle.py)."""
