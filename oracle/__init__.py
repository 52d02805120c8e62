"""CPU oracle (test infrastructure only; see voila_oracle)."""
