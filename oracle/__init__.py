"""CPU oracle (test infrastructure only; see arrabit_oracle)."""
