"""FP64 CPU oracle (test infrastructure only; see tlda_oracle)."""
