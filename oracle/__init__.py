"""FP64 CPU oracle (test infrastructure only; see qbe_oracle module docstring)."""
