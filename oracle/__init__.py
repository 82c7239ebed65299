"""FP64 CPU oracle (test infrastructure only; see fpm_oracle)."""
