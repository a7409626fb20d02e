"""FP64 CPU oracle (test infrastructure only; see oracle/mbh_oracle.c)."""
