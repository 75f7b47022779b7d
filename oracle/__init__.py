"""FP64 CPU oracle (test infrastructure only; see wf_oracle.py)."""
