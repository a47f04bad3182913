"""FP64 CPU oracle for the flip-free ADMM: test infrastructure, never used by the library."""
