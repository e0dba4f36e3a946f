"""Plain FP64 CPU oracle for the PF-LB-FD step (test infrastructure only)."""
