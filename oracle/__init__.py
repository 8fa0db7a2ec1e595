"""FP64 CPU oracle of the LB + raspberry-coupling step (test infrastructure only)."""
