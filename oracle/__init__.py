"""FP64 CPU oracle of the acoustic FD propagator (test infrastructure only)."""
