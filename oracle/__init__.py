"""FP64 CPU oracle of the MLMC dispersion path (test infrastructure only)."""
