"""Plain FP64 CPU oracle of Fourier-accelerated Landau gauge fixing (test infrastructure only)."""
