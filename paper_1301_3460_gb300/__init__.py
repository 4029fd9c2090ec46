"""GB300-native Fourier-accelerated steepest-descent Landau gauge fixing (arXiv:1301.3460)."""
