"""GB300-native FFT-accelerated boundary element operator (Benad, arXiv:1809.00845)."""
