"""GB300-native Fast Haar wavelet transform (arXiv:1002.2184)."""
