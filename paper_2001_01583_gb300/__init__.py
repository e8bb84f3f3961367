"""GB300-native NFFT (the gridding NFFT of the HP-NFFT paper on one GPU)."""
