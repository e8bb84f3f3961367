"""CPU oracle for the NFFT library: plain, slow, FP64 reference code.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package; only the tests, the smoke check and the
benchmark's CPU-baseline leg use it.  It shares no code with the CUDA path.

Contents
--------
ndft        direct NDFT, Eq. 5 (adjoint) and Eq. 6 (forward), plain C with
            POSIX threads, FP64 (the definitions written out).
nfft_steps  the gridding NFFT of Section 2 (spread -> FFT -> scale, and
            subdivide -> inverse FFT -> interpolate) step by step in numpy FP64,
            with the window functions and their Fourier coefficients.
ewald       direct Ewald sum (Eqs. 10-12) and the reciprocal-space energy.
mlp         FP64 forward/backward of the small parameter-picker network.
"""
