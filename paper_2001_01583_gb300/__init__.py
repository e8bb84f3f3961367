"""GB300-native NFFT: the gridding NFFT of the HP-NFFT paper on one GPU.

    from paper_2001_01583_gb300 import Plan
    plan = Plan(N=(64, 64, 64), M=10**6, sigma=2.0, m=4, window="kaiser_bessel", precision="fp32")
    plan.set_points(x)            # (M, 3) float64 CUDA tensor
    fhat = plan.adjoint(f)        # Eq. 5
    g = plan.forward(fhat)        # Eq. 6

The CUDA library (libgbnfft.so) is loaded on first use; importing this
package alone (for example for the input generators) needs no GPU.
"""

__all__ = ["Plan", "Batch", "plan_params", "ewald_real_space", "ewald_real_space_forces"]


def __getattr__(name):
    if name in ("Plan", "Batch", "plan_params", "ewald_real_space", "ewald_real_space_forces"):
        from . import nfft
        return getattr(nfft, name)
    raise AttributeError(name)
