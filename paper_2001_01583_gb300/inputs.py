"""Seeded synthetic inputs shaped like the HP-NFFT paper's workloads.

This module holds input generators only (numpy, no transform arithmetic).
The tests, the smoke check and the benchmark feed the same arrays to the CUDA
library and to the CPU oracle, so generator details never affect parity.

Recipes
-------
uniform_points     x_j iid uniform in [-1/2, 1/2)^d          (Section 1, Pi^d)
clustered_points   K cluster centres uniform in Pi^d; each point picks a centre
                   uniformly, adds N(0, std^2) per coordinate, wraps into Pi^d
complex_normal     real and imaginary parts iid N(0, 1)
fluorite           the CaF2 crystal of Section 5: L_c^3 cubic cells of edge l,
                   Ca2+ (charge +2) on the 4 fcc sites, F- (charge -1) on the 8
                   sites (1/4 or 3/4)^3 l; lengths in units of the Ca-F distance
                   r0 = sqrt(3) l / 4, so l = 4 / sqrt(3) and L = L_c l
batch_items        count transforms, N_t drawn from a set per item, M
                   log-uniform in [M_lo, M_hi]
"""
import math

import numpy as np


def _wrap(x):
    return x - np.floor(x + 0.5)


def uniform_points(M: int, d: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.random((M, d)) - 0.5


def clustered_points(M: int, d: int, n_clusters: int, std: float, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    centres = rng.random((n_clusters, d)) - 0.5
    which = rng.integers(0, n_clusters, size=M)
    x = centres[which] + std * rng.standard_normal((M, d))
    return _wrap(x)


def complex_normal(shape, seed: int = 0, dtype=np.complex128) -> np.ndarray:
    rng = np.random.default_rng(seed)
    shape = (shape,) if isinstance(shape, int) else tuple(shape)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return z.astype(dtype)


# fractional positions inside one fluorite cell (units of the cell edge l)
_CA_SITES = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
_F_SITES = np.array([[a, b, c] for a in (0.25, 0.75) for b in (0.25, 0.75) for c in (0.25, 0.75)])

# fractional positions inside one rock-salt (NaCl) cell: a textbook lattice
# used to check the Ewald code on a second crystal
_NA_SITES = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
_CL_SITES = _NA_SITES + np.array([0.5, 0.0, 0.0])


def _lattice(Lc, sites, charges, edge):
    cells = np.stack(np.meshgrid(*[np.arange(Lc)] * 3, indexing="ij"), -1).reshape(-1, 1, 3)
    frac = (cells + sites[None, :, :]).reshape(-1, 3)
    q = np.tile(charges, Lc ** 3)
    return frac * edge, q.astype(np.float64), Lc * edge


def fluorite(Lc: int):
    """Returns (r, q, L): positions (n_ions x 3, units of r0), charges, box length."""
    edge = 4.0 / math.sqrt(3.0)
    sites = np.concatenate([_CA_SITES, _F_SITES])
    charges = np.array([2.0] * 4 + [-1.0] * 8)
    return _lattice(Lc, sites, charges, edge)


def rock_salt(Lc: int):
    """NaCl lattice with nearest-neighbour distance 1: (r, q, L)."""
    edge = 2.0
    sites = np.concatenate([_NA_SITES, _CL_SITES])
    charges = np.array([1.0] * 4 + [-1.0] * 4)
    return _lattice(Lc, sites, charges, edge)


def box_points(r, L):
    """Map positions in a periodic box [0, L)^3 to NFFT points in [-1/2, 1/2)^3."""
    return _wrap(np.asarray(r, dtype=np.float64) / L - 0.5)


def batch_items(count: int, N_choices=(32, 64), M_lo: int = 1000, M_hi: int = 100000, d: int = 3, seed: int = 0):
    """Per item: dict(N=(N,)*d, M=int, seed=int)."""
    rng = np.random.default_rng(seed)
    Ns = rng.choice(np.asarray(N_choices), size=count)
    Ms = np.exp(rng.uniform(math.log(M_lo), math.log(M_hi), size=count)).astype(np.int64)
    return [dict(N=(int(Ns[i]),) * d, M=int(Ms[i]), seed=int(seed + 1 + i)) for i in range(count)]
