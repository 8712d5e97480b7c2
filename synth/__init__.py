"""Seeded synthetic inputs for the directional SLSHT.

The one module that both the oracle tests and the CUDA path use.  It holds
none of the method's arithmetic: it only draws coefficient vectors, lists of
(l, m) pairs and grid sizes, and reads the two stored elliptical
concentration windows of workloads 2 and 5 (inputs of the transform,
Sec. III-D of the paper), which tests/golden/make_windows.py wrote with the
oracle's window generator.

Layouts: coefficient vectors are complex128 with flat index l*l + l + m and
EXCLUSIVE band limits (f_lm = 0 for l >= Lf).  Pair lists are int32 [n, 2]
holding (l, m).

Recipe of every workload (the paper's public Earth / Mars topography models
are not available here; these synthetic inputs stand in for them with the
same shapes: power-law, topography-like spectra and elliptical eigenfunction
windows, Sec. V):
  * ``signal_cn_real``   f_lm ~ CN(0,1) with the real-field symmetry
                         f_{l,-m} = (-1)^m conj(f_lm); f_l0 real N(0,1).
  * ``signal_powerlaw``  same symmetry, per-coefficient variance
                         C_l = (l+1)^-2 (topography-like).
  * ``window_cn``        h_pq ~ CN(0,1) / (p+1)^decay for every order (no
                         symmetry, azimuthally asymmetric), unit energy.
  * ``stored_window``    the most concentrated band-limited function in the
                         elliptical region R_(theta_c, a) at the north pole
                         (Eq. region_def), real-valued, unit energy, h00 > 0:
                         L_h = 8 in the 20 x 10 degree ellipse (workload 2),
                         L_h = 64 in the 8 x 3 degree ellipse (workload 5).
"""

import json
import os
from math import pi

import numpy as np

_GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")


def ellipse_from_axes(a_deg, b_deg):
    """(theta_c, a) in radians from the semi-major and semi-minor arcs of an
    ellipse centred on the pole: the foci lie on the major axis at colatitude
    theta_c, and cos(a) = cos(theta_c) cos(b) (spherical Pythagoras)."""
    a = np.deg2rad(a_deg)
    b = np.deg2rad(b_deg)
    return float(np.arccos(np.cos(a) / np.cos(b))), float(a)


def stored_window(workload):
    """(h, concentration) of the stored elliptical window of workload 2 or 5
    (complex128 [L_h*L_h], flat index p*p+p+q)."""
    d = json.load(open(os.path.join(_GOLDEN, "workload%d_window.json" % workload)))
    return np.array(d["re"]) + 1j * np.array(d["im"]), float(d["concentration"])


def _cn(rng, size):
    """Circular complex normal CN(0, 1): E|z|^2 = 1."""
    return (rng.standard_normal(size) + 1j * rng.standard_normal(size)) / np.sqrt(2.0)


def signal_real_symmetric(L, seed, variance=None):
    """Coefficients of a real-valued signal: f_{l,-m} = (-1)^m conj(f_lm).

    variance(l) gives E|f_lm|^2 (default 1)."""
    rng = np.random.default_rng(seed)
    f = np.zeros(L * L, dtype=np.complex128)
    for l in range(L):
        v = 1.0 if variance is None else float(variance(l))
        sd = np.sqrt(v)
        f[l * l + l] = rng.standard_normal() * sd
        z = _cn(rng, l) * sd
        for m in range(1, l + 1):
            f[l * l + l + m] = z[m - 1]
            f[l * l + l - m] = (-1) ** m * np.conj(z[m - 1])
    return f


def signal_cn_real(L, seed):
    return signal_real_symmetric(L, seed)


def signal_powerlaw(L, seed):
    return signal_real_symmetric(L, seed, variance=lambda l: (l + 1.0) ** -2)


def signal_uniform(L, seed):
    """Re, Im ~ U[0, 1] independently (the timing signals of Sec. V-A)."""
    rng = np.random.default_rng(seed)
    return rng.random(L * L) + 1j * rng.random(L * L)


def window_cn(L, seed, decay=0.0):
    """h_pq ~ CN(0,1)/(p+1)^decay for all |q| <= p < L, normalised to unit energy
    (<h, h> = 1, Definition 1)."""
    rng = np.random.default_rng(seed)
    h = _cn(rng, L * L)
    p = np.floor(np.sqrt(np.arange(L * L))).astype(np.float64)
    h = h / (p + 1.0) ** decay
    return h / np.linalg.norm(h)


def pairs_all(L):
    """All (l, m) with l < L."""
    return np.array([(l, m) for l in range(L) for m in range(-l, l + 1)], dtype=np.int32)


def pairs_bands(bands):
    """All orders of each listed degree."""
    return np.array([(l, m) for l in bands for m in range(-l, l + 1)], dtype=np.int32)


def pairs_random(L, n, seed):
    """n distinct (l, m) with l < L, drawn uniformly over the pairs."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(L * L, size=n, replace=False)
    l = np.floor(np.sqrt(idx)).astype(np.int64)
    m = idx - l * l - l
    return np.stack([l, m], axis=1).astype(np.int32)


def subsample_pairs(pairs, frac, seed):
    """A seeded subset (at least one) of a pair list, in the original order."""
    rng = np.random.default_rng(seed)
    n = max(1, int(round(frac * len(pairs))))
    idx = np.sort(rng.choice(len(pairs), size=n, replace=False))
    return pairs[idx]


# --------------------------------------------------------------------------
# the five workloads (band limits exclusive)
# --------------------------------------------------------------------------

CONFIGS = {
    # FP64, one map, all l < 16, CN(0,1) real-symmetric f, CN(0,1) window
    1: dict(name="fp64 L_f=16 L_h=4 all l<16, grid 31x16x7",
            Lf=16, Lh=4, grid=(31, 16, 7), maps=1),
    # FP64, one map, power-law f, 20x10 deg elliptical eigenfunction window
    2: dict(name="fp64 L_f=64 L_h=8 all l<64, ellipse 20x10 deg, grid 127x64x15",
            Lf=64, Lh=8, grid=(127, 64, 15), maps=1),
    # 4 maps, L_f=256, L_h=16, l in {16,64,128,255} all m, power-law f,
    # CN(0,1)/(l+1) asymmetric windows
    3: dict(name="4 maps L_f=256 L_h=16 l in {16,64,128,255} all m, grid 511x256x31",
            Lf=256, Lh=16, grid=(511, 256, 31), maps=4, bands=(16, 64, 128, 255)),
    # 16 pairs at L_f=2048, L_h=64, 8x3 deg ellipse window
    5: dict(name="L_f=2048 L_h=64 16 pairs, ellipse 8x3 deg, grid 4095x2048x127",
            Lf=2048, Lh=64, grid=(4095, 2048, 127), maps=1, npairs=16),
}


def config_inputs(cfg, map_index=0, window_cache=None):
    """(f, h, pairs) for map ``map_index`` of workload ``cfg`` (seed 1000*cfg + map)."""
    c = CONFIGS[cfg]
    seed = 1000 * cfg + map_index
    Lf, Lh = c["Lf"], c["Lh"]
    if cfg == 1:
        return signal_cn_real(Lf, seed), window_cn(Lh, seed + 500), pairs_all(Lf)
    if cfg == 2:
        h = window_cache if window_cache is not None else stored_window(2)[0]
        return signal_powerlaw(Lf, seed), h, pairs_all(Lf)
    if cfg == 3:
        return signal_powerlaw(Lf, seed), window_cn(Lh, seed + 500, decay=1.0), pairs_bands(c["bands"])
    if cfg == 5:
        h = window_cache if window_cache is not None else stored_window(5)[0]
        return signal_powerlaw(Lf, seed), h, pairs_random(Lf, c["npairs"], seed)
    raise KeyError(cfg)


def samples_per_pair(grid):
    Na, Nb, Ng = grid
    return Na * Nb * Ng


def grid_native(Lh):
    """The paper's tessellation E_{Lh-1} for a window of exclusive band limit Lh."""
    return (2 * Lh - 1, Lh, 2 * Lh - 1)


__all__ = [
    "signal_real_symmetric", "signal_cn_real", "signal_powerlaw", "signal_uniform",
    "window_cn", "stored_window", "ellipse_from_axes", "pairs_all", "pairs_bands",
    "pairs_random", "subsample_pairs", "CONFIGS", "config_inputs", "samples_per_pair",
    "grid_native", "pi",
]
