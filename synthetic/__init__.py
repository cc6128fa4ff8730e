"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds only input generation -- random targets and starting fields -- and none
of the descriptor, loss, gradient or optimiser arithmetic.  It stands in for the paper's
pyMKS-generated media and the micrographs of Li et al. (Sec. 4.2), which are not
available here: thresholded periodic Gaussian random fields (GRF), optionally with discs,
and checkerboards (Sec. 4.1).

Recipes
-------
* GRF: i.i.d. N(0, 1) white noise (numpy PCG64, seeded), periodically convolved with the
  Gaussian kernel exp(-sum_a x_a^2 / (2 l_a^2)), l_a the correlation length per axis.
* Exact-count threshold: the round(vf * N) largest values become phase 1; ties go to the
  lower linear index (stable sort).
* Discs: radius uniform integer in [rmin, rmax], centre uniform; a disc is rejected if it
  overlaps a placed one (periodic distance); placement stops when the discs cover
  ``cover`` of the domain or after ``max_reject`` rejections.  Disc pixels are set to 1.
* Starting field: uniform[0, 1) from the SplitMix64 generator (Steele, Lea & Flood,
  OOPSLA 2014), counter based: value_i = top 24 bits of splitmix64(seed, i) * 2^-24, so the
  same seed gives the same field on every device and in every language.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """SplitMix64 output for state seed + (index + 1) * golden-gamma, vectorised (uint64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + (np.asarray(index, dtype=np.uint64) + np.uint64(1)) * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_field(shape, seed: int) -> np.ndarray:
    """Counter-based uniform[0,1) field (float32-exact values k * 2^-24)."""
    n = int(np.prod(shape))
    z = splitmix64(seed, np.arange(n, dtype=np.uint64))
    return ((z >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).reshape(shape)


def gaussian_random_field(shape, corr_len, seed: int) -> np.ndarray:
    shape = tuple(int(s) for s in shape)
    if np.isscalar(corr_len):
        corr_len = (float(corr_len),) * len(shape)
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    kern = np.ones(shape)
    for ax, (n, l) in enumerate(zip(shape, corr_len)):
        x = np.arange(n)
        x = np.minimum(x, n - x).astype(np.float64)
        k1 = np.exp(-x * x / (2.0 * l * l))
        sh = [1] * len(shape)
        sh[ax] = n
        kern = kern * k1.reshape(sh)
    return np.real(np.fft.ifftn(np.fft.fftn(noise) * np.fft.fftn(kern)))


def threshold_count(field: np.ndarray, vf: float) -> np.ndarray:
    flat = np.asarray(field).ravel()
    k = int(round(vf * flat.size))
    order = np.argsort(-flat, kind="stable")
    out = np.zeros(flat.size)
    out[order[:k]] = 1.0
    return out.reshape(np.shape(field))


def add_discs(img: np.ndarray, seed: int, rmin=6, rmax=20, cover=0.10, max_reject=10000) -> np.ndarray:
    img = np.array(img, dtype=np.float64)
    n0, n1 = img.shape
    rng = np.random.default_rng(seed)
    discs = []
    area = 0.0
    rejects = 0
    yy, xx = np.mgrid[0:n0, 0:n1]
    while area < cover * n0 * n1 and rejects < max_reject:
        r = int(rng.integers(rmin, rmax + 1))
        c0, c1 = float(rng.uniform(0, n0)), float(rng.uniform(0, n1))
        ok = True
        for (d0, d1, dr) in discs:
            e0 = abs(c0 - d0); e0 = min(e0, n0 - e0)
            e1 = abs(c1 - d1); e1 = min(e1, n1 - e1)
            if e0 * e0 + e1 * e1 < (r + dr) ** 2:
                ok = False
                break
        if not ok:
            rejects += 1
            continue
        discs.append((c0, c1, r))
        area += np.pi * r * r
        e0 = np.abs(yy - c0); e0 = np.minimum(e0, n0 - e0)
        e1 = np.abs(xx - c1); e1 = np.minimum(e1, n1 - e1)
        img[e0 * e0 + e1 * e1 <= r * r] = 1.0
    return img


def checkerboard(n: int, a: int, ndim: int = 2) -> np.ndarray:
    idx = np.indices((n,) * ndim)
    return (np.sum(idx // a, axis=0) % 2).astype(np.float64)


# ----------------------------------------------------------------------------- workloads

def target_2d_grf(n: int, corr_len: float, vf: float, seed: int) -> np.ndarray:
    return threshold_count(gaussian_random_field((n, n), corr_len, seed), vf)


def target_small_2d(seed: int = 1000) -> np.ndarray:
    """64x64 GRF (l = 4 px) thresholded to vf 0.30."""
    return target_2d_grf(64, 4.0, 0.30, seed)


def target_large_2d(seed: int = 2000) -> np.ndarray:
    """512x512 GRF (l = 12 px, vf 0.40) united with periodic non-overlapping discs r 6..20."""
    base = target_2d_grf(512, 12.0, 0.40, seed)
    return add_discs(base, seed + 1)


def target_3d(n: int = 128, seed: int = 3000, corr=(6.0, 6.0, 12.0), vf=0.25) -> np.ndarray:
    """n^3 GRF with anisotropic correlation lengths, thresholded to vf."""
    return threshold_count(gaussian_random_field((n, n, n), corr, seed), vf)


def batch_instances(count: int = 256, seed: int = 4000, sizes=(64, 128, 256, 512), pmin=16, pmax=64):
    """Mixed-size 2-D instances: size uniform over ``sizes``, vf ~ U[0.1, 0.5], window
    uniform in [pmin, pmax] capped at n/2.  Returns a list of (target, window, seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        vf = float(rng.uniform(0.1, 0.5))
        P = int(min(rng.integers(pmin, pmax + 1), n // 2))
        tgt = target_2d_grf(n, max(n / 32.0, 2.0), vf, seed + 1 + i)
        out.append((tgt, P, seed + 1 + i))
    return out


def multiphase_grf(shape, corr_len, fractions, seed: int) -> np.ndarray:
    """Phase indicator stack (n_phase, *shape) of a periodic GRF cut at exact quantiles:
    the highest fractions[0] of the values are phase 0, the next fractions[1] phase 1, ...,
    the rest the last phase (n_phase = len(fractions) + 1).  Every position lies in exactly
    one phase."""
    g = gaussian_random_field(shape, corr_len, seed).ravel()
    order = np.argsort(-g, kind="stable")
    labels = np.full(g.size, len(fractions), dtype=np.int64)
    start = 0
    for a, fr in enumerate(fractions):
        k = int(round(fr * g.size))
        labels[order[start:start + k]] = a
        start += k
    out = np.zeros((len(fractions) + 1, g.size))
    out[labels, np.arange(g.size)] = 1.0
    return out.reshape((len(fractions) + 1,) + tuple(int(s) for s in shape))
