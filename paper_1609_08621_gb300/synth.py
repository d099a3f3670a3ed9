"""Seeded synthetic particle sets for the FMM force solve.

This module only draws inputs: positions in the isolated unit box [0,1)^3 and
masses.  It contains none of the solver's arithmetic, so both the CUDA path and
the CPU oracle can be fed from it.  Every set is a pure function of its seed
(numpy's PCG64 stream, uniform draws only, so the stream is stable across numpy
versions).

The structures stand in for the paper's clustered cosmological particle
distributions (Sec. 4, late-time LCDM), which are not available here:

* ``clustered_plummer``: a uniform background plus Plummer spheres (the small
  and batched workloads);
* ``clustered_nfw``: a uniform background plus NFW halos whose masses follow a
  power law (the 128^3 workload);
* a few degenerate sets for edge cases (coincident points, a line, tiny N).

Softening follows the paper's rule of 1/50 of the mean inter-particle
separation (Sec. 3.1), available as :func:`paper_softening`.

Arrays: ``pos`` is float64 of shape (3, N) (structure of arrays x|y|z);
``mass`` is float32 of shape (N,), all equal and summing to 1.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "paper_softening",
    "uniform_box",
    "clustered_plummer",
    "clustered_nfw",
    "coincident",
    "batch_boxes",
    "make",
    "to_fixed",
    "WORKLOADS",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def paper_softening(n: int) -> float:
    """1/50 of the mean inter-particle separation of n particles in a unit box (Sec. 3.1)."""
    return 1.0 / (50.0 * float(n) ** (1.0 / 3.0))


def _equal_masses(n: int) -> np.ndarray:
    return np.full(n, 1.0 / max(n, 1), dtype=np.float32)


def _isotropic(rng: np.random.Generator, r: np.ndarray) -> np.ndarray:
    """Points at radius r with isotropic directions, shape (3, len(r))."""
    k = r.shape[0]
    cz = 2.0 * rng.random(k) - 1.0
    ph = 2.0 * np.pi * rng.random(k)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([r * sz * np.cos(ph), r * sz * np.sin(ph), r * cz])


def _inside(p: np.ndarray) -> np.ndarray:
    return np.all((p >= 0.0) & (p < 1.0), axis=0)


def _resample(rng, draw, n: int) -> np.ndarray:
    """Call draw(rng, k) -> (3, k) until n points inside the unit box are collected."""
    out = np.empty((3, n), dtype=np.float64)
    got = 0
    while got < n:
        k = n - got
        p = draw(rng, k)
        p = p[:, _inside(p)]
        take = min(k, p.shape[1])
        out[:, got:got + take] = p[:, :take]
        got += take
    return out


def uniform_box(n: int, seed: int):
    rng = _rng(seed)
    pos = rng.random((3, n))
    return pos, _equal_masses(n)


def _plummer_radius(rng, a: float, k: int) -> np.ndarray:
    # inverse of the Plummer cumulative mass M(<r)/M = r^3 / (r^2 + a^2)^{3/2}
    u = rng.random(k)
    u = np.clip(u, 1e-12, 1.0 - 1e-12)
    return a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)


def clustered_plummer(n: int, seed: int, n_spheres: int = 4, scale: float = 0.02,
                      uniform_frac: float = 0.5):
    """Uniform background plus ``n_spheres`` Plummer spheres of scale radius ``scale``.

    Sphere centres are uniform in [0.2, 0.8]^3; each sphere gets an equal share of the
    clustered particles (remainder to the first spheres).  Points that fall outside
    the unit box are redrawn.
    """
    rng = _rng(seed)
    n_uni = int(round(uniform_frac * n))
    n_cl = n - n_uni
    centres = 0.2 + 0.6 * rng.random((3, n_spheres))
    parts = [rng.random((3, n_uni))]
    base, rem = divmod(n_cl, n_spheres)
    for s in range(n_spheres):
        k = base + (1 if s < rem else 0)
        c = centres[:, s:s + 1]
        parts.append(_resample(rng, lambda g, kk: c + _isotropic(g, _plummer_radius(g, scale, kk)), k))
    pos = np.concatenate(parts, axis=1)
    # interleave so that the input order is not grouped by structure
    perm = rng.permutation(n)
    return np.ascontiguousarray(pos[:, perm]), _equal_masses(n)


def _nfw_mu(x):
    return np.log1p(x) - x / (1.0 + x)


def _nfw_radius(rng, c: float, rvir: float, k: int) -> np.ndarray:
    """Radii inside r_vir from the NFW enclosed mass M(<r)/M(<r_vir) = mu(r c / r_vir) / mu(c),
    mu(x) = ln(1 + x) - x / (1 + x), inverted by bisection (60 halvings of [0, c])."""
    target = rng.random(k) * _nfw_mu(c)
    a = np.zeros(k)
    b = np.full(k, c)
    for _ in range(60):
        mid = 0.5 * (a + b)
        below = _nfw_mu(mid) < target
        a = np.where(below, mid, a)
        b = np.where(below, b, mid)
    return 0.5 * (a + b) * (rvir / c)


def clustered_nfw(n: int, seed: int, n_halos: int = 200, uniform_frac: float = 0.3,
                  slope: float = 1.9, decades: float = 3.0, rvir_max: float = 0.05):
    """Uniform background plus NFW halos.

    Halo masses follow dN/dM ~ M^-slope over ``decades`` decades (inverse CDF);
    particle counts are proportional to halo mass (largest-remainder rounding);
    concentrations are uniform in [5, 15]; r_vir = rvir_max * (M/M_max)^(1/3);
    radii inside r_vir are drawn from the NFW enclosed-mass profile by bisection.
    """
    rng = _rng(seed)
    n_uni = int(round(uniform_frac * n))
    n_cl = n - n_uni
    lo, hi = 1.0, 10.0 ** decades
    e = 1.0 - slope
    u = rng.random(n_halos)
    m = (lo ** e + u * (hi ** e - lo ** e)) ** (1.0 / e)
    share = m / m.sum() * n_cl
    cnt = np.floor(share).astype(np.int64)
    left = n_cl - int(cnt.sum())
    order = np.argsort(-(share - cnt), kind="stable")
    cnt[order[:left]] += 1
    conc = 5.0 + 10.0 * rng.random(n_halos)
    rvir = rvir_max * (m / m.max()) ** (1.0 / 3.0)
    centres = rng.random((3, n_halos))
    parts = [rng.random((3, n_uni))]
    for h in range(n_halos):
        k = int(cnt[h])
        if k == 0:
            continue
        c = centres[:, h:h + 1]
        ch, rv = conc[h], rvir[h]

        def draw(g, kk, c=c, ch=ch, rv=rv):
            return c + _isotropic(g, _nfw_radius(g, ch, rv, kk))

        parts.append(_resample(rng, draw, k))
    pos = np.concatenate(parts, axis=1)
    perm = rng.permutation(n)
    return np.ascontiguousarray(pos[:, perm]), _equal_masses(n)


def coincident(n: int, seed: int, n_points: int = 1):
    """n particles on n_points distinct random locations (degenerate duplicate keys)."""
    rng = _rng(seed)
    pts = 0.1 + 0.8 * rng.random((3, n_points))
    idx = rng.integers(0, n_points, n)
    return np.ascontiguousarray(pts[:, idx]), _equal_masses(n)


def batch_boxes(n_boxes: int, seed: int, n_lo: int = 32 ** 3, n_hi: int = 96 ** 3):
    """Independent boxes, each a ``clustered_plummer`` set with N uniform in [n_lo, n_hi].

    Returns (list of (pos, mass), offsets) with offsets of length n_boxes + 1.
    """
    rng = _rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, n_boxes)
    boxes = [clustered_plummer(int(k), seed * 1000 + i + 1) for i, k in enumerate(ns)]
    off = np.zeros(n_boxes + 1, dtype=np.int64)
    off[1:] = np.cumsum(ns)
    return boxes, off


# Named workloads: the shapes and parameters of the five measured configurations.
WORKLOADS = {
    "plummer4096": dict(n=4096, kind="plummer", seed=1, eps=1e-3, theta=0.7),
    "nfw2m": dict(n=128 ** 3, kind="nfw", seed=2, eps=paper_softening(128 ** 3), theta=0.55),
    "batch64": dict(n=None, kind="batch", seed=3, eps=1e-3, theta=0.7, boxes=64),
    "rungs16m": dict(n=256 ** 3, kind="plummer", seed=4, eps=paper_softening(256 ** 3), theta=0.55),
    "learned134m": dict(n=512 ** 3, kind="plummer", seed=5, eps=paper_softening(512 ** 3), theta=0.55),
    "periodic2m": dict(n=128 ** 3, kind="nfw", seed=2, eps=paper_softening(128 ** 3), theta=0.55, nrep=1),
    "compressed704": dict(n=704 ** 3, kind="plummer", seed=6, eps=paper_softening(704 ** 3), theta=0.55),
}


def make(kind: str, n: int, seed: int):
    """Dispatch by structure name: 'uniform', 'plummer', 'nfw', 'coincident'."""
    if kind == "uniform":
        return uniform_box(n, seed)
    if kind == "plummer":
        return clustered_plummer(n, seed)
    if kind == "nfw":
        return clustered_nfw(n, seed)
    if kind == "coincident":
        return coincident(n, seed)
    raise ValueError(f"unknown structure {kind!r}")


def to_fixed(pos: np.ndarray) -> np.ndarray:
    """Positions in [0, 1) as 32-bit fixed-point coordinates u (x ~ u 2^-32, nearest, capped at
    2^32 - 1): the compressed storage of Sec. 3.4, an input format."""
    u = np.rint(np.asarray(pos, dtype=np.float64) * 4294967296.0)
    return np.minimum(u, 4294967295.0).astype(np.uint32)
