"""Seeded synthetic problems for the multi-channel integrator.

This module only *draws* problem parameters (which coordinates each channel
maps, with which kind of map, masses, widths, peak weights, run schedules).
It holds none of the integration method's arithmetic: no maps, densities,
grids or estimators.  Both the CPU oracle and the CUDA library consume the
arrays it returns, so it is the one module they share.

Workload shapes follow the paper's ranges: dimension d between 2 and 25 and
channel counts from one upwards (§2), a few tens of bins per axis (§3.2),
narrow resonances mapped by Breit-Wigner channels (§2, §3.4).  The paper's
physics processes and matrix elements are not available, so these synthetic
integrands stand in for them:

* ``single_gauss``: one Gaussian peak (sigma 0.1, centre 0.5) in d=4,
  a single identity channel, 20 bins, 5 iterations of 1e4 calls.
* ``bw_gauss``: d=8, six channels each applying a Breit-Wigner map to one
  coordinate; the integrand is a Dirichlet-weighted sum of six matching
  Breit-Wigner x Gaussian(sigma 0.2) peaks; 50 bins; 10 x 1e6 calls.
* ``collider``: d=14, 64 channels mapping 2-4 distinct coordinates each by
  Breit-Wigner or power-law maps; 64 matching peaks with widths log-uniform
  in [1e-4, 1e-2]; 100 bins; 15 x 1e7 calls, then 1e6 unweighted events.
* ``batch_instance(i)``: one of 256 uneven instances (d in 2..16,
  channels log-uniform in 1..64, calls log-uniform in 1e4..1e7, bins in
  {20, 50, 100}), each built like ``bw_gauss``.
* ``serving_stream``: Poisson arrivals of integrate-then-generate requests.
* ``signed_pair`` / ``signed_bw_gauss``: integrands of both signs (peaks
  with negative weights), as NLO matrix elements can be (§3.1).
* ``ring``: channels that are images of one another under a cyclic shift
  of coordinates (and mirror-symmetric on every axis), with the channel
  equivalences that say so (§3.5).

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64), which
gives identical streams on x86-64 and AArch64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MAP_ID = 0
MAP_BW = 1
MAP_POW = 2

GAUSS_NORM_REAL_LINE = 0  # Gaussian normalised on the whole real line
GAUSS_NORM_UNIT = 1       # Gaussian normalised on [0, 1]

MAX_MAPPED = 4            # mapped coordinates per channel / peak

# per-axis kinds of a channel equivalence (§3.5)
EQ_IDENTITY = 0
EQ_INVERT = 1
EQ_SYMMETRIC = 2
EQ_INVARIANT = 3


@dataclasses.dataclass
class MapSet:
    """K channel maps (or K integrand peaks) in struct-of-arrays form.

    Slot s < n_mapped[k] of row k maps coordinate coord[k, s] with map kind
    kind[k, s]; for a Breit-Wigner slot a = mass m and b = width Gamma, for
    a power-law slot b = the width delta of the integrand factor (the
    channel map itself is the pure x**5).
    """

    n_mapped: np.ndarray  # int32[K]
    coord: np.ndarray     # int32[K, 4]
    kind: np.ndarray      # int32[K, 4]
    a: np.ndarray         # float64[K, 4]
    b: np.ndarray         # float64[K, 4]

    @staticmethod
    def identity(k: int) -> "MapSet":
        return MapSet(np.zeros(k, np.int32), np.zeros((k, MAX_MAPPED), np.int32),
                      np.zeros((k, MAX_MAPPED), np.int32),
                      np.zeros((k, MAX_MAPPED), np.float64),
                      np.zeros((k, MAX_MAPPED), np.float64))

    def copy(self) -> "MapSet":
        return MapSet(*(np.array(getattr(self, f.name)) for f in dataclasses.fields(self)))

    def __len__(self) -> int:
        return int(self.n_mapped.shape[0])


@dataclasses.dataclass
class Problem:
    """One integration problem plus its run schedule (all plain data)."""

    name: str
    d: int
    n_bins: int
    channels: MapSet
    peak_weight: np.ndarray   # float64[P]
    peaks: MapSet
    gauss_sigma: float
    gauss_centre: float
    gauss_norm: int
    seed: int                 # 64-bit Philox key of the sampling RNG
    request_id: int = 0
    grid_alpha: float = 1.5   # damping power of the rebinning measure
    beta: float = 0.5         # power of the channel-weight update
    n_min: int = 10           # lower threshold of calls per live channel
    smooth: int = 0           # 1: neighbour-average the bin d-values
    omega_mode: int = 0       # 0: channel variance, 1: second moment
    gen_batch: int = 1 << 20  # calls per generation batch
    iterations: int = 1
    calls: int = 10_000
    adapt_grid: bool = True
    adapt_alpha: bool = True
    combine_from: int = 0     # first iteration entering the combination
    n_events: int = 0
    stratified: int = 0       # 1: pseudo-stratified sampling in r space (§3.3)
    # channel equivalences (§3.5): int32[n_equiv, 2 + 2d], each row
    # (c, c', π_0..π_{d-1}, kind_0..kind_{d-1}): axis k of channel c takes
    # the bin weights of axis π_k of channel c' with kind EQ_*
    equivalences: np.ndarray | None = None

    @property
    def n_channels(self) -> int:
        return len(self.channels)

    @property
    def n_peaks(self) -> int:
        return len(self.peaks)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def _dirichlet1(rng: np.random.Generator, k: int) -> np.ndarray:
    e = rng.exponential(1.0, size=k)
    return e / e.sum()


def _log_uniform(rng: np.random.Generator, lo: float, hi: float, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


def single_gauss(seed: int = 1) -> Problem:
    """d=4 single-channel VEGAS problem: one Gaussian (sigma 0.1, centre 0.5)."""
    return Problem(name="single_gauss_d4", d=4, n_bins=20,
                   channels=MapSet.identity(1), peak_weight=np.ones(1),
                   peaks=MapSet.identity(1), gauss_sigma=0.1, gauss_centre=0.5,
                   gauss_norm=GAUSS_NORM_REAL_LINE, seed=seed, grid_alpha=1.5,
                   iterations=5, calls=10_000, adapt_grid=True, adapt_alpha=False,
                   combine_from=2)


def _bw_gauss_maps(rng, d: int, k: int, with_replacement: bool) -> MapSet:
    ms = MapSet.identity(k)
    if with_replacement or k > d:
        coords = rng.integers(0, d, size=k)
    else:
        coords = rng.choice(d, size=k, replace=False)
    masses = rng.uniform(0.2, 0.8, size=k)
    widths = _log_uniform(rng, 1e-3, 1e-2, size=k)
    ms.n_mapped[:] = 1
    ms.coord[:, 0] = coords
    ms.kind[:, 0] = MAP_BW
    ms.a[:, 0] = masses
    ms.b[:, 0] = widths
    return ms


def bw_gauss(problem_seed: int = 2, rng_seed: int = 2) -> Problem:
    """d=8, six Breit-Wigner x Gaussian peaks with six matching channels."""
    rng = np.random.default_rng(problem_seed)
    maps = _bw_gauss_maps(rng, 8, 6, with_replacement=False)
    w = _dirichlet1(rng, 6)
    return Problem(name="bw_gauss_d8_k6", d=8, n_bins=50, channels=maps,
                   peak_weight=w, peaks=maps.copy(), gauss_sigma=0.2,
                   gauss_centre=0.5, gauss_norm=GAUSS_NORM_UNIT, seed=rng_seed,
                   iterations=10, calls=1_000_000, adapt_grid=True,
                   adapt_alpha=True, combine_from=4)


def collider(problem_seed: int = 3, rng_seed: int = 3) -> Problem:
    """d=14, 64 channels mapping 2-4 coordinates each (Breit-Wigner or power)."""
    rng = np.random.default_rng(problem_seed)
    d, k = 14, 64
    ms = MapSet.identity(k)
    for c in range(k):
        nm = int(rng.integers(2, 5))
        coords = rng.choice(d, size=nm, replace=False)
        ms.n_mapped[c] = nm
        for s in range(nm):
            ms.coord[c, s] = coords[s]
            if rng.uniform() < 0.5:
                ms.kind[c, s] = MAP_BW
                ms.a[c, s] = rng.uniform(0.2, 0.8)
            else:
                ms.kind[c, s] = MAP_POW
                ms.a[c, s] = 0.0
            ms.b[c, s] = float(_log_uniform(rng, 1e-4, 1e-2))
    w = _dirichlet1(rng, k)
    return Problem(name="collider_d14_k64", d=d, n_bins=100, channels=ms,
                   peak_weight=w, peaks=ms.copy(), gauss_sigma=0.2,
                   gauss_centre=0.5, gauss_norm=GAUSS_NORM_UNIT, seed=rng_seed,
                   iterations=15, calls=10_000_000, adapt_grid=True,
                   adapt_alpha=True, combine_from=5, n_events=1_000_000)


def batch_instance(i: int) -> Problem:
    """Instance i of the 256-instance uneven batch (problem seed 1000 + i)."""
    rng = np.random.default_rng(1000 + i)
    d = int(rng.integers(2, 17))
    k = max(1, int(round(float(_log_uniform(rng, 1.0, 64.0)))))
    calls = int(round(float(_log_uniform(rng, 1e4, 1e7))))
    n_bins = int(rng.choice([20, 50, 100]))
    maps = _bw_gauss_maps(rng, d, k, with_replacement=k > d)
    w = _dirichlet1(rng, k)
    return Problem(name=f"batch_{i:03d}", d=d, n_bins=n_bins, channels=maps,
                   peak_weight=w, peaks=maps.copy(), gauss_sigma=0.2,
                   gauss_centre=0.5, gauss_norm=GAUSS_NORM_UNIT,
                   seed=1000 + i, request_id=i, iterations=10, calls=calls,
                   adapt_grid=True, adapt_alpha=True, combine_from=4)


def batch(n_instances: int = 256) -> list[Problem]:
    return [batch_instance(i) for i in range(n_instances)]


@dataclasses.dataclass
class Request:
    arrival_s: float
    problem: Problem


def serving_stream(rate_per_s: float = 200.0, duration_s: float = 60.0,
                   seed: int = 5, max_requests: int | None = None) -> list[Request]:
    """Poisson arrivals of integrate-then-generate requests.

    Each request is drawn like a batch instance, plus a log-uniform number of
    unweighted events in [1e3, 1e5].
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out: list[Request] = []
    idx = 0
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t >= duration_s:
            break
        sub = int(rng.integers(0, 2**31 - 1))
        r2 = np.random.default_rng(sub)
        d = int(r2.integers(2, 17))
        k = max(1, int(round(float(_log_uniform(r2, 1.0, 64.0)))))
        calls = int(round(float(_log_uniform(r2, 1e4, 1e7))))
        n_bins = int(r2.choice([20, 50, 100]))
        maps = _bw_gauss_maps(r2, d, k, with_replacement=k > d)
        w = _dirichlet1(r2, k)
        n_ev = int(round(float(_log_uniform(r2, 1e3, 1e5))))
        p = Problem(name=f"req_{idx:05d}", d=d, n_bins=n_bins, channels=maps,
                    peak_weight=w, peaks=maps.copy(), gauss_sigma=0.2,
                    gauss_centre=0.5, gauss_norm=GAUSS_NORM_UNIT, seed=sub,
                    request_id=idx, iterations=10, calls=calls, adapt_grid=True,
                    adapt_alpha=True, combine_from=4, n_events=n_ev)
        out.append(Request(t, p))
        idx += 1
        if max_requests is not None and idx >= max_requests:
            break
    return out


def special_case(kind: str, d: int = 2, n_bins: int = 10, seed: int = 7,
                 **kw) -> Problem:
    """Small problems with closed-form answers (used by tests).

    * ``"const"``: f = 1 on the unit cube, one identity channel.
    * ``"bw"``: f = one normalised Breit-Wigner in coordinate 0 (others
      uniform), the channel applies the same Breit-Wigner map.
    * ``"pow"``: f = the power-law density in coordinate 0 with delta = 0,
      the channel applies the x**5 map.
    """
    ch = MapSet.identity(1)
    pk = MapSet.identity(1)
    if kind == "const":
        pass
    elif kind == "bw":
        m, g = kw.get("mass", 0.37), kw.get("width", 3e-3)
        for ms in (ch, pk):
            ms.n_mapped[0] = 1
            ms.coord[0, 0] = 0
            ms.kind[0, 0] = MAP_BW
            ms.a[0, 0] = m
            ms.b[0, 0] = g
    elif kind == "pow":
        for ms in (ch, pk):
            ms.n_mapped[0] = 1
            ms.coord[0, 0] = 0
            ms.kind[0, 0] = MAP_POW
            ms.b[0, 0] = 0.0
    else:
        raise ValueError(kind)
    # sigma = 0 switches the Gaussian factor off (factor 1 on every
    # coordinate that the peak does not map): the integrand is then exactly
    # the product of the mapped factors.
    return Problem(name=f"special_{kind}", d=d, n_bins=n_bins, channels=ch,
                   peak_weight=np.ones(1), peaks=pk, gauss_sigma=0.0,
                   gauss_centre=0.5, gauss_norm=GAUSS_NORM_UNIT, seed=seed,
                   iterations=3, calls=5000, adapt_grid=True, adapt_alpha=False)


def signed_pair(weights=(1.3, -0.3), d: int = 1, masses=(0.3, 0.7), width: float = 0.05,
                seed: int = 13) -> Problem:
    """f = w_0 BW(p_0; m_0) + w_1 BW(p_0; m_1) (factor 1 on other coordinates),
    two channels with the matching Breit-Wigner maps.  A negative weight makes
    f < 0 around its mass; the integral is w_0 + w_1."""
    ms = MapSet.identity(2)
    ms.n_mapped[:] = 1
    ms.coord[:, 0] = 0
    ms.kind[:, 0] = MAP_BW
    ms.a[:, 0] = masses
    ms.b[:, 0] = width
    return Problem(name=f"signed_pair_d{d}", d=d, n_bins=20, channels=ms,
                   peak_weight=np.asarray(weights, np.float64), peaks=ms.copy(),
                   gauss_sigma=0.0, gauss_centre=0.5, gauss_norm=GAUSS_NORM_UNIT, seed=seed,
                   iterations=5, calls=20_000, adapt_grid=True, adapt_alpha=True, combine_from=2)


def signed_bw_gauss(problem_seed: int = 2, rng_seed: int = 2) -> Problem:
    """``bw_gauss`` with the last peak's weight negated: f < 0 near its
    resonance; the integral is the signed sum of the weights."""
    pr = bw_gauss(problem_seed, rng_seed)
    w = np.array(pr.peak_weight)
    w[5] *= -1.0
    return pr.replace(name="signed_bw_gauss_d8_k6", peak_weight=w)


def ring(n_ring: int = 3, d: int = 6, width: float = 3e-3, seed: int = 11,
         equivalences: bool = True, kind: int = EQ_IDENTITY) -> Problem:
    """Channels related by symmetry, with their equivalences (§3.5).

    Channel c < n_ring applies a Breit-Wigner map (mass 0.5, common width)
    to coordinate c; the integrand is the equal-weight sum of the matching
    peaks times Gaussians (sigma 0.2, centre 0.5) on the other coordinates.
    A cyclic shift of coordinates 0..n_ring-1 permutes the peaks, and
    p_k -> 1 - p_k leaves every factor unchanged, so channel c' samples
    like channel c with its axes shifted by c' - c.  With ``equivalences``
    every ordered pair (c, c'), c != c', is listed with that permutation
    and the per-axis kind ``kind``.
    """
    ms = MapSet.identity(n_ring)
    ms.n_mapped[:] = 1
    ms.coord[:, 0] = np.arange(n_ring)
    ms.kind[:, 0] = MAP_BW
    ms.a[:, 0] = 0.5
    ms.b[:, 0] = width
    eq = rotation_equivalences(n_ring, d, kind) if equivalences else None
    return Problem(name=f"ring_d{d}_k{n_ring}", d=d, n_bins=20, channels=ms,
                   peak_weight=np.full(n_ring, 1.0 / n_ring), peaks=ms.copy(),
                   gauss_sigma=0.2, gauss_centre=0.5, gauss_norm=GAUSS_NORM_UNIT,
                   seed=seed, iterations=5, calls=30_000, adapt_grid=True,
                   adapt_alpha=True, combine_from=2, equivalences=eq)


def rotation_equivalences(n_ring: int, d: int, kind: int = EQ_IDENTITY) -> np.ndarray:
    """Equivalences of ``ring``: axis k < n_ring of channel c matches axis
    (k + c' - c) mod n_ring of channel c'; the other axes match themselves."""
    rows = []
    for c in range(n_ring):
        for cp in range(n_ring):
            if cp == c:
                continue
            perm = [(k + cp - c) % n_ring if k < n_ring else k for k in range(d)]
            rows.append([c, cp] + perm + [kind] * d)
    return np.array(rows, np.int32).reshape(-1, 2 + 2 * d)


CONFIGS = {
    "single_gauss": single_gauss,
    "bw_gauss": bw_gauss,
    "collider": collider,
}
