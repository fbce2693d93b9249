"""Seeded synthetic inputs for CTD workloads.

This module only draws random tensors.  It holds none of the decomposition's
arithmetic, so both the CUDA path and the FP64 oracle can take their inputs
from it without sharing any of the method.

All tensors are 3-way count tensors in coordinate (COO) form with distinct
coordinates, the sparse-unordered layout that Section 2.1 of the paper
assumes.  Index vectors are int32 and 0-based; values are int32 counts.

Workloads imitate the paper's network-traffic tensor
(source x destination x time, Section 5): source and destination ids follow
a truncated Zipf law whose ranks are mapped through a seeded permutation,
time is uniform, values are small positive counts.

Rules (one reading, fixed here so every consumer sees the same bytes):
  * Zipf(a) over n ids: P(rank r) proportional to r**-a, r = 1..n; the id
    of rank r is perm[r-1] for a seeded permutation perm of range(n).
  * Distinct coordinates: coordinates are drawn in batches; the tensor keeps
    the first `nnz` distinct coordinates in draw order.
  * Entries are shuffled into a seeded random order (the input is unordered).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Iterator, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Coo3:
    """A 3-way sparse tensor in SoA COO form (0-based int32 indices)."""

    dims: tuple
    i: np.ndarray
    j: np.ndarray
    k: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.val.shape[0])

    def subset(self, mask: np.ndarray) -> "Coo3":
        return Coo3(self.dims, self.i[mask], self.j[mask], self.k[mask], self.val[mask])


class _Zipf:
    """Truncated Zipf(a) over n ids with a seeded rank -> id permutation."""

    def __init__(self, perm_rng: np.random.Generator, n: int, a: float):
        w = np.arange(1, n + 1, dtype=np.float64) ** (-a)
        cdf = np.cumsum(w)
        self.cdf = cdf / cdf[-1]
        self.perm = perm_rng.permutation(n).astype(np.int64)
        self.n = n

    def sampler(self, rng: np.random.Generator) -> Callable[[int], np.ndarray]:
        def draw(size: int) -> np.ndarray:
            r = np.searchsorted(self.cdf, rng.random(size), side="right")
            return self.perm[np.minimum(r, self.n - 1)]

        return draw


def _uniform_sampler(rng: np.random.Generator, n: int) -> Callable[[int], np.ndarray]:
    def draw(size: int) -> np.ndarray:
        return rng.integers(0, n, size=size, dtype=np.int64)

    return draw


def _distinct(rng: np.random.Generator, dims, nnz: int, di, dj, dk) -> tuple:
    """First `nnz` distinct coordinates of a stream of (di, dj, dk) draws."""
    I, J, K = (int(d) for d in dims)
    cells = I * J * K
    if nnz > cells:
        raise ValueError("more nonzeros than cells")
    keys_parts: List[np.ndarray] = []
    have = np.empty(0, dtype=np.int64)
    first_pos = np.empty(0, dtype=np.int64)
    drawn = 0
    batch = max(int(nnz * 1.1) + 16, 64)
    for _ in range(200):
        ii = di(batch)
        jj = dj(batch)
        kk = dk(batch)
        key = ii + I * (jj + J * kk)
        keys_parts.append(key)
        allk = np.concatenate(keys_parts)
        uniq, idx = np.unique(allk, return_index=True)
        drawn = allk.shape[0]
        if uniq.shape[0] >= nnz:
            order = np.argsort(idx, kind="stable")[:nnz]
            have = uniq[order]
            first_pos = idx[order]
            break
        missing = nnz - uniq.shape[0]
        batch = max(int(missing * 2.0) + 64, batch // 2)
    else:  # pragma: no cover - only for degenerate laws
        raise RuntimeError("could not draw enough distinct coordinates")
    del first_pos, drawn
    ii = have % I
    rest = have // I
    jj = rest % J
    kk = rest // J
    return ii, jj, kk


def _finish(rng, dims, ii, jj, kk, vals) -> Coo3:
    perm = rng.permutation(ii.shape[0])
    return Coo3(
        tuple(int(d) for d in dims),
        np.ascontiguousarray(ii[perm], dtype=np.int32),
        np.ascontiguousarray(jj[perm], dtype=np.int32),
        np.ascontiguousarray(kk[perm], dtype=np.int32),
        np.ascontiguousarray(vals[perm], dtype=np.int32),
    )


def uniform_counts(dims, nnz: int, lam: float, seed: int) -> Coo3:
    """Distinct uniform coordinates, values Poisson(lam)+1."""
    rng = np.random.default_rng(seed)
    I, J, K = dims
    cells = I * J * K
    lin = rng.choice(cells, size=nnz, replace=False).astype(np.int64)
    ii = lin % I
    jj = (lin // I) % J
    kk = lin // (I * J)
    vals = rng.poisson(lam, size=nnz) + 1
    return _finish(rng, dims, ii, jj, kk, vals)


def traffic(dims, nnz: int, a_src: float, a_dst: float, values: str, seed: int,
            vparam: float) -> Coo3:
    """Source x destination x time counts: Zipf ids, uniform time."""
    rng = np.random.default_rng(seed)
    I, J, K = dims
    di = _Zipf(rng, I, a_src).sampler(rng)
    dj = _Zipf(rng, J, a_dst).sampler(rng)
    dk = _uniform_sampler(rng, K)
    ii, jj, kk = _distinct(rng, dims, nnz, di, dj, dk)
    vals = _values(rng, values, vparam, ii.shape[0])
    return _finish(rng, dims, ii, jj, kk, vals)


def traffic_device(dims, nnz: int, a_src: float, a_dst: float, values: str, vparam: float,
                   seed: int, device: str = "cuda"):
    """The law of `traffic` drawn on the GPU (for timing runs of workloads
    too large to draw on the host in reasonable time).

    Same rules as above -- Zipf ids through a seeded rank -> id permutation,
    uniform time, the first `nnz` distinct coordinates of the draw stream,
    Geometric or Poisson+1 counts, a seeded shuffle -- with draws from a
    seeded torch generator on `device`, so the tensors follow the same
    distributions as `traffic`'s but are not the same draws.  Returns int32
    tensors (i, j, k, val) on the device."""
    import torch
    I, J, K = (int(d) for d in dims)
    if nnz > I * J * K:
        raise ValueError("more nonzeros than cells")
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))

    def zipf(n, a):
        w = torch.arange(1, n + 1, device=device, dtype=torch.float64).pow(-a)
        cdf = torch.cumsum(w, 0)
        cdf = cdf / cdf[-1]
        perm = torch.randperm(n, generator=g, device=device)

        def draw(m):
            u = torch.rand(m, generator=g, device=device, dtype=torch.float64)
            return perm[torch.searchsorted(cdf, u, right=True).clamp_(max=n - 1)]
        return draw

    di, dj = zipf(I, a_src), zipf(J, a_dst)
    keys = torch.empty(0, dtype=torch.int64, device=device)
    batch = int(nnz * 1.1) + 16
    for _ in range(64):
        ii = di(batch)
        jj = dj(batch)
        kk = torch.randint(0, K, (batch,), generator=g, device=device)
        keys = torch.cat([keys, ii + I * (jj + J * kk)])
        uniq, inv = torch.unique(keys, sorted=True, return_inverse=True)
        if uniq.numel() >= nnz:
            break
        # draws are cheap here: ask for plenty more than the shortfall
        batch = max(8 * (nnz - uniq.numel()) + 1024, batch)
    else:  # pragma: no cover - only for degenerate laws
        raise RuntimeError("could not draw enough distinct coordinates")
    first = torch.full((uniq.numel(),), keys.numel(), dtype=torch.int64, device=device)
    first.scatter_reduce_(0, inv, torch.arange(keys.numel(), device=device), reduce="amin")
    key = uniq[torch.argsort(first)[:nnz]]
    del keys, inv, first, uniq
    if values == "geometric":
        v = torch.empty(nnz, device=device, dtype=torch.float64).geometric_(vparam, generator=g)
    elif values == "poisson1":
        v = torch.poisson(torch.full((nnz,), float(vparam), device=device), generator=g) + 1
    else:
        raise ValueError(values)
    order = torch.randperm(nnz, generator=g, device=device)
    key = key[order]
    v = v[order]
    ii = (key % I).to(torch.int32)
    rest = key // I
    return ii, (rest % J).to(torch.int32), (rest // J).to(torch.int32), v.to(torch.int32)


def _values(rng, kind: str, p: float, n: int) -> np.ndarray:
    if kind == "geometric":
        return rng.geometric(p, size=n)
    if kind == "poisson1":
        return rng.poisson(p, size=n) + 1
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def small_uniform(seed: int = 1001) -> Coo3:
    """100 x 100 x 50, 5,000 distinct uniform coordinates, Poisson(3)+1."""
    return uniform_counts((100, 100, 50), 5000, 3.0, seed)


def traffic_10m(seed: int = 1002, scale: float = 1.0) -> Coo3:
    """10^4 x 10^4 x 10^3 traffic tensor, 10^7 nonzeros, Zipf(1.2), Geometric(0.3).

    `scale` < 1 shrinks every mode and the nonzero count together (for tests).
    """
    I = max(8, int(round(10000 * scale)))
    J = max(8, int(round(10000 * scale)))
    K = max(2, int(round(1000 * scale)))
    nnz = max(16, int(round(10_000_000 * scale ** 3)))
    return traffic((I, J, K), nnz, 1.2, 1.2, "geometric", seed, 0.3)


@dataclasses.dataclass
class SliceStream:
    """A time-ordered stream of source x destination slices (K = 1 each)."""

    dims2: tuple
    steps: int
    nnz: int
    a: float
    lam: float
    seed: int
    planted_steps: Sequence[int] = ()
    planted_src: Optional[np.ndarray] = None
    planted_dst: Optional[np.ndarray] = None
    planted_lam: float = 0.0

    def slice(self, t: int) -> Coo3:
        I, J = self.dims2
        rng = np.random.default_rng([self.seed, t])
        # the id permutations are fixed per stream; the draws are per slice
        di_t = _Zipf(np.random.default_rng([self.seed, 0x5A]), I, self.a).sampler(rng)
        dj_t = _Zipf(np.random.default_rng([self.seed, 0x5B]), J, self.a).sampler(rng)
        dk = lambda size: np.zeros(size, dtype=np.int64)  # noqa: E731
        ii, jj, kk = _distinct(rng, (I, J, 1), self.nnz, di_t, dj_t, dk)
        vals = rng.poisson(self.lam, size=ii.shape[0]) + 1
        if t in set(self.planted_steps) and self.planted_src is not None:
            src = np.repeat(self.planted_src, self.planted_dst.shape[0])
            dst = np.tile(self.planted_dst, self.planted_src.shape[0])
            add = rng.poisson(self.planted_lam, size=src.shape[0])
            key_bg = ii + I * jj
            key_pl = src + I * dst
            allk = np.concatenate([key_bg, key_pl])
            allv = np.concatenate([vals, add])
            uk, inv = np.unique(allk, return_inverse=True)
            summed = np.zeros(uk.shape[0], dtype=np.int64)
            np.add.at(summed, inv, allv)
            keep = summed != 0
            uk = uk[keep]
            vals = summed[keep]
            ii = uk % I
            jj = uk // I
            kk = np.zeros_like(ii)
        return _finish(rng, (I, J, 1), ii, jj, kk, vals)

    def __iter__(self) -> Iterator[Coo3]:
        for t in range(self.steps):
            yield self.slice(t)


def traffic_stream_20k(seed: int = 1003, scale: float = 1.0, steps: int = 100) -> SliceStream:
    """100 slices of 2*10^4 x 2*10^4 with 5*10^5 nonzeros each (Zipf(1.1),
    Poisson(2)+1), plus a planted 200 x 50 block of Poisson(40) counts added
    at steps 40..45.  `scale` shrinks the slice side, the nonzero count (by
    scale**2) and the planted block together."""
    I = J = max(16, int(round(20000 * scale)))
    nnz = max(32, int(round(500_000 * scale ** 2)))
    rng = np.random.default_rng([seed, 0xB10C])
    ns = max(2, int(round(200 * scale)))
    nd = max(1, int(round(50 * scale)))
    src = np.sort(rng.choice(I, size=min(ns, I), replace=False)).astype(np.int64)
    dst = np.sort(rng.choice(J, size=min(nd, J), replace=False)).astype(np.int64)
    planted = [t for t in range(40, 46) if t < steps]
    return SliceStream((I, J), steps, nnz, 1.1, 2.0, seed, planted, src, dst, 40.0)


@dataclasses.dataclass
class BatchSpec:
    dims: tuple
    nnz: int
    s: int
    seed: int

    def tensor(self) -> Coo3:
        return traffic(self.dims, self.nnz, 1.2, 1.2, "poisson1", self.seed, 3.0)


def batch_256(seed: int = 1004, count: int = 256, nnz_cap: Optional[int] = None) -> List[BatchSpec]:
    """256 tensors of uneven size: I, J log-uniform in [500, 2*10^4], K in
    [10, 500], nnz log-uniform in [10^4, 2*10^6] (at most a quarter of the
    cells), Zipf(1.2) ids, Poisson(3)+1 counts, s = floor(min(I, J) / 20)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        I = int(round(np.exp(rng.uniform(np.log(500), np.log(20000)))))
        J = int(round(np.exp(rng.uniform(np.log(500), np.log(20000)))))
        K = int(round(np.exp(rng.uniform(np.log(10), np.log(500)))))
        nnz = int(round(np.exp(rng.uniform(np.log(1e4), np.log(2e6)))))
        nnz = min(nnz, (I * J * K) // 4)
        if nnz_cap is not None:
            nnz = min(nnz, nnz_cap)
        out.append(BatchSpec((I, J, K), nnz, max(1, min(I, J) // 20), seed * 1000 + b))
    return out


@dataclasses.dataclass
class Request:
    stream: int
    step: int
    arrival_s: float
    nnz: int
    seed: int

    def slice(self, dims2=(5000, 5000), a: float = 1.1, lam: float = 3.0) -> Coo3:
        return traffic((dims2[0], dims2[1], 1), self.nnz, a, a, "poisson1", self.seed, lam)


def serving_requests(seed: int = 1005, streams: int = 64, rate_hz: float = 2000.0,
                     duration_s: float = 2.0, nnz_lo: float = 1e4, nnz_hi: float = 1e6) -> List[Request]:
    """Poisson arrivals at `rate_hz` in total, spread uniformly over `streams`
    streams; each request is one 5,000 x 5,000 slice whose nonzero count is
    log-uniform in [nnz_lo, nnz_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    steps = [0] * streams
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        st = int(rng.integers(0, streams))
        nnz = int(round(np.exp(rng.uniform(np.log(nnz_lo), np.log(nnz_hi)))))
        out.append(Request(st, steps[st], t, nnz, seed * 100000 + len(out)))
        steps[st] += 1
    return out


def tiny(dims=(6, 5, 4), nnz: int = 30, seed: int = 7, vmax: int = 5, signed: bool = False) -> Coo3:
    """Small uniform tensor for brute-force checks."""
    rng = np.random.default_rng(seed)
    I, J, K = dims
    lin = rng.choice(I * J * K, size=nnz, replace=False).astype(np.int64)
    ii = lin % I
    jj = (lin // I) % J
    kk = lin // (I * J)
    vals = rng.integers(1, vmax + 1, size=nnz)
    if signed:
        vals = vals * rng.choice([-1, 1], size=nnz)
    return _finish(rng, dims, ii, jj, kk, vals)


def nway_uniform(dims, nnz: int, seed: int, vmax: int = 5, signed: bool = False):
    """An N-way tensor with `nnz` distinct uniform coordinates and values in
    1 .. vmax (random signs if `signed`): (list of N int32 index arrays,
    int32 values), in a seeded random order."""
    rng = np.random.default_rng(seed)
    cells = int(np.prod([int(d) for d in dims]))
    lin = rng.choice(cells, size=nnz, replace=False).astype(np.int64)
    idx, rest = [], lin
    for d in dims:
        idx.append(np.ascontiguousarray(rest % int(d), dtype=np.int32))
        rest = rest // int(d)
    val = rng.integers(1, vmax + 1, size=nnz)
    if signed:
        val = val * rng.choice([-1, 1], size=nnz)
    return idx, np.ascontiguousarray(val, dtype=np.int32)


def nway_real(dims, nnz: int, seed: int, spread: float = 1.5):
    """An N-way tensor with `nnz` distinct uniform coordinates and real FP32
    values sign * exp(N(0, spread^2)) (magnitudes spread over several
    octaves): (list of N int32 index arrays, float32 values)."""
    idx, _ = nway_uniform(dims, nnz, seed)
    rng = np.random.default_rng([seed, 0xF32])
    mag = np.exp(rng.normal(0.0, spread, size=nnz))
    val = mag * rng.choice([-1.0, 1.0], size=nnz)
    return idx, np.ascontiguousarray(val, dtype=np.float32)
