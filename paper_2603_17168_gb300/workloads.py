"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5.1).

This module holds no arithmetic of the hash table: only random keys, scores
and values. Tests feed the same arrays to the CUDA library and to the CPU
oracle; the benchmark uses them for every configuration.

Key streams (Sec. 5.1, Exp. 1 and 3c): the paper uses uniform random keys
for its load-factor sweeps and Zipf-distributed keys for cache-quality runs.
A Zipf rank r in [1, N] is drawn by rejection-inversion (Hoermann and
Derflinger, 1996, "Rejection-inversion to generate variates from monotone
discrete distributions") and mapped to a key by the bijection
key = (r * 0x9E3779B97F4A7C15) mod 2^63, so keys are never 0 and never in
the reserved range [2^63, 2^64). Uniform keys over an N-key universe use the
same mapping on uniform ranks. Values are N(0, 1) fp32.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
KEY_MASK = np.uint64((1 << 63) - 1)
SEED_BASE = 0x484B5600


def seed_for(config: int, batch: int = 0) -> int:
    return SEED_BASE + config * 1_000_003 + batch


def rank_to_key(ranks: np.ndarray) -> np.ndarray:
    r = np.asarray(ranks, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return (r * GOLDEN) & KEY_MASK


def uniform_keys(rng: np.random.Generator, n: int, universe: int | None = None,
                 distinct: bool = False) -> np.ndarray:
    """n keys: uniform over [1, 2^63) when universe is None, else the keys of
    uniform ranks in [1, universe]. distinct=True redraws collisions."""
    def draw(m):
        if universe is None:
            return rng.integers(1, 1 << 63, size=m, dtype=np.uint64)
        return rank_to_key(rng.integers(1, universe + 1, size=m, dtype=np.uint64))

    k = draw(n)
    if distinct:
        k = np.unique(k)
        while k.size < n:
            k = np.unique(np.concatenate([k, draw(n - k.size + 16)]))
        k = rng.permutation(k)[:n]
    return k


class Zipf:
    """Zipf(alpha) ranks on [1, N] by rejection-inversion; alpha > 0, != 1."""

    def __init__(self, alpha: float, n_elements: int):
        if alpha <= 0 or alpha == 1.0:
            raise ValueError("alpha must be positive and != 1")
        self.s = float(alpha)
        self.N = int(n_elements)
        self.h_x1 = self._H(1.5) - 1.0
        self.h_n = self._H(self.N + 0.5)
        self.cut = 2.0 - self._Hinv(self._H(2.5) - self._h(2.0))

    # H(x) = (x^(1-s) - 1) / (1 - s), an antiderivative of h(x) = x^-s
    def _H(self, x):
        lx = np.log(x)
        t = (1.0 - self.s) * lx
        return np.where(np.abs(t) > 1e-8, np.expm1(t) / np.where(t == 0, 1, t), 1.0) * lx

    def _Hinv(self, y):
        t = (1.0 - self.s) * y
        return np.exp(np.where(np.abs(t) > 1e-8, np.log1p(t) / np.where(t == 0, 1, t), 1.0) * y)

    def _h(self, x):
        return np.exp(-self.s * np.log(x))

    def ranks(self, rng: np.random.Generator, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint64)
        todo = np.arange(n)
        while todo.size:
            u = self.h_n + rng.random(todo.size) * (self.h_x1 - self.h_n)
            x = self._Hinv(u)
            k = np.clip(np.floor(x + 0.5), 1, self.N)
            ok = (k - x <= self.cut) | (u >= self._H(k + 0.5) - self._h(k))
            out[todo[ok]] = k[ok].astype(np.uint64)
            todo = todo[~ok]
        return out

    def keys(self, rng: np.random.Generator, n: int) -> np.ndarray:
        return rank_to_key(self.ranks(rng, n))


def normal_values(rng: np.random.Generator, n: int, dim: int) -> np.ndarray:
    return rng.standard_normal((n, dim), dtype=np.float32)


def lognormal_sizes(rng: np.random.Generator, n: int, median: float, sigma: float,
                    lo: int, hi: int) -> np.ndarray:
    s = np.exp(np.log(median) + sigma * rng.standard_normal(n))
    return np.clip(np.rint(s), lo, hi).astype(np.int64)


# Configuration shapes (sizes only).
TINY = dict(name="tiny", num_buckets=512, dim=8, batches=16, batch=4096, finds=4096)
SINGLE = dict(name="single", num_buckets=1 << 19, dim=32, batch=1 << 20, zipf_alpha=1.05,
              universe=1 << 32, lambdas=(0.50, 0.75, 0.90, 1.00))
MULTI_DIMS = (16, 32, 64, 64, 128, 128, 256, 8)
MULTI_SLOTS = (1 << 25, 1 << 25, 1 << 24, 1 << 24, 1 << 23, 1 << 23, 1 << 22, 1 << 25)
TIERED = dict(name="tiered", slots=1 << 28, dim=128, hbm_value_bytes=48 << 30, zipf_alpha=0.99,
              universe=1 << 34, batch=1 << 20)


# ---------------------------------------------------------------------------
# Device-side twins of the generators (torch on the GPU), for benchmark
# inputs too large to draw on the host quickly. Same constructions as above;
# the streams differ from numpy's, so parity tests use the numpy versions.

def rank_to_key_torch(ranks):
    import torch
    g = torch.tensor(int(GOLDEN) - (1 << 64), dtype=torch.int64, device=ranks.device)
    return (ranks.to(torch.int64) * g) & ((1 << 63) - 1)


def key_to_rank_torch(keys):
    """Inverse of rank_to_key_torch: the rank of each key (mod 2^63)."""
    import torch
    inv = pow(int(GOLDEN), -1, 1 << 63)  # < 2^63: fits an int64
    g = torch.tensor(inv, dtype=torch.int64, device=keys.device)
    return (keys.to(torch.int64) * g) & ((1 << 63) - 1)


def uniform_keys_torch(gen, n: int, universe: int, device="cuda"):
    import torch
    r = torch.randint(1, universe + 1, (n,), dtype=torch.int64, device=device, generator=gen)
    return rank_to_key_torch(r)


def zipf_ranks_torch(gen, z: Zipf, n: int, device="cuda"):
    import torch
    out = torch.empty(n, dtype=torch.int64, device=device)
    todo = torch.arange(n, device=device)
    s = z.s

    def H(x):
        lx = torch.log(x)
        t = (1.0 - s) * lx
        return torch.where(t.abs() > 1e-8, torch.expm1(t) / torch.where(t == 0, 1.0, t), 1.0) * lx

    def Hinv(y):
        t = (1.0 - s) * y
        return torch.exp(torch.where(t.abs() > 1e-8, torch.log1p(t) / torch.where(t == 0, 1.0, t),
                                     1.0) * y)

    while todo.numel():
        u = z.h_n + torch.rand(todo.numel(), dtype=torch.float64, device=device,
                               generator=gen) * (z.h_x1 - z.h_n)
        x = Hinv(u)
        k = torch.clamp(torch.floor(x + 0.5), 1, z.N)
        ok = (k - x <= z.cut) | (u >= H(k + 0.5) - torch.exp(-s * torch.log(k)))
        out[todo[ok]] = k[ok].to(torch.int64)
        todo = todo[~ok]
    return out


def zipf_keys_torch(gen, z: Zipf, n: int, device="cuda"):
    return rank_to_key_torch(zipf_ranks_torch(gen, z, n, device))
