"""Seeded synthetic inputs for DPF-PIR tests and benchmarks.

This module holds no DPF or AES arithmetic.  It draws the tables, target
indices and key randomness that both the oracle and the CUDA library consume,
so that the two sides see identical inputs while sharing no method code.

Tables stand in for the paper's embedding tables (Sec. 2, Tables 1-2: rows of
64-1024 bytes); no dataset is read.  Table entries are uniform u32 drawn from
the SplitMix64 stream (Steele, Lea and Flood, OOPSLA 2014; constants from the
published reference generator):

    T[r][w] = low32(splitmix64_output(seed + (r * W + w + 1) * GAMMA))

which is the (r*W + w)-th output of a SplitMix64 generator started at `seed`.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# Workload shapes (rows, width in u32 words).  Names say what they are.
PLAIN_SINGLE = dict(rows=1 << 16, width=16, batch=1)            # 4 MiB table, 1 key pair
BATCHED_1M = dict(rows=1 << 20, width=64, batch=256)             # 256 MiB table, 2048-bit entries
MULTI_TABLE_ROWS = [1 << 16, 1 << 17, 1 << 18, 1 << 19, 1 << 20, 1 << 20, 1 << 21, 1 << 22]
MULTI_TABLE_WIDTHS = [16, 32, 32, 64, 64, 128, 32, 16]
MULTI_TABLE_QUERIES = 2048
LARGE_16M = dict(rows=1 << 24, width=32, batch=1024)             # 2 GiB table
SERVING_TABLES = [(1 << 18, 64), (1 << 20, 32), (1 << 22, 32), (1 << 24, 16)]
# hot/full split serving: a full table, its 2^18 most popular rows as the hot
# table, requests of HOTFULL_WANTED rows each (Zipf 1.1 popularity), fixed
# budgets of hot and full queries per request
HOTFULL_FULL = (1 << 22, 32)
HOTFULL_HOT_ROWS = 1 << 18
HOTFULL_WANTED = 10
HOTFULL_Q_HOT, HOTFULL_Q_FULL = 10, 3


def splitmix64_stream(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start..start+count-1 of SplitMix64 seeded with `seed` (uint64)."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + i * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        z = z ^ (z >> np.uint64(31))
    return z


def table_u32(seed: int, rows: int, width: int, chunk_rows: int = 1 << 16) -> np.ndarray:
    """The seeded table T[rows][width] of uniform u32 (host, numpy)."""
    out = np.empty((rows, width), dtype=np.uint32)
    for r0 in range(0, rows, chunk_rows):
        r1 = min(rows, r0 + chunk_rows)
        z = splitmix64_stream(seed, r0 * width, (r1 - r0) * width)
        out[r0:r1] = (z & np.uint64(0xFFFFFFFF)).astype(np.uint32).reshape(r1 - r0, width)
    return out


def table_rows_u32(seed: int, width: int, rows: np.ndarray) -> np.ndarray:
    """Selected rows of the same seeded table, without building all of it."""
    rows = np.asarray(rows, dtype=np.uint64)
    out = np.empty((rows.size, width), dtype=np.uint32)
    for i, r in enumerate(rows.tolist()):
        z = splitmix64_stream(seed, int(r) * width, width)
        out[i] = (z & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return out


def _signed64(v: int) -> int:
    v &= MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def table_u32_torch(seed: int, rows: int, width: int, device, chunk_rows: int = 1 << 18):
    """The same table built with torch int64 ops on `device` (bit-identical to
    table_u32); returned as torch.int32 holding the u32 bit patterns."""
    import torch

    out = torch.empty((rows, width), dtype=torch.int32, device=device)
    g = torch.tensor(_signed64(GAMMA), dtype=torch.int64, device=device)
    m1 = torch.tensor(_signed64(MIX1), dtype=torch.int64, device=device)
    m2 = torch.tensor(_signed64(MIX2), dtype=torch.int64, device=device)
    s = torch.tensor(_signed64(seed), dtype=torch.int64, device=device)

    def lsr(x, k):  # logical right shift on int64 bit patterns
        return (x >> k) & ((1 << (64 - k)) - 1)

    for r0 in range(0, rows, chunk_rows):
        r1 = min(rows, r0 + chunk_rows)
        i = torch.arange(r0 * width + 1, r1 * width + 1, dtype=torch.int64, device=device)
        z = s + i * g
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        z = z ^ lsr(z, 31)
        lo = z & 0xFFFFFFFF
        lo = ((lo ^ 0x80000000) - 0x80000000).to(torch.int32)
        out[r0:r1] = lo.view(r1 - r0, width)
    return out


def alphas(seed: int, rows: int, count: int) -> np.ndarray:
    """Target indices alpha, uniform in [0, rows)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, rows, size=count, dtype=np.uint64)


def key_randomness(seed: int, n: int, count: int):
    """Per key pair: (root0, root1, codeword randomness C_0 of n*2*16 bytes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        raw = rng.integers(0, 256, size=32 + 32 * n, dtype=np.uint8).tobytes()
        out.append((raw[:16], raw[16:32], raw[32:]))
    return out


def zipf_assignment(seed: int, ntables: int, count: int, s: float = 1.1) -> np.ndarray:
    """Table index per query, P(rank k) proportional to k^-s over k = 1..ntables
    (rank 1 = table 0)."""
    p = np.arange(1, ntables + 1, dtype=np.float64) ** (-s)
    p /= p.sum()
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.choice(ntables, size=count, p=p).astype(np.int32)


class ZipfRows:
    """Row popularity of an embedding table: rank k (1-based) is drawn with
    probability proportional to k^-s, and rank k is row perm[k-1] of a seeded
    permutation, so popular rows are scattered over the table."""

    def __init__(self, seed: int, rows: int, s: float = 1.1):
        rng = np.random.Generator(np.random.PCG64(seed))
        self.perm = rng.permutation(rows)
        w = np.arange(1, rows + 1, dtype=np.float64) ** (-s)
        self.cdf = np.cumsum(w)
        self.cdf /= self.cdf[-1]

    def top(self, k: int) -> np.ndarray:
        """The k most popular rows, increasing."""
        return np.sort(self.perm[:k]).astype(np.uint64)

    def sample(self, seed: int, count: int) -> np.ndarray:
        rng = np.random.Generator(np.random.PCG64(seed))
        ranks = np.searchsorted(self.cdf, rng.random(count), side="right")
        return self.perm[np.minimum(ranks, self.perm.size - 1)].astype(np.uint64)


def poisson_arrivals(seed: int, rate_qps: float, count: int) -> np.ndarray:
    """Arrival times in seconds of a Poisson process with the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_qps, size=count))


def uniform_tables(seed: int, ntables: int, count: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, ntables, size=count, dtype=np.int32)


def domain_bits(rows: int) -> int:
    """n = ceil(log2 rows), at least 1."""
    return max(1, (int(rows) - 1).bit_length())
