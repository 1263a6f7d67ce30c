"""The seeded input generators: host and torch paths agree bit for bit, and
the SplitMix64 stream matches the published generator's sequential form."""
import numpy as np

import workloads as wl

M64 = (1 << 64) - 1


def _splitmix64_sequential(seed, count):
    # the published generator: state += GAMMA, then mix (plain Python ints)
    out, state = [], seed
    for _ in range(count):
        state = (state + wl.GAMMA) & M64
        z = state
        z = ((z ^ (z >> 30)) * wl.MIX1) & M64
        z = ((z ^ (z >> 27)) * wl.MIX2) & M64
        out.append(z ^ (z >> 31))
    return out


def test_stream_matches_sequential_generator():
    got = wl.splitmix64_stream(12345, 0, 50).tolist()
    assert got == _splitmix64_sequential(12345, 50)
    assert wl.splitmix64_stream(12345, 10, 5).tolist() == got[10:15]


def test_torch_table_equals_numpy_table():
    import torch

    a = wl.table_u32(77, 3000, 12)
    b = wl.table_u32_torch(77, 3000, 12, "cpu", chunk_rows=1000).numpy().view(np.uint32)
    assert np.array_equal(a, b)
    assert np.array_equal(wl.table_rows_u32(77, 12, [0, 1234, 2999]), a[[0, 1234, 2999]])
    assert a.dtype == np.uint32 and len(np.unique(a)) > 35000


def test_zipf_assignment_follows_rank_order():
    t = wl.zipf_assignment(1, 8, 20000)
    counts = np.bincount(t, minlength=8)
    assert all(counts[i] > counts[i + 1] for i in range(7))
    assert 0.38 < counts[0] / t.size < 0.42  # 1 / H_{8,1.1} ~ 0.398


def test_poisson_rate():
    t = wl.poisson_arrivals(3, 1000.0, 20000)
    assert abs(t[-1] - 20.0) < 0.6
