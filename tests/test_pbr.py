"""Partial batch retrieval (Sec. 4, batch PIR) and batch key generation on
the host: the oracle's bin plan against a worked example, the oracle's bin
answers against the reconstruction closed form, and the library's client
side (pir_keygen_batch, pir_pbr_keygen) against the oracle.  No GPU needed."""
import numpy as np
import pytest

import workloads as wl

M32 = 0xFFFFFFFF


@pytest.fixture(scope="module")
def pir():
    import __graft_entry__ as g

    g.build_library()
    import paper_2301_10904_gb300 as pir

    return pir


def test_pbr_plan_worked_example(orc):
    # 10 rows in bins of 4: {0..3}, {4..7}, {8, 9}.  Index 5 claims bin 1, 1 claims
    # bin 0, 6 falls in bin 1 again and is dropped, 9 claims bin 2.
    alphas, betas, kept = orc.pbr_plan(10, 4, [5, 1, 6, 9])
    assert alphas == [1, 1, 1] and betas == [1, 1, 1] and kept == [True, True, False, True]
    # nobody asks for bin 1: it gets the dummy query
    alphas, betas, kept = orc.pbr_plan(10, 4, [2, 8])
    assert alphas == [2, 0, 0] and betas == [1, 0, 1] and kept == [True, True]
    assert orc.pbr_plan(8, 4, []) == ([0, 0], [0, 0], [])


def test_pbr_answer_reconstructs_kept_rows_and_zero_for_dummies(orc):
    rows, bin_rows, W = 1000, 128, 5  # 8 bins, the last of 104 rows
    T = wl.table_u32(9, rows, W)
    n = (bin_rows - 1).bit_length()
    wanted = [130, 999, 3, 140, 500]
    alphas, betas, kept = orc.pbr_plan(rows, bin_rows, wanted)
    rnd = wl.key_randomness(10, n, len(alphas))
    pairs = [orc.gen(n, a, b, r0, r1, c0) for (r0, r1, c0), a, b in zip(rnd, alphas, betas)]
    s0 = orc.pbr_answer([p[0] for p in pairs], T, bin_rows)
    s1 = orc.pbr_answer([p[1] for p in pairs], T, bin_rows)
    rec = (s0.astype(np.uint64) + s1) & M32
    for i, idx in enumerate(wanted):
        if kept[i]:
            assert np.array_equal(rec[idx // bin_rows], T[idx])
    for b in range(len(alphas)):
        if betas[b] == 0:
            assert not rec[b].any()
    assert kept == [True, True, True, False, True]


def _ctr_seed_blocks(master: bytes, count: int) -> list[bytes]:
    """32-byte blocks of AES-128-CTR keyed by master[:16], counter block master[16:]
    read little-endian and incremented per block (the library's documented stream)."""
    Cipher = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    algorithms = Cipher.algorithms
    modes = Cipher.modes
    enc = Cipher.Cipher(algorithms.AES(master[:16]), modes.ECB()).encryptor()
    ctr = int.from_bytes(master[16:], "little")
    stream = b"".join(enc.update(((ctr + i) % (1 << 128)).to_bytes(16, "little")) for i in range(2 * count))
    return [stream[32 * i:32 * i + 32] for i in range(count)]


def test_keygen_batch_equals_single_keygen_with_derived_seeds(pir):
    n, count = 9, 13
    master = bytes(range(32))
    alphas = [(i * 37) % 512 for i in range(count)]
    betas = [i * 1000 + 1 for i in range(count)]
    k0, k1 = pir.pir_keygen_batch(n, alphas, betas, seed=master, threads=3)
    kb = pir.pir_key_bytes(n)
    seeds = _ctr_seed_blocks(master, count)
    for i in range(count):
        a0, a1 = pir.pir_keygen_prf(n, alphas[i], betas[i], pir.PIR_PRF_AES128, seeds[i])
        assert k0[i * kb:(i + 1) * kb] == a0 and k1[i * kb:(i + 1) * kb] == a1
    # thread count does not change the keys
    assert pir.pir_keygen_batch(n, alphas, betas, seed=master, threads=1) == (k0, k1)


def test_keygen_batch_keys_satisfy_identity_under_oracle(pir, orc):
    n = 6
    alphas = [0, 63, 17, 17, 40]
    k0, k1 = pir.pir_keygen_batch(n, alphas, None, prf=pir.PIR_PRF_CHACHA20, seed=b"\x07" * 32)
    kb = pir.pir_key_bytes(n)
    for i, a in enumerate(alphas):
        s = (orc.full_eval(k0[i * kb:(i + 1) * kb], 64).astype(np.uint64) +
             orc.full_eval(k1[i * kb:(i + 1) * kb], 64)) & M32
        want = np.zeros(64, np.uint64)
        want[a] = 1
        assert np.array_equal(s, want)


@pytest.mark.parametrize("rows,bin_rows", [(1000, 128), (4096, 1024), (37, 2), (300, 300), (301, 300)])
def test_library_pbr_keys_follow_the_oracle_plan(pir, orc, rows, bin_rows):
    rng = np.random.Generator(np.random.PCG64(rows + bin_rows))
    wanted = rng.integers(0, rows, 12).tolist()
    k0, k1, kept = pir.pir_pbr_keygen(rows, bin_rows, wanted, seed=b"\x01" * 32)
    alphas, betas, want_kept = orc.pbr_plan(rows, bin_rows, wanted)
    assert kept.tolist() == want_kept
    nb = pir.pir_domain_bits(bin_rows)
    kb = pir.pir_key_bytes(nb)
    nbins = len(alphas)
    assert len(k0) == len(k1) == nbins * kb
    T = wl.table_u32(rows, rows, 3)
    keys0 = [k0[b * kb:(b + 1) * kb] for b in range(nbins)]
    keys1 = [k1[b * kb:(b + 1) * kb] for b in range(nbins)]
    rec = (orc.pbr_answer(keys0, T, bin_rows).astype(np.uint64) + orc.pbr_answer(keys1, T, bin_rows)) & M32
    for b in range(nbins):
        lo = b * bin_rows
        want = T[lo + alphas[b]] if betas[b] else np.zeros(3, np.uint32)
        assert np.array_equal(rec[b], want), b


def test_pbr_keygen_errors(pir):
    with pytest.raises(pir.PirError):
        pir.pir_pbr_keygen(100, 1, [3])  # bins of one row
    with pytest.raises(pir.PirError):
        pir.pir_pbr_keygen(100, 10, [100])  # index past the table
