"""Pins for the oracle's DPF (Sec. 3.1, Eqs. p1-p3) and server answer.

None of these restates the oracle's arithmetic: they check what the paper and
the mathematics fix — the DPF correctness identity (Sec. 3.1) by brute force,
agreement of two different evaluation orders, the paper's L=4 dependency
example, the key-size law of Table 4, linearity over index ranges
(Sec. 3.2.7), and reconstruction of T[alpha] (Sec. 3.1).
"""
import numpy as np
import pytest

import workloads as wl
from conftest import read_golden

M32 = 0xFFFFFFFF


def _keys(orc, n, alpha, beta, seed):
    r0, r1, c0 = wl.key_randomness(seed, n, 1)[0]
    return orc.gen(n, alpha, beta, r0, r1, c0)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_correctness_identity_every_alpha(orc, n):
    # Eval(k_a, j) + Eval(k_b, j) = beta * [j == alpha] for every alpha, j.
    L = 1 << n
    rng = np.random.Generator(np.random.PCG64(n))
    for alpha in range(L):
        beta = int(rng.integers(0, 1 << 32))
        k0, k1 = _keys(orc, n, alpha, beta, 1000 * n + alpha)
        s = (orc.full_eval(k0, L).astype(np.uint64) + orc.full_eval(k1, L)) & M32
        want = np.zeros(L, np.uint64)
        want[alpha] = beta
        assert np.array_equal(s, want), (n, alpha)


@pytest.mark.parametrize("n", [7, 10])
def test_correctness_identity_brute_force_larger_domains(orc, n):
    L = 1 << n
    alphas = range(L) if n <= 7 else wl.alphas(77, L, 48).tolist() + [0, L - 1]
    for alpha in alphas:
        k0, k1 = _keys(orc, n, int(alpha), 1, int(alpha) + 7)
        s = (orc.full_eval(k0, L).astype(np.uint64) + orc.full_eval(k1, L)) & M32
        nz = np.nonzero(s)[0]
        assert nz.tolist() == [alpha] and s[alpha] == 1


def test_beta_extremes_and_domain_edges(orc):
    for n in (1, 3, 9):
        L = 1 << n
        for alpha in (0, L - 1):
            for beta in (0, 1, M32, 0x80000000):
                k0, k1 = _keys(orc, n, alpha, beta, alpha + beta % 97)
                s = (orc.full_eval(k0, L).astype(np.uint64) + orc.full_eval(k1, L)) & M32
                want = np.zeros(L, np.uint64)
                want[alpha] = beta
                assert np.array_equal(s, want)


def test_shares_alone_look_nothing_like_the_indicator(orc):
    # Each share vector on its own is pseudorandom: no party sees the point.
    k0, k1 = _keys(orc, 10, 333, 1, 5)
    y0 = orc.full_eval(k0, 1024)
    assert len(np.unique(y0)) > 1000


@pytest.mark.parametrize("n", [3, 8])
def test_tree_order_equals_branch_order(orc, n):
    # FullEval (every node once, level by level) == Eval(k, j) per index
    # (root-to-leaf walk), for both parties.
    L = 1 << n
    for seed in range(3):
        for k in _keys(orc, n, seed * 5 % L, 12345, seed):
            full = orc.full_eval(k, L)
            point = np.array([orc.eval_point(k, j) for j in range(L)], np.uint32)
            assert np.array_equal(full, point)


def test_off_path_nodes_equal_on_path_control_bits_differ(orc):
    # BGI16 invariant behind the identity: below depth d, the two keys'
    # nodes agree off the alpha path; on it their control bits (lsb) differ.
    n = 6
    for alpha in (0, 21, 63):
        k0, k1 = _keys(orc, n, alpha, 1, alpha)
        for d in range(0, n + 1):
            for j in range(1 << d):
                a = orc.node(k0, d, j)
                b = orc.node(k1, d, j)
                if j == alpha >> (n - d):
                    assert (a[0] ^ b[0]) & 1 == 1
                else:
                    assert a == b


def test_paper_l4_example_dependency(orc):
    # Sec. 3.1 worked example, L = 4: Eval(k, 3) = P(2, 3) needs P(1, 1),
    # which needs P(0, 0).  So the depth-1 codewords for child bit 1 can
    # change only leaves 2 and 3, and the depth-2 codewords for child bit 1
    # only the odd leaves.
    k0, _ = _keys(orc, 2, 1, 1, 3)
    base = orc.full_eval(k0, 4)
    for d, b, expect_changed in ((1, 1, {2, 3}), (1, 0, {0, 1}), (2, 1, {1, 3}), (2, 0, {0, 2})):
        union = set()
        for t in (0, 1):
            mutated = bytearray(k0)
            off = 32 + 64 * (d - 1) + 32 * t + 16 * b
            for i in range(16):
                mutated[off + i] ^= 0x5A
            after = orc.full_eval(bytes(mutated), 4)
            union |= {j for j in range(4) if after[j] != base[j]}
        assert union == expect_changed, (d, b, union)


def test_child_is_aes_of_parent_xor_codeword(orc):
    # Independent AES (OpenSSL): P(1, b) = AES_{P(0,0)}(b || 0^120) ^ C_t[b][1],
    # t = lsb(P(0,0)).  Pins the PRF's orientation and plaintext encoding.
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    for party_key in _keys(orc, 3, 5, 1, 11):
        root = party_key[16:32]
        t = root[0] & 1
        for b in (0, 1):
            enc = ciphers.Cipher(ciphers.algorithms.AES(root), ciphers.modes.ECB()).encryptor()
            prf = enc.update(bytes([b]) + bytes(15)) + enc.finalize()
            off = 32 + 32 * t + 16 * b
            want = bytes(x ^ y for x, y in zip(prf, party_key[off:off + 16]))
            assert orc.node(party_key, 1, b) == want


@pytest.mark.parametrize("row", read_golden("key_size_table4.txt"), ids=lambda r: r[0])
def test_key_size_law_table4(orc, row):
    entries, n, paper_bytes = (int(x) for x in row)
    assert wl.domain_bits(entries) == n
    assert orc.key_bytes(n) - 32 == paper_bytes
    k0, k1 = _keys(orc, n, entries - 1, 1, n)
    assert len(k0) == len(k1) == 32 + paper_bytes


def test_reconstruction_returns_the_row(orc):
    # Sec. 3.1: T x (Eval(k_a) + Eval(k_b)) = T x I(alpha) = T[alpha].
    for L, W in ((1 << 9, 16), (1000, 5), (2, 1), (777, 64)):
        n = wl.domain_bits(L)
        T = wl.table_u32(99, L, W)
        for alpha in (0, L - 1, L // 3):
            for beta in (1, 7):
                k0, k1 = _keys(orc, n, alpha, beta, alpha + L)
                got = orc.reconstruct(orc.answer(k0, T), orc.answer(k1, T))
                want = (T[alpha].astype(np.uint64) * beta) & M32
                assert np.array_equal(got, want.astype(np.uint32))


def test_answer_is_linear_over_index_ranges(orc):
    # Sec. 3.2.7: the final reduction is a sum, so shares over disjoint index
    # ranges add up to the full share.
    L, W = 1 << 10, 8
    T = wl.table_u32(5, L, W)
    k0, _ = _keys(orc, 10, 600, 1, 2)
    full = orc.answer(k0, T)
    cuts = [0, 1, 255, 256, 700, 1023, 1024]
    parts = np.zeros(W, np.uint64)
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        parts += orc.answer(k0, T, lo, hi)
    assert np.array_equal((parts & M32).astype(np.uint32), full)


def test_non_power_of_two_domain_ignores_padding_leaves(orc):
    # L = 1000 uses n = 10; leaves 1000..1023 exist in the tree but are unused.
    L = 1000
    k0, k1 = _keys(orc, 10, 999, 3, 8)
    y0 = orc.full_eval(k0, L)
    assert np.array_equal(y0, orc.full_eval(k0, 1024)[:L])
    s = (y0.astype(np.uint64) + orc.full_eval(k1, L)) & M32
    assert s[999] == 3 and np.count_nonzero(s) == 1


def test_key_rejects_garbage(orc):
    k0, _ = _keys(orc, 4, 3, 1, 1)
    bad = bytearray(k0)
    bad[0] = ord("X")
    with pytest.raises(ValueError):
        orc.eval_point(bytes(bad), 0)
    bad = bytearray(k0)
    bad[6] = 2
    with pytest.raises(ValueError):
        orc.full_eval(bytes(bad), 16)


def test_contract_one_hot_selects_rows_and_agrees_with_answer(orc):
    # closed form: a one-hot share matrix selects table rows (times beta)
    L, W = 300, 9
    T = wl.table_u32(12, L, W)
    S = np.zeros((3, L), np.uint32)
    S[0, 0] = 1
    S[1, L - 1] = M32  # -1 mod 2^32
    S[2, 7] = 3
    out = orc.contract(S, T)
    assert np.array_equal(out[0], T[0])
    assert np.array_equal(out[1], ((-T[L - 1].astype(np.int64)) & M32).astype(np.uint32))
    assert np.array_equal(out[2], ((T[7].astype(np.uint64) * 3) & M32).astype(np.uint32))
    # the product with a full share vector is the server answer
    k0, _ = _keys(orc, wl.domain_bits(L), 5, 1, 9)
    assert np.array_equal(orc.contract(orc.full_eval(k0, L)[None, :], T)[0], orc.answer(k0, T))


def test_contract_wraps_like_python_integers(orc):
    rng = np.random.Generator(np.random.PCG64(3))
    S = rng.integers(0, 1 << 32, (4, 50), dtype=np.uint64).astype(np.uint32)
    T = rng.integers(0, 1 << 32, (50, 3), dtype=np.uint64).astype(np.uint32)
    out = orc.contract(S, T)
    for b in range(4):
        for w in range(3):
            assert int(out[b, w]) == sum(int(S[b, k]) * int(T[k, w]) for k in range(50)) % (1 << 32)
