"""The library's client side (host C++): keys from pir_keygen are checked by
the oracle's evaluation against the DPF identity (Sec. 3.1), and the oracle's
keys are accepted by the library's key validation.  No GPU needed."""
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


def _seed(i):
    return bytes((i * 37 + k) & 0xFF for k in range(32))


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_library_keys_satisfy_identity_under_oracle(pir, orc, n):
    L = 1 << n
    for alpha in sorted({0, L - 1, L // 2, (L * 3) // 5}):
        for beta in (1, M32, 0x12345678):
            k0, k1 = pir.pir_keygen(n, alpha, beta, _seed(alpha + n))
            s = (orc.full_eval(k0, L).astype(np.uint64) + orc.full_eval(k1, L)) & M32
            want = np.zeros(L, np.uint64)
            want[alpha] = beta
            assert np.array_equal(s, want)


def test_library_keys_reconstruct_table_row_under_oracle(pir, orc):
    L, W = 1000, 7
    T = wl.table_u32(3, L, W)
    n = pir.pir_domain_bits(L)
    for alpha in (0, 999, 512):
        k0, k1 = pir.pir_keygen(n, alpha, 1, _seed(alpha))
        s = pir.pir_reconstruct(orc.answer(k0, T), orc.answer(k1, T))
        assert np.array_equal(s, T[alpha])


def test_keygen_is_deterministic_per_seed_and_random_without(pir):
    a = pir.pir_keygen(10, 5, 1, _seed(1))
    b = pir.pir_keygen(10, 5, 1, _seed(1))
    c = pir.pir_keygen(10, 5, 1, _seed(2))
    d = pir.pir_keygen(10, 5, 1, None)
    e = pir.pir_keygen(10, 5, 1, None)
    assert a == b and a != c and d != e


def test_key_layout_matches_oracle_parse(pir, orc):
    k0, k1 = pir.pir_keygen(12, 100, 9, _seed(4))
    assert len(k0) == pir.pir_key_bytes(12) == orc.key_bytes(12)
    n0, p0, cw0 = orc.key_parse(k0)
    n1, p1, cw1 = orc.key_parse(k1)
    assert (n0, p0, n1, p1) == (12, 0, 12, 1) and cw0 == cw1
    assert k0[32:] == k1[32:]  # both servers receive the same codewords
    assert pir.pir_key_check(k0) == (12, 0) and pir.pir_key_check(k1) == (12, 1)


def test_library_accepts_oracle_keys_and_rejects_garbage(pir, orc):
    r0, r1, c0 = wl.key_randomness(1, 6, 1)[0]
    k0, k1 = orc.gen(6, 17, 1, r0, r1, c0)
    assert pir.pir_key_check(k0) == (6, 0)
    assert pir.pir_key_check(k1) == (6, 1)
    bad = bytearray(k0)
    bad[1] = 0
    with pytest.raises(pir.PirError):
        pir.pir_key_check(bytes(bad))
    bad = bytearray(k0)
    bad[6] = 3
    with pytest.raises(pir.PirError):
        pir.pir_key_check(bytes(bad))
    with pytest.raises(pir.PirError):
        pir.pir_key_check(k0[:-1])


def test_keygen_argument_errors(pir):
    with pytest.raises(pir.PirError):
        pir.pir_keygen(4, 16, 1, None)  # alpha >= 2^n
    with pytest.raises(pir.PirError):
        pir.pir_keygen(0, 0, 1, None)


def test_reconstruct_wraps_mod_2_32(pir):
    s = pir.pir_reconstruct(np.array([M32, 5], np.uint32), np.array([2, M32], np.uint32))
    assert s.tolist() == [1, 4]


def test_library_chacha_keys_satisfy_identity_under_oracle(pir, orc):
    for n in (1, 4, 9):
        L = 1 << n
        for alpha in (0, L - 1, L // 3):
            k0, k1 = pir.pir_keygen_prf(n, alpha, 5, pir.PIR_PRF_CHACHA20, _seed(alpha + 3 * n))
            assert k0[7] == 1 and k1[7] == 1 and pir.pir_key_check(k0) == (n, 0)
            s = (orc.full_eval(k0, L).astype(np.uint64) + orc.full_eval(k1, L)) & M32
            want = np.zeros(L, np.uint64)
            want[alpha] = 5
            assert np.array_equal(s, want)


def test_keygen_rejects_unknown_prf(pir):
    with pytest.raises(pir.PirError):
        pir.pir_keygen_prf(4, 1, 1, 7, None)
