"""Pins for the oracle's ChaCha20 PRF (the alternative PRF of Sec. 3.2.6,
Table 5): RFC 8439 vectors, OpenSSL's ChaCha20 on random inputs, and the DPF
correctness identity with ChaCha20 in place of AES-128."""
import numpy as np
import pytest

import workloads as wl
from conftest import read_golden

M32 = 0xFFFFFFFF


def test_rfc8439_vectors(orc):
    for row in read_golden("chacha20_rfc8439.txt"):
        if row[0] == "qr":
            words = [int(x, 16) for x in row[1:]]
            assert orc.chacha_quarter_round(*words[:4]) == tuple(words[4:])
        else:
            _, key, ctr, nonce, block = row
            assert orc.chacha20_block(bytes.fromhex(key), int(ctr), bytes.fromhex(nonce)).hex() == block


def test_block_matches_openssl(orc):
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    rng = np.random.Generator(np.random.PCG64(8439))
    for _ in range(32):
        key = rng.integers(0, 256, 32, dtype=np.uint8).tobytes()
        nonce = rng.integers(0, 256, 12, dtype=np.uint8).tobytes()
        ctr = int(rng.integers(0, 1 << 32))
        enc = ciphers.Cipher(ciphers.algorithms.ChaCha20(key, ctr.to_bytes(4, "little") + nonce), mode=None).encryptor()
        assert orc.chacha20_block(key, ctr, nonce) == enc.update(bytes(64))


def test_prf_is_block_zero_under_seed_and_zero_half(orc):
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    seed = bytes(range(100, 116))
    enc = ciphers.Cipher(ciphers.algorithms.ChaCha20(seed + bytes(16), bytes(16)), mode=None).encryptor()
    ks = enc.update(bytes(32))
    assert orc.prf(seed, 0, orc.PRF_CHACHA20) == ks[:16]
    assert orc.prf(seed, 1, orc.PRF_CHACHA20) == ks[16:32]


@pytest.mark.parametrize("n", [1, 3, 6])
def test_identity_with_chacha_every_alpha(orc, n):
    L = 1 << n
    for alpha in range(L):
        r0, r1, c0 = wl.key_randomness(50 * n + alpha, n, 1)[0]
        k0, k1 = orc.gen(n, alpha, 7, r0, r1, c0, orc.PRF_CHACHA20)
        assert k0[7] == 1 and k1[7] == 1
        s = (orc.full_eval(k0, L).astype(np.uint64) + orc.full_eval(k1, L)) & M32
        want = np.zeros(L, np.uint64)
        want[alpha] = 7
        assert np.array_equal(s, want)


def test_chacha_tree_equals_branch_and_differs_from_aes(orc):
    r0, r1, c0 = wl.key_randomness(3, 8, 1)[0]
    kc, _ = orc.gen(8, 100, 1, r0, r1, c0, orc.PRF_CHACHA20)
    ka, _ = orc.gen(8, 100, 1, r0, r1, c0, orc.PRF_AES128)
    full = orc.full_eval(kc, 256)
    assert np.array_equal(full, np.array([orc.eval_point(kc, j) for j in range(256)], np.uint32))
    assert not np.array_equal(full, orc.full_eval(ka, 256))


def test_child_under_chacha_is_block_slice_xor_codeword(orc):
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    r0, r1, c0 = wl.key_randomness(4, 3, 1)[0]
    for key in orc.gen(3, 5, 1, r0, r1, c0, orc.PRF_CHACHA20):
        root = key[16:32]
        t = root[0] & 1
        enc = ciphers.Cipher(ciphers.algorithms.ChaCha20(root + bytes(16), bytes(16)), mode=None).encryptor()
        ks = enc.update(bytes(32))
        for b in (0, 1):
            off = 32 + 32 * t + 16 * b
            assert orc.node(key, 1, b) == bytes(x ^ y for x, y in zip(ks[16 * b:16 * b + 16], key[off:off + 16]))
