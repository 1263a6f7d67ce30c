"""Pins for the oracle's AES-128 (the PRF of Sec. 3.2.6) against FIPS-197.

Each check is independent of the oracle's own code: published vectors
(tests/golden/), and a second AES implementation (Python `cryptography`,
i.e. OpenSSL) run on random keys and blocks where it is installed.
"""
import os

import numpy as np
import pytest

from conftest import read_golden


def test_gf_mul_and_sbox_examples(orc):
    for op, a, b, res in read_golden("gf256_fips197.txt"):
        if op == "mul":
            assert orc.gf_mul(int(a, 16), int(b, 16)) == int(res, 16)
        else:
            assert orc.sbox()[int(a, 16)] == int(res, 16)


def test_sbox_is_a_permutation_with_no_fixed_points(orc):
    # FIPS-197 Sec. 5.1.1: the S-box is invertible; its affine constant makes
    # S(x) != x and S(x) != ~x for every byte (a property of the published box).
    s = orc.sbox()
    assert sorted(s) == list(range(256))
    assert all(s[x] != x and s[x] != (x ^ 0xFF) for x in range(256))


def test_key_expansion_appendix_a1(orc):
    rows = read_golden("aes128_keyexp_fips197.txt")
    key = bytes.fromhex(rows[0][1])
    w = orc.aes128_key_expansion(key)
    for idx, word in rows[1:]:
        i = int(idx)
        assert w[4 * i:4 * i + 4].hex() == word


@pytest.mark.parametrize("row", read_golden("aes128_fips197.txt"), ids=lambda r: r[0])
def test_cipher_known_answers(orc, row):
    _, key, pt, ct = row
    assert orc.aes128_encrypt(bytes.fromhex(key), bytes.fromhex(pt)).hex() == ct


def test_cipher_matches_openssl_on_random_blocks(orc):
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    rng = np.random.Generator(np.random.PCG64(1234))
    for _ in range(64):
        key = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
        blk = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
        enc = ciphers.Cipher(ciphers.algorithms.AES(key), ciphers.modes.ECB()).encryptor()
        assert orc.aes128_encrypt(key, blk) == enc.update(blk) + enc.finalize()


def test_prf_is_aes_keyed_by_node_on_child_bit(orc):
    # Sec. 3.1, Eq. p3: PRF_s(x) is a cipher keyed by s applied to the message x.
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    seed = bytes(range(16, 32))
    for x in (0, 1):
        enc = ciphers.Cipher(ciphers.algorithms.AES(seed), ciphers.modes.ECB()).encryptor()
        msg = bytes([x]) + bytes(15)
        assert orc.prf(seed, x) == enc.update(msg) + enc.finalize()
