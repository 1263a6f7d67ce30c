"""The oracle's pins must catch plausible mistakes.

Each case copies the oracle into a temporary tree, plants one mistake in the
copy of dpf_oracle.c (on the CPU; the real oracle is untouched), and runs the
oracle pin tests there.  The pin suite has to fail for every mutant.
"""
import os
import shutil
import subprocess
import sys

import pytest

from conftest import ROOT

MUTANTS = {
    # dropped term: the codeword is not applied during the tree expansion
    "drop_codeword_fulleval": ("next[16 * jd + i] = (uint8_t)(prf[i] ^ cw[i]);",
                               "next[16 * jd + i] = (uint8_t)(prf[i]);"),
    # wrong sign: party 1 does not negate its leaf share
    "no_party_negation": ("return party ? (uint32_t)(0u - y) : y;", "return y;"),
    # wrong index: codeword selected by the child bit instead of the parent's control bit
    "codeword_by_child_bit": ("const uint8_t* cw = codeword(key, d, lsb(parent), b);",
                              "const uint8_t* cw = codeword(key, d, b, b);"),
    # wrong index: path bits taken least-significant first in the branch walk
    "lsb_first_path": ("int b = (int)((j >> (n - d)) & 1); /* \"j mod 2\"",
                       "int b = (int)((j >> (d - 1)) & 1); /* \"j mod 2\""),
    # transposed operands: PRF keyed by the message instead of the node
    "prf_key_message_swapped": ("orc_aes128_encrypt(s, msg, out);", "orc_aes128_encrypt(msg, s, out);"),
    # wrong constant in MixColumns
    "mixcolumns_coefficient": ("state[0][c] = (uint8_t)(mul2(s0) ^ mul3(s1) ^ s2 ^ s3);",
                               "state[0][c] = (uint8_t)(mul2(s0) ^ mul2(s1) ^ s2 ^ s3);"),
    # wrong reduction polynomial in xtime
    "xtime_polynomial": ("return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1b : 0x00));",
                         "return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1d : 0x00));"),
    # wrong round-constant progression
    "rcon_step": ("rcon = gf_mul(rcon, 0x02);", "rcon = gf_mul(rcon, 0x03);"),
    # output correction without the control-bit sign
    "cw_out_sign": ("uint32_t cw_out = lsb(v[1]) ? (uint32_t)(0u - diff) : diff;", "uint32_t cw_out = diff;"),
    # inner product against the wrong column
    "answer_wrong_column": ("out[w] += y[j] * row[w];", "out[w] += y[j] * row[0];"),
    # ChaCha20 quarter round with a wrong rotation
    "chacha_rotation": ("*b ^= *c; *b = rotl32(*b, 12);", "*b ^= *c; *b = rotl32(*b, 13);"),
    # ChaCha20 PRF taking the wrong slice of the block
    "chacha_slice": ("memcpy(out, block + 16 * x, 16);", "memcpy(out, block + 32 * x, 16);"),
    # ShiftRows in the wrong direction
    "shiftrows_direction": ("tmp[r][c] = state[r][(c + r) % 4];", "tmp[r][c] = state[r][(c + 4 - r) % 4];"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "dpf_oracle.c")).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    for sub in ("oracle", "workloads"):
        shutil.copytree(os.path.join(ROOT, sub), tmp_path / sub,
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
    (tmp_path / "tests").mkdir()
    for f in ("conftest.py", "test_oracle_aes.py", "test_oracle_dpf.py", "test_oracle_chacha.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tmp_path / "tests" / "golden")
    (tmp_path / "oracle" / "dpf_oracle.c").write_text(src.replace(old, new))
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "tests"],
                         cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert res.returncode == 1, f"mutant {name} survived the pins:\n{res.stdout[-2000:]}"
