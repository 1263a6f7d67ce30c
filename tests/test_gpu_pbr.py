"""Partial batch retrieval on the GPU (pir_server_eval_pbr): every bin's share
bit-exact against the oracle (keys from the oracle and from the library's
client side), ragged last bins, tiny and wide bins, every bin-group size the
planner picks (by row width), reconstruction of every kept row, dummy bins
reconstructing to zero, bad keys, and refused layouts; one full-size case
(2^22 rows x 32 words, 1024 bins) checked by reconstruction and sampled bins."""
import numpy as np
import pytest

import workloads as wl
from test_gpu_parity import dev_keys, dev_table

pytestmark = pytest.mark.gpu
M32 = 0xFFFFFFFF


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    import oracle
    import paper_2301_10904_gb300 as pir

    return torch, pir, oracle


def _oracle_keys(orc, rows, bin_rows, wanted, seed):
    alphas, betas, kept = orc.pbr_plan(rows, bin_rows, wanted)
    n = (bin_rows - 1).bit_length()
    rnd = wl.key_randomness(seed, n, len(alphas))
    pairs = [orc.gen(n, a, b, r0, r1, c0) for (r0, r1, c0), a, b in zip(rnd, alphas, betas)]
    return [p[0] for p in pairs], [p[1] for p in pairs], alphas, betas, kept


def _run(torch, pir, table, bin_rows, keys, W, status=None):
    out = torch.full((len(keys), W), 7, dtype=torch.int32, device="cuda")
    pir.pir_server_eval_pbr(table, bin_rows, dev_keys(torch, keys), out, status)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("rows,bin_rows,W", [
    (4096, 1024, 64), (5000, 1024, 16), (1 << 14, 256, 32), (3000, 2, 4), (100, 64, 128), (2000, 512, 256),
    (1500, 700, 1024), (9 * 4096 + 5, 4096, 8), ((1 << 15) + 3, 1 << 11, 64),
    # bins of 1,000 rows are not a multiple of the scan's chunk: the bins kernel runs, and on 152 SMs the
    # planner cuts the 11 items past the first round (163 items of 8 bins) into 8 pieces each
    (1300 * 1000, 1000, 16)])
def test_pbr_matches_oracle(env, rows, bin_rows, W):
    torch, pir, orc = env
    T = wl.table_u32(rows + W, rows, W)
    rng = np.random.Generator(np.random.PCG64(rows * 7 + bin_rows))
    wanted = rng.integers(0, rows, max(1, rows // bin_rows)).tolist()
    ks0, ks1, alphas, betas, kept = _oracle_keys(orc, rows, bin_rows, wanted, rows + bin_rows)
    table = dev_table(torch, T)
    got0 = _run(torch, pir, table, bin_rows, ks0, W)
    got1 = _run(torch, pir, table, bin_rows, ks1, W)
    nbins = len(ks0)
    check = range(nbins) if nbins <= 64 else sorted({0, nbins - 1, *rng.integers(0, nbins, 24).tolist()})
    for b in check:
        lo = b * bin_rows
        assert np.array_equal(got0[b], orc.answer(ks0[b], T[lo:lo + bin_rows])), b
        assert np.array_equal(got1[b], orc.answer(ks1[b], T[lo:lo + bin_rows])), b
    rec = (got0.astype(np.uint64) + got1) & M32
    for i, idx in enumerate(wanted):
        if kept[i]:
            assert np.array_equal(rec[idx // bin_rows], T[idx])
    for b in range(nbins):
        if betas[b] == 0:
            assert not rec[b].any()


def test_pbr_with_library_client_keys_chacha(env):
    torch, pir, orc = env
    rows, bin_rows, W = 1 << 13, 512, 32
    T = wl.table_u32(77, rows, W)
    wanted = [0, 511, 512, 8191, 4000, 4001]
    k0, k1, kept = pir.pir_pbr_keygen(rows, bin_rows, wanted, prf=pir.PIR_PRF_CHACHA20, seed=b"\x05" * 32)
    # 511 shares bin 0 with 0, and 4001 bin 7 with 4000: both dropped
    assert kept.tolist() == [True, False, True, True, True, False]
    nbins, kb = rows // bin_rows, pir.pir_key_bytes(pir.pir_domain_bits(bin_rows))
    table = dev_table(torch, T)
    outs = []
    for keys in (k0, k1):
        out = torch.empty((nbins, W), dtype=torch.int32, device="cuda")
        pir.pir_server_eval_pbr(table, bin_rows, torch.frombuffer(bytearray(keys), dtype=torch.uint8).cuda(), out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy().view(np.uint32))
    for b in (0, 7, nbins - 1):
        assert np.array_equal(outs[0][b], orc.answer(k0[b * kb:(b + 1) * kb], T[b * bin_rows:(b + 1) * bin_rows]))
    rec = (outs[0].astype(np.uint64) + outs[1]) & M32
    for i, idx in enumerate(wanted):
        if kept[i]:
            assert np.array_equal(rec[idx // bin_rows], T[idx])


def test_pbr_bad_key_zero_share_and_status(env):
    torch, pir, orc = env
    rows, bin_rows, W = 2048, 256, 16
    T = wl.table_u32(5, rows, W)
    ks0, _, _, _, _ = _oracle_keys(orc, rows, bin_rows, [3, 700], 5)
    bad = bytearray(ks0[2])
    bad[0] ^= 0xFF  # magic
    ks0[2] = bytes(bad)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = _run(torch, pir, dev_table(torch, T), bin_rows, ks0, W, status)
    assert not got[2].any() and int(status.item()) & pir.PIR_STATUS_BAD_KEY
    assert np.array_equal(got[1], orc.answer(ks0[1], T[256:512]))


def test_pbr_refuses_bad_layouts(env):
    torch, pir, _ = env
    keys = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    out = torch.empty((8, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(pir.PirError) as e:
        pir.pir_server_eval_pbr(torch.zeros((64, 5), dtype=torch.int32, device="cuda"), 8, keys, out)
    assert e.value.code == -8  # rows not 16-byte multiples
    with pytest.raises(pir.PirError) as e:
        pir.pir_server_eval_pbr(torch.zeros((64, 8), dtype=torch.int32, device="cuda"), 1, keys, out)
    assert e.value.code == -1  # bins of one row


def test_pbr_full_size(env):
    """2^22 rows x 32 words (512 MiB), bins of 2^12 rows: 1024 bins in one launch."""
    torch, pir, orc = env
    rows, bin_rows, W = 1 << 22, 1 << 12, 32
    table = wl.table_u32_torch(42, rows, W, "cuda")
    rng = np.random.Generator(np.random.PCG64(42))
    wanted = rng.integers(0, rows, 1500).tolist()
    k0, k1, kept = pir.pir_pbr_keygen(rows, bin_rows, wanted, seed=b"\x2a" * 32)
    nbins, kb = rows // bin_rows, pir.pir_key_bytes(12)
    outs = []
    for keys in (k0, k1):
        out = torch.empty((nbins, W), dtype=torch.int32, device="cuda")
        pir.pir_server_eval_pbr(table, bin_rows, torch.frombuffer(bytearray(keys), dtype=torch.uint8).cuda(), out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy().view(np.uint32))
    rec = ((outs[0].astype(np.uint64) + outs[1]) & M32).astype(np.uint32)
    idx = np.array([w for w, k in zip(wanted, kept) if k], dtype=np.int64)
    want = table[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint32)
    assert np.array_equal(rec[idx // bin_rows], want)
    assert kept.sum() < len(wanted)  # 1500 draws over 1024 bins collide
    for b in (0, 511, nbins - 1):
        T = table[b * bin_rows:(b + 1) * bin_rows].cpu().numpy().view(np.uint32)
        assert np.array_equal(outs[0][b], orc.answer(k0[b * kb:(b + 1) * kb], T))


@pytest.mark.parametrize("rows,bin_rows,W", [(1 << 16, 1 << 10, 64), (5000, 1000, 16), (3000, 2, 4)])
def test_pbr_one_launch_equals_the_two_launch_forms(env, rows, bin_rows, W):
    """A dense table takes the one-launch kernel (trees breadth first, then each
    CTA's own rows); the same rows at a padded stride take the expand-and-scan
    or the bins kernel.  Both give the oracle's shares word for word, with a
    bad key among the bins (zero share, status bit), and the status words agree."""
    torch, pir, orc = env
    T = wl.table_u32(rows + bin_rows + W, rows, W)
    rng = np.random.Generator(np.random.PCG64(rows + W))
    wanted = rng.integers(0, rows, max(1, rows // bin_rows)).tolist()
    ks0, _, _, _, _ = _oracle_keys(orc, rows, bin_rows, wanted, rows + 3)
    bad = bytearray(ks0[1])
    bad[0] ^= 0xFF  # magic
    ks0[1] = bytes(bad)
    dense = dev_table(torch, T)
    padded_full = torch.zeros((rows, W + 4), dtype=torch.int32, device="cuda")
    padded_full[:, :W] = dense
    padded = padded_full[:, :W]
    outs, stats = [], []
    for table in (dense, padded):
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        outs.append(_run(torch, pir, table, bin_rows, ks0, W, status))
        stats.append(int(status.item()))
    assert np.array_equal(outs[0], outs[1])
    assert stats[0] == stats[1] and stats[0] & pir.PIR_STATUS_BAD_KEY
    assert not outs[0][1].any()
    nbins = len(ks0)
    for b in sorted({0, nbins - 1, *rng.integers(0, nbins, 6).tolist()} - {1}):
        lo = b * bin_rows
        assert np.array_equal(outs[0][b], orc.answer(ks0[b], T[lo:lo + bin_rows])), b
