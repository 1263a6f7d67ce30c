"""The materialised baseline (expansion to a share matrix in HBM, then the
share-matrix x table product) against the oracle, and against the fused path."""
import numpy as np
import pytest

import workloads as wl
from test_gpu_parity import dev_keys, dev_table, make_keys

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


@pytest.mark.parametrize("rows,batch,pad", [(2, 1, 0), (3, 2, 1), (1000, 9, 3), (4096, 8, 0), ((1 << 15) + 17, 5, 4),
                                            (1 << 14, 17, 0)])
def test_materialised_shares_match_oracle_full_eval(env, rows, batch, pad):
    torch, pir, orc = env
    n = pir.pir_domain_bits(rows)
    alphas = wl.alphas(rows + 1, rows, batch)
    ks0, _ = make_keys(orc, n, alphas, [1] * batch, rows + 2)
    ld = rows + pad
    S = torch.full((batch, ld), -1, dtype=torch.int32, device="cuda")
    pir.pir_expand_materialise(rows, dev_keys(torch, ks0), batch, S)
    torch.cuda.synchronize()
    got = S.cpu().numpy().view(np.uint32)
    for q in range(batch):
        assert np.array_equal(got[q, :rows], orc.full_eval(ks0[q], rows)), q
        assert (got[q, rows:] == M32).all()  # padding untouched


@pytest.mark.parametrize("rows,batch,pad", [(1024, 1024, 0), (1000, 300, 1), (8192, 152, 0), (5, 7, 0), (2, 64, 3),
                                            (3, 200, 0), (8191, 153, 2)])
def test_many_small_trees_match_oracle_full_eval(env, rows, batch, pad):
    """Batches of keys over small domains (partial batch retrieval's bins) run
    breadth first, several keys per CTA, where a CTA's keys fit its level
    buffers (8191 x 153 does not: two keys of 2^13 leaves per CTA, the item
    kernel instead).  Every share vector equals the oracle's FullEval, with
    AES-128 and ChaCha20 keys mixed in one batch, padded rows (odd ld) and one
    bad key, whose vector is zero and which sets the status bit."""
    torch, pir, orc = env
    n = pir.pir_domain_bits(rows)
    alphas = wl.alphas(rows + 3, rows, batch)
    rnd = wl.key_randomness(rows + batch, n, batch)
    keys = [orc.gen(n, int(a), 1 + q, r0, r1, c0, q % 2)[q % 3 == 1] for q, ((r0, r1, c0), a) in
            enumerate(zip(rnd, alphas))]
    bad_q = batch // 2
    bad = bytearray(keys[bad_q])
    bad[6] = 2  # party byte out of range
    keys[bad_q] = bytes(bad)
    ld = rows + pad
    S = torch.full((batch, ld), -1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    pir.pir_expand_materialise(rows, dev_keys(torch, keys), batch, S, status)
    torch.cuda.synchronize()
    got = S.cpu().numpy().view(np.uint32)
    for q in range(batch):
        if q == bad_q:
            assert not got[q, :rows].any()
        else:
            assert np.array_equal(got[q, :rows], orc.full_eval(keys[q], rows)), q
        assert (got[q, rows:] == M32).all()  # padding untouched
    assert int(status.item()) & pir.PIR_STATUS_BAD_KEY


def test_materialised_bad_key_gives_zero_vector_and_status(env):
    torch, pir, orc = env
    rows = 2000
    n = pir.pir_domain_bits(rows)
    ks0, _ = make_keys(orc, n, [3, 4], [1, 1], 5)
    bad = bytearray(ks0[1])
    bad[4] = 9  # version
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    S = torch.full((2, rows), 7, dtype=torch.int32, device="cuda")
    pir.pir_expand_materialise(rows, dev_keys(torch, [ks0[0], bytes(bad)]), 2, S, status)
    torch.cuda.synchronize()
    got = S.cpu().numpy().view(np.uint32)
    assert np.array_equal(got[0], orc.full_eval(ks0[0], rows))
    assert not got[1].any() and int(status.item()) & 1


@pytest.mark.parametrize("engine", [0, 1, 3, 4], ids=["imad", "mma_u8", "tc_f16", "auto"])
@pytest.mark.parametrize("B,L,W", [(1, 1, 1), (3, 100, 5), (64, 4096, 64), (70, 3000, 65), (256, 1 << 14, 16),
                                   (5, 777, 128), (9, 20000, 32), (6, 4096, 32), (20, 4096, 64),
                                   (32, 2048, 16), (33, 2048, 16),  # both sides of the AUTO switch, narrow rows
                                   (16, 2048, 64), (17, 2048, 64)])  # and wide rows
def test_contract_matches_oracle(env, B, L, W, engine):
    torch, pir, orc = env
    rng = np.random.Generator(np.random.PCG64(B * L + W))
    S = rng.integers(0, 1 << 32, (B, L), dtype=np.uint64).astype(np.uint32)
    if L >= 20000:
        S[:, :] = 0xFFFFFFFF  # every limb at its maximum: the largest accumulator values
    T = wl.table_u32(W, L, W)
    if L >= 20000:
        T[:, :] = 0xFFFFFFFF
    out = torch.empty((B, W), dtype=torch.int32, device="cuda")
    pir.pir_contract_u32(torch.from_numpy(S.view(np.int32)).cuda(), B, dev_table(torch, T), out, engine=engine)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), orc.contract(S, T))


def test_materialised_pipeline_equals_fused_and_oracle(env):
    torch, pir, orc = env
    rows, width, batch = (1 << 13) + 5, 32, 12
    n = pir.pir_domain_bits(rows)
    T = wl.table_u32(31, rows, width)
    alphas = wl.alphas(31, rows, batch)
    ks0, ks1 = make_keys(orc, n, alphas, [1] * batch, 31)
    table = dev_table(torch, T)
    outs = []
    for keys in (ks0, ks1):
        dk = dev_keys(torch, keys)
        S = torch.empty((batch, rows), dtype=torch.int32, device="cuda")
        pir.pir_expand_materialise(rows, dk, batch, S)
        mat = torch.empty((batch, width), dtype=torch.int32, device="cuda")
        pir.pir_contract_u32(S, batch, table, mat)
        mma = torch.empty_like(mat)
        pir.pir_contract_u32(S, batch, table, mma, engine=pir.PIR_CONTRACT_MMA_U8)
        tc = torch.empty_like(mat)
        pir.pir_contract_u32(S, batch, table, tc, engine=pir.PIR_CONTRACT_TC_F16)
        fused = torch.empty_like(mat)
        pir.pir_server_eval_device(table, dk, batch, fused)
        torch.cuda.synchronize()
        m = mat.cpu().numpy().view(np.uint32)
        assert np.array_equal(m, fused.cpu().numpy().view(np.uint32))
        assert torch.equal(mma, mat)
        assert torch.equal(tc, mat)
        for q in (0, batch - 1):
            assert np.array_equal(m[q], orc.answer(keys[q], T))
        outs.append(m)
    rec = (outs[0].astype(np.uint64) + outs[1]) & M32
    assert np.array_equal(rec.astype(np.uint32), T[alphas])


# The tcgen05 engine has two kernels with one result: for 16-byte-aligned operands
# the raw tiles arrive by tensor-map copies, otherwise (or with
# PIR_TC_TENSOR_MAPS=0) the conversion warps load them.  The tests below run both.
KERNELS = {"tensor_maps": "1", "loads": "0"}


@pytest.fixture(params=sorted(KERNELS))
def tc_kernel(request, monkeypatch):
    monkeypatch.setenv("PIR_TC_TENSOR_MAPS", KERNELS[request.param])
    return request.param


def _tc_contract(torch, pir, S, T, pad=0):
    B, L = S.shape
    Sd = torch.zeros((B, L + pad), dtype=torch.int32)
    Sd[:, :L] = torch.from_numpy(S.view(np.int32))
    out = torch.full((B, T.shape[1]), 5, dtype=torch.int32, device="cuda")
    pir.pir_contract_u32(Sd.cuda()[:, :L], B, dev_table(torch, T), out, engine=pir.PIR_CONTRACT_TC_F16)
    torch.cuda.synchronize()
    flags = pir.pir_device_status(clear=True)
    assert flags == 0, flags
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("B,L,W,pad", [
    (200, (1 << 16) + 77, 48, 0),   # 2 query tiles, several 256-k accumulator chunks per CTA, ragged k tail
    (200, (1 << 16) + 77, 48, 3),   # the same with 16-byte-aligned share rows
    (129, 5000, 96, 0),             # one row in the second query tile; two word tiles, the second ragged
    (128, 20000, 32, 0),            # the 32-word tile shape
    (37, 3001, 33, 2),              # unaligned rows (ld % 4 != 0: scalar loads), ragged everywhere
    (300, 256, 64, 0),              # exactly one chunk per CTA
    (5, 1000, 16, 0),               # batch and width below one tile: copies mostly past the edges
    (1, 4, 4, 0),                   # k below one 32-value stage
    (3, 70, 8, 2),                  # ragged k stage, aligned rows
    (150, 3000, 32, 0),             # 32-word tiles, the second query tile 22 rows deep
])
def test_tc_contract_matches_oracle(env, tc_kernel, B, L, W, pad):
    torch, pir, orc = env
    rng = np.random.Generator(np.random.PCG64(B * 7 + L + W))
    S = rng.integers(0, 1 << 32, (B, L), dtype=np.uint64).astype(np.uint32)
    T = wl.table_u32(W + 1, L, W)
    assert np.array_equal(_tc_contract(torch, pir, S, T, pad), orc.contract(S, T))


@pytest.mark.parametrize("pad", [0, 3], ids=["ld_odd", "ld_aligned"])
def test_tc_contract_exact_at_the_accumulator_bound(env, tc_kernel, pad):
    """0x7F7F7F80 splits into four signed limbs of -128, so every limb product
    is +2^14 and a class-3 accumulator reaches 4 * 2^14 * 256 = 2^24 just
    before it is drained: the largest value the exactness argument allows."""
    torch, pir, orc = env
    B, L, W = 130, 76 * 512 + 37, 40  # three 256-k chunks per CTA
    S = np.full((B, L), 0x7F7F7F80, dtype=np.uint32)
    T = np.full((L, W), 0x7F7F7F80, dtype=np.uint32)
    S[3, :] = 0x80808080  # limbs of mixed sign in one row
    T[:, 7] = 0xFFFFFFFF
    assert np.array_equal(_tc_contract(torch, pir, S, T, pad), orc.contract(S, T))


@pytest.mark.parametrize("B,L,W,nrows,ncols", [(256, 1 << 20, 64, 6, 16), (1024, 1 << 24, 32, 4, 6)],
                         ids=["batched_2^20x64", "large_2^24x32"])
def test_tc_contract_full_size_sampled_outputs(env, tc_kernel, B, L, W, nrows, ncols):
    """The bench's full-size shapes, in the launch configuration the bench
    times: seeded random shares and table on the device, the tcgen05 product,
    and the oracle's product for a seeded sample of outputs (query rows x
    table words, the first and last of each included)."""
    torch, pir, orc = env
    free = torch.cuda.mem_get_info()[0]
    if (B + W) * L * 4 > 0.6 * free:
        pytest.skip("not enough device memory for this shape")
    gen = torch.Generator(device="cuda").manual_seed(B * 131 + W)
    S = torch.randint(-2**31, 2**31 - 1, (B, L), dtype=torch.int32, device="cuda", generator=gen)
    T = torch.randint(-2**31, 2**31 - 1, (L, W), dtype=torch.int32, device="cuda", generator=gen)
    out = torch.empty((B, W), dtype=torch.int32, device="cuda")
    pir.pir_contract_u32(S, B, T, out, engine=pir.PIR_CONTRACT_TC_F16)
    torch.cuda.synchronize()
    assert pir.pir_device_status(clear=True) == 0
    got = out.cpu().numpy().view(np.uint32)
    rng = np.random.Generator(np.random.PCG64(L + B))
    rows = sorted({0, B - 1, *rng.integers(0, B, nrows - 2).tolist()})
    cols = sorted({0, W - 1, *rng.integers(0, W, ncols - 2).tolist()})
    Sh = S[rows].cpu().numpy().view(np.uint32)
    Th = T[:, cols].cpu().numpy().view(np.uint32)
    want = orc.contract(Sh, Th)
    assert np.array_equal(got[np.ix_(rows, cols)], want)
    del S, T
    torch.cuda.empty_cache()
