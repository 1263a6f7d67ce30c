"""The streaming scan engine of the share-matrix x table product
(PIR_CONTRACT_SCAN): bit-exact against the oracle's contraction on ragged
shapes, padded strides, the widest and narrowest rows, more than eight queries
(several passes), extreme operands, and against the tile engines at full
size; unsupported layouts are refused, and no bounded wait gives up."""
import numpy as np
import pytest

import workloads as wl
from test_gpu_parity import dev_table

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

    pir.pir_device_status(clear=True)
    return torch, pir, oracle


def _padded(torch, A, cols):
    """Device copy of A (rows x w, uint32) inside a rows x cols buffer; returns the view."""
    full = torch.full((A.shape[0], cols), -1, dtype=torch.int32, device="cuda")
    full[:, :A.shape[1]] = torch.from_numpy(np.ascontiguousarray(A).view(np.int32)).cuda()
    return full[:, :A.shape[1]]


@pytest.mark.parametrize("B,L,W,ld_pad,stride_pad", [
    (1, 1, 4, 0, 0), (1, 2, 4, 4, 0), (3, 5, 4, 0, 4), (2, 7, 8, 4, 4), (8, 1000, 16, 0, 0), (9, 4097, 64, 4, 0),
    (13, 20000, 32, 0, 4), (5, 777, 128, 8, 0), (2, 3000, 1024, 0, 0), (8, (1 << 16) + 77, 4, 4, 4),
    (4, 513, 12, 0, 0), (16, 1 << 14, 64, 0, 0)])
def test_scan_matches_oracle(env, B, L, W, ld_pad, stride_pad):
    torch, pir, orc = env
    rng = np.random.Generator(np.random.PCG64(B * L + W + ld_pad))
    S = rng.integers(0, 1 << 32, (B, L), dtype=np.uint64).astype(np.uint32)
    T = wl.table_u32(W + 1, L, W)
    dS = _padded(torch, S, (L + 3) // 4 * 4 + ld_pad)  # the engine needs ld % 4 == 0
    dT = _padded(torch, T, W + stride_pad)
    out = torch.full((B, W), 5, dtype=torch.int32, device="cuda")
    pir.pir_contract_u32(dS, B, dT, out, engine=pir.PIR_CONTRACT_SCAN)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), orc.contract(S, T))
    assert pir.pir_device_status() == 0


def test_scan_extreme_operands(env):
    torch, pir, orc = env
    B, L, W = 8, 12345, 32
    S = np.full((B, L), M32, np.uint32)
    T = np.full((L, W), M32, np.uint32)
    out = torch.empty((B, W), dtype=torch.int32, device="cuda")
    pir.pir_contract_u32(_padded(torch, S, (L + 3) // 4 * 4), B, dev_table(torch, T), out,
                         engine=pir.PIR_CONTRACT_SCAN)
    torch.cuda.synchronize()
    # sum of L products (2^32-1)^2 = 1 (mod 2^32) each
    assert (out.cpu().numpy().view(np.uint32) == (L & M32)).all()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), orc.contract(S, T))


def test_scan_refuses_unsupported_layouts(env):
    torch, pir, _ = env
    L = 100
    S = torch.zeros((2, L + 4), dtype=torch.int32, device="cuda")
    T = torch.zeros((L, 16), dtype=torch.int32, device="cuda")
    out = torch.empty((2, 16), dtype=torch.int32, device="cuda")
    with pytest.raises(pir.PirError) as e:  # shares not 16-byte aligned
        pir.pir_contract_u32(S[:, 1:L + 1], 2, T, out, engine=pir.PIR_CONTRACT_SCAN)
    assert e.value.code == -8
    T5 = torch.zeros((L, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(pir.PirError) as e:  # width not a multiple of 4
        pir.pir_contract_u32(S[:, :L], 2, T5, torch.empty((2, 5), dtype=torch.int32, device="cuda"),
                             engine=pir.PIR_CONTRACT_SCAN)
    assert e.value.code == -8
    Tw = torch.zeros((L, 1028), dtype=torch.int32, device="cuda")
    with pytest.raises(pir.PirError) as e:  # rows wider than the stage limit
        pir.pir_contract_u32(S[:, :L], 2, Tw, torch.empty((2, 1028), dtype=torch.int32, device="cuda"),
                             engine=pir.PIR_CONTRACT_SCAN)
    assert e.value.code == -8


def test_scan_equals_tile_engines_at_full_size(env):
    """2^24 rows x 32 words (2 GiB table), eight queries: the scan agrees with
    the CUDA-core tile engine word for word, and sampled words with the oracle."""
    torch, pir, orc = env
    rows, width, B = 1 << 24, 32, 8
    table = wl.table_u32_torch(24, rows, width, "cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    S = torch.randint(-(1 << 31), 1 << 31, (B, rows), dtype=torch.int32, device="cuda", generator=g)
    a = torch.empty((B, width), dtype=torch.int32, device="cuda")
    b = torch.empty_like(a)
    pir.pir_contract_u32(S, B, table, a, engine=pir.PIR_CONTRACT_SCAN)
    pir.pir_contract_u32(S, B, table, b, engine=pir.PIR_CONTRACT_IMAD)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # one word per query recomputed on the host from sampled rows of a small slice
    lo, hi = 5_000_000, 5_000_000 + 4096
    Ts = table[lo:hi].cpu().numpy().view(np.uint32)
    Ss = S[:, lo:hi].cpu().numpy().view(np.uint32)
    part = torch.empty((B, width), dtype=torch.int32, device="cuda")
    pir.pir_contract_u32(S[:, lo:hi], B, table[lo:hi], part, engine=pir.PIR_CONTRACT_SCAN)
    torch.cuda.synchronize()
    assert np.array_equal(part.cpu().numpy().view(np.uint32), orc.contract(Ss, Ts))
    assert pir.pir_device_status() == 0
