"""The redzone harness of the GPU out-of-bounds tests, checked on the CPU with
planted faults: a write one word before or after a payload, or into a table's
row padding, is reported; an untouched buffer is not; a read past a row's width
or past a buffer's end sees random words rather than neighbouring data."""
import numpy as np
import pytest

from test_gpu_redzones import GUARD, Guarded, guarded_table, intact


@pytest.fixture(scope="module")
def torch():
    return pytest.importorskip("torch")


def test_untouched_buffer_passes(torch):
    buf = Guarded(torch, 100, 1, device="cpu")
    assert buf.guards_intact() and buf.unchanged() and intact(buf)
    buf.words()[:] = 7  # writing the whole payload is in bounds
    assert buf.guards_intact() and not buf.unchanged()


@pytest.mark.parametrize("where", [GUARD - 1, GUARD + 100, 0, 2 * GUARD + 99])
def test_write_outside_the_payload_is_caught(torch, where):
    buf = Guarded(torch, 100, 2, device="cpu")
    buf.dev[where] ^= 1  # a planted out-of-bounds write
    assert not buf.guards_intact() and not intact(buf)


def test_write_into_row_padding_is_caught(torch):
    T = np.arange(40, dtype=np.uint32).reshape(10, 4)
    tbuf, view = guarded_table(torch, T, 3, 3, device="cpu")
    assert np.array_equal(view.numpy().view(np.uint32), T) and view.stride(0) == 7
    assert tbuf.unchanged()
    tbuf.words().view(10, 7)[4, 5] += 1  # a planted write past row 4's width
    assert tbuf.guards_intact() and not tbuf.unchanged()


def test_reads_past_the_width_or_the_end_see_random_words(torch):
    rows, W, pad = 64, 4, 4
    T = np.arange(rows * W, dtype=np.uint32).reshape(rows, W)
    tbuf, view = guarded_table(torch, T, pad, 4, device="cpu")
    full = tbuf.words().view(rows, W + pad).numpy().view(np.uint32)
    padding = full[:, W:]
    assert len(np.unique(padding)) > padding.size // 2  # random, not a copy of the table
    assert not np.isin(padding, T).all()
    after = tbuf.dev[GUARD + rows * (W + pad):].numpy().view(np.uint32)
    assert len(np.unique(after)) > GUARD // 2
    # a product that reads one word past each row's width no longer matches
    ones = np.ones((1, rows), np.uint64)
    good = (ones @ full[:, :W].astype(np.uint64)) & 0xFFFFFFFF
    shifted = (ones @ full[:, 1:W + 1].astype(np.uint64)) & 0xFFFFFFFF
    assert not np.array_equal(good, shifted)
