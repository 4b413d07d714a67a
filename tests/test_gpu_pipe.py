"""The host-resident pipeline (spv_pipe_run): a batch in host memory, split
into chunks whose uploads, kernels and downloads overlap, gives exactly the
oracle's statuses, error rows, encoded words and text for the whole batch,
whatever the chunking; a text capacity smaller than the text is filled to
the byte and not past it."""
import numpy as np
import pytest

import oracle
from paper_2305_09493_b300 import synth
from tests import spvhand as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gpu():
    from paper_2305_09493_b300 import build, spvgpu
    build.build()
    spvgpu.load()
    return spvgpu


def _batch(n, seed, corrupt=True):
    n_instr, n_k = synth.batch_shape(n, seed, median=800, lo=200, hi=6000)
    w, off = synth.batch(n_instr, n_k, seed)
    if corrupt:
        rng = np.random.default_rng(seed)
        for m in range(0, n, 7):
            w[int(rng.integers(off[m] + 5, off[m + 1]))] = int(rng.integers(0, 2 ** 32))
    return w, off


def _outputs(n_mod, n_words, cap, pinned):
    mk = (lambda n, dt: torch.empty(n, dtype=dt).pin_memory()) if pinned else (lambda n, dt: torch.empty(n, dtype=dt))
    return (mk(n_mod, torch.int32), mk(n_mod, torch.int64), mk(n_mod + 1, torch.int64), mk(cap, torch.uint8),
            mk(max(1, n_words), torch.int32), mk(max(1, n_mod), torch.int32))


def _check(gpu, w, off, chunk_words, depth=3, pinned=True, cap=None, inline=True, header=True):
    st_o, er_o = oracle.validate(w, off)
    d = oracle.decode(w, off)
    enc_o = oracle.encode(w, off, d, True)
    text_o, toff_o = oracle.disassemble(w, off, inline, header)
    cap = len(text_o) if cap is None else cap
    n_mod = len(off) - 1
    status, err, toff, text, out, dstat = _outputs(n_mod, len(w), cap + 64, pinned)
    text.fill_(0xAB)
    words = torch.from_numpy(w.view(np.int32))
    mod_off = torch.from_numpy(off)
    if pinned:
        words, mod_off = words.pin_memory(), mod_off.pin_memory()
    p = gpu.Pipe(chunk_words=chunk_words, depth=depth, inline_names=inline, header=header)
    try:
        total = p.run(words, mod_off, status, err, toff, text[:cap], out_words=out, dis_status=dstat)
    finally:
        p.close()
    assert total == len(text_o)
    assert np.array_equal(status.numpy().view(np.uint32), st_o)
    assert np.array_equal(err.numpy(), er_o)
    assert np.array_equal(toff.numpy().view(np.uint64), toff_o)
    got = bytes(text.numpy()[:min(cap, total)])
    assert got == text_o[:cap]
    assert (text.numpy()[min(cap, total):] == 0xAB).all()          # nothing written past the capacity
    assert np.array_equal(out.numpy()[:len(w)].view(np.uint32), enc_o)
    assert (dstat.numpy()[:n_mod] == 0).all()


@pytest.mark.parametrize("chunk_words,depth", [(60_000, 3), (250_000, 2), (1 << 24, 3), (20_000, 8)])
def test_pipe_matches_oracle_for_any_chunking(gpu, chunk_words, depth):
    w, off = _batch(120, 3)
    _check(gpu, w, off, chunk_words, depth)


def test_pipe_pageable_memory_and_header_off(gpu):
    w, off = _batch(40, 5)
    _check(gpu, w, off, 50_000, pinned=False, inline=False, header=False)


def _wordy_text_module(n_rows, name_len):
    """Few words, much text: an id named by a long OpName and used by every
    row, so each 4-word row prints the whole name."""
    body = H.minimal_body()
    body = body[:7] + [H.ins(H.OpName, 2, H.s("n" * name_len))] + \
        [H.ins(H.OpConstant, 2, 100 + k, k) for k in range(n_rows)] + body[7:]
    return H.module(body, bound=100 + n_rows + 1)


def test_pipe_module_larger_than_a_chunk(gpu):
    # a string-heavy module several times a chunk, between ordinary ones
    big, boff, _, _ = synth.large_module(4, n_instr=150_000, n_funcs=20)
    small, soff = _batch(6, 7, corrupt=False)
    mods = [small[soff[i]:soff[i + 1]] for i in range(3)] + [big] + [small[soff[i]:soff[i + 1]] for i in range(3, 6)]
    w, off = H.batch(mods)
    _check(gpu, w, off, 100_000)


def test_pipe_text_outgrows_the_slot_buffer(gpu):
    # chunks of at most 100,000 words get a first text buffer of about 1 MB;
    # this module prints about 6 MB from 12,546 words
    small, soff = _batch(12, 8, corrupt=False)
    mods = [small[soff[i]:soff[i + 1]] for i in range(12)]
    mods.insert(5, _wordy_text_module(3000, 2000))
    w, off = H.batch(mods)
    _check(gpu, w, off, 100_000)


def test_pipe_text_capacity_below_total(gpu):
    w, off = _batch(30, 9)
    text_o, _ = oracle.disassemble(w, off, True, True)
    for cap in (0, 1, len(text_o) // 3 + 7, len(text_o) - 1):
        _check(gpu, w, off, 40_000, cap=cap)


def test_pipe_handle_reuse_and_empty_batch(gpu):
    p = gpu.Pipe(chunk_words=30_000)
    try:
        for n, seed in ((0, 0), (10, 11), (60, 12), (5, 13)):
            w, off = _batch(n, seed) if n else (np.zeros(0, np.uint32), np.zeros(1, np.int64))
            text_o, toff_o = oracle.disassemble(w, off, True, True)
            st_o, er_o = oracle.validate(w, off)
            status, err, toff, text, out, dstat = _outputs(n, len(w), len(text_o) + 1, True)
            total = p.run(torch.from_numpy(w.view(np.int32)), torch.from_numpy(off), status, err, toff, text)
            assert total == len(text_o)
            assert np.array_equal(toff.numpy().view(np.uint64), toff_o)
            assert bytes(text.numpy()[:total]) == text_o
            assert np.array_equal(status.numpy()[:n].view(np.uint32), st_o)
            assert np.array_equal(err.numpy()[:n], er_o)
    finally:
        p.close()


def test_pipe_rejects_bad_offsets(gpu):
    w, off = _batch(4, 1)
    bad = off.copy()
    bad[2] = bad[1] - 1
    status, err, toff, text, _, _ = _outputs(4, len(w), 16, False)
    p = gpu.Pipe()
    try:
        with pytest.raises(gpu.SpvError):
            p.run(w, bad, status, err, toff, text)
    finally:
        p.close()
