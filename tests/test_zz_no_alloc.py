"""spv_process_batch_noalloc: the entry point for callers that cannot
allocate device memory (a runtime that owns all device memory through its
own pool, a serving loop that must not call cudaMalloc). It runs the same
kernels with the library's fixed device scratch instead of a caller
workspace; its results must equal spv_process_batch's, call after call,
although every call shares (and leaves behind) the same scratch.

Collected last on purpose, and self-contained so it passes alone in a fresh
process as well as after the other tests."""
import ctypes

import numpy as np
import pytest

from paper_2305_09493_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gpu():
    from paper_2305_09493_b300 import build, spvgpu
    build.build()
    spvgpu.load()
    return spvgpu


def _batches():
    # batch A: generated modules with corruptions (duplicate ids, bad words) so
    # the id sets and the fixup pass run; batch B: different shapes, clean
    n_instr, n_k = synth.batch_shape(40, 77, median=1500, lo=200, hi=12000)
    wa, offa = synth.batch(n_instr, n_k, 77)
    rng = np.random.default_rng(3)
    wa = wa.copy()
    for m in range(0, 40, 4):
        lo, hi = int(offa[m]) + 5, int(offa[m + 1])
        wa[int(rng.integers(lo, hi))] = int(rng.integers(0, 2 ** 32))
    n_instr, n_k = synth.batch_shape(25, 91, median=2500, lo=200, hi=20000)
    wb, offb = synth.batch(n_instr, n_k, 91)
    wl, offl, _, _ = synth.large_module(13, n_instr=80_000, n_funcs=8)
    wb = np.concatenate([wb, wl])
    offb = np.concatenate([offb, offb[-1] + offl[1:]])
    return [(wa, offa), (wb, offb)]


def _noalloc(gpu, words_t, off_t):
    m = off_t.numel() - 1
    table = gpu.Table(m, words_t.numel(), words_t.device)
    status = torch.empty(m, dtype=torch.int32, device=words_t.device)
    err = torch.empty(m, dtype=torch.int64, device=words_t.device)
    out = torch.empty_like(words_t)
    rc = gpu.spv_process_batch_noalloc(gpu.batch_of(words_t, off_t), table.c(), ctypes.c_void_p(status.data_ptr()),
                                       ctypes.c_void_p(err.data_ptr()), 1, ctypes.c_void_p(out.data_ptr()), 1, None,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == gpu.SPV_SUCCESS
    return table, status, err, out


def test_no_alloc_matches_workspace_entry_point_two_calls_in_a_row(gpu):
    for words, offs in _batches() * 2:     # A, B, A, B: each call follows another on the shared scratch
        w = torch.from_numpy(words.view(np.int32)).cuda()
        o = torch.from_numpy(offs).cuda()
        ws = gpu.spv_workspace_bytes(len(offs) - 1, len(words))
        assert ws <= gpu.SPV_NOALLOC_SCRATCH_BYTES
        t1, s1, e1, out1 = _noalloc(gpu, w, o)
        ref = gpu.process(w, o, validate=True, encode=True)
        torch.cuda.synchronize()
        a, b = t1.to_numpy(), ref["table"].to_numpy()
        n = int(b["first_row"][-1])
        assert int(a["first_row"][-1]) == n
        for k in ("op", "wc", "off", "rtype", "rid", "mod", "first_row", "n_instr"):
            assert np.array_equal(a[k], b[k]), k
        assert torch.equal(s1, ref["status"]) and torch.equal(e1, ref["err_row"])
        assert torch.equal(out1, ref["out"])
        assert (s1 != 0).any() or len(offs) < 41   # batch A carries errors


def test_no_alloc_rejects_batches_beyond_its_scratch(gpu):
    w = torch.zeros(16, dtype=torch.int32, device="cuda")
    o = torch.zeros(2, dtype=torch.int64, device="cuda")
    big = gpu.SpvBatch(w.data_ptr(), o.data_ptr(), 1, 20_000_000)   # workspace for 20M words: too large
    table = gpu.Table(1, 16, w.device)
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    er = torch.empty(1, dtype=torch.int64, device="cuda")
    rc = gpu.spv_process_batch_noalloc(big, table.c(), ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(er.data_ptr()),
                                       1, None, 0, None, None)
    assert rc == gpu.SPV_E_WORKSPACE
    assert gpu.spv_workspace_bytes(1, 20_000_000) > gpu.SPV_NOALLOC_SCRATCH_BYTES
