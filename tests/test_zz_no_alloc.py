"""spv_process_batch_noalloc: the entry point for callers that cannot
allocate device memory (a runtime that owns all device memory through its
own pool, a serving loop that must not call cudaMalloc). It runs the same
kernels with the library's fixed device scratch instead of a caller
workspace; its results must equal spv_process_batch's and the oracle's,
call after call, although every call shares (and leaves behind) the same
scratch.

Collected last on purpose, and self-contained so it passes alone in a fresh
process as well as after the other tests."""
import ctypes

import numpy as np
import pytest

import oracle
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


def _near_limit_batch(gpu, limit):
    """Generated modules, as many as keep the workspace at or under `limit`
    bytes, then the last one cut down (a module's tail words dropped) to come
    as close to the limit as a few tiles allow: the scratch array's tail end
    is used."""
    n_instr, n_k = synth.batch_shape(400, 5, median=2500, lo=200, hi=20000)
    w, off = synth.batch(n_instr, n_k, 500)
    m = len(off) - 1
    while m > 1 and gpu.spv_workspace_bytes(m, int(off[m])) > limit:
        m -= 1
    # grow the last module word by word (in steps) up to the limit; a module
    # cut short still decodes (its tail is a framing error the oracle names too)
    extra = 0
    nxt = int(off[m + 1]) if m < len(off) - 1 else int(off[m])
    step = 1024
    while step >= 1:
        while int(off[m]) + extra + step <= nxt and gpu.spv_workspace_bytes(m + 1, int(off[m]) + extra + step) <= limit:
            extra += step
        step //= 2
    if extra:
        words = np.ascontiguousarray(w[:int(off[m]) + extra])
        offs = np.concatenate([off[:m + 1], [int(off[m]) + extra]]).astype(np.int64)
    else:
        words = np.ascontiguousarray(w[:int(off[m])])
        offs = np.ascontiguousarray(off[:m + 1])
    return words, offs


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


def _check_against_oracle(words, offs, table, status, err, out):
    """The allocation-free call's table, statuses, error rows and encoded
    words, element by element against the oracle."""
    m = len(offs) - 1
    d = oracle.decode(words, offs)
    t = table.to_numpy()
    n = d["n_rows"]
    assert int(t["first_row"][m]) == n
    for k in ("op", "wc", "off", "rtype", "rid", "mod"):
        assert np.array_equal(t[k][:n], d[k]), k
    assert np.array_equal(t["first_row"][:m], d["first_row"])
    assert np.array_equal(t["n_instr"][:m], d["n_instr"])
    st, er = oracle.validate(words, offs)
    assert np.array_equal(status.cpu().numpy().view(np.uint32), st)
    assert np.array_equal(err.cpu().numpy(), er)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.encode(words, offs, d, True))


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
        _check_against_oracle(words, offs, t1, s1, e1, out1)


def test_no_alloc_batch_just_under_the_scratch_size(gpu):
    """A batch whose workspace fills the scratch array to within a few tiles
    of its end, twice in a row: exact against the oracle and against
    spv_process_batch."""
    limit = gpu.SPV_NOALLOC_SCRATCH_BYTES
    words, offs = _near_limit_batch(gpu, limit)
    need = gpu.spv_workspace_bytes(len(offs) - 1, len(words))
    assert limit - 4096 * 64 <= need <= limit
    w = torch.from_numpy(words.view(np.int32)).cuda()
    o = torch.from_numpy(offs).cuda()
    for _ in range(2):
        t1, s1, e1, out1 = _noalloc(gpu, w, o)
        torch.cuda.synchronize()
        _check_against_oracle(words, offs, t1, s1, e1, out1)
    ref = gpu.process(w, o, validate=True, encode=True)
    torch.cuda.synchronize()
    assert torch.equal(s1, ref["status"]) and torch.equal(out1, ref["out"])


def test_no_alloc_rejects_batches_beyond_its_scratch(gpu):
    # every batch here is backed by device buffers of its full size, so even a
    # call that wrongly went ahead would read only memory it owns
    n_big = 20_000_000
    w = torch.zeros(n_big, dtype=torch.int32, device="cuda")
    o = torch.tensor([0, n_big], dtype=torch.int64, device="cuda")
    big = gpu.batch_of(w, o)                          # workspace for 20M words: too large
    table = gpu.Table(1, n_big, w.device)
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    er = torch.empty(1, dtype=torch.int64, device="cuda")
    rc = gpu.spv_process_batch_noalloc(big, table.c(), ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(er.data_ptr()),
                                       1, None, 0, None, None)
    assert rc == gpu.SPV_E_WORKSPACE
    assert gpu.spv_workspace_bytes(1, n_big) > gpu.SPV_NOALLOC_SCRATCH_BYTES
    # a null output argument is an argument error whatever the batch's size
    rc = gpu.spv_process_batch_noalloc(big, table.c(), None, ctypes.c_void_p(er.data_ptr()), 1, None, 0, None, None)
    assert rc == gpu.SPV_E_ARG
    del w, table
    # a batch only a few tiles past the limit is refused too
    words, offs = _near_limit_batch(gpu, gpu.SPV_NOALLOC_SCRATCH_BYTES)
    words = np.concatenate([words, np.zeros(4 * 4096, np.uint32)])
    offs = offs.copy()
    offs[-1] = len(words)
    m = len(offs) - 1
    assert gpu.spv_workspace_bytes(m, len(words)) > gpu.SPV_NOALLOC_SCRATCH_BYTES
    w2 = torch.from_numpy(words.view(np.int32)).cuda()
    o2 = torch.from_numpy(offs).cuda()
    table = gpu.Table(m, len(words), w2.device)
    st = torch.empty(m, dtype=torch.int32, device="cuda")
    er = torch.empty(m, dtype=torch.int64, device="cuda")
    rc = gpu.spv_process_batch_noalloc(gpu.batch_of(w2, o2), table.c(), ctypes.c_void_p(st.data_ptr()),
                                       ctypes.c_void_p(er.data_ptr()), 1, None, 0, None, None)
    assert rc == gpu.SPV_E_WORKSPACE
