"""The serving handle (continuous batching): every module's result, taken
from a mix of concurrently submitted modules, equals its result alone and the
oracle's; admission by footprint refuses what does not fit and admits again
after release; the decoded rows stay on the device until release."""
import time

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


def _modules(n, seed):
    n_instr, n_k = synth.batch_shape(n, seed, median=800, lo=200, hi=6000)
    w, off = synth.batch(n_instr, n_k, seed)
    mods = [w[off[i]:off[i + 1]].copy() for i in range(n)]
    rng = np.random.default_rng(seed)
    for i in range(0, n, 5):                       # some corrupted modules in the mix
        mods[i][int(rng.integers(5, len(mods[i])))] = int(rng.integers(0, 2 ** 32))
    return mods


def _expected(m):
    off = np.array([0, len(m)], np.int64)
    st, er = oracle.validate(m, off)
    text, _ = oracle.disassemble(m, off, True, True)
    d = oracle.decode(m, off)
    return int(st[0]), int(er[0]), text, d


def test_results_alone_equal_in_mix_and_oracle(gpu):
    mods = _modules(120, 31)
    srv = gpu.Server(hbm_cap_bytes=1 << 30, max_batch_modules=64)
    try:
        # alone: one module at a time
        alone = []
        for m in mods[:12]:
            t = srv.submit(m)
            r = srv.wait(t)
            alone.append((r.status, r.err_row, gpu.Server.text_of(r)))
            srv.release(t)
        # in a mix: everything submitted back to back, then collected
        tickets = [srv.submit(m) for m in mods]
        assert all(t is not None for t in tickets)
        results = []
        for t in tickets:
            r = srv.wait(t)
            assert r is not None and r.error == 0
            results.append(r)
        assert max(r.batch_modules for r in results) > 1        # modules really were batched together
        for i, (m, r) in enumerate(zip(mods, results)):
            st, er, text, d = _expected(m)
            assert (r.status, r.err_row) == (st, er), i
            assert gpu.Server.text_of(r) == text, i
            if i < 12:
                assert alone[i] == (r.status, r.err_row, gpu.Server.text_of(r))
            # decoded rows stay on the device until release
            n = r.n_instr
            assert n == d["n_rows"]
            if n:
                op = torch.empty(n, dtype=torch.int16, device="cuda")
                torch.cuda.synchronize()
                import ctypes
                cudart = ctypes.CDLL("libcudart.so")
                cudart.cudaMemcpy(ctypes.c_void_p(op.data_ptr()), ctypes.c_void_p(r.op), ctypes.c_size_t(2 * n), 3)
                assert np.array_equal(op.cpu().numpy().view(np.uint16), d["op"])
        for t in tickets:
            srv.release(t)
    finally:
        srv.close()


def test_admission_by_footprint(gpu):
    mods = _modules(20, 5)
    need = sum(28 * len(m) + 64 for m in mods[:5])
    srv = gpu.Server(hbm_cap_bytes=need, max_batch_modules=8)
    try:
        tickets = [srv.submit(m) for m in mods[:5]]
        assert all(t is not None for t in tickets)
        assert srv.submit(mods[5]) is None             # over the cap: refused, nothing changes
        for t in tickets:
            assert srv.wait(t) is not None
        srv.release(tickets[0])
        t = srv.submit(mods[0])                         # room again after a release
        assert t is not None
        assert srv.wait(t).status == _expected(mods[0])[0]
        srv.release(t)
        for t in tickets[1:]:
            srv.release(t)
    finally:
        srv.close()


def test_one_module_per_launch_mode(gpu):
    mods = _modules(10, 9)
    srv = gpu.Server(hbm_cap_bytes=1 << 28, max_batch_modules=1)
    try:
        tickets = [srv.submit(m) for m in mods]
        for t, m in zip(tickets, mods):
            r = srv.wait(t)
            assert r.batch_modules == 1
            st, er, text, _ = _expected(m)
            assert (r.status, r.err_row, gpu.Server.text_of(r)) == (st, er, text)
            srv.release(t)
    finally:
        srv.close()


def test_poll_and_latency_stamps(gpu):
    mods = _modules(4, 13)
    srv = gpu.Server(hbm_cap_bytes=1 << 28)
    try:
        t = srv.submit(mods[0])
        deadline = time.time() + 10
        r = None
        while r is None and time.time() < deadline:
            r = srv.poll(t)
        assert r is not None and r.done_ns >= r.submit_ns
        srv.release(t)
        with pytest.raises(Exception):
            srv.release(t)
    finally:
        srv.close()


def test_replay_reports_every_module(gpu):
    """spv_serve_replay submits on its own thread at the scheduled times and
    collects in order: every module gets a latency no shorter than its time
    in the server, batches form under load, and the server stays usable."""
    mods = _modules(60, 21)
    srv = gpu.Server(hbm_cap_bytes=1 << 30)
    try:
        arrive = (np.arange(60, dtype=np.int64) * 20_000)        # one module every 20 us
        lat, srv_ns, bm, busy = srv.replay(mods, arrive)
        assert (srv_ns > 0).all() and (lat >= srv_ns - 1_000_000).all()
        assert bm.max() >= 1 and busy >= 0
        t = srv.submit(mods[0])
        r = srv.wait(t)
        st, er, text, _ = _expected(mods[0])
        assert (r.status, r.err_row, gpu.Server.text_of(r)) == (st, er, text)
        srv.release(t)
        with pytest.raises(Exception):
            srv.replay(mods[:3], np.array([5, 3, 9], np.int64))  # arrivals must not decrease
    finally:
        srv.close()
