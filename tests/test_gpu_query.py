"""spv_query_sizes: the row bound holds for every batch and the text size is
exactly the disassembler's total (and the oracle's text length), for both
option settings, on a batch with a bad module."""
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


@pytest.mark.parametrize("inline,header", [(True, True), (False, False)])
def test_query_sizes(gpu, inline, header):
    n_instr, n_k = synth.batch_shape(30, 41, median=800, lo=200, hi=4000)
    w, off = synth.batch(n_instr, n_k, 41)
    w = w.copy()
    w[off[3]] = 0x12345678                                   # module 3: bad magic, no text
    wd = torch.from_numpy(w.view(np.int32)).cuda()
    od = torch.from_numpy(off).cuda()
    rows, text = gpu.query_sizes(wd, od, inline_names=inline, header=header)
    want, _ = oracle.disassemble(w, off, inline, header)
    assert text == len(want)
    d = oracle.decode(w, off)
    assert rows == len(w) - 5 * (len(off) - 1) and rows >= d["n_rows"]
    r = gpu.process(wd, od)
    t, toff, _ = gpu.disassemble(wd, od, r["table"], inline_names=inline, header=header)
    assert int(toff[-1].item()) == text


def test_query_sizes_empty(gpu):
    wd = torch.zeros(1, dtype=torch.int32, device="cuda")
    od = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert gpu.query_sizes(wd[:0], od) == (0, 0)
