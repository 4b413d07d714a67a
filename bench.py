"""Benchmark of the batched SPIR-V hot path on B300.

One step = the whole hot path over one batch of synthetic modules:
decode + validate + encode in one persistent launch (spv_process_batch),
then disassembly with inline names and header lines (spv_disassemble_batch).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload batch|large|single]
                    [--impl gpu|reference]

The default workload is the batch of 10,000 synthetic kernel modules
(instruction counts lognormal, median 1,500, 1-8 kernels each; ~122M words).
Prints one JSON line (rank 0). Under torchrun each rank processes its own
batch of the same shape (different seeds): weak scaling, no data-path
collective.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPIR-V GB/s decode+validate+disasm, batched vs per-module; serve p50/p99 latency"
L2_BYTES = 126 * 2**20


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="batch", choices=["batch", "large", "single", "bins"],
                    help="bins: 4 size bins x 1,000 modules, tile-shape sweep and autotuned CUDA-graph replay per bin")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-per-module", action="store_true", help="skip the per-module comparison leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bins", action="store_true", help="skip the size-bin leg (tile sweep, autotuner, CUDA graph)")
    ap.add_argument("--modules", type=int, default=10_000, help="modules in the batch workload")
    ap.add_argument("--serve-rates", default="5000,10000,20000,50000",
                    help="Poisson arrival rates of the serve legs (modules/s, comma-separated)")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="duration of each continuous-batching serve leg (0: skip)")
    ap.add_argument("--serve-per-launch-seconds", type=float, default=0.5,
                    help="duration of each one-module-per-launch comparison leg")
    ap.add_argument("--serve-cap-gb", type=float, default=8.0, help="admission cap of the server's device-resident tables")
    ap.add_argument("--e2e-chunk-words", type=int, default=0, help="chunk size of the end-to-end pipeline (0: library default)")
    return ap.parse_args(argv)


def workload(name, rank, n_mod=10_000):
    from paper_2305_09493_b300 import synth
    if name == "batch":
        w, off = synth.module_batch(n_mod, seed0=rank * n_mod)
        cfg = {"workload": f"batch of {n_mod:,} synthetic kernel modules", "modules": n_mod,
               "instr_per_module": "lognormal median 1500 sigma 1.0 clip [200, 50000]", "kernels_per_module": "1-8"}
    elif name == "large":
        w, off, _, _ = synth.large_module(seed=rank)
        cfg = {"workload": "one module of 4M instructions, 500 functions, 10% OpString/OpName", "modules": 1}
    else:
        w, off, _, _ = synth.single_module(seed=rank)
        cfg = {"workload": "one ~10k-word kernel module (2,000-instruction function, 40 blocks)", "modules": 1}
    cfg["words"] = int(len(w))
    return w, off, cfg


def dist_setup(n):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    return rank, world


def max_over_ranks(values, world):
    """Each value reduced to its maximum over all ranks (the step time of the
    slowest rank). The tensor lives where the process group's backend wants
    it: host memory under gloo, the current GPU under NCCL."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    dev = torch.device("cpu") if dist.get_backend() == "gloo" else torch.device("cuda", torch.cuda.current_device())
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu().tolist()]


def job_gbs(world, words_per_rank, ms):
    """Whole-job input throughput: every rank processes its own batch of
    words_per_rank words in (at most) ms milliseconds."""
    return world * 4 * words_per_rank / (ms * 1e-3) / 1e9


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# the device-code sources each measured kernel is built from
KERNEL_SOURCES = {
    "k_dis_main": ("spv_dis.cu", "spv_device.cuh", "spv_tables.cuh"),
    "k_tile": ("spv_batch.cu", "spv_device.cuh", "spv_tables.cuh"),
    "k_asm_measure": ("spv_asm.cu", "spv_tables.cuh"),
}


def source_hash(kernel):
    """Hash of the kernel's device-code sources: a stored ncu figure is used
    only while these are unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2305_09493_b300", "csrc")
    for f in KERNEL_SOURCES.get(kernel, sorted(os.listdir(csrc))):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        # bounded: an nvidia-smi blocked inside the driver must not hold the
        # bench (terminate, then kill, then go on with the samples written)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                pass
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].strip() == "Active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# algorithmic bytes per launch of each kernel (W words, N rows, L text bytes, M modules)
def algorithmic_bytes(kernel, W, N, L, M):
    return {
        "k_tile": 4 * W + 4 * W + 24 * N,                # words in; encoded words + 24-byte rows out
        "k_dis_main": 4 * W + 12 * N + L,                # words + op/wc/off columns in; text out
        "k_dis_ids": 20 * N,                             # op/wc/off/mod/rid columns
        "k_dis_namelen": 4 * N,                          # op column (OpName rows are few)
        "k_dis_clear": 0, "k_tile_setup": 0, "k_prepass_mod": 40 * M, "k_prepass_scan": 24 * M, "k_finalize": 64 * M,
    }.get(kernel, 0)


def issue_roofline(warp_inst, ms, clk):
    """Instruction-issue view of the dominant kernel: its warp instructions
    per launch (an ncu count for the same source and workload) over the live
    launch time, against 148 SMs x 4 schedulers x one warp instruction per
    cycle at the sampled SM clock."""
    mhz = clk.get("sm_mhz") if clk else None
    if not warp_inst or not mhz:
        return None
    peak = 148 * 4 * mhz * 1e6
    achieved = warp_inst / (ms * 1e-3)
    return {"unit": "warp instructions/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
            "warp_instructions_per_launch": warp_inst, "sm_mhz": mhz}


def serve_leg(spvgpu, w_np, off_np, rate, seconds, max_batch_modules=0, pool_size=2000, cap=8 << 30):
    """Poisson arrivals at `rate` modules/s for `seconds`, modules drawn in
    turn from the batch workload (its size distribution), replayed by the
    library's native load thread (spv_serve_replay: each module submitted at
    its scheduled time, retried while admission refuses it, collected in
    order). Latency is reported from submission to completion (the server,
    library clock), and from each module's scheduled arrival to its
    completion, which adds any time the one load thread ran behind its
    schedule or waited for admission. Throughput is the
    modules over the span from the first scheduled arrival to the last
    completion."""
    m_total = len(off_np) - 1
    pool = [np.ascontiguousarray(w_np[off_np[i]:off_np[i + 1]]) for i in range(min(pool_size, m_total))]
    srv = spvgpu.Server(hbm_cap_bytes=cap, max_batch_modules=max_batch_modules)
    srv.replay(pool[:8], np.arange(8, dtype=np.int64) * 1000)        # warm up the server's kernels
    rng = np.random.default_rng(12345)
    n = max(1, int(rate * seconds))
    arrive_ns = (np.cumsum(rng.exponential(1.0 / rate, n)) * 1e9).astype(np.int64)
    mods = [pool[i % len(pool)] for i in range(n)]
    lat, srv_ns, bm, busy = srv.replay(mods, arrive_ns)
    srv.close()
    # the server's own span: from the first scheduled arrival to the last
    # completion (the library's clock), not the caller's set-up around it
    elapsed = float(np.max(arrive_ns + lat) - arrive_ns[0]) / 1e9
    words_done = sum(len(m) for m in mods)
    lat_ms, srv_ms = lat / 1e6, srv_ns / 1e6
    return {"rate_per_s": rate, "seconds": seconds, "modules": n,
            "latency": "submit to completion (the server)",
            "p50_ms": float(np.percentile(srv_ms, 50)), "p99_ms": float(np.percentile(srv_ms, 99)),
            "from_arrival_p50_ms": float(np.percentile(lat_ms, 50)),
            "from_arrival_p99_ms": float(np.percentile(lat_ms, 99)),
            "mean_batch_modules": float(np.mean(bm)),
            "throughput_modules_per_s": n / elapsed, "gbs": 4 * words_done / elapsed / 1e9,
            "admission_retries": int(busy)}


def cpu_baseline(words, mod_off, budget_s=15.0):
    """The oracle (plain sequential C, one thread) on a bounded sample: the
    first modules of the batch, as many as fit the time budget."""
    import oracle
    m_total = len(mod_off) - 1
    k = max(1, min(m_total, 200))
    t0 = time.perf_counter()
    while True:
        sub = words[mod_off[0]:mod_off[k]]
        off = mod_off[:k + 1] - mod_off[0]
        t = time.perf_counter()
        d = oracle.decode(sub, off)
        oracle.validate(sub, off)
        oracle.encode(sub, off, d, True)
        oracle.disassemble(sub, off, True, True)
        dt = time.perf_counter() - t
        if dt > budget_s / 2 or k == m_total or time.perf_counter() - t0 > 2 * budget_s:
            break
        k = min(m_total, int(k * max(2.0, budget_s / max(dt, 1e-3))))
    gbs = 4 * len(sub) / dt / 1e9
    return {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"first {k} of {m_total} modules ({len(sub)} words): decode+validate+encode+disassemble, "
                      f"{dt:.2f} s on one host core", "k": k, "seconds": dt}


def _oracle_chunk(args):
    """One process's share of the all-cores oracle run: its modules, timed."""
    import oracle
    sub, off = args
    t = time.perf_counter()
    d = oracle.decode(sub, off)
    oracle.validate(sub, off)
    oracle.encode(sub, off, d, True)
    oracle.disassemble(sub, off, True, True)
    return time.perf_counter() - t


def cpu_all_cores(words, mod_off, k):
    """The same oracle on the same first k modules, split over one process
    per host core (spawned, each with a contiguous share of the modules of
    about equal words); the wall time of the parallel run."""
    import multiprocessing as mproc
    n = max(1, min(os.cpu_count() or 1, k, 64))
    total = mod_off[k] - mod_off[0]
    cuts = [0]
    for i in range(1, n):
        cuts.append(int(np.searchsorted(mod_off[:k + 1], mod_off[0] + total * i // n)))
    cuts.append(k)
    cuts = sorted(set(cuts))
    parts = [(words[mod_off[a]:mod_off[b]], mod_off[a:b + 1] - mod_off[a]) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
    from concurrent.futures import ProcessPoolExecutor
    try:
        # a worker that cannot start ends the pool with an error, never a wait
        with ProcessPoolExecutor(len(parts), mp_context=mproc.get_context("spawn")) as pool:
            list(pool.map(_oracle_chunk, [(w[:0], np.zeros(1, np.int64)) for w, _ in parts]))   # start the workers
            t = time.perf_counter()
            list(pool.map(_oracle_chunk, parts))
            dt = time.perf_counter() - t
    except Exception as e:                                                                  # noqa: BLE001
        return {"unavailable": f"process pool: {type(e).__name__}"}
    return {"value": 4 * total / dt / 1e9, "unit": "GB/s", "cores": len(parts), "kind": "oracle",
            "sample": f"the same first {k} modules in {len(parts)} processes, {dt:.2f} s wall"}


def run_reference(args):
    """The oracle as it stands, on one host core: each step is a bounded
    sample of the workload (its first modules, about 8 s of work), so the
    whole run ends within minutes. ms_per_step is the time of the work each
    step actually did; the whole-batch time at the sampled rate is reported
    apart, as a projection."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, off, cfg = workload(args.workload, 0, args.modules)
    for _ in range(args.warmup):
        cpu_baseline(w, off, budget_s=2.0)
    vals, times, words = [], [], []
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(w, off, budget_s=8.0)
        k = last.pop("k", None)
        vals.append(last["value"])
        times.append(last.pop("seconds"))
        words.append(int(off[k] - off[0]))
    v = float(np.median(vals))
    ms_step = 1e3 * float(np.mean(times))
    sample_cfg = dict(cfg)
    sample_cfg.update({"workload": f"first {k:,} modules of the {cfg['workload']}", "modules": k,
                       "words": words[-1], "sample_of": cfg["workload"]})
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": sample_cfg,
            "projection": {"scope": "the whole workload at the sampled rate (not measured)",
                           "words": int(len(w)), "ms_per_step": 1e3 * 4.0 * len(w) / (v * 1e9) if v > 0 else None},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": last["sample"], "value": v, "unit": "GB/s"},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BIN_INSTR = (200, 2_000, 20_000, 50_000)


def bins_leg(args, spvgpu, synth, dev):
    """Size bins (1,000 modules each at 200 / 2k / 20k / 50k instructions, 1-8
    kernels): per bin every tile shape of spv_process_batch timed, the
    autotuner's pick, and the whole step (decode + validate + encode with the
    picked shape, then disassemble) captured once in a CUDA graph and
    replayed; against the same decode + validate + encode with one launch
    sequence per module. Returns (bins, words, step ms, launches)."""
    import torch
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    bins, tot_words, tot_ms = [], 0, 0.0
    launches = 0
    for b, ni in enumerate(BIN_INSTR):
        rng = np.random.default_rng(100 + b)
        n_instr = np.full(1000, ni, np.int64)
        n_k = rng.integers(1, 9, 1000).astype(np.int32)
        w_np, off_np = synth.batch(n_instr, n_k, 1_000_000 * (b + 1))
        W, M = len(w_np), len(off_np) - 1
        words = torch.from_numpy(w_np.view(np.int32)).to(dev)
        mod_off = torch.from_numpy(off_np).to(dev)
        table = spvgpu.Table(M, W, dev)
        out = torch.empty_like(words)
        sweep = {}
        for tw, nt in spvgpu.TILE_SHAPES:
            c = spvgpu.make_config(tw, nt)
            ws = spvgpu.Workspace(M, W, dev, 0, c)
            for _ in range(2):
                spvgpu.process(words, mod_off, encode=True, table=table, workspace=ws, out=out, cfg=c)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t = 0.0
            for _ in range(3):
                flush.zero_()
                e0.record()
                spvgpu.process(words, mod_off, encode=True, table=table, workspace=ws, out=out, cfg=c)
                e1.record()
                torch.cuda.synchronize()
                t += e0.elapsed_time(e1)
            sweep[f"{tw}x{nt}"] = t / 3
            del ws
        best, best_ms, _ = spvgpu.autotune(words, mod_off, table=table, out=out, reps=3)
        ws = spvgpu.Workspace(M, W, dev, 0, best)
        dws = spvgpu.DisWorkspace(M, W, W, dev)
        _, toff, _ = spvgpu.disassemble(words, mod_off, table, workspace=dws)
        L = int(toff[-1].item())
        text = torch.empty(L + 16, dtype=torch.uint8, device=dev)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            spvgpu.process(words, mod_off, encode=True, table=table, workspace=ws, out=out, cfg=best)
            spvgpu.disassemble(words, mod_off, table, workspace=dws, text=text, sync=False)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            r = spvgpu.process(words, mod_off, encode=True, table=table, workspace=ws, out=out, cfg=best)
            _, _, dst = spvgpu.disassemble(words, mod_off, table, workspace=dws, text=text, sync=False)
        for _ in range(max(3, args.warmup)):
            g.replay()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        step_ms = float(np.median(ts))
        ok = bool((r["status"] == 0).all().item()) and bool((dst == 0).all().item())
        # decode + validate + encode, one launch sequence per module
        pm = spvgpu.make_config(per_module=1)
        wsp = spvgpu.Workspace(M, W, dev, 0, pm)
        spvgpu.process(words, mod_off, encode=True, table=table, workspace=wsp, out=out, cfg=pm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        spvgpu.process(words, mod_off, encode=True, table=table, workspace=wsp, out=out, cfg=pm)
        torch.cuda.synchronize()
        pm_ms = (time.perf_counter() - t0) * 1e3
        launches += args.steps * 14
        bins.append({"instr_per_module": ni, "modules": M, "words": W, "text_bytes": L,
                     "sweep_process_ms": {k: round(v, 4) for k, v in sweep.items()},
                     "autotuned": f"{best.tile_words}x{best.threads}", "autotuned_process_ms": best_ms,
                     "graph_step_ms": step_ms, "graph_step_gbs": 4 * W / (step_ms * 1e-3) / 1e9,
                     "process_gbs": 4 * W / (best_ms * 1e-3) / 1e9,
                     "per_module_process_gbs": 4 * W / (pm_ms * 1e-3) / 1e9, "all_status_ok": ok})
        tot_words += W
        tot_ms += step_ms
        del words, mod_off, table, out, ws, wsp, dws, text, g, r, dst
        torch.cuda.empty_cache()
    return bins, tot_words, tot_ms, launches


def run_bins(args):
    """The size-bin workload alone (bins_leg), as its own JSON line."""
    import torch
    from paper_2305_09493_b300 import build, spvgpu, synth
    build.build()
    spvgpu.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    clocks = Clocks(torch.cuda.current_device())
    bins, tot_words, tot_ms, launches = bins_leg(args, spvgpu, synth, dev)
    clk = clocks.stop()
    line = {"metric": METRIC, "value": 4 * tot_words / (tot_ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "4 size bins x 1,000 modules at 200 / 2k / 20k / 50k instructions",
                       "parallelism": "1 GPU", "graph": "each bin's step captured once in a CUDA graph, replayed",
                       "l2": "L2 flushed (252 MiB write) before every timed replay"},
            "bins": bins, "clocks": clk, "gpu_launches": launches}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "bins":
        run_bins(args)
        return
    import torch
    rank, world = dist_setup(args.gpus)
    from paper_2305_09493_b300 import build, spvgpu
    build.build()
    spvgpu.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    w_np, off_np, cfg = workload(args.workload, rank, args.modules)
    W, M = len(w_np), len(off_np) - 1
    words = torch.from_numpy(w_np.view(np.int32)).to(dev)
    mod_off = torch.from_numpy(off_np).to(dev)
    stream = torch.cuda.current_stream()

    # resident outputs and workspaces, reused by every step
    table = spvgpu.Table(M, W, dev)
    ws = spvgpu.Workspace(M, W, dev)
    out = torch.empty_like(words)
    dws = spvgpu.DisWorkspace(M, W, W, dev)
    r = spvgpu.process(words, mod_off, encode=True, table=table, workspace=ws, out=out)
    text, text_off, dst = spvgpu.disassemble(words, mod_off, table, workspace=dws)
    torch.cuda.synchronize()
    N = int(table.mod_first_row[-1].item())
    Ltext = int(text_off[-1].item())
    status_ok = bool((r["status"] == 0).all().item()) and bool((dst == 0).all().item())
    text_buf = torch.empty(Ltext + 1, dtype=torch.uint8, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev) if 4 * W < 2 * L2_BYTES else None

    def step():
        spvgpu.process(words, mod_off, encode=True, table=table, workspace=ws, out=out)
        spvgpu.disassemble(words, mod_off, table, workspace=dws, text=text_buf, sync=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    clocks = Clocks(torch.cuda.current_device())
    spvgpu.profile_enable(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        if flush is not None:
            flush.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    prof = spvgpu.profile_read()
    spvgpu.profile_enable(False)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_ms = float(np.sum(step_ms))
    t_ms = max_over_ranks([t_ms], world)[0]
    ms_per_step = t_ms / args.steps
    value = job_gbs(world, W, ms_per_step)

    # roofline of the dominant kernel, and of the decode + validate + encode
    # kernel. A kernel's time is its time per step: k_tile launches twice per
    # step, the second launch a guarded redo that returns at once unless an
    # entry guess failed.
    launches = sum(v[0] for v in prof.values())
    top = max(prof.items(), key=lambda kv: kv[1][1])
    peak, peak_kind = measured_peaks()
    tj = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    tjd = json.load(open(tj)) if os.path.exists(tj) else {}

    def kernel_roofline(kname):
        kl, kms = prof[kname]
        step_ms_k = kms / args.steps
        alg = algorithmic_bytes(kname, W, N, Ltext, M)
        traffic, inst = None, None
        kt = tjd.get("kernels", {}).get(kname, {})
        if kt.get("source_sha") == source_hash(kname) and tjd.get("workload") == args.workload and \
                tjd.get("modules") == M:
            traffic = kt.get("bytes_per_launch")
            inst = kt.get("warp_instructions_per_launch")
        ach = alg / (step_ms_k * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": kname, "achieved": ach, "peak": peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": ach / peak, "traffic": traffic, "algorithmic_bytes_per_launch": alg,
                "ms_per_launch": step_ms_k, "launches_per_step": kl / args.steps,
                "issue": issue_roofline(inst, step_ms_k, clk)}
    kernels = {k: {"launches": v[0], "ms_per_step": v[1] / args.steps} for k, v in
               sorted(prof.items(), key=lambda kv: -kv[1][1])}

    # end to end through spv_pipe_run: the batch in pinned host memory, the
    # results back in pinned host memory; uploads, kernels and downloads of
    # successive chunks overlap. The serial chain (one upload, the step, one
    # download, on one stream) is timed beside it for comparison.
    h_words = torch.from_numpy(w_np.view(np.int32)).pin_memory()
    h_off = torch.from_numpy(off_np).pin_memory()
    h_status = torch.empty(M, dtype=torch.int32).pin_memory()
    h_err = torch.empty(M, dtype=torch.int64).pin_memory()
    h_toff = torch.empty(M + 1, dtype=torch.int64).pin_memory()
    h_text = torch.empty(Ltext + 1, dtype=torch.uint8).pin_memory()
    pipe = spvgpu.Pipe(chunk_words=args.e2e_chunk_words)
    pipe.run(h_words, h_off, h_status, h_err, h_toff, h_text)
    # the pipeline's downloaded results against the resident step's, byte for
    # byte: text, text offsets, statuses and error rows
    e2e_ok = bool(torch.equal(h_text[:Ltext], text_buf[:Ltext].cpu())) and \
        bool(torch.equal(h_toff, text_off.cpu())) and \
        bool(torch.equal(h_status, r["status"].cpu())) and bool(torch.equal(h_err, r["err_row"].cpu()))
    ksteps = max(1, min(args.steps, 5))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ksteps):
        pipe.run(h_words, h_off, h_status, h_err, h_toff, h_text)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / ksteps
    pipe.close()
    chunk_words = args.e2e_chunk_words or (8 << 20)
    n_chunks, a = 0, 0
    while a < M:                                   # the library's chunking: whole modules, ~chunk_words words
        b = a + 1
        while b < M and off_np[b + 1] - off_np[a] <= chunk_words:
            b += 1
        n_chunks, a = n_chunks + 1, b
    e_words = torch.empty_like(words)
    e_off = torch.empty_like(mod_off)

    def serial_step():
        e_words.copy_(h_words, non_blocking=True)
        e_off.copy_(h_off, non_blocking=True)
        rr = spvgpu.process(e_words, e_off, encode=True, table=table, workspace=ws, out=out)
        _, toff, _ = spvgpu.disassemble(e_words, e_off, table, workspace=dws, text=text_buf, sync=False)
        h_status.copy_(rr["status"], non_blocking=True)
        h_err.copy_(rr["err_row"], non_blocking=True)
        h_toff.copy_(toff, non_blocking=True)
        h_text.copy_(text_buf, non_blocking=True)

    serial_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(ksteps):
        serial_step()
    e1.record(stream)
    torch.cuda.synchronize()
    serial_ms = e0.elapsed_time(e1) / ksteps
    e2e_ms, serial_ms = max_over_ranks([e2e_ms, serial_ms], world)
    e2e = {"value": job_gbs(world, W, e2e_ms), "unit": "GB/s",
           "h2d_bytes_per_step": 4 * W + 8 * (M + n_chunks),
           "d2h_bytes_per_step": 4 * M + 8 * M + 8 * (M + n_chunks) + Ltext,
           "ms_per_step": e2e_ms, "api": "spv_pipe_run", "chunks": n_chunks, "results_exact": e2e_ok,
           "serial_one_stream": {"ms_per_step": serial_ms, "value": job_gbs(world, W, serial_ms)}}

    # logical layout and scopes over the decoded table (spv_layout_batch):
    # reads the op column (2 bytes per row) and the module row offsets
    lay_ms = []
    lws = torch.empty(max(1, spvgpu.load().spv_layout_workspace_bytes(M, table.capacity_rows)), dtype=torch.uint8,
                      device=dev)
    for k in range(6):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if flush is not None:
            flush.zero_()
        a.record(stream)
        lst, _ = spvgpu.layout(table, M, workspace=lws)
        b.record(stream)
        torch.cuda.synchronize()
        if k:
            lay_ms.append(a.elapsed_time(b))
    lay = float(np.median(lay_ms))
    layout_leg = {"scope": "section order and function / block nesting over the decoded table",
                  "ms": lay, "rows_per_s": N / (lay * 1e-3), "achieved_gbs": (2 * N + 8 * M) / (lay * 1e-3) / 1e9,
                  "all_clean": bool((lst == 0).all().item())}

    # assembler (spv_assemble_batch): the step's own text back to words, which
    # must be the input words; reads the text (L bytes), writes 4 W bytes
    aws = spvgpu.AsmWorkspace(M, Ltext, dev)
    a_words = torch.empty_like(words)
    a_text = text_buf[:Ltext]
    spvgpu.assemble(a_text, text_off, words=a_words, workspace=aws)
    asm_ms = []
    spvgpu.profile_enable(True)
    for k in range(6):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if flush is not None:
            flush.zero_()
        a.record(stream)
        _, a_off, a_st, _ = spvgpu.assemble(a_text, text_off, words=a_words, workspace=aws, sync=False)
        b.record(stream)
        torch.cuda.synchronize()
        if k:
            asm_ms.append(a.elapsed_time(b))
    aprof = spvgpu.profile_read()
    spvgpu.profile_enable(False)
    asm_t = float(np.median(asm_ms))
    asm_kernels = {k: {"launches": v[0], "ms_per_call": v[1] / 6} for k, v in
                   sorted(aprof.items(), key=lambda kv: -kv[1][1])[:8]}
    # the dominant kernel: reads the text and 12 bytes per line (line start,
    # module), writes 41 bytes per line (word count, names, flags, 32-byte slot)
    n_lines, _ = spvgpu.spv_asm_required(spvgpu._ptr(aws.buf))
    mk_l, mk_ms = aprof["k_asm_measure"]
    meas_ms = mk_ms / mk_l
    meas_alg = Ltext + 53 * n_lines
    meas_traffic, meas_inst = None, None
    if os.path.exists(tj):
        kt = json.load(open(tj)).get("kernels", {}).get("k_asm_measure", {})
        if kt.get("source_sha") == source_hash("k_asm_measure") and kt.get("lines") == n_lines:
            meas_traffic, meas_inst = kt.get("bytes_per_launch"), kt.get("warp_instructions_per_launch")
    asm_leg = {"scope": "the step's disassembly text back to words (named ids, types, constants, headers)",
               "ms": asm_t, "text_gbs": Ltext / (asm_t * 1e-3) / 1e9,
               "achieved_gbs": (Ltext + 4 * W) / (asm_t * 1e-3) / 1e9,
               "round_trip_exact": bool(torch.equal(a_words, words)) and bool(torch.equal(a_off, mod_off))
               and bool((a_st == 0).all().item()),
               "lines": n_lines,
               "roofline": {"bound": "hbm", "kernel": "k_asm_measure",
                            "achieved": meas_alg / (meas_ms * 1e-3) / 1e9, "peak": peak, "peak_kind": peak_kind,
                            "unit": "GB/s", "frac": meas_alg / (meas_ms * 1e-3) / 1e9 / peak,
                            "traffic": meas_traffic, "algorithmic_bytes_per_launch": meas_alg,
                            "ms_per_launch": meas_ms, "issue": issue_roofline(meas_inst, meas_ms, clk)},
               "kernels": asm_kernels}

    # builder (spv_build_batch): the batch's own op lists, the rows a JIT
    # backend hands over, back to modules. Algorithmic bytes: per row the
    # opcode (2) and operand offset (8), per operand its value (4) and kind
    # (1), per output word 4.
    bld_leg = None
    if args.workload == "batch":
        from paper_2305_09493_b300 import synth
        ol = synth.oplist_module_batch(M, seed0=rank * M)
        d_ol = (torch.from_numpy(ol["op"].view(np.int16)).to(dev), torch.from_numpy(ol["opd_off"]).to(dev),
                torch.from_numpy(ol["opd"].view(np.int32)).to(dev), torch.from_numpy(ol["opd_ref"]).to(dev),
                torch.from_numpy(ol["row_off"]).to(dev))
        bws = spvgpu.BuildWorkspace(M, len(ol["op"]), dev)
        b_words = torch.empty_like(words)
        spvgpu.build_modules(*d_ol, version=0x00010200, generator=32, words=b_words, workspace=bws)
        bld_ms = []
        spvgpu.profile_enable(True)
        for k in range(6):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if flush is not None:
                flush.zero_()
            a.record(stream)
            _, b_off, b_st, _, _ = spvgpu.build_modules(*d_ol, version=0x00010200, generator=32, words=b_words,
                                                       workspace=bws, sync=False)
            b.record(stream)
            torch.cuda.synchronize()
            if k:
                bld_ms.append(a.elapsed_time(b))
        bprof = spvgpu.profile_read()
        spvgpu.profile_enable(False)
        bt = float(np.median(bld_ms))
        n_rows, n_opd = len(ol["op"]), len(ol["opd"])
        balg = 10 * n_rows + 5 * n_opd + 4 * W + 8 * M
        # the built modules are the batch up to a renaming of ids: the same
        # offsets, the same non-id words (the generator marks the id words)
        got = b_words.cpu().numpy().view(np.uint32)
        keep = ol["is_id"] == 0
        keep[(off_np[:-1, None] + np.arange(5)).ravel()] = False
        same = bool(np.array_equal(b_off.cpu().numpy(), off_np)) and bool((b_st == 0).all().item()) and \
            bool(np.array_equal(got[keep], w_np[keep]))
        bk = sorted(bprof.items(), key=lambda kv: -kv[1][1])
        bld_leg = {"scope": "the batch's op lists (rows with references) to modules, ids by a scan",
                   "rows": n_rows, "operands": n_opd, "ms": bt, "words_gbs": 4 * W / (bt * 1e-3) / 1e9,
                   "achieved_gbs": balg / (bt * 1e-3) / 1e9, "algorithmic_bytes": balg,
                   "frac_of_hbm": balg / (bt * 1e-3) / 1e9 / peak, "modules_equal_up_to_id_renaming": same,
                   "kernels": {k: {"launches": v[0], "ms_per_call": v[1] / 6} for k, v in bk[:6]}}
        del d_ol, bws, b_words, ol

    # batched vs per-module launches (decode+validate+encode, same exact output)
    cmp = None
    if not args.no_per_module and world == 1:
        def process_only(cfg_):
            spvgpu.process(words, mod_off, encode=True, table=table, workspace=ws, out=out, cfg=cfg_)
        res = {}
        for label, cfg_ in (("batched", None), ("per_module", spvgpu.make_config(per_module=1))):
            process_only(cfg_)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3 if label == "batched" else 1
            if flush is not None:
                flush.zero_()
            a.record(stream)
            for _ in range(reps):
                process_only(cfg_)
            b.record(stream)
            torch.cuda.synchronize()
            res[label] = 4 * W / (a.elapsed_time(b) / reps * 1e-3) / 1e9
        cmp = {"scope": "decode+validate+encode", "batched_gbs": res["batched"], "per_module_gbs": res["per_module"],
               "speedup": res["batched"] / res["per_module"]}

    serve = None
    if args.serve_seconds > 0 and world == 1:
        cap = int(args.serve_cap_gb * (1 << 30))
        legs = []
        for rate in (float(x) for x in args.serve_rates.split(",") if x):
            legs.append({"rate_per_s": rate,
                         "continuous_batching": serve_leg(spvgpu, w_np, off_np, rate, args.serve_seconds, cap=cap),
                         "one_module_per_launch": serve_leg(spvgpu, w_np, off_np, rate, args.serve_per_launch_seconds,
                                                            max_batch_modules=1, cap=cap)})
        serve = {"scope": "decode+validate+disassemble per module, Poisson arrivals, latency from arrival to completion",
                 "cap_gb": args.serve_cap_gb, "seconds_per_rate": args.serve_seconds,
                 "per_launch_seconds_per_rate": args.serve_per_launch_seconds, "legs": legs}
    bins = None
    if not args.no_bins and world == 1 and args.workload == "batch":
        from paper_2305_09493_b300 import synth as _synth
        del table, ws, out, dws, text_buf, e_words, e_off, words, mod_off, aws, a_words
        torch.cuda.empty_cache()
        b_list, b_words, b_ms, b_launch = bins_leg(args, spvgpu, _synth, dev)
        bins = {"scope": "4 size bins x 1,000 modules; per bin the tile-shape sweep, the autotuner's pick, the "
                         "whole step in one CUDA graph, and one launch sequence per module",
                "graph_steps_gbs": 4 * b_words / (b_ms * 1e-3) / 1e9, "bins": b_list}
    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w_np, off_np)
        cpu.pop("seconds")
        cpu["all_cores"] = cpu_all_cores(w_np, off_np, cpu.pop("k"))
    cfg.update({"rows": N, "text_bytes": Ltext, "l2": "inputs larger than L2" if flush is None else
                "L2 flushed (252 MiB write) between timed steps", "parallelism": f"{world} GPU(s), one batch each",
                "all_status_ok": status_ok})
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": cfg,
        "roofline": kernel_roofline(top[0]),
        "roofline_decode_validate_encode": kernel_roofline("k_tile") if "k_tile" in prof else None,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "batched_vs_per_module": cmp,
        "layout": layout_leg,
        "assemble": asm_leg,
        "build": bld_leg,
        "serve": serve,
        "size_bins": bins,
        "clocks": clk,
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()


if __name__ == "__main__":
    main()
