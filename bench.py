#!/usr/bin/env python
"""Benchmark: compress + decompress throughput of the cuSZ+ data-parallel path on GB300.

One step = compress one synthetic field (device-resident FP32) to an archive and
decompress it back, through the library's C ABI.  Default workload: the largest
single-field configuration, a 3-D 512^3 log-normal density exp(1.5 g) (g a GRF with
spectrum k^-2.5), value-range-relative eb 1e-4, exhaustive per-block choice between
Huffman, RLE and RLE+Huffman.  The field (537 MB) is larger than L2, and L2 is also
flushed before every timed step.

Prints one JSON line (rank 0).  `--impl reference` times the scalar CPU oracle on
the host cores instead (bounded samples of the same workload, one slab per core).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

L2_BYTES = 129 * 1024 * 1024
FLUSH_BYTES = 256 * 1024 * 1024


def flush_l2(buf: torch.Tensor, sink: torch.Tensor, i: int) -> None:
    """Evict the previous step's data from L2 (untimed): write a buffer twice the L2,
    then read it back, so the lines L2 holds afterwards are clean flush data (the
    write-back of the flush's dirty lines happens here, not inside the timed step)."""
    buf.fill_(float(i))
    torch.sum(buf, dim=0, out=sink)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["2d", "1d", "3d"], default="3d")
    p.add_argument("--select", default="exhaustive")
    p.add_argument("--n3d", type=int, default=512, help="side of the 3-D workload")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain comparison")
    p.add_argument("--batch-scale", type=float, default=1.0, help="size factor of the 256-field batch")
    return p.parse_args()


def workload_spec(name, rank=0, n3d=512):
    from paper_2105_12912_gb300 import synth
    if name == "2d":
        return synth.workload_2d(seed=2 + 1000 * rank)
    if name == "1d":
        return synth.workload_1d(seed=1 + 1000 * rank)
    return synth.workload_3d(n=n3d, seed=3 + 1000 * rank, eb=1e-4)


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def fused_block_fraction(codec, dims):
    """Fraction of the field's elements in blocks whose decoding and reconstruction run
    fused (Huffman-coded blocks of full codec-block extent)."""
    blk = {1: (4096,), 2: (64, 64), 3: (16, 16, 16)}[len(dims)]
    g = [-(-d // b) for d, b in zip(dims, blk)]
    full = np.ones(g, dtype=bool)
    for ax, (d, b) in enumerate(zip(dims, blk)):
        if d % b:
            idx = [slice(None)] * len(dims)
            idx[ax] = -1
            full[tuple(idx)] = False
    fused = full.ravel() & (codec == 0)
    return float(fused.sum()) * int(np.prod(blk)) / float(np.prod(dims))


def algorithmic_bytes(kernel, n, nslots, nblk, hdr, fused_frac=0.0):
    """Bytes a kernel must move per launch: the input it reads and the output it
    writes once (codes 2 B per slot, records 8 B, the payload), nothing re-read.  The
    entropy decoder reconstructs fused blocks itself: for those it writes the floats
    (4 B per element) instead of codes."""
    payload, n_rec = hdr["payload"], hdr["n_rec"]
    nh, nr, nrh = hdr["n_codec"]
    huff_frac = nh / max(1, nblk)
    if kernel == "range":
        return 4 * n
    if kernel == "construct":
        return 4 * n + 2 * nslots + 8 * n_rec
    if kernel == "encode":
        return 2 * nslots + payload + 5 * nblk
    if kernel == "stream_decode":
        return payload + int(4 * n * fused_frac) + int(2 * n * max(0.0, huff_frac - fused_frac))
    if kernel == "rle_expand":
        return int(2 * n * (1 - huff_frac))
    if kernel == "reconstruct":
        slow = 1.0 - fused_frac
        return int((2 * nslots + 4 * n) * slow) + 8 * n_rec
    return 0


SELECTORS = {"huff": 0, "rle": 1, "rle_huff": 2, "heuristic": 3, "exhaustive": 4}
SLAB_ROWS = {"3d": 16, "2d": 128, "1d": 1 << 18}  # rows of the slowest axis per oracle slab


def _save_sample(x_cpu, rows):
    """The first `rows` rows of the field as a .npy file the oracle workers map."""
    import tempfile
    d = tempfile.mkdtemp(prefix="cszp_oracle_")
    path = os.path.join(d, "field.npy")
    np.save(path, np.ascontiguousarray(x_cpu[:rows].numpy()))
    return path


def run_reference(args):
    """Reference arm: the scalar C oracle, unchanged, on the host cores (rank 0 only):
    every step is one round trip of `cores` independent slabs of the same field, one
    oracle process per core."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import timing
    from paper_2105_12912_gb300 import synth
    spec = workload_spec(args.workload, 0, args.n3d)
    x = synth.make_field(spec, "cpu")
    cores = timing.host_cores()
    rows = SLAB_ROWS[args.workload]
    nslab = max(1, min(cores, x.shape[0] // rows))
    path = _save_sample(x, rows * nslab)
    bounds = [(i * rows, (i + 1) * rows) for i in range(nslab)]
    mode = 1 if spec.eb_mode == "rel" else 0
    sel = SELECTORS[args.select]
    per_slab = 4 * int(np.prod(x.shape[1:])) * rows
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(nslab) as pool:
        pool.map(timing._warm, range(nslab))
        work = [(path, lo, hi, mode, spec.eb, sel) for lo, hi in bounds]
        for _ in range(args.warmup):
            pool.map(timing._round_trip, work, chunksize=1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(timing._round_trip, work, chunksize=1)
        t = time.perf_counter() - t0
    gbs = args.steps * per_slab * nslab / t / 1e9
    line = {"impl": "reference", "metric": "compress+decompress GB/s (FP32 in)", "value": gbs, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": spec.name, "dims": list(spec.dims), "eb_mode": spec.eb_mode, "eb": spec.eb,
                       "select": args.select},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": nslab, "kind": "oracle",
                             "sample": f"per step, {nslab} independent slabs of {rows} rows of the field "
                                       f"({per_slab // 4} floats each), one oracle process per core"},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(spec, x_cpu, select, workload):
    """The oracle, unchanged, on bounded samples of the field (independent slabs along
    the slowest axis, each compressed and decompressed as a field of its own):
    single-threaded over 8 slabs, and with one process per host core over two slabs
    per core.  Data generation and process start-up are not timed."""
    from oracle import timing
    mode = 1 if spec.eb_mode == "rel" else 0
    sel = SELECTORS.get(select, 4)
    cores = timing.host_cores()
    rows = SLAB_ROWS[workload]
    nrows = x_cpu.shape[0]
    nslab = max(1, min(nrows // rows, max(8, 2 * cores)))
    path = _save_sample(x_cpu, rows * nslab)
    bounds = [(i * rows, (i + 1) * rows) for i in range(nslab)]
    per_slab = 4 * int(np.prod(x_cpu.shape[1:])) * rows
    n1 = min(8, nslab)
    t1, _ = timing.time_slabs(path, bounds[:n1], mode, spec.eb, sel, 1)
    tp, _ = timing.time_slabs(path, bounds, mode, spec.eb, sel, cores)
    try:
        os.remove(path)
        os.rmdir(os.path.dirname(path))
    except OSError:
        pass
    single = n1 * per_slab / t1 / 1e9
    par = nslab * per_slab / tp / 1e9
    return {"value": par, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{nslab} independent slabs of {rows} rows ({per_slab // 4} floats each), compressed and "
                      f"decompressed by {cores} oracle processes side by side ({tp:.1f} s wall)",
            "single_thread": {"value": single, "unit": "GB/s", "cores": 1,
                              "sample": f"{n1} of the same slabs, one after another ({t1:.1f} s)"}}


def batched_comparison(args, dev, flush):
    """256 seeded fields of uneven shape and dimensionality (1-D 1e4-3e8, 2-D up to
    4096^2, 3-D up to 256x512x512, spectra k^-2..k^-4, 0-50% zero blocks, rel eb in
    {1e-2, 1e-3, 1e-4}): the plain per-field path (csz_compress per field, exhaustive
    selection) against the batched path (one launch per stage, CUDA graph) with the
    learned selector and with exhaustive selection.  Compression only."""
    sink = torch.empty((), dtype=torch.float32, device=dev)
    from paper_2105_12912_gb300 import api, selector, synth
    specs = synth.workload_batch(256, scale=args.batch_scale)
    xs = [synth.make_field(sp, dev) for sp in specs]
    ebs = [sp.eb for sp in specs]
    modes = [sp.eb_mode for sp in specs]
    n_in = sum(4 * x.numel() for x in xs)
    caps = [min(api.max_archive_bytes(tuple(x.shape)), 6 * x.numel() + (1 << 20)) for x in xs]
    # selector weights: trained on the method's own sizes from separately seeded fields
    # of the same mix (seeds 9000+, a twentieth of the size) and 3-D zero-block fields
    train_specs = synth.workload_batch(48, seed0=9000, scale=0.05)
    rows = selector.collect_rows(
        [(lambda sp=sp: synth.make_field(sp, dev), sp.eb, sp.eb_mode) for sp in train_specs] +
        [(lambda s=s: synth.make_field(synth.workload_selector(s, dims=(48, 160, 160)), dev), 1e-3, "rel")
         for s in range(1000, 1008)])
    w, _, _ = selector.train(rows, seed=0, steps=3000, lr=1e-2)
    stream = torch.cuda.current_stream()
    ws = api.Workspace(dev)
    arc = torch.empty(max(caps), dtype=torch.uint8, device=dev)

    def plain():
        tot = 0
        for x, eb, m in zip(xs, ebs, modes):
            _, nb, _ = api.compress(x, eb, m, select="exhaustive", out=arc[:min(arc.numel(), 6 * x.numel() + (1 << 20))],
                                    workspace=ws)
            tot += nb
        return tot

    def timed(fn, reps):
        out = []
        for i in range(reps):
            flush_l2(flush, sink, i)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = fn()
            b.record(stream)
            torch.cuda.synchronize()
            out.append((a.elapsed_time(b), r))
        return out

    plain_bytes = plain()
    t_plain = [t for t, _ in timed(plain, 3)]
    # plain round trip: per-field compress + decompress
    outs = [torch.empty_like(x) for x in xs]

    def plain_rt():
        for x, eb, m, o in zip(xs, ebs, modes, outs):
            ar, nb, _ = api.compress(x, eb, m, select="exhaustive", out=arc[:min(arc.numel(), 6 * x.numel() + (1 << 20))],
                                     workspace=ws)
            api.decompress(ar, nb, out=o, dims=tuple(x.shape), workspace=ws)
    t_plain_rt = [t for t, _ in timed(plain_rt, 3)]
    res = {}
    for sel, wt in (("learned", w), ("exhaustive", None)):
        bc = api.BatchCompressor(xs, ebs, modes, select=sel, weights=wt, archive_caps=caps)
        bc.run()
        sizes, stats = bc.results()
        if any(stats):
            raise RuntimeError(f"batched {sel}: field status {stats}")
        t_b = [t for t, _ in timed(bc.run, 5)]
        bd = api.BatchDecompressor(bc.archives, [tuple(x.shape) for x in xs], archive_bytes=caps, outs=outs)
        res_warps, _ = bd.tune()
        bd.run()
        dstats = bd.results()
        if any(dstats):
            raise RuntimeError(f"batched decompression: field status {dstats}")

        def rt():
            bc.run()
            bd.run()
        t_rt = [t for t, _ in timed(rt, 5)]
        ok = all(float((x.double() - o.double()).abs().max()) <= api.header(a)["eb_f"]
                 for x, o, a in zip(xs, outs, bc.archives))
        if not ok:
            raise RuntimeError("batched round trip outside the error bound")
        res[sel] = {"gbs": n_in / (np.mean(t_b) * 1e-3) / 1e9, "ms": float(np.mean(t_b)),
                    "rt_gbs": n_in / (np.mean(t_rt) * 1e-3) / 1e9,
                    "bytes": int(sum(sizes)), "tuning": bc.info(), "decoder_warps": res_warps}
        del bd, bc
    plain_gbs = n_in / (np.mean(t_plain) * 1e-3) / 1e9
    plain_rt_gbs = n_in / (np.mean(t_plain_rt) * 1e-3) / 1e9
    return {
        "workload": "batch256_mixed_1d2d3d", "fields": len(xs), "input_bytes": n_in,
        "plain_per_field_gbs": plain_gbs, "plain_ms": float(np.mean(t_plain)), "plain_cr": n_in / plain_bytes,
        "plain_round_trip_gbs": plain_rt_gbs,
        "batched_learned_gbs": res["learned"]["gbs"], "batched_learned_ms": res["learned"]["ms"],
        "batched_learned_cr": n_in / res["learned"]["bytes"],
        "batched_learned_round_trip_gbs": res["learned"]["rt_gbs"],
        "batched_exhaustive_gbs": res["exhaustive"]["gbs"], "batched_exhaustive_cr": n_in / res["exhaustive"]["bytes"],
        "batched_exhaustive_round_trip_gbs": res["exhaustive"]["rt_gbs"],
        "speedup_learned_batched_vs_plain": res["learned"]["gbs"] / plain_gbs,
        "speedup_round_trip_learned_batched_vs_plain": res["learned"]["rt_gbs"] / plain_rt_gbs,
        "cr_loss_learned_vs_plain": res["learned"]["bytes"] / plain_bytes - 1.0,
        "construct_grid": res["learned"]["tuning"]["construct_grid"],
        "decoder_warps_per_cta": res["learned"]["decoder_warps"],
        # the compression plan the autotuner kept (one persistent launch, or one launch
        # per stage) and the batch times it measured for each with 1..4 CTAs per SM
        "plan": {sel: ("persistent" if res[sel]["tuning"]["persistent"] else "staged") for sel in res},
        "autotune_ms": res["learned"]["tuning"]["tuned_ms"],
        "autotune_persistent_ms": {sel: res[sel]["tuning"]["persist_ms"] for sel in res},
        "autotune_staged_ms": {sel: res[sel]["tuning"]["tuned_ms"] for sel in res},
        "note": "GB/s of FP32 input; every timed pass is preceded by a 256 MiB L2 flush; the plain path "
                "synchronises once per call (it returns each size / status to the host); round trips "
                "are compression then decompression",
    }


def kernel_source_rev():
    """Hash of the CUDA sources: DRAM counters taken from an ncu capture are reported
    only while the kernels they measured are unchanged."""
    import hashlib
    root = os.path.join(ROOT, "paper_2105_12912_gb300", "csrc")
    h = hashlib.sha1()
    for f in sorted(os.listdir(root)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(f.encode())
            with open(os.path.join(root, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def whole_job(step_ms, world, bytes_per_rank_step, dist=None, device=None):
    """Whole-job throughput of `world` replicas: each rank's timed steps (ms) are
    summed, the slowest rank's total bounds the job (max over ranks), and the value
    counts the bytes all ranks processed.  Returns (GB/s, total ms of the slowest)."""
    total_ms = float(np.sum(step_ms))
    if dist is not None:
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * len(step_ms) * bytes_per_rank_step / (total_ms * 1e-3) / 1e9, total_ms


def roofline_entry(name, k, peak, peak_kind, traffic):
    return {"bound": "hbm", "kernel": name, "achieved": k["gbs"], "peak": peak, "unit": "GB/s",
            "frac": (k["gbs"] / peak) if k["gbs"] else None, "traffic": traffic,
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json), of measured",
            "note": "achieved = algorithmic bytes per launch / mean launch time (CUDA events)"}


def load_traffic(workload):
    """DRAM bytes per launch from profiles/traffic.json, when its captures were taken
    on the current kernel sources (else no figure)."""
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tpath):
        return {}
    try:
        tj = json.load(open(tpath))
    except Exception:
        return {}
    if tj.get("source_rev") != kernel_source_rev():
        return {}
    out = {}
    for key, ent in tj.get("entries", {}).items():
        wl, _, kern = key.partition(":")
        if wl == workload:
            out[kern] = ent.get("bytes_per_launch")
    return out


def run_ours(args):
    from paper_2105_12912_gb300 import api, synth
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()

    spec = workload_spec(args.workload, rank, args.n3d)
    x = synth.make_field(spec, dev)
    n = x.numel()
    bytes_in = 4 * n
    dims = tuple(x.shape)
    ws = api.Workspace(dev)
    # archive buffer: twice the input is ample for these fields (the worst-case bound,
    # csz_max_archive_bytes, is 32 B per element); a smaller buffer is an error, not UB
    arc = torch.empty(min(api.max_archive_bytes(dims), 8 * n + (1 << 20)), dtype=torch.uint8, device=dev)
    rec = torch.empty_like(x)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)

    # The timed step: one round trip through the public calls -- compression (one host
    # synchronisation, which returns the size and the header) and decompression with
    # no host round trip (its status stays on the device until after the timed region).
    dstatus = torch.zeros(1, dtype=torch.int32, device=dev)

    def step():
        ar, nb, hb = api.compress_with_header(x, spec.eb, spec.eb_mode, select=args.select, out=arc,
                                              workspace=ws)
        api.decompress_async(ar, nb, hb, rec, dstatus, workspace=ws)
        return nb

    for _ in range(args.warmup):
        nb = step()
    torch.cuda.synchronize()
    # correctness guard on the measured configuration
    assert int(dstatus.item()) == 0
    err = float((x.double() - rec.double()).abs().max())
    hdr = api.header(arc)
    assert err <= hdr["eb_f"], (err, hdr["eb_f"])
    hdr_bytes = bytes(arc[:128].cpu().numpy().tobytes())
    codec = arc[128:128 + hdr["nblk"]].cpu().numpy()

    def timed(fn, steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush_l2(flush, sink, i)  # evict the previous step's data from L2 (untimed)
            evs[i][0].record(stream)
            fn()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    api.trace_read(reset=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_round = timed(step, args.steps)
    launches = sum(c for _, c in api.trace_read(reset=True).values())
    torch.cuda.synchronize()
    assert int(dstatus.item()) == 0
    if dist:
        dist.barrier()
    ms_step = float(np.mean(t_round))
    value, total_ms = whole_job(t_round, world, bytes_in, dist, dev)

    # compress-only and decompress-only throughput of the same calls
    t_c = timed(lambda: api.compress(x, spec.eb, spec.eb_mode, select=args.select, out=arc, workspace=ws),
                max(10, args.steps // 2))
    t_d = timed(lambda: api.decompress_async(arc, nb, hdr_bytes, rec, dstatus, workspace=ws),
                max(10, args.steps // 2))
    assert int(dstatus.item()) == 0

    # The same round trip replayed as CUDA graphs through the batch calls with one
    # field (no host synchronisation at all); archive and reconstruction checked
    # identical to the plain calls'.
    bc = api.BatchCompressor([x], spec.eb, spec.eb_mode, select=args.select, archive_caps=[arc.numel()])
    bc.run()
    gsizes, gstat = bc.results()
    assert gstat == [0] and gsizes[0] == nb and torch.equal(bc.archives[0][:nb], arc[:nb])
    bd = api.BatchDecompressor(bc.archives, [dims], archive_bytes=[nb])
    dec_warps, _ = bd.tune()
    bd.run()
    assert bd.results() == [0] and torch.equal(bd.outs[0].view(torch.int32), rec.view(torch.int32))

    def graph_step():
        bc.run()
        bd.run()

    for _ in range(3):
        graph_step()
    t_graph = timed(graph_step, max(10, args.steps // 2))
    t_gc = timed(bc.run, max(10, args.steps // 2))
    t_gd = timed(bd.run, max(10, args.steps // 2))
    assert bc.results()[1] == [0] and bd.results() == [0]
    del bd, bc

    # per-kernel durations of the timed step (CUDA events around each launch on the
    # launching stream)
    api.trace_enable(True)
    api.trace_read(reset=True)
    timed(step, max(10, args.steps // 2))
    tr = api.trace_read(reset=True)
    api.trace_enable(False)
    assert int(dstatus.item()) == 0
    nslots = 4096 * hdr["nblk"]
    peak, peak_kind = measured_peak_hbm()
    fused_frac = fused_block_fraction(codec, dims)
    kernels = {}
    for name, (ms, cnt) in tr.items():
        if cnt == 0:
            continue
        avg_ms = ms / cnt
        ab = algorithmic_bytes(name, n, nslots, hdr["nblk"], hdr, fused_frac)
        kernels[name] = {"launches": cnt, "avg_us": 1e3 * avg_ms, "share": None,
                         "alg_bytes": ab, "gbs": (ab / (avg_ms * 1e-3) / 1e9) if ab and avg_ms > 0 else None}
    tot = sum(v["avg_us"] * v["launches"] for v in kernels.values())
    for v in kernels.values():
        v["share"] = v["avg_us"] * v["launches"] / tot if tot else None
    dom = max(kernels, key=lambda k: kernels[k]["avg_us"] * kernels[k]["launches"])
    traffic = load_traffic(args.workload)
    roofline = roofline_entry(dom, kernels[dom], peak, peak_kind, traffic.get(dom))
    # the Lorenzo kernels of the method (construct; reconstruct, which runs inside the
    # entropy decoder for fused blocks) each against the same peak
    roofline["lorenzo"] = {k: roofline_entry(k, kernels[k], peak, peak_kind, traffic.get(k))
                           for k in ("construct", "reconstruct", "stream_decode") if k in kernels}

    # end to end through the public API with host buffers (pinned), copies timed.
    # Serial: one step at a time (field in, compress, archive out and back in,
    # decompress, reconstruction out).  Streamed: the same steps issued on two streams
    # with their own buffers and workspaces, as a compressor that streams fields would
    # run, so that one step's reconstruction copy to the host overlaps the next step's
    # field copy to the device and its compression (the host link is full duplex);
    # K steps are timed as one region and every step's copies are inside it.
    e2e = None
    if not args.no_e2e:
        xh = x.cpu().pin_memory()
        slots = []
        for _ in range(2):
            slots.append({
                "s": torch.cuda.Stream(), "ws": api.Workspace(dev), "xd": torch.empty_like(x),
                "arc": torch.empty_like(arc), "ard": torch.empty_like(arc),
                "arh": torch.empty(arc.numel(), dtype=torch.uint8, pin_memory=True),
                "rec": torch.empty_like(x), "outh": torch.empty(dims, dtype=torch.float32, pin_memory=True),
                "st": torch.zeros(1, dtype=torch.int32, device=dev)})
        nb_box = [0]

        def e2e_one(S):
            s = S["s"]
            with torch.cuda.stream(s):
                S["xd"].copy_(xh, non_blocking=True)
                ar, nbe, hb = api.compress_with_header(S["xd"], spec.eb, spec.eb_mode, select=args.select,
                                                       out=S["arc"], workspace=S["ws"], stream=s)
                S["arh"][:nbe].copy_(ar[:nbe], non_blocking=True)
                S["ard"][:nbe].copy_(S["arh"][:nbe], non_blocking=True)
                api.decompress_async(S["ard"], nbe, hb, S["rec"], S["st"], workspace=S["ws"], stream=s)
                S["outh"].copy_(S["rec"], non_blocking=True)
            nb_box[0] = nbe

        for S in slots:  # warm-up: sizes the workspaces
            e2e_one(S)
        torch.cuda.synchronize()
        # serial
        main = torch.cuda.current_stream()

        def serial_step():
            slots[0]["s"].wait_stream(main)
            e2e_one(slots[0])
            main.wait_stream(slots[0]["s"])

        t_e = timed(serial_step, max(10, args.steps // 2))
        torch.cuda.synchronize()
        # streamed: K steps alternating between the two slots
        K = max(10, args.steps)
        flush_l2(flush, sink, 0)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(main)
        for S in slots:
            S["s"].wait_stream(main)
        for i in range(K):
            e2e_one(slots[i % 2])
        for S in slots:
            main.wait_stream(S["s"])
        ev1.record(main)
        torch.cuda.synchronize()
        t_stream = ev0.elapsed_time(ev1) / K
        for S in slots:
            assert int(S["st"].item()) == 0
            assert torch.equal(S["outh"], rec.cpu())
        e2e = {"value": world * bytes_in / (t_stream * 1e-3) / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": bytes_in + nb_box[0], "d2h_bytes_per_step": nb_box[0] + bytes_in,
               "mode": "streamed: two streams, steps overlap (field in, compress, archive out and in, decompress, "
                       "reconstruction out per step; every step's copies inside the timed region)",
               "steps": K, "ms_per_step": t_stream,
               "serial": {"value": world * bytes_in / (np.mean(t_e) * 1e-3) / 1e9, "unit": "GB/s",
                          "ms_per_step": float(np.mean(t_e))}}
        del xh, slots

    # the same field under global (unchunked) Lorenzo prediction, and as a double field
    def side_leg(xin, global_lorenzo=False):
        out = torch.empty_like(xin)
        arc2 = torch.empty(min(api.max_archive_bytes(dims), 8 * n + (1 << 20)), dtype=torch.uint8, device=dev)

        def comp():
            return api.compress(xin, spec.eb, spec.eb_mode, select=args.select, out=arc2, workspace=ws,
                                global_lorenzo=global_lorenzo)[1]

        nb2 = comp()
        api.decompress(arc2, nb2, out=out, workspace=ws)
        torch.cuda.synchronize()
        h2 = api.header(arc2)
        bound = h2["eb_d"] if xin.dtype == torch.float64 else h2["eb_f"]
        e2 = float((xin.double() - out.double()).abs().max())
        assert e2 <= bound, (e2, bound)
        reps = max(5, args.steps // 4)
        tc = timed(comp, reps)
        td = timed(lambda: api.decompress(arc2, nb2, out=out, workspace=ws), reps)
        nbytes_in = xin.numel() * xin.element_size()
        del arc2, out
        return {"gbs": world * nbytes_in / ((np.mean(tc) + np.mean(td)) * 1e-3) / 1e9,
                "compress_gbs": world * nbytes_in / (np.mean(tc) * 1e-3) / 1e9,
                "decompress_gbs": world * nbytes_in / (np.mean(td) * 1e-3) / 1e9,
                "cr": nbytes_in / nb2, "max_abs_err": e2, "bound": bound,
                "note": "plain calls (each synchronises once); GB/s of input bytes"}

    global_leg = side_leg(x, global_lorenzo=True)
    global_leg["cr_chunked"] = bytes_in / nb
    f64_leg = side_leg(x.double())
    f64_leg["workload"] = spec.name + " as float64"

    batched = None
    if not args.no_batched:
        del flush
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        batched = batched_comparison(args, dev, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(spec, x.cpu(), args.select, args.workload)

    line = {
        "metric": "compress+decompress GB/s (FP32 in)",
        "value": value,
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": spec.name, "dims": list(dims), "eb_mode": spec.eb_mode, "eb": spec.eb,
                   "radius": 512, "select": args.select, "parallelism": f"replicas{world}",
                   "path": "csz_compress_with_header (one host synchronisation) + csz_decompress_async "
                           "(status read after the timed region), device-resident field and archive",
                   "l2": "inputs larger than L2, and L2 flushed (256 MiB written, then read back) before every "
                         "timed step, outside the step's events"},
        "compress_gbs": world * bytes_in / (np.mean(t_c) * 1e-3) / 1e9,
        "decompress_gbs": world * bytes_in / (np.mean(t_d) * 1e-3) / 1e9,
        "graph_replay": {"note": "the same round trip as CUDA graph replays of the batch calls with one field "
                                 f"(decoder CTAs of {dec_warps} warps, tuned)",
                         "gbs": world * bytes_in / (np.mean(t_graph) * 1e-3) / 1e9,
                         "compress_gbs": world * bytes_in / (np.mean(t_gc) * 1e-3) / 1e9,
                         "decompress_gbs": world * bytes_in / (np.mean(t_gd) * 1e-3) / 1e9},
        "cr": bytes_in / nb,
        "archive_bytes": nb,
        "codec_blocks": {"huff": hdr["n_codec"][0], "rle": hdr["n_codec"][1], "rle_huff": hdr["n_codec"][2]},
        "max_abs_err": err,
        "eb_abs": hdr["eb_f"],
        "roofline": roofline,
        "kernels": kernels,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": launches,
        "batched": batched,
        "global_lorenzo": global_leg,
        "f64": f64_leg,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
