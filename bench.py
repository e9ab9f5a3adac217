#!/usr/bin/env python3
"""Benchmark: read bases/s of Genome-on-Diet seeding on one GB300 (and N replicas).

One step = one pass of the whole hot path over one synthetic batch: build the
compressed seed index of the 100 Mbp reference (sparsify, 2-bit code, hash,
minimizers, radix-sort index, filter, hash table; plus the learned index with
its on-GPU root training when --index learned), then seed all 2,000,000
150 bp reads in one batched pass (pattern alignment over both shifts, lookups,
anchors, per-read sorted anchor lists). value = read bases / step time with
the reference and reads already in HBM; e2e = the same step through the C ABI
with pinned host buffers, H2D of the inputs and D2H of the anchors inside the
timed region.

Multi-GPU (torchrun): reads are independent, so every rank seeds its own batch
(weak scaling) against its own copy of the index; no data-path collective.
The reference arm (--impl reference) times the plain C++ oracle on the host.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2211_08157_gb300 import synth  # noqa: E402

METRIC = "read bases/sec & anchors/sec on 1 GB300, learned vs hash index, bit-exact anchors"
L2_BYTES = 129 * 1024 * 1024


# ALU roofline of the sketch kernel. Peak: the issue-limited 32-bit integer rate
# from the unit counts and clock: 152 SMs x 4 schedulers x 32 lanes x 2.07 GHz.
ALU_PEAK_TOPS = 152 * 4 * 32 * 2.07e9 / 1e12


def sketch_ops_per_base(k: int) -> int:
    """32-bit integer operations the method needs per patterned base (counted
    from its arithmetic, not from the kernel): 2-bit code (4), forward and
    reverse-complement k-mer update (14 for 64-bit codes, 7 for 32-bit),
    canonical choice and strand (5), Wang hash (46 in 64-bit, 23 in 32-bit),
    window minimum and maximum by van Herk / Gil-Werman (24 / 12), the
    minimizer test (2)."""
    if k > 16:
        return 4 + 14 + 5 + 46 + 24 + 2
    return 4 + 7 + 5 + 23 + (12 if k <= 15 else 24) + 2


SKETCH_SOURCES = {"sketch": "sketch.cu", "sketch_seg": "sketch_seg.cu"}


def recorded_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes (read + write) of `kernel` from the committed ncu
    summary, if it was captured on this workload and on the current kernel
    source (source hash matches), else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    src = os.path.join(ROOT, "paper_2211_08157_gb300", "csrc", SKETCH_SOURCES.get(kernel, "sketch.cu"))
    try:
        d = json.load(open(path))
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if d.get("source_sha256") != h or d.get("workload") != workload:
            return None
        return {"bytes_per_launch": d["bytes_per_launch"], "source": d.get("command", path)}
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return out
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower() == "active"})
        out.update(sm_mhz=statistics.median(r[0] for r in rows), sm_max_mhz=max(r[1] for r in rows),
                   reasons=reasons, samples=len(rows))
        return out


def make_workload(name: str, n_reads: int | None, rank: int):
    wl = synth.WORKLOADS[name]
    ref = wl.make_reference()
    # rank r seeds its own batch: reads drawn from stream 2 + 10 r
    reads, offs, _ = wl.make_reads(ref, n=n_reads, seed_stream=2 + 10 * rank)
    return wl, ref, reads, offs


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return ws, rank, local


def dist_max(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- CPU oracle
def oracle_step(idx_args, reads, offs, t: int, threads: int):
    """One oracle step over the whole batch: index build of the whole reference
    (single-threaded, as the oracle stands) + seeding of every read over
    `threads` host threads. Returns (index s, seeding s, anchors)."""
    import oracle
    t0 = time.perf_counter()
    idx = oracle.Index(*idx_args)
    t_index = time.perf_counter() - t0
    t0 = time.perf_counter()
    a, _ = idx.seed(reads, offs, t, threads=threads)
    t_seed = time.perf_counter() - t0
    idx.close()
    return t_index, t_seed, int(a.size)


def run_reference(args, ws, rank):
    """The oracle as the reference arm: the same step (index build + seeding of
    the whole batch) on the host cores; rank 0 only."""
    if rank != 0:
        return
    wl, ref, reads, offs = make_workload(args.workload, args.n_reads, 0)
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    bases = float(offs[-1])
    n = offs.size - 1
    idx_args = (ref, wl.pattern, wl.k, wl.w, wl.max_occ)
    for _ in range(args.warmup):
        oracle_step(idx_args, reads, offs, wl.t, threads)
    steps = []
    t_run0 = time.perf_counter()
    for _ in range(args.steps):
        steps.append(oracle_step(idx_args, reads, offs, wl.t, threads))
    wall = time.perf_counter() - t_run0
    step_s = statistics.mean(ti + ts for ti, ts, _ in steps)
    t_index = statistics.mean(ti for ti, _, _ in steps)
    t_seed = statistics.mean(ts for _, ts, _ in steps)
    n_anchors = steps[-1][2]
    value = bases / step_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "read bases/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/u64 integer", "data": "synthetic",
        "config": {"workload": wl.name, "reads": n, "read_bases": int(bases), "ref_bases": int(ref.size),
                   "pattern": wl.pattern, "k": wl.k, "w": wl.w, "max_occ": wl.max_occ, "pa_t": wl.t,
                   "step": "index build + seeding of all reads"},
        "anchors_per_s": n_anchors / step_s, "anchors_per_step": n_anchors,
        "cpu_baseline": {"value": value, "unit": "read bases/s", "cores": threads, "kind": "oracle",
                         "sample": f"the whole batch every step: oracle index of the {ref.size} bp reference on "
                                   f"1 thread ({t_index:.2f} s) + oracle seeding of all {n} reads "
                                   f"({int(bases)} bases) on {threads} threads ({t_seed:.2f} s)"},
        "e2e": {"value": value, "unit": "read bases/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "timed_wall_s": wall,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- serving
def serving_pool(ref, long_max=300, seed=5):
    """Request payloads: short-read batches (1k-50k x 150 bp) and long-read batches
    (HiFi-like and ONT-like, 10-long_max reads), each kind a third of the stream."""
    return synth.serving_requests(ref, 8, long_max, seed)


def seed_host(god, idx, reads, offs, via):
    """god_seed_into with host buffers and an explicit lookup path (grows the
    output on GOD_ERANGE)."""
    cap = max(1024, int(offs[-1]) // 8)
    while True:
        out = np.empty((cap, 4), np.uint32)
        try:
            m = god.god_seed_into(idx, reads, offs, out, via=via)
            return out[:m]
        except god.GodError as e:
            if e.rc != -5:
                raise
            cap = max(cap * 2, int(getattr(e, "needed", 0) or 0))


def run_serving(god, idx, pool, rate, duration, mode, slots=4, seed=11, saturate=False, via=None):
    """Poisson arrivals at `rate`/s for `duration` s. mode 'server': the
    continuous-batching server; 'plain': one god_seed call per request, FIFO
    (index path `via`). saturate: every request arrives at time 0 (the
    throughput the path sustains; latency then includes the queue)."""
    import queue
    rng = np.random.default_rng(seed)
    kinds = ["short", "hifi", "ont"]
    arrivals, t = [], 0.0
    while t < duration:
        t += rng.exponential(1.0 / rate)
        kind = kinds[int(rng.integers(0, 3))]
        arrivals.append((0.0 if saturate else t, pool[kind][int(rng.integers(0, len(pool[kind])))]))
    lat, bases = [], 0
    t0 = time.perf_counter()
    if mode == "server":
        srv = god.GodServer(idx, slots=slots)
        ids = []

        def waiter(q):
            while True:
                item = q.get()
                if item is None:
                    return
                _, l = srv.wait(item, with_latency=True)
                lat.append(l)

        q = queue.Queue()
        th = threading.Thread(target=waiter, args=(q,))
        th.start()
        for at, (r, o) in arrivals:
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            q.put(srv.submit(r, o))
            bases += int(o[-1])
        q.put(None)
        th.join()
        stats = srv.stats()
        srv.close()
    else:
        stats = {}
        for at, (r, o) in arrivals:
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            if via is None:
                god.god_seed(idx, r, o)
            else:
                seed_host(god, idx, r, o, via)
            lat.append(time.perf_counter() - t0 - at)
            bases += int(o[-1])
    wall = time.perf_counter() - t0
    lat = np.array(lat)
    return {"requests": len(arrivals), "read_bases_per_s": bases / wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "wall_s": wall, **({"merged_requests": stats["merged_requests"],
            "batches": stats["batches"], "max_inflight_batches": stats["max_inflight_batches"],
            "worker_seconds": {k: round(stats[k], 4) for k in ("gather_s", "pin_alloc_s", "device_s", "copy_back_s")}}
            if stats else {})}


# ----------------------------------------------------------------------------- other workloads
def time_events(stream, flush, fn, reps=3):
    """Mean CUDA-event milliseconds of fn() on `stream`, L2 flushed before each."""
    import torch
    tt = []
    for _ in range(reps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        tt.append(e0.elapsed_time(e1))
    return statistics.mean(tt)


def vote_line(god, torch, dev, stream, flush, idx, d_reads, d_offs, bases, long_reads):
    """Location voting over one seeding result on the device: D = 100, V = 3
    and 8 winners per read for long reads, D = 50, V = 2 and 4 for short
    ones (Sec. 3.4 steps 4 / 5)."""
    D, V, max_out = (100, 3, 8) if long_reads else (50, 2, 4)
    ptr, m = god.god_seed_device(idx, d_reads, d_offs, stream=stream)
    n = d_offs.numel() - 1
    d_out = torch.empty((n * max_out, 10), dtype=torch.int32, device=dev)
    d_cnt = torch.empty(n, dtype=torch.int32, device=dev)

    def vote():
        god.god_vote((ptr, m), d_offs, D, V, max_out, out=d_out, counts=d_cnt, stream=stream)

    vote()
    ms = time_events(stream, flush, vote)
    winners = int(d_cnt.sum().item())
    god.god_free(ptr)
    return {"D": D, "V": V, "max_out": max_out, "anchors": m, "ms": ms, "anchors_per_s": m / (ms / 1e3),
            "read_bases_per_s": bases / (ms / 1e3), "records": winners}


def workload_line(god, torch, dev, stream, flush, name, ref=None):
    """Seeding throughput of one stated workload at its full size with a resident
    index (inputs in HBM), hash against learned lookups, plus each index's build
    time. Returns (line, reference array)."""
    wl = synth.WORKLOADS[name]
    t0 = time.perf_counter()
    if ref is None:
        ref = wl.make_reference()
    reads, offs, _ = wl.make_reads(ref)
    gen_s = time.perf_counter() - t0
    bases = float(offs[-1])
    d_ref = torch.from_numpy(ref).to(dev)
    d_reads = torch.from_numpy(reads).to(dev)
    d_offs = torch.from_numpy(offs.view(np.int64)).to(dev)
    out = {"reads": int(offs.size - 1), "read_bases": int(bases), "ref_bases": int(ref.size), "pattern": wl.pattern,
           "k": wl.k, "w": wl.w, "max_occ": wl.max_occ, "pa_t": wl.t, "input_generation_s": gen_s}
    for nm, kd in (("hash", god.GOD_INDEX_HASH), ("learned", god.GOD_INDEX_LEARNED)):
        prm = god.god_params_init(index_kind=kd, pa_t=wl.t)
        holder = {}

        def build():
            if "idx" in holder:
                holder.pop("idx").close()
            holder["idx"] = god.god_build_index(d_ref, wl.pattern, wl.k, wl.w, wl.max_occ, params=prm,
                                                stream=stream)

        build_ms = time_events(stream, flush, build, reps=2)
        idx = holder["idx"]
        res = {}

        def seed():
            ptr, m = god.god_seed_device(idx, d_reads, d_offs, stream=stream)
            res["m"] = m
            god.god_free(ptr)

        seed()
        ms = time_events(stream, flush, seed)
        info = idx.info
        out[nm] = {"read_bases_per_s": bases / (ms / 1e3), "anchors_per_s": res["m"] / (ms / 1e3),
                   "anchors": res["m"], "seed_ms": ms, "index_build_ms": build_ms}
        if nm == "hash":
            out["vote"] = vote_line(god, torch, dev, stream, flush, idx, d_reads, d_offs, bases, long_reads=True)
            if wl.lengths.kind != "fixed":
                seg = {}

                def seed_seg():
                    ptr, m = god.god_seed_device(idx, d_reads, d_offs, stream=stream, seg_len=30_000)
                    seg["m"] = m
                    god.god_free(ptr)

                seed_seg()
                sms = time_events(stream, flush, seed_seg)
                out["segmented_30kb"] = {"read_bases_per_s": bases / (sms / 1e3), "anchors": seg["m"],
                                         "seed_ms": sms, "note": "hash index, reads cut into 30,000-base "
                                                                 "segments, each pattern-aligned on its own"}
        if nm == "learned":
            out[nm].update(rmi_mean_eps=info["rmi_mean_eps"], rmi_leaves=info["rmi_leaves"],
                           rmi_fallback_key_frac=info["rmi_fallback_key_frac"])
        idx.close()
    out["learned_over_hash"] = out["learned"]["read_bases_per_s"] / out["hash"]["read_bases_per_s"]
    del d_ref, d_reads, d_offs
    torch.cuda.empty_cache()
    return out, ref


# ----------------------------------------------------------------------------- seed matching evaluation
def seed_match_line(god, torch, dev, stream, flush, n_pairs=100_000, length=1000, seed=77):
    """The evaluation of Sec. 2.1.1 on the GPU: n_pairs 1000-base pairs, each a
    random sequence and a copy with 0-300 substitutions at random positions;
    Levenshtein distance and the matched / total seeds of the four seeding
    algorithms at k = 8, w = 6, pattern 100 (spaced seeds with 100 repeated).
    Reports pairs/s, and per algorithm the share of pairs accepted at a few
    edit-distance thresholds (threshold rate = the smallest matching rate of
    the pairs within the distance; accepted = pairs at or above it)."""
    rng = np.random.default_rng(seed)
    S = synth.ACGT[rng.integers(0, 4, (n_pairs, length))]
    T = S.copy()
    n_sub = rng.integers(0, 301, n_pairs)
    for i in range(n_pairs):
        pos = rng.choice(length, int(n_sub[i]), replace=False)
        T[i, pos] = synth.ACGT[(np.searchsorted(synth.ACGT, T[i, pos]) + rng.integers(1, 4, pos.size)) % 4]
    seqs = np.stack([S, T], axis=1).reshape(-1)
    offs = np.arange(0, 2 * n_pairs * length + 1, length, dtype=np.uint64)
    d_seqs = torch.from_numpy(seqs).to(dev)
    d_offs = torch.from_numpy(offs.view(np.int64)).to(dev)
    ed = torch.empty(n_pairs, dtype=torch.int32, device=dev)
    mt = torch.empty((n_pairs, 4), dtype=torch.int32, device=dev)
    tt = torch.empty((n_pairs, 4), dtype=torch.int32, device=dev)
    L = god.load()
    import ctypes as C

    def run():
        god.check(L.god_seed_match(C.c_void_p(d_seqs.data_ptr()), C.c_void_p(d_offs.data_ptr()), n_pairs, b"100",
                                   b"100", 8, 6, C.c_void_p(ed.data_ptr()), C.c_void_p(mt.data_ptr()),
                                   C.c_void_p(tt.data_ptr()), C.c_void_p(stream.cuda_stream)))

    run()
    ms = time_events(stream, flush, run)
    e = ed.cpu().numpy()
    rate = mt.cpu().numpy() / np.maximum(tt.cpu().numpy(), 1)
    accepted = {}
    for thr in (20, 50, 100, 138, 200, 295):
        within = e <= thr
        row = {}
        for a, name in enumerate(("all", "minimizer", "spaced", "god")):
            cut = rate[within, a].min() if within.any() else 1.0
            row[name] = float((rate[:, a] >= cut).mean())
        accepted[str(thr)] = row
    return {"pairs": n_pairs, "length": length, "k": 8, "w": 6, "pattern": "100", "spaced": "100",
            "substitutions": "uniform 0-300 per pair", "ms": ms, "pairs_per_s": n_pairs / (ms / 1e3),
            "dp_cells_per_s": n_pairs * length * length / (ms / 1e3),
            "accepted_share_by_edit_distance_threshold": accepted}


# ----------------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--index", default="hash", choices=["hash", "learned"])
    ap.add_argument("--workload", default="short_100mbp_2m")
    ap.add_argument("--n-reads", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the other index kind's seed-only line")
    ap.add_argument("--no-seed-match", action="store_true", help="skip the seed matching evaluation line")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the HiFi-like and human-scale ONT-like seeding lines")
    ap.add_argument("--serving-seconds", type=float, default=3.0, help="0 skips the serving measurement")
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--serving-workload", default="ont_3100mbp_100k",
                    help="reference of the served index (the 3.1 Gbp one by default)")
    ap.add_argument("--serving-long-max", type=int, default=2000, help="largest long-read request (reads)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    import paper_2211_08157_gb300 as god
    torch.cuda.set_device(local)
    god.load()
    wl, ref, reads, offs = make_workload(args.workload, args.n_reads, rank)
    n = offs.size - 1
    bases = float(offs[-1])
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    d_ref = torch.from_numpy(ref).to(dev)
    d_reads = torch.from_numpy(reads).to(dev)
    d_offs = torch.from_numpy(offs.view(np.int64)).to(dev)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    kind = god.GOD_INDEX_LEARNED if args.index == "learned" else god.GOD_INDEX_HASH
    params = god.god_params_init(index_kind=kind, pa_t=wl.t, tune=1)
    cap = max(int(bases // 4), 1 << 20)
    d_out = torch.empty((cap, 4), dtype=torch.int32, device=dev)

    def step(out):
        idx = god.god_build_index(d_ref, wl.pattern, wl.k, wl.w, wl.max_occ, params=params, stream=stream)
        m = god.god_seed_into(idx, d_reads, d_offs, out, stream=stream)
        idx.close()
        return m

    # warm-up (also sizes the output)
    n_anchors = 0
    for _ in range(args.warmup):
        try:
            n_anchors = step(d_out)
        except god.GodError as e:
            if e.rc != -5:
                raise
            cap *= 2
            d_out = torch.empty((cap, 4), dtype=torch.int32, device=dev)
            n_anchors = step(d_out)
    torch.cuda.synchronize(dev)

    # ---- timed region: K steps, L2 flushed between steps (untimed)
    clocks = ClockSampler(local)
    clocks.start()
    god.god_prof_reset()
    god.god_prof_enable(2)           # only the sketch kernel's launches carry timing events
    launches0 = god.god_launch_count()
    step_ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        barrier(ws)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n_anchors = step(d_out)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize(dev)
        barrier(ws)
        step_ms.append(e0.elapsed_time(e1))
    launches = god.god_launch_count() - launches0
    god.god_prof_enable(False)
    prof = god.god_prof_report()
    clk = clocks.stop()
    # per-kernel breakdown from separate steps with every launch timed (the
    # event pairs add a little to those steps, which are not the timed ones)
    prof_steps = 2
    god.god_prof_reset()
    god.god_prof_enable(1)
    for _ in range(prof_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        step(d_out)
    torch.cuda.synchronize(dev)
    god.god_prof_enable(False)
    prof_all = god.god_prof_report()
    ms = statistics.mean(step_ms)
    ms_max = dist_max(ms, ws)
    total_bases = dist_sum(bases, ws)
    total_anchors = dist_sum(float(n_anchors), ws)
    value = total_bases / (ms_max / 1e3)

    # ---- dominant kernel roofline (CUDA events on the library's stream)
    hbm, peak_src = peaks()
    # the dominant kernel by the per-kernel breakdown; its launch duration from
    # the timed steps when it is the one timed there (the sketch kernel)
    tname = max(prof_all.items(), key=lambda kv: kv[1][1])[0]
    tl, tms, tbytes, tunits = prof[tname] if tname in prof else prof_all[tname]
    per_launch_s = (tms / tl) / 1e3
    if tname in ("sketch", "sketch_seg"):
        # algorithmic bytes: 1 B per patterned base read + 16 B per minimizer
        # record written; the integer-issue view of the same launches beside it
        bpl = tbytes / tl
        achieved = bpl / per_launch_s / 1e9
        ops = sketch_ops_per_base(wl.k) * tunits / tl            # algorithmic int32 ops per launch
        tr = recorded_traffic(tname, wl.name)
        roof = {"kernel": tname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": tr["bytes_per_launch"] if tr else None,
                "traffic_source": tr["source"] if tr else "no capture on the current kernel source",
                "peak_source": peak_src, "bytes_per_launch": bpl, "ms_per_launch": tms / tl,
                "alu_view": {"achieved": ops / per_launch_s / 1e12, "peak": ALU_PEAK_TOPS,
                             "unit": "Tops/s (int32, issue-limited)",
                             "frac": ops / per_launch_s / 1e12 / ALU_PEAK_TOPS,
                             "ops_per_patterned_base": sketch_ops_per_base(wl.k),
                             "peak_source": "derived from 152 SMs x 128 lanes x 2.07 GHz"}}
    elif tbytes > 0:
        achieved = (tbytes / tl) / per_launch_s / 1e9
        roof = {"kernel": tname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None, "peak_source": peak_src,
                "bytes_per_launch": tbytes / tl, "ms_per_launch": tms / tl}
    else:
        roof = {"kernel": tname, "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
                "traffic": None, "peak_source": peak_src, "ms_per_launch": tms / tl}
    # both sketch kernels of a step together: the reference's (tile kernel) and
    # the reads' (per-segment kernel when their segments are short)
    sks = [prof[n] for n in ("sketch", "sketch_seg") if n in prof]
    sketch_roof = None
    if sks and sum(x[2] for x in sks) > 0:
        sk_ms = sum(x[1] for x in sks)
        a = sum(x[2] for x in sks) / (sk_ms / 1e3) / 1e9
        sketch_roof = {"hbm_achieved_gbs": a, "hbm_frac": a / hbm, "ms_per_step": sk_ms / args.steps,
                       "patterned_bases_per_s": sum(x[3] for x in sks) / (sk_ms / 1e3),
                       "per_kernel_ms_per_step": {n: prof[n][1] / args.steps for n in ("sketch", "sketch_seg")
                                                  if n in prof}}
    kernels = {k: {"launches_per_step": v[0] / prof_steps, "ms_per_step": v[1] / prof_steps,
                   "share": v[1] / sum(x[1] for x in prof_all.values())} for k, v in
               sorted(prof_all.items(), key=lambda kv: -kv[1][1])}

    # ---- index build alone, then seed-only throughput with a resident index
    # (hash and learned; the learned build includes training its model)
    seed_only = {}
    index_build = {}
    if not args.no_compare:
        for nm, kd in (("hash", god.GOD_INDEX_HASH), ("learned", god.GOD_INDEX_LEARNED),
                       ("learned_readout_only", god.GOD_INDEX_LEARNED)):
            prm = god.god_params_init(index_kind=kd, pa_t=wl.t)
            if nm == "learned_readout_only":
                prm.rmi_train_steps = 0          # the least-squares output layer without the Adam steps
            bt = []
            idx = None
            for _ in range(3):
                if idx is not None:
                    idx.close()
                with torch.cuda.stream(stream):
                    flush.zero_()
                stream.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                idx = god.god_build_index(d_ref, wl.pattern, wl.k, wl.w, wl.max_occ, params=prm, stream=stream)
                e1.record(stream)
                e1.synchronize()
                bt.append(e0.elapsed_time(e1))
            index_build[nm] = {"ref_bases_per_s": float(ref.size) / (statistics.mean(bt) / 1e3),
                               "ms": statistics.mean(bt)}
            god.god_seed_into(idx, d_reads, d_offs, d_out, stream=stream)
            tt = []
            for _ in range(3):
                with torch.cuda.stream(stream):
                    flush.zero_()
                stream.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                god.god_seed_into(idx, d_reads, d_offs, d_out, stream=stream)
                e1.record(stream)
                e1.synchronize()
                tt.append(e0.elapsed_time(e1))
            info = idx.info
            seed_only[nm] = {"read_bases_per_s": bases / (statistics.mean(tt) / 1e3),
                             "ms": statistics.mean(tt)}
            if nm == "hash":
                seed_only["vote"] = vote_line(god, torch, dev, stream, flush, idx, d_reads, d_offs, bases,
                                              long_reads=False)
            if nm.startswith("learned"):
                seed_only[nm].update(rmi_mean_eps=info["rmi_mean_eps"], rmi_leaves=info["rmi_leaves"],
                                     rmi_fallback_key_frac=info["rmi_fallback_key_frac"],
                                     rmi_final_loss=info["rmi_final_loss"])
            idx.close()

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        h_ref = torch.from_numpy(ref).pin_memory()
        h_reads = torch.from_numpy(reads).pin_memory()
        h_offs = torch.from_numpy(offs.view(np.int64)).pin_memory()
        h_out = torch.empty((max(n_anchors, 1) + 1024, 4), dtype=torch.int32).pin_memory()
        ref_np, reads_np, offs_np = h_ref.numpy(), h_reads.numpy(), h_offs.numpy().view(np.uint64)
        out_np = h_out.numpy()

        def e2e_step():
            idx = god.god_build_index(ref_np, wl.pattern, wl.k, wl.w, wl.max_occ, params=params, stream=stream)
            m = god.god_seed_into(idx, reads_np, offs_np, out_np, stream=stream)
            idx.close()
            return m

        e2e_step()
        tt = []
        for _ in range(max(2, min(args.steps, 3))):
            with torch.cuda.stream(stream):
                flush.zero_()
            stream.synchronize()
            t0 = time.perf_counter()
            m = e2e_step()
            tt.append(time.perf_counter() - t0)
        e2e_s = dist_max(statistics.mean(tt), ws)
        e2e = {"value": total_bases / e2e_s, "unit": "read bases/s",
               "h2d_bytes_per_step": int(ref.nbytes + reads.nbytes + offs.nbytes),
               "d2h_bytes_per_step": int(m * 16), "ms_per_step": e2e_s * 1e3}

    # ---- serving: request streams against a resident index; the server (the
    # index's learned lookups, continuous batching) against the plain path (one
    # god_seed call per request, hash lookups)
    # ---- the other stated workloads at full size (rank 0): 200,000 HiFi-like
    # reads on the 100 Mbp reference, 100,000 ONT-like reads on the 3.1 Gbp one
    workloads = None
    refs = {wl.name: ref}
    # (the one-GPU lines: left out when several GPUs are held for the scaling run)
    if rank == 0 and ws == 1 and not args.no_workloads:
        workloads = {}
        for wname in ("hifi_100mbp_200k", "ont_3100mbp_100k"):
            r0 = None
            wref_cfg = synth.WORKLOADS[wname].ref_config or synth.WORKLOADS[wname].config
            for nm0, r in refs.items():
                w0 = synth.WORKLOADS[nm0]
                if (w0.ref_config or w0.config) == wref_cfg and w0.ref_len == synth.WORKLOADS[wname].ref_len:
                    r0 = r
            workloads[wname], refs[wname] = workload_line(god, torch, dev, stream, flush, wname, r0)

    seed_match = None
    if rank == 0 and ws == 1 and not args.no_seed_match:
        seed_match = seed_match_line(god, torch, dev, stream, flush)

    serving = None
    if args.serving_seconds > 0 and rank == 0 and ws == 1:
        swl = synth.WORKLOADS[args.serving_workload]
        sref = refs.get(swl.name)
        if sref is None:
            sref = swl.make_reference()
        pool = serving_pool(sref, long_max=args.serving_long_max)
        sp = god.god_params_init(index_kind=god.GOD_INDEX_LEARNED, pa_t=swl.t)
        t0 = time.perf_counter()
        sidx = god.god_build_index(sref, swl.pattern, swl.k, swl.w, swl.max_occ, params=sp)
        build_s = time.perf_counter() - t0
        # warm-up (untimed): a short stream and a saturated burst, so that the
        # process's page-locked buffer cache holds what the timed streams reuse
        run_serving(god, sidx, pool, args.serving_rate, 0.5, "server")
        run_serving(god, sidx, pool, args.serving_rate, 0.5, "server", saturate=True)
        n_sat = max(1, int(args.serving_rate * args.serving_seconds))
        serving = {"workload": swl.name, "ref_bases": int(sref.size), "index": "learned (server) / hash (plain)",
                   "index_build_s_from_host": build_s, "index_info": {k: sidx.info[k] for k in
                                                                      ("n_keys", "n_entries", "rmi_mean_eps")},
                   "mix": f"1/3 short (1k-50k x 150 bp), 1/3 HiFi-like, 1/3 ONT-like (10-{args.serving_long_max} "
                          f"reads) per request",
                   "warm_up": "untimed: a 0.5 s stream and a 0.5 s saturated burst before the timed streams",
                   "poisson": {"rate_per_s": args.serving_rate, "seconds": args.serving_seconds,
                               "continuous_batching": run_serving(god, sidx, pool, args.serving_rate,
                                                                  args.serving_seconds, "server"),
                               "plain_hash_one_at_a_time": run_serving(god, sidx, pool, args.serving_rate,
                                                                       args.serving_seconds, "plain", via=0)},
                   "saturated": {"requests": n_sat, "note": "every request submitted at time 0",
                                 "continuous_batching": run_serving(god, sidx, pool, args.serving_rate,
                                                                    args.serving_seconds, "server",
                                                                    saturate=True),
                                 "plain_hash_one_at_a_time": run_serving(god, sidx, pool, args.serving_rate,
                                                                         args.serving_seconds, "plain",
                                                                         saturate=True, via=0)}}
        sidx.close()

    # ---- CPU oracle baseline (rank 0, N = 1 only): one oracle step over the
    # whole batch, as the oracle stands
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        t_index, t_seed, _ = oracle_step((ref, wl.pattern, wl.k, wl.w, wl.max_occ), reads, offs, wl.t, threads)
        cpu = {"value": bases / (t_index + t_seed), "unit": "read bases/s", "cores": threads, "kind": "oracle",
               "sample": f"the whole batch once: oracle index of the {ref.size} bp reference on 1 thread "
                         f"({t_index:.2f} s) + oracle seeding of all {n} reads ({int(bases)} bases) on {threads} "
                         f"threads ({t_seed:.2f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "read bases/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8/u64 integer", "data": "synthetic",
            "config": {"workload": wl.name, "reads_per_gpu": n, "read_bases_per_gpu": int(bases),
                       "ref_bases": int(ref.size), "pattern": wl.pattern, "k": wl.k, "w": wl.w,
                       "max_occ": wl.max_occ, "pa_t": wl.t, "index": args.index,
                       "step": "index build + batched seeding of all reads",
                       "l2": "flushed between timed steps (256 MiB write); inputs 400 MB > L2",
                       "parallelism": f"replicas x{ws}"},
            "anchors_per_s": total_anchors / (ms_max / 1e3), "anchors_per_step": int(total_anchors),
            "autotune": god.god_autotune_report(),
            "gpu_launches": int(launches),
            "roofline": roof, "sketch_roofline": sketch_roof, "kernels": kernels,
            "kernels_note": f"per-step means over {prof_steps} extra steps with every launch timed by CUDA events",
            "seed_only_resident_index": seed_only, "index_build_resident_reference": index_build, "workloads": workloads, "seed_match": seed_match, "serving": serving, "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
