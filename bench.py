#!/usr/bin/env python3
"""Benchmark of the motion-estimation hot path on the 1080p workload.

Workload: 1920x1080 luma padded to 1088 rows, 16x16 blocks, p = 32,
Qp = 28 (lambda_q8 = 6595), a 60-frame synthetic sequence (panned textured
background, 20 objects moving at up to 24 px/frame, noise sigma 2, 10% of
block slots per frame overwritten with noise).  One step = every frame pair
of the sequence through the whole hot path: FSBM of all pairs in one launch
(me_fsbm_sequence) and ACBM of all pairs in one persistent launch
(me_acbm_sequence: padding, Intra_SAD, PBM, the two conditions and the
full-search fallback, the field of each pair feeding the next as temporal
predictors, pairs overlapping on the GPU).  The per-pair calls (me_fsbm,
me_acbm with its graph-replayed wave launches) are timed beside it for the
per-pair latency, and their outputs compared with the step's.  Frames stay
resident in device memory; L2 is flushed between timed steps (the flush
itself is not timed).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W, H, H_PAD, P, N, M, QP = 1920, 1080, 1088, 32, 16, 16, 28
SEQ_FRAMES = 60
BW, BH = W // N, H_PAD // M
NBLK = BW * BH
NCAND = (2 * P + 1) ** 2
ABSDIFF_PER_FRAME = NBLK * NCAND * N * M          # 8.83e9 for FSBM
# ncu dram__bytes_read.sum + dram__bytes_write.sum of each pipelined FSBM
# kernel the tuner may pick for the sequence, on 13 frames (12 pairs), per
# frame of the sequence: k_fsbm_pipe<16,16,13> 27.202560 MB + 0 B,
# k_fsbm_pipe_tab<16,16> 27.203840 MB + 0 B (every frame read once)
FSBM_SEQ_DRAM_BYTES_PER_FRAME = {"k_fsbm_pipe": 27.202560e6 / 13, "k_fsbm_pipe_tab": 27.203840e6 / 13}
# the kernel behind each full-search form of the tuner's record
FSBM_FORM_KERNEL = (("pipetab", "k_fsbm_pipe_tab"), ("pipe", "k_fsbm_pipe"), ("group", "k_fsbm_seq"))
WORKLOAD = "1080p 1920x1088 16x16 p=32 Qp=28, 60-frame synthetic sequence"
# one metric string for both arms (the native step and the oracle's), so the
# two lines can be divided; candidate-SADs/s, the roofline and p99 are keys
METRIC = "1080p frames/s & candidate-SADs/s (FSBM, ACBM) vs int-pipe roofline; p99 ms"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--frames", type=int, default=SEQ_FRAMES)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-legs", action="store_true",
                    help="skip the batch64 and serve legs of the default line")
    ap.add_argument("--workload", default="1080p",
                    choices=["1080p", "batch64", "serve", "loadtable", "configs"],
                    help="1080p: the default line; batch64 / serve: the multi-stream forms; "
                         "loadtable: ACBM load per block vs Qp on QCIF scenes (Table 1 layout)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: requests per second")
    ap.add_argument("--seconds", type=float, default=10.0, help="serve: arrival window")
    ap.add_argument("--rate-sweep", action="store_true",
                    help="serve: every rate of 2000..12000 req/s in turn (--seconds each)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed
def dist_setup(n_gpus, backend: str = "nccl"):
    """Replicas only: one process per GPU (RANK / WORLD_SIZE / LOCAL_RANK from
    the launcher); the ranks meet only at the timing barrier and the
    max-over-ranks reduction.  `backend` "gloo" runs the same logic on CPU."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def replica_seed(rank: int) -> int:
    """Each rank times an independent synthetic sequence of its own."""
    return 2026 + rank


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v: float) -> float:
    if pg is None:
        return v
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle legs
def oracle_sample(frames, n_pairs: int, threads: int):
    """The oracle on n_pairs frame pairs: FSBM (OpenMP over blocks) + ACBM
    (sequential, as the method orders it).  Returns seconds per frame."""
    import oracle
    lam = oracle.lambda_q8(QP)
    prm = oracle.params(qp=QP)
    prev = None
    t0 = time.perf_counter()
    for t in range(1, n_pairs + 1):
        oracle.fsbm(frames[t], frames[t - 1], N, M, P, lam, nthreads=threads)
        prev = oracle.acbm(frames[t], frames[t - 1], N, M, P, lam, prm, prev)[0]
    return (time.perf_counter() - t0) / n_pairs


def parse_tune_log(text: str) -> list:
    """me_tune_log lines as dicts: shape, whether timed, the model's and the
    chosen form, and every candidate form's best time in ms."""
    out = []
    for ln in text.splitlines():
        head, _, rest = ln.partition(" | ")
        if not rest:
            continue
        what, _, choice = head.rpartition(": ")
        kind = "tuned" if what.endswith(" tuned") else "modelled"
        what = what.rsplit(" ", 1)[0]
        model = choice.split(" chosen=")[0].replace("model=", "")
        chosen = choice.split(" chosen=")[1] if " chosen=" in choice else model
        times = {}
        for c in (head.split(" | ")[1:] + rest.split(" | ")):
            name, _, t = c.strip().rpartition(" ")
            if name.endswith(" ms") or t == "ms":
                name, _, t = name.rpartition(" ")
            try:
                times[name] = float(t)
            except ValueError:
                pass
        out.append({"shape": what, "kind": kind, "model": model, "chosen": chosen, "ms": times})
    return out


def cpu_model() -> str:
    """The host CPU's model name (x86 /proc/cpuinfo, else lscpu on Arm)."""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ main
def _item(me, cur, ref, prev, out, lam, prm):
    it = me.BatchItem()
    it.cur, it.ref = cur.data_ptr(), ref.data_ptr()
    it.prev_mv = None if prev is None else prev.data_ptr()
    it.mv_out, it.J_out, it.mask_out = out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr()
    it.sad_out, it.load_out = out[3].data_ptr(), out[4].data_ptr()
    it.lambda_q8 = lam
    it.prm = prm
    return it


def batch64_measure(n_steps: int, gpu_index: int = 0):
    """The 64-stream mix (24 QCIF p16, 24 CIF p16, 12 720p p32, 4 2160p p64):
    one persistent launch per step (captured graph) against the plain per-frame
    ACBM/FSBM calls on the same frames; outputs compared.  Returns the
    per-mode timings, the mix's FSBM absdiff rate and the clock record."""
    import torch
    import synth
    import paper_0710_4819_gb300 as me
    specs = synth.batch_mix()
    n_frames = 1 + max(2, n_steps)
    seqs = [torch.from_numpy(synth.stream_frames(s, n_frames)).cuda() for s in specs]
    lam = me.me_lambda_q8(QP)
    prm = me.params(qp=QP)

    def outs(s):
        BH, BW = s.height // M, s.w // N
        return [torch.empty((BH, BW, 2), dtype=torch.int16, device="cuda"),
                torch.empty((BH, BW), dtype=torch.int32, device="cuda"),
                torch.empty((BH, BW), dtype=torch.uint8, device="cuda"),
                torch.empty((BH, BW), dtype=torch.int32, device="cuda"),
                torch.empty((BH, BW), dtype=torch.int32, device="cuda")]

    res = {}
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(gpu_index)
    clocks.start()
    for mode, name in ((0, "fsbm"), (1, "acbm")):
        b = me.Batch()
        for s in specs:
            b.add_stream(s.w, s.height, N, M, s.p)
        o_b = [[outs(s) for s in specs] for _ in range(n_frames)]
        o_p = [[outs(s) for s in specs] for _ in range(n_frames)]

        def batch_step(t):
            items = [_item(me, seqs[i][t], seqs[i][t - 1],
                           o_b[t - 1][i][0] if (mode == 1 and t >= 2) else None, o_b[t][i], lam, prm)
                     for i in range(len(specs))]
            b.run(mode, items)

        def plain_step(t):
            for i, s in enumerate(specs):
                o = o_p[t][i]
                if mode == 0:
                    me.me_fsbm(seqs[i][t], seqs[i][t - 1], N, M, s.p, lam, out=(o[0], o[1], o[3]))
                else:
                    prev = o_p[t - 1][i][0] if t >= 2 else None
                    me.me_acbm(seqs[i][t], seqs[i][t - 1], N, M, s.p, lam, prm, prev_mv=prev,
                               out=tuple(o))
        for fn in (batch_step, plain_step):       # warm-up (plans, graphs)
            fn(1)
        b.sync()
        torch.cuda.synchronize()
        timings = {}
        for fn, key in ((batch_step, "batched"), (plain_step, "plain")):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for t in range(1, n_frames):
                fn(t)
            e1.record(stream)
            torch.cuda.synchronize()
            timings[key] = e0.elapsed_time(e1) / (n_frames - 1)
        b.sync()
        same = all(torch.equal(x, y) for t in range(1, n_frames) for i in range(len(specs))
                   for k, (x, y) in enumerate(zip(o_b[t][i], o_p[t][i])) if mode == 1 or k in (0, 1, 3))
        b.close()
        res[name] = {"batched_ms_per_step": timings["batched"], "plain_ms_per_step": timings["plain"],
                     "batched_frames_per_s": len(specs) / (timings["batched"] * 1e-3),
                     "plain_frames_per_s": len(specs) / (timings["plain"] * 1e-3),
                     "speedup": timings["plain"] / timings["batched"], "outputs_identical": same}
    res["clocks"] = clocks.stop()
    absd = sum((s.w // N) * (s.height // M) * (2 * s.p + 1) ** 2 * N * M for s in specs)
    res["fsbm_absdiff_per_s_T"] = absd / (res["fsbm"]["batched_ms_per_step"] * 1e-3) / 1e12
    res["steps"] = n_frames - 1
    return res


BATCH64_WORKLOAD = "batch64: 24 QCIF p16, 24 CIF p16, 12 720p p32, 4 2160p p64, 16x16, Qp 28"


def run_batch64(args):
    res = batch64_measure(args.steps)
    line = {"metric": "64-stream mix frames/s (one persistent launch per step vs plain per-frame calls)",
            "value": res["acbm"]["batched_frames_per_s"], "unit": "frames/s", "n_gpus": 1,
            "steps": res["steps"], "higher_is_better": True, "dtype": "u8", "data": "synthetic",
            "config": {"workload": BATCH64_WORKLOAD},
            "fsbm": res["fsbm"], "acbm": res["acbm"],
            "fsbm_absdiff_per_s_T": res["fsbm_absdiff_per_s_T"], "clocks": res["clocks"]}
    print(json.dumps(line))


def run_configs(args):
    """Each single-stream workload (QCIF p=16, CIF p=16 at Qp 22/28/34/40,
    1080p p=32) through the GPU sequence forms (FSBM and ACBM of all pairs,
    one launch each; frames resident, L2 flushed, median of 5) beside the
    oracle on a bounded sample of the same frames (FSBM on one thread and on
    all host threads, ACBM on one thread: it is sequential per frame)."""
    import numpy as np
    import torch
    import oracle
    import synth
    import paper_0710_4819_gb300 as me
    thr = cpu_threads()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    lanes = me.me_sad_peak(0)[1]
    rows = []
    for name, p, frames_n, qps, sample in (("qcif", 16, 10, (28,), 3), ("cif", 16, 31, (22, 28, 34, 40), 2),
                                            ("1080p", 32, 60, (28,), 1)):
        seq = synth.config_sequence(name, seed=2026, n_frames=frames_n)
        H, W = seq.shape[1:]
        K = frames_n - 1
        fr = torch.from_numpy(seq).cuda()
        for qp in qps:
            lam = me.me_lambda_q8(qp)
            prm = me.params(qp=qp)
            res = {}
            clocks = ClockSampler(0)
            clocks.start()
            for key, fn in (("fsbm", lambda: me.me_fsbm_sequence(fr, N, M, p, lam)),
                            ("acbm", lambda: me.me_acbm_sequence(fr, N, M, p, lam, prm))):
                for _ in range(3):
                    fn()
                ts = []
                for _ in range(5):
                    flush.fill_(1)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record()
                    fn()
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                res[key] = statistics.median(ts) / K
            ck = clocks.stop()
            absd = (W // N) * (H // M) * (2 * p + 1) ** 2 * N * M
            clk = ck.get("sm_mhz") or ck.get("sm_max_mhz") or 2070.0
            peak = n_sm * 4 * lanes * clk * 1e6
            olam = oracle.lambda_q8(qp)
            t0 = time.perf_counter()
            for t in range(1, sample + 1):
                oracle.fsbm(seq[t], seq[t - 1], N, M, p, olam, nthreads=1)
            f1 = (time.perf_counter() - t0) / sample
            t0 = time.perf_counter()
            for t in range(1, sample + 1):
                oracle.fsbm(seq[t], seq[t - 1], N, M, p, olam, nthreads=thr)
            fa = (time.perf_counter() - t0) / sample
            t0 = time.perf_counter()
            prev = None
            for t in range(1, sample + 1):
                prev = oracle.acbm(seq[t], seq[t - 1], N, M, p, olam, oracle.params(qp=qp), prev)[0]
            a1 = (time.perf_counter() - t0) / sample
            rows.append({"workload": f"{name} {W}x{H} 16x16 p={p} Qp={qp}", "pairs": K,
                         "gpu_fsbm_ms_per_pair": res["fsbm"], "gpu_acbm_ms_per_pair": res["acbm"],
                         "gpu_frames_per_s": 1e3 / (res["fsbm"] + res["acbm"]),
                         "gpu_fsbm_frac_of_peak": absd / (res["fsbm"] * 1e-3) / peak,
                         "oracle_fsbm_ms_1core": 1e3 * f1, "oracle_fsbm_ms_allcores": 1e3 * fa,
                         "oracle_acbm_ms_1core": 1e3 * a1,
                         "oracle_frames_per_s_1core": 1.0 / (f1 + a1),
                         "oracle_frames_per_s_allcores": 1.0 / (fa + a1), "oracle_sample_pairs": sample,
                         "sm_mhz": clk, "clock_reasons": ck.get("reasons")})
    line = {"metric": "per-config frames/s: GPU sequence forms vs the oracle (1 core / all cores)",
            "value": rows[-1]["gpu_frames_per_s"], "unit": "frames/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "QCIF p16, CIF p16 at Qp 22/28/34/40, 1080p p32; 16x16"},
            "cores": thr, "cpu_model": cpu_model(), "rows": rows}
    print(json.dumps(line))


LOAD_QPS = (30, 28, 26, 24, 22, 20, 18, 16)
LOAD_P = 15                       # the paper's search range (961 + 8 half-pel = 969 positions)


def load_cell(me, frames, qp, prm=None):
    """ACBM of a QCIF sequence (16x16, p = 15, lambda from Qp) in one launch:
    returns (average integer positions per block, full-search fraction, sum J,
    sum SAD)."""
    import numpy as np
    import torch
    lam = me.me_lambda_q8(qp)
    a = me.me_acbm_sequence(frames, N, M, LOAD_P, lam, prm if prm is not None else me.params(qp=qp))
    torch.cuda.synchronize()
    load = a.load.double().mean().item()
    fs = a.mask.double().mean().item()
    J = a.J.cpu().numpy().view(np.uint32).astype(np.int64).sum()
    sad = a.sad.cpu().numpy().view(np.uint32).astype(np.int64).sum()
    return load, fs, int(J), int(sad)


def run_load_table(args):
    """The Table 1 layout on synthetic QCIF scenes: ACBM's average candidate
    positions per block (integer positions, and +8 for the half-pel step the
    paper's count of 969 for FSBM includes) for Qp 30..16 at 30 and 10 fps,
    alpha, beta, gamma = 1000, 8, 1/4; then one-at-a-time sweeps of alpha,
    beta and gamma at Qp 28 with the load and the cost relative to FSBM."""
    import numpy as np
    import torch
    import synth
    import paper_0710_4819_gb300 as me
    stream = torch.cuda.current_stream()
    seqs = {(name, fps): torch.from_numpy(synth.load_sequence(name, fps, seed=500)).cuda()
            for name in synth.LOAD_RECIPES for fps in (30, 10)}
    for f in seqs.values():                      # warm-up (plans)
        load_cell(me, f, 28)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    table = {}
    for (name, fps), f in seqs.items():
        for qp in LOAD_QPS:
            load, fs, _, _ = load_cell(me, f, qp)
            table.setdefault(name, {}).setdefault(str(fps), {})[str(qp)] = {
                "positions": round(load, 2), "positions_with_halfpel": round(load + 8, 2),
                "fullsearch_fraction": round(fs, 4)}
    e1.record(stream)
    torch.cuda.synchronize()
    table_ms = e0.elapsed_time(e1)
    # sweeps at Qp 28: cost of ACBM relative to FSBM's (the method's objective)
    base = dict(alpha=1000, beta=8, gamma_num=1, gamma_den=4)
    variants = ([("alpha", v, dict(base, alpha=v)) for v in (0, 250, 500, 2000, 4000, 16000)] +
                [("beta", v, dict(base, beta=v)) for v in (0, 2, 4, 16, 32)] +
                [("gamma", f"{n}/{d}", dict(base, gamma_num=n, gamma_den=d))
                 for n, d in ((0, 1), (1, 8), (1, 2), (1, 1))] +
                [("paper", "1000, 8, 1/4", base)])
    fsbm_J, fsbm_sad = {}, {}
    for key, f in seqs.items():
        r = me.me_fsbm_sequence(f, N, M, LOAD_P, me.me_lambda_q8(28))
        torch.cuda.synchronize()
        fsbm_J[key] = int(r.J.cpu().numpy().view(np.uint32).astype(np.int64).sum())
        fsbm_sad[key] = int(r.sad.cpu().numpy().view(np.uint32).astype(np.int64).sum())
    sweep = []
    for which, v, kw in variants:
        prm = me.AcbmParams(kw["alpha"], kw["beta"], kw["gamma_num"], kw["gamma_den"], 28, 1)
        loads, dJ, dS = [], [], []
        for key, f in seqs.items():
            load, _, J, sad = load_cell(me, f, 28, prm)
            loads.append(load)
            dJ.append(J / fsbm_J[key] - 1.0)
            dS.append(sad / fsbm_sad[key] - 1.0)
        sweep.append({"vary": which, "value": v, "positions": round(float(np.mean(loads)), 2),
                      "J_over_fsbm_pct": round(100 * float(np.mean(dJ)), 3),
                      "SAD_over_fsbm_pct": round(100 * float(np.mean(dS)), 3)})
    cells = [c["positions_with_halfpel"] for r in table.values() for fr in r.values() for c in fr.values()]
    line = {"metric": "ACBM average candidate positions per 16x16 block incl. 8 half-pel (Table 1 layout)",
            "value": float(np.mean(cells)), "unit": "positions/block", "n_gpus": 1,
            "steps": len(cells), "higher_is_better": False, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "load table: 4 synthetic QCIF scenes x {30, 10} fps x Qp 30..16, "
                                   "10 frames, 16x16, p=15, alpha/beta/gamma = 1000/8/1/4",
                       "fsbm_positions_with_halfpel": (2 * LOAD_P + 1) ** 2 + 8},
            "table_ms": table_ms, "table": table, "sweep_qp28": sweep}
    print(json.dumps(line))


class ServeRig:
    """The serving mix: 200 streams (CIF p16 : 720p p32 : 1080p p32 =
    50 : 35 : 15) opened on one continuous-batching server, each primed with
    its first frame; a few distinct looping sequences per resolution are
    shared round-robin."""

    def __init__(self, n_streams: int = 200):
        import numpy as np
        import synth
        import paper_0710_4819_gb300 as me
        specs = synth.serving_mix(n_streams)
        pool = {}
        for kind in ("cif", "720p", "1080p"):
            ex = [s for s in specs if s.name == kind][:4]
            pool[kind] = [synth.stream_frames(s, 6)[:, :s.height] for s in ex]
        self.specs = specs
        self.srv = me.Server(40 << 30, max_inflight=2, mode=1)
        self.ids = [self.srv.open_stream(s.w, s.height, s.p, qp=QP) for s in specs]
        self.seq_of = [pool[s.name][i % len(pool[s.name])] for i, s in enumerate(specs)]
        self.frame_no = [0] * len(specs)
        self.rng = np.random.default_rng(11)
        prime = [self.srv.submit(self.ids[i], self.seq_of[i][0]) for i in range(len(specs))]
        for i, r in enumerate(prime):
            self.srv.wait(r, self.ids[i], 60000)
            self.frame_no[i] = 1

    def run(self, rate: float, seconds: float, gpu_index: int = 0) -> dict:
        """Poisson arrivals at `rate` requests/s for `seconds`, every result
        waited for.  Latency = submit to results ready, per request, as the
        server measures it; a request's completion time is its submit time
        plus that latency, so reading the results back on the host (after the
        window) does not count against the server.  The server keeps up when
        it completes requests as fast as they are submitted and its latency
        does not grow over the window; otherwise it is saturated."""
        n_req = max(1, int(rate * seconds))
        gaps = self.rng.exponential(1.0 / rate, size=n_req)
        which = self.rng.integers(0, len(self.specs), size=n_req)
        reqs, t_sub = [], []
        clocks = ClockSampler(gpu_index)
        clocks.start()
        t0 = time.perf_counter()
        t_next = t0
        for k in range(n_req):
            t_next += gaps[k]
            while True:
                now = time.perf_counter()
                if now >= t_next:
                    break
                if t_next - now > 0.0005:
                    time.sleep(t_next - now - 0.0003)
            i = int(which[k])
            f = self.seq_of[i][self.frame_no[i] % self.seq_of[i].shape[0]]
            self.frame_no[i] += 1
            t_sub.append(time.perf_counter() - t0)
            reqs.append((i, self.srv.submit(self.ids[i], f)))
        sub_s = time.perf_counter() - t0
        lat = []
        for i, r in reqs:
            has, ms, _ = self.srv.wait(r, self.ids[i], 120000)
            lat.append(ms)
        clk = clocks.stop()
        last_done = max(t + ms * 1e-3 for t, ms in zip(t_sub, lat))
        done_rate = len(reqs) / last_done
        sub_rate = len(reqs) / sub_s
        dec = max(1, len(lat) // 10)
        first_p50 = sorted(lat[:dec])[dec // 2]
        last_p50 = sorted(lat[-dec:])[dec // 2]
        srt = sorted(lat)
        return {"offered_rate": rate, "requests": len(reqs), "seconds": seconds,
                "submitted_per_s": sub_rate, "frames_per_s": done_rate,
                "p50_ms": srt[len(srt) // 2], "p99_ms": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
                "max_ms": srt[-1], "first_decile_p50_ms": first_p50, "last_decile_p50_ms": last_p50,
                "saturated": bool(done_rate < 0.97 * sub_rate or last_p50 > 3 * first_p50 + 1.0),
                "submit_kept_up": bool(sub_rate >= 0.97 * rate), "clocks": clk}

    def close(self):
        self.srv.close()


SERVE_WORKLOAD = "serve: 200 streams CIF p16 50% / 720p p32 35% / 1080p p32 15%, Poisson arrivals, budget 40 GB"
SERVE_SWEEP = (2000, 4000, 6000, 8000, 10000, 12000)
SERVE_BEYOND = (16000, 20000, 24000, 32000)   # past the configured range, to find saturation


def run_serve(args):
    """Continuous-batching server over the 200-stream mix: Poisson arrivals
    at --rate for --seconds, or (--rate-sweep) at each rate of the configured
    range 2000..12000 req/s in turn, reporting the curve and the highest rate
    the server keeps up with."""
    rig = ServeRig()
    if args.rate_sweep:
        curve = [rig.run(r, args.seconds) for r in SERVE_SWEEP]
        beyond = []
        for r in SERVE_BEYOND:
            c = rig.run(r, args.seconds)
            beyond.append(c)
            if c["saturated"] or not c["submit_kept_up"]:
                break
        rig.close()
        kept = [c["offered_rate"] for c in curve + beyond if not c["saturated"] and c["submit_kept_up"]]
        line = {"metric": "serving: frames/s and latency vs offered rate (continuous batching, 200 streams)",
                "value": max(c["frames_per_s"] for c in curve), "unit": "frames/s", "n_gpus": 1,
                "higher_is_better": True, "dtype": "u8", "data": "synthetic",
                "config": {"workload": SERVE_WORKLOAD + f", {args.seconds:.1f} s per rate"},
                "highest_rate_kept_up": max(kept) if kept else None, "curve": curve,
                "beyond_configured_range": beyond}
    else:
        r = rig.run(args.rate, args.seconds)
        rig.close()
        line = {"metric": "serving: frames/s and latency (continuous batching, 200 streams)",
                "value": r["frames_per_s"], "unit": "frames/s", "n_gpus": 1, "higher_is_better": True,
                "dtype": "u8", "data": "synthetic",
                "config": {"workload": SERVE_WORKLOAD + f", {args.rate:.0f} req/s for {args.seconds:.1f} s"},
                **{k: v for k, v in r.items() if k != "frames_per_s"}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.workload != "1080p" and args.impl == "native":
        import torch
        torch.cuda.set_device(0)
        import paper_0710_4819_gb300 as me
        me.load_library(build_if_missing=True)
        {"batch64": run_batch64, "serve": run_serve, "loadtable": run_load_table,
         "configs": run_configs}[args.workload](args)
        return
    rank, world, local, pg = dist_setup(args.gpus)
    import numpy as np
    import synth

    frames_np = synth.config_sequence("1080p", seed=replica_seed(rank), n_frames=args.frames)
    pairs = frames_np.shape[0] - 1

    if args.impl == "reference":
        if rank != 0:
            return
        thr = cpu_threads()
        sec = []
        for i in range(args.warmup + args.steps):
            s = oracle_sample(frames_np, 1, thr)
            if i >= args.warmup:
                sec.append(s)
        fps = 1.0 / statistics.mean(sec)
        line = {
            "impl": "reference", "metric": METRIC,
            "value": fps, "unit": "frames/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(sec),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "1 frame pair per step"},
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": thr, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": "1 frame pair per step: FSBM on all cores + ACBM on one"},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line))
        return

    import torch
    import paper_0710_4819_gb300 as me

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    me.load_library(build_if_missing=True)
    lam = me.me_lambda_q8(QP)
    prm = me.params(qp=QP)
    frames = torch.from_numpy(frames_np).to(dev)
    stream = torch.cuda.current_stream()

    # outputs: one field per pair (ACBM chains through them)
    f_mv = torch.empty((pairs, BH, BW, 2), dtype=torch.int16, device=dev)
    f_J = torch.empty((pairs, BH, BW), dtype=torch.int32, device=dev)
    f_sad = torch.empty((pairs, BH, BW), dtype=torch.int32, device=dev)
    a_mv = torch.empty_like(f_mv)
    a_J = torch.empty_like(f_J)
    a_sad = torch.empty_like(f_sad)
    a_mask = torch.empty((pairs, BH, BW), dtype=torch.uint8, device=dev)
    a_load = torch.empty_like(f_J)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    f_out = (f_mv, f_J, f_sad)
    a_out = (a_mv, a_J, a_mask, a_sad, a_load)

    def step():
        # every pair of the sequence: FSBM in one launch, ACBM in one
        # persistent launch with the pairs overlapping
        me.me_fsbm_sequence(frames, N, M, P, lam, out=f_out)
        me.me_acbm_sequence(frames, N, M, P, lam, prm, out=a_out)

    for _ in range(args.warmup):
        step()
    me.me_acbm_sequence_status(W, H_PAD, N, M, P, pairs)

    gpu_index = (int(os.environ["CUDA_VISIBLE_DEVICES"])
                 if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    clocks = ClockSampler(gpu_index)
    step_ms, fsbm_ms, acbm_ms = [], [], []
    clocks.start()
    for _ in range(args.steps):
        flush.fill_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        barrier(pg)
        torch.cuda.synchronize()
        ev[0].record(stream)
        me.me_fsbm_sequence(frames, N, M, P, lam, out=f_out)
        ev[1].record(stream)
        me.me_acbm_sequence(frames, N, M, P, lam, prm, out=a_out)
        ev[2].record(stream)
        torch.cuda.synchronize()
        barrier(pg)
        step_ms.append(ev[0].elapsed_time(ev[2]))
        fsbm_ms.append(ev[0].elapsed_time(ev[1]))
        acbm_ms.append(ev[1].elapsed_time(ev[2]))
    clk = clocks.stop()
    me.me_acbm_sequence_status(W, H_PAD, N, M, P, pairs)
    seq_out = [x.clone() for x in a_out + f_out]
    acbm_load = int(a_load.to(torch.int64).sum().item())
    # positions PBM evaluated: the load of blocks that passed, the 22-position
    # bound (14 predictors + 8 ring) for blocks that went on to a full search
    pbm_positions = int(torch.where(a_mask.bool(), torch.full_like(a_load, 22),
                                    a_load).to(torch.int64).sum().item())
    fs_frac = float(a_mask.float().mean().item())

    total_ms = max_over_ranks(pg, sum(step_ms))
    frames_done = pairs * args.steps * world
    fps = frames_done / (total_ms * 1e-3)

    # per-pair forms: plain ACBM (wave launches replayed from a graph) and
    # single-pair FSBM, for latency per pair and to check identical outputs
    def run_pair(t):
        me.me_fsbm(frames[t], frames[t - 1], N, M, P, lam,
                   out=(f_mv[t - 1], f_J[t - 1], f_sad[t - 1]))
        prev = a_mv[t - 2] if t >= 2 else None
        me.me_acbm(frames[t], frames[t - 1], N, M, P, lam, prm, prev_mv=prev,
                   out=(a_mv[t - 1], a_J[t - 1], a_mask[t - 1], a_sad[t - 1], a_load[t - 1]))
    for t in range(1, pairs + 1):
        run_pair(t)
    torch.cuda.synchronize()
    ep = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(pairs)]
    for t in range(1, pairs + 1):
        ep[t - 1][0].record(stream)
        me.me_fsbm(frames[t], frames[t - 1], N, M, P, lam,
                   out=(f_mv[t - 1], f_J[t - 1], f_sad[t - 1]))
        ep[t - 1][1].record(stream)
        prev = a_mv[t - 2] if t >= 2 else None
        me.me_acbm(frames[t], frames[t - 1], N, M, P, lam, prm, prev_mv=prev,
                   out=(a_mv[t - 1], a_J[t - 1], a_mask[t - 1], a_sad[t - 1], a_load[t - 1]))
        ep[t - 1][2].record(stream)
    torch.cuda.synchronize()
    pair_fsbm_ms = [e[0].elapsed_time(e[1]) for e in ep]
    pair_acbm_ms = [e[1].elapsed_time(e[2]) for e in ep]
    identical = all(torch.equal(x, y) for x, y in zip(seq_out, a_out + f_out))

    # half-pel refinement of the full-search field (Sec. 2.2/2.3; next to the
    # step, not part of it): all pairs in one launch
    h_out = (torch.empty_like(f_mv), torch.empty_like(f_J), torch.empty_like(f_sad))
    for _ in range(3):
        me.me_halfpel_sequence(frames, N, M, P, lam, f_mv, out=h_out)
    torch.cuda.synchronize()
    hp_ms = []
    for _ in range(10):
        flush.fill_(1)
        eh0, eh1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        eh0.record(stream)
        me.me_halfpel_sequence(frames, N, M, P, lam, f_mv, out=h_out)
        eh1.record(stream)
        torch.cuda.synchronize()
        hp_ms.append(eh0.elapsed_time(eh1))
    hp_frame_ms = statistics.median(hp_ms) / pairs

    # SAD_min / SAD_deviation (Sec. 3.1) of one 1080p pair: the FSBM engine
    # with the SAD sum and minimum reduced beside the winning key
    # (timed as single launches after an L2 flush, beside me_fsbm timed the same way)
    ss_ms, fs1_ms = [], []
    for i in range(13):
        for fn, acc in ((lambda c, r: me.me_sad_deviation(c, r, N, M, P, lam), ss_ms),
                        (lambda c, r: me.me_fsbm(c, r, N, M, P, lam, out=(f_mv[0], f_J[0], f_sad[0])),
                         fs1_ms)):
            flush.fill_(1)
            es0, es1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            es0.record(stream)
            fn(frames[1 + i % pairs], frames[i % pairs])
            es1.record(stream)
            torch.cuda.synchronize()
            if i >= 3:
                acc.append(es0.elapsed_time(es1))
    ss_frame_ms = statistics.median(ss_ms)
    fs_single_ms = statistics.median(fs1_ms)
    # FSBM with the rate coded against the median predictor (a wavefront):
    # the whole sequence in two launches, and one pair alone
    pr_out = (torch.empty_like(f_mv), torch.empty_like(f_J), torch.empty_like(f_sad))
    for _ in range(2):
        me.me_fsbm_pred_sequence(frames, N, M, P, lam, out=pr_out)
        me.me_fsbm_pred(frames[1], frames[0], N, M, P, lam, out=(f_mv[0], f_J[0], f_sad[0]))
    torch.cuda.synchronize()
    pr_seq_ms, pr_one_ms = [], []
    for i in range(5):
        for fn, acc in ((lambda: me.me_fsbm_pred_sequence(frames, N, M, P, lam, out=pr_out), pr_seq_ms),
                        (lambda: me.me_fsbm_pred(frames[1 + i], frames[i], N, M, P, lam,
                                                 out=(pr_out[0][0], pr_out[1][0], pr_out[2][0])),
                         pr_one_ms)):
            flush.fill_(1)
            ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ep0.record(stream)
            fn()
            ep1.record(stream)
            torch.cuda.synchronize()
            acc.append(ep0.elapsed_time(ep1))
    pred_ok = me.me_fsbm_pred_status(W, H_PAD, N, M, P, pairs) == 0
    pred_frame_ms = statistics.median(pr_seq_ms) / pairs
    pred_pair_ms = statistics.median(pr_one_ms)

    # the known-motion experiment of Sec. 3.1 / Fig. 3 (CIF, nine moved
    # frames, 16x16, p = 16, lambda = 0): one launch, then its error classes
    st_frames, st_g = synth.global_motion_sequence(41, 352, 288)
    st_f, st_gd = torch.from_numpy(st_frames).cuda(), torch.from_numpy(st_g).cuda()
    for _ in range(3):
        st = me.me_motion_study(st_f, st_gd, 16, 16, 16, 0)
    torch.cuda.synchronize()
    et0, et1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    et0.record(stream)
    st = me.me_motion_study(st_f, st_gd, 16, 16, 16, 0)
    et1.record(stream)
    torch.cuda.synchronize()
    study_ms = et0.elapsed_time(et1)
    st_err = st.err.cpu().numpy().astype(np.int64)
    st_intra = st.intra.cpu().numpy().view(np.uint32) / 256.0    # Intra_SAD (N*M = 256 scale)
    st_dev = st.sad_dev.cpu().numpy().view(np.uint32)
    st_cls = np.minimum(st_err, 5)
    study_classes = [{"error": (str(c) if c < 5 else ">=5"), "blocks": int((st_cls == c).sum()),
                      "median_intra_sad": float(np.median(st_intra[st_cls == c])) if (st_cls == c).any() else None,
                      "median_sad_deviation": float(np.median(st_dev[st_cls == c])) if (st_cls == c).any() else None}
                     for c in range(6)]

    # kernel-only FSBM timing (the SAD engine) for the roofline, same stream
    reps = 20
    ek0, ek1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ek0.record(stream)
    for i in range(reps):
        me.me_fsbm(frames[1 + i % pairs], frames[i % pairs], N, M, P, lam,
                   out=(f_mv[0], f_J[0], f_sad[0]))
    ek1.record(stream)
    torch.cuda.synchronize()
    fsbm_kernel_ms = ek0.elapsed_time(ek1) / reps
    # peak: this device's SMs x the packed-SAD lane rate per SM per clock
    # measured by the library's probe (4 absdiffs per lane-op) x the median
    # SM clock sampled during the timed steps
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    lanes_per_clk = me.me_sad_peak(0)[1]
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    peak_absdiff = n_sm * 4 * lanes_per_clk * sm_mhz * 1e6
    seq_fsbm_ms = statistics.mean(fsbm_ms) / pairs
    achieved = ABSDIFF_PER_FRAME / (seq_fsbm_ms * 1e-3)

    # end-to-end through the C ABI with host buffers: host frames copied in,
    # the step's calls, results copied out, all inside the timed region.  The
    # frames go up in four chunks on a copy stream and the full search of each
    # chunk's pairs starts as soon as its frames are in (pairs are
    # independent); ACBM, whose pairs chain, starts when all frames are in,
    # and the full-search results go down while it runs.
    host_frames = torch.from_numpy(frames_np).pin_memory()
    h_out = [torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in a_out + f_out]
    d_frames = torch.empty_like(frames)
    copy_stream = torch.cuda.Stream()
    n_chunks = 4
    cuts = [round(c * pairs / n_chunks) for c in range(n_chunks + 1)]

    def e2e_once():
        arrived = []
        with torch.cuda.stream(copy_stream):
            for c in range(n_chunks):
                f0 = 0 if c == 0 else cuts[c] + 1       # pairs cuts[c]..cuts[c+1]-1 need
                f1 = cuts[c + 1] + 1                    # frames cuts[c]..cuts[c+1]
                d_frames[f0:f1].copy_(host_frames[f0:f1], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
                arrived.append(ev)
        for c in range(n_chunks):
            stream.wait_event(arrived[c])
            lo, hi = cuts[c], cuts[c + 1]
            me.me_fsbm_sequence(d_frames[lo:hi + 1], N, M, P, lam,
                                out=(f_mv[lo:hi], f_J[lo:hi], f_sad[lo:hi]))
        fs_done = torch.cuda.Event()
        fs_done.record(stream)
        me.me_acbm_sequence(d_frames, N, M, P, lam, prm, out=a_out)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(fs_done)
            for h, d in zip(h_out[len(a_out):], f_out):
                h.copy_(d, non_blocking=True)
        for h, d in zip(h_out[:len(a_out)], a_out):
            h.copy_(d, non_blocking=True)
        torch.cuda.synchronize()

    e2e_once()                                      # warm-up (the chunk shapes' plans)
    e2e_times = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_once()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(pg, statistics.median(e2e_times))
    same_e2e = all(torch.equal(h, d.cpu()) for h, d in zip(h_out, a_out + f_out))
    h2d = host_frames.numel()
    d2h = sum(x.numel() * x.element_size() for x in h_out)
    e2e_fps = pairs * world / e2e_s

    # the batched and served forms, compact legs beside the step: the 64-stream
    # mix (one persistent launch per step against per-frame plain calls,
    # outputs compared) and a Poisson serve run, each with its clock record
    legs = {}
    if rank == 0 and world == 1 and not args.no_extra_legs:
        b64 = batch64_measure(4, gpu_index)
        legs["batch64"] = {"workload": BATCH64_WORKLOAD, "steps": b64["steps"],
                           "acbm": b64["acbm"], "fsbm": b64["fsbm"],
                           "fsbm_absdiff_per_s_T": b64["fsbm_absdiff_per_s_T"], "clocks": b64["clocks"]}
        rig = ServeRig()
        legs["serve"] = dict(rig.run(4000.0, 3.0, gpu_index), workload=SERVE_WORKLOAD)
        rig.close()

    # the autotuner's record for the shapes this run used: model's and chosen
    # launch form and every candidate's time (first call of each shape)
    tuning = parse_tune_log(me.me_tune_log())
    # the dominant kernel: the full-search form the tuner chose for the step
    fs_form = next((t["chosen"] for t in tuning
                    if t["shape"] == f"fsbm {W}x{H_PAD} {N}x{M} p={P} K={pairs}"), "pipe")
    fs_kernel = next(k for pre, k in FSBM_FORM_KERNEL if fs_form.startswith(pre))
    fs_traffic = FSBM_SEQ_DRAM_BYTES_PER_FRAME.get(fs_kernel)

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        thr = cpu_threads()
        sec = oracle_sample(frames_np, 2, thr)
        cpu_base = {"value": 1.0 / sec, "unit": "frames/s", "cores": thr, "kind": "oracle",
                    "cpu_model": cpu_model(),
                    "sample": "frame pairs 1-2 of the sequence: oracle FSBM (OpenMP over "
                              f"blocks, {thr} threads) + oracle ACBM (one thread)"}

    if rank != 0:
        return
    fsbm_mean = statistics.mean(fsbm_ms) / pairs
    acbm_mean = statistics.mean(acbm_ms) / pairs

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]

    pair_ms = [f + a for f, a in zip(pair_fsbm_ms, pair_acbm_ms)]
    line = {
        "metric": METRIC,
        "value": fps, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames_per_step": pairs, "l2": "flushed between steps",
                   "parallelism": f"replicas x{world} (independent sequences, no collective)"},
        "fsbm": {"form": "me_fsbm_sequence (one launch for all pairs)",
                 "frames_per_s": 1e3 / fsbm_mean, "cand_sads_per_s": NBLK * NCAND / (fsbm_mean * 1e-3),
                 "ms_per_frame": fsbm_mean, "single_pair_kernel_ms": fsbm_kernel_ms},
        "acbm": {"form": "me_acbm_sequence (one persistent launch, pairs overlapping)",
                 "frames_per_s": 1e3 / acbm_mean,
                 "cand_sads_per_s": acbm_load / pairs / (acbm_mean * 1e-3),
                 "ms_per_frame": acbm_mean, "fullsearch_fraction": fs_frac,
                 "avg_positions_per_block": acbm_load / (pairs * NBLK),
                 # PBM stages' algorithmic bytes: the current frame, N*M
                 # reference bytes per position PBM evaluated, 12-byte outputs
                 # per block (the full searches read their windows from shared
                 # memory); the true bound is the latency of the dependency chain
                 "pbm_algorithmic_gb_per_s": (W * H_PAD + pbm_positions / pairs * N * M + 12 * NBLK)
                                             / (acbm_mean * 1e-3) / 1e9},
        "halfpel": {"form": "me_halfpel_sequence on the full-search field (one launch)",
                    "ms_per_frame": hp_frame_ms, "frames_per_s": 1e3 / hp_frame_ms,
                    "positions_per_block": 9,
                    # algorithmic bytes: each frame read as current and as reference
                    "algorithmic_gb_per_s": 2 * W * H_PAD / (hp_frame_ms * 1e-3) / 1e9},
        "sad_deviation": {"form": "me_sad_deviation, one 1080p pair (FSBM + SAD_min + SAD_deviation)",
                          "ms_per_frame": ss_frame_ms, "me_fsbm_same_timing_ms": fs_single_ms,
                          "absdiff_per_s": ABSDIFF_PER_FRAME / (ss_frame_ms * 1e-3) / 1e12,
                          "frac_of_peak": ABSDIFF_PER_FRAME / (ss_frame_ms * 1e-3) / peak_absdiff,
                          "unit": "T absdiff/s"},
        "fsbm_pred": {"form": "me_fsbm_pred_sequence: rate against the median predictor "
                              "(SAD volume + persistent wavefront), all pairs in two launches",
                      "ms_per_frame": pred_frame_ms, "frames_per_s": 1e3 / pred_frame_ms,
                      "single_pair_ms": pred_pair_ms, "status_ok": pred_ok},
        "motion_study": {"form": "me_motion_study: CIF original + 9 frames moved by known global "
                                 "vectors, 16x16, p=16, lambda=0, one launch",
                         "ms": study_ms, "classes": study_classes},
        "per_pair": {"form": "me_fsbm + me_acbm per pair (each in the form the tuner chose)",
                     "frames_per_s": 1e3 / statistics.mean(pair_ms),
                     "acbm_ms": statistics.mean(pair_acbm_ms), "fsbm_ms": statistics.mean(pair_fsbm_ms),
                     "p50_ms": pct(pair_ms, 0.5), "p99_ms": pct(pair_ms, 0.99),
                     "outputs_identical_to_sequence": identical},
        "p99_ms": pct(pair_ms, 0.99),
        "roofline": {"bound": "alu", "kernel": fs_kernel, "form": fs_form, "achieved": achieved / 1e12,
                     "peak": peak_absdiff / 1e12, "unit": "T absdiff/s",
                     "frac": achieved / peak_absdiff,
                     # DRAM bytes of one launch over the whole sequence: ncu
                     # dram__bytes_read+write of the same kernel on the 13-frame
                     # case (27.20 MB, every frame read once), scaled by frames
                     "traffic": None if fs_traffic is None else fs_traffic * (pairs + 1),
                     "traffic_unit": "bytes/launch",
                     "algorithmic_bytes": (pairs + 1) * W * H_PAD,
                     "peak_source": f"{n_sm} SMs x {lanes_per_clk:.2f} packed-SAD lanes/clk/SM "
                                    f"(measured by me_sad_peak) x 4 absdiffs x {sm_mhz:.0f} MHz "
                                    "(median SM clock sampled during the timed steps)"},
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "outputs_identical": same_e2e,
                "form": "frames up in 4 chunks on a copy stream, each chunk's full search "
                        "as soon as it is in; median of 3"},
        "gpu_launches": 4 * args.steps,   # the full search; k_seq_begin, k_seq_prologue, k_acbm_seq
        "clocks": clk,
        "cpu_baseline": cpu_base,
        "tuning": tuning,
        **legs,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
