#!/usr/bin/env python
"""Throughput of the symmetry-blocked M2L translation on one GB300.

Workload (the symmetry-blocked FP64/FP32 configuration): a uniform octree of
[-1,1]^3 holding N = 2,000,000 particles U([-1,1]^3) with leaf level 5, so
levels 2..5 are full grids (64 .. 32768 cells, 6,039,504 far-field
interactions in total); Chebyshev order ell = 5 (125 nodes), kernel 1/r.
Multipole vectors are seeded N(0,1) stand-ins for the upward pass (the values
do not change the work).

One step = one pass of the whole hot path:
  a2     m2l_ops_rebuild_tables     (the permutation tables, on device)
  a1     m2l_ops_rebuild_operators  (the 16 operators) and m2l_ops_prepare (their kernel images)
  a3     m2l_plan_classify          (per level 2..5, on the level's stream, after the tables)
  a4-a6  m2l_plan_apply             (per level 2..5, the fused kernel, after the images)
value = far-field interactions of levels 2..5 / step time, summed over ranks.
"""
from __future__ import annotations

import argparse
import platform
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ELL = 5
LEVELS = (2, 3, 4, 5)
KERNEL = 0  # 1/r
N_PARTICLES = 2_000_000
SEED = 2
WORKLOAD = ("uniform octree of [-1,1]^3, N=2,000,000 particles U([-1,1]^3), leaf level 5 (levels 2-5 full: "
            "64/512/4096/32768 cells), ell=5 (125 nodes), kernel 1/r, multipoles N(0,1) seed 2")
METRIC = "M2L interactions/s (levels 2-5, one pass of the hot path)"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
NOMINAL = {"bf16": 2250.0, "tf32": 1100.0}
FLOPS_PER_INTERACTION = 2 * (ELL ** 3) ** 2


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return PEAKS_FALLBACK, "fallback"


def full_interactions(level):
    n = 1 << level
    a = sum(1 for x in range(n) for y in range(n) if abs((x >> 1) - (y >> 1)) <= 1)
    b = 3 * n - 2
    return a ** 3 - b ** 3


class ClockSampler:
    """nvidia-smi clock samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_selector(device):
    """nvidia-smi -i argument of the GPU torch runs on (its UUID when torch knows it)."""
    import torch
    props = torch.cuda.get_device_properties(device)
    u = getattr(props, "uuid", None)
    if u is not None:
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        return vis.split(",")[device.index or 0].strip()
    return str(device.index or 0)


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "gloo":
        device = torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------------------------
def cpu_oracle_sample(ntargets=2048, seed=11, with_locals=False):
    """The oracle, as it stands, on a bounded sample of the level-5 workload:
    the 316 directly assembled operators plus the cell-by-cell M2L of
    `ntargets` random level-5 target cells with their full lists."""
    import numpy as np

    import oracle
    from paper_1210_7292_gb300 import synth
    cells = synth.full_grid(5)
    w = synth.gaussian_vectors(len(cells), ELL ** 3, seed=SEED)
    rng = np.random.default_rng(seed)
    samp = np.sort(rng.choice(len(cells), ntargets, replace=False))
    off, src = oracle.interaction_lists(cells[samp], cells)
    t0 = time.perf_counter()
    ops = oracle.operator_table(ELL, KERNEL, 0.0, 5)
    loc = oracle.m2l_apply(ops, cells[samp], cells, off, src, w)
    dt = time.perf_counter() - t0
    nint = int(off[-1])
    out = {"value": nint / dt, "unit": "interactions/s", "cores": 1, "kind": "oracle",
           "sample": "%d random level-5 target cells (%d interactions) of the workload, 316 operators "
                     "assembled directly, single-threaded C loops, %.1f s" % (ntargets, nint, dt),
           "gflops": nint * FLOPS_PER_INTERACTION / dt / 1e9}
    if with_locals:
        return out, loc
    return out


def host_info():
    """Host cores and CPU model, for the CPU baselines."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu_count": os.cpu_count(), "model": model, "machine": platform.machine()}


def cpu_nablk_sample(ntargets=2048, seed=11, ref=None):
    """The paper's blocked method on the host cores (a paper-style CPU baseline, not
    the oracle): per sampled level-5 target cell the full list, classified by the 16
    unique operators (Sec. 4.2.1), gathered and permuted per class, one BLAS matrix
    product per class (Sec. 4.2.3, NumPy's multithreaded BLAS), un-permuted and
    summed per target.  Operators and tables are built from the oracle's definitions
    inside the timed region, as the GPU step rebuilds them."""
    import numpy as np

    import oracle
    from paper_1210_7292_gb300 import synth
    n3 = ELL ** 3
    cells = synth.full_grid(5)
    w = synth.gaussian_vectors(len(cells), n3, seed=SEED)
    rng = np.random.default_rng(seed)
    samp = np.sort(rng.choice(len(cells), ntargets, replace=False))
    off, src = oracle.interaction_lists(cells[samp], cells)
    tgt = np.repeat(np.arange(len(samp)), np.diff(off))
    t0 = time.perf_counter()
    kp = np.stack([oracle.operator_for_t(ELL, KERNEL, 0.0, 5, t) for t in oracle.t_sym_list()])
    sig = oracle.sigma_tables(ELL)
    lut = oracle.lut343().astype(np.int64)
    t = cells[samp][tgt] - cells[src]
    code = lut[(t[:, 0] + 3) + 7 * (t[:, 1] + 3) + 49 * (t[:, 2] + 3)]
    p, g = code & 0xFF, code >> 8
    order = np.argsort(p, kind="stable")
    bounds = np.searchsorted(p[order], np.arange(17))
    loc = np.zeros((len(samp), n3))
    for q in range(16):
        sel = order[bounds[q]:bounds[q + 1]]
        if len(sel) == 0:
            continue
        sg = sig[g[sel]]
        wp = np.empty((len(sel), n3))
        np.put_along_axis(wp, sg, w[src[sel]], axis=1)       # W[sigma(b)] = w[b]
        f = np.take_along_axis(wp @ kp[q].T, sg, axis=1)     # F = K_p W; f[a] = F[sigma(a)]
        tq = tgt[sel]                                        # ascending within the class
        starts = np.flatnonzero(np.r_[True, tq[1:] != tq[:-1]])
        loc[tq[starts]] += np.add.reduceat(f, starts, axis=0)
    dt = time.perf_counter() - t0
    nint = int(off[-1])
    out = {"value": nint / dt, "unit": "interactions/s", "cores": os.cpu_count(),
           "kind": "paper-style blocked CPU (NumPy BLAS, all host cores; not the oracle)",
           "sample": "the same %d level-5 target cells (%d interactions), %.2f s" % (ntargets, nint, dt),
           "gflops": nint * FLOPS_PER_INTERACTION / dt / 1e9}
    if ref is not None:
        out["rel_l2_vs_oracle"] = float(np.linalg.norm(loc - ref) / np.linalg.norm(ref))
    return out


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle  # noqa: F401  (built by build(); compiled here if missing)
    oracle.build_c()
    ntg = 256
    for _ in range(args.warmup):
        cpu_oracle_sample(ntargets=64)
    vals, times = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = cpu_oracle_sample(ntargets=ntg)
        times.append(time.perf_counter() - t0)
        vals.append(r["value"])
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 (CPU oracle)", "l2_policy": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": 1, "kind": "oracle",
                             "sample": "per step: %d random level-5 target cells with full lists, 316 directly "
                                       "assembled operators, single-threaded C loops" % ntg},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------------------------
def level_streams(device):
    """One stream per level; the largest level's, the step's critical path, at high
    priority so that its classification and apply go ahead of the smaller levels'."""
    import torch
    return {L: torch.cuda.Stream(device=device, priority=-1 if L == max(LEVELS) else 0) for L in LEVELS}


def rebuild_on(m2l, ops, precision, cur):
    """Tables (a2), then operators (a1) and their kernel images, on stream `cur`;
    returns the events after the tables (classification may start) and after the
    images (applies may start)."""
    import torch
    tables, ready = torch.cuda.Event(), torch.cuda.Event()
    m2l.m2l_ops_rebuild_tables(ops, cur)
    tables.record(cur)
    m2l.m2l_ops_rebuild_operators(ops, cur)
    m2l.m2l_ops_prepare(ops, precision, cur)
    ready.record(cur)
    return tables, ready


class Workload:
    def __init__(self, m2l, device, precision, seed):
        import numpy as np
        import torch

        from paper_1210_7292_gb300 import synth
        self.m2l, self.device, self.precision = m2l, device, precision
        self.ops = m2l.m2l_precompute(m2l.M2L_K_INV_R, ELL)
        self.dt_in = torch.float64 if precision == "fp64" else torch.float32
        self.levels, self.mp, self.loc = {}, {}, {}
        self.host = {}
        self.nint = {}
        for L in LEVELS:
            cells = synth.full_grid(L)
            ijk = torch.from_numpy(cells).to(device)
            off, src = m2l.m2l_build_lists(ijk, ijk)
            self.levels[L] = m2l.Level(2.0 / (1 << L), ijk, ijk, off, src, L)
            w = synth.gaussian_vectors(len(cells), ELL ** 3, seed=seed + 100 * L)
            self.mp[L] = torch.from_numpy(w).to(device, self.dt_in)
            self.loc[L] = torch.zeros(len(cells), ELL ** 3, dtype=self.dt_in, device=device)
            self.nint[L] = self.levels[L].nnz
            # pinned host copies for the end-to-end leg
            self.host[L] = {"mp": torch.from_numpy(w).to(self.dt_in).pin_memory(),
                            "ijk": torch.from_numpy(cells).pin_memory(),
                            "off": off.cpu().pin_memory(), "src": src.cpu().pin_memory(),
                            "loc": torch.zeros(len(cells), ELL ** 3, dtype=self.dt_in).pin_memory()}
        self.total = sum(self.nint.values())
        self.local_nint = dict(self.nint)
        assert self.nint[5] == full_interactions(5)
        # M2L at one level reads only that level's multipoles and lists and writes only its
        # locals, so the levels run concurrently: one stream and one plan (its own bucket
        # buffers) per level, classified again in every step
        self.plans = {L: m2l.m2l_plan_create(self.ops, self.levels[L]) for L in LEVELS}
        self.streams = level_streams(device)
        self.copy_streams = {L: torch.cuda.Stream(device=device) for L in LEVELS}
        torch.cuda.synchronize(device)

    def rebuild(self, cur):
        return rebuild_on(self.m2l, self.ops, self.precision, cur)

    def step(self, kev=None):
        """One pass of the hot path: tables (a2) and operators (a1) on the current stream,
        then per level, on its own stream, classification (a3, once the tables are done)
        and the fused apply (a4-a6, once the operators are); the current stream waits for
        every level."""
        import torch
        m2l = self.m2l
        cur = torch.cuda.current_stream(self.device)
        tables, ready = self.rebuild(cur)
        for L in sorted(LEVELS, reverse=True):   # the largest level first: it is the critical path
            s = self.streams[L]
            s.wait_event(tables)
            if kev is not None:
                kev[L][2].record(s)
            m2l.m2l_plan_classify(self.plans[L], self.levels[L], s)
            if kev is not None:
                kev[L][3].record(s)
            s.wait_event(ready)
            if kev is not None:
                kev[L][0].record(s)
            m2l.m2l_plan_apply(self.plans[L], self.mp[L], self.loc[L], self.precision, stream=s)
            if kev is not None:
                kev[L][1].record(s)
            done = torch.cuda.Event()
            done.record(s)
            cur.wait_event(done)

    def e2e_step(self):
        """The same step through the public API from pinned host buffers: every level,
        on its own stream, copies its inputs in, re-classifies its plan from the copied
        lists, applies, and copies its locals out, all inside the timed region."""
        import torch
        m2l = self.m2l
        cur = torch.cuda.current_stream(self.device)
        tables, ready = self.rebuild(cur)
        dev_lv = {}
        for L in sorted(LEVELS, reverse=True):   # the largest level first
            s = self.streams[L]
            s.wait_event(tables)
            h = self.host[L]
            with torch.cuda.stream(s):
                ijk = h["ijk"].to(self.device, non_blocking=True)
                off = h["off"].to(self.device, non_blocking=True)
                src = h["src"].to(self.device, non_blocking=True)
                lv = m2l.Level(2.0 / (1 << L), ijk, ijk, off, src, L)
                loc = torch.zeros(lv.struct.ncells_tgt, ELL ** 3, dtype=self.dt_in, device=self.device)
                m2l.m2l_plan_classify(self.plans[L], lv, s)
            # the multipoles are read by the apply only: they are copied on a stream of
            # their own, beside the lists' copies and the classification
            c = self.copy_streams[L]
            c.wait_event(tables)   # within this step, as every other copy
            with torch.cuda.stream(c):
                mp = h["mp"].to(self.device, non_blocking=True)
            mp.record_stream(s)
            mp_done = torch.cuda.Event()
            mp_done.record(c)
            with torch.cuda.stream(s):
                s.wait_event(mp_done)
                s.wait_event(ready)
                m2l.m2l_plan_apply(self.plans[L], mp, loc, self.precision, stream=s)
                h["loc"].copy_(loc, non_blocking=True)
            dev_lv[L] = (lv, mp, loc)
            done = torch.cuda.Event()
            done.record(s)
            cur.wait_event(done)
        return dev_lv

    def e2e_bytes(self):
        h2d = d2h = 0
        for L in LEVELS:
            h = self.host[L]
            h2d += sum(t.numel() * t.element_size() for t in (h["mp"], h["ijk"], h["off"], h["src"]))
            d2h += h["loc"].numel() * h["loc"].element_size()
        return h2d, d2h


class ShardedWorkload:
    """The same hot path split by target ranges over the ranks (one process per
    GPU): every level's target cells are cut into contiguous ranges; a rank
    owns the multipoles and locals of its range and applies the level's lists
    of its targets.  Per step and level: one all-gather of the level's
    multipoles (the only exchange: sources lie within three cells of a target,
    Sec. 3.2), then the rank's classification and apply on its shard."""

    def __init__(self, m2l, device, precision, seed, rank, world):
        import numpy as np
        import torch

        from paper_1210_7292_gb300 import shard, synth
        self.m2l, self.device, self.precision, self.rank, self.world = m2l, device, precision, rank, world
        self.shard = shard
        self.ops = m2l.m2l_precompute(m2l.M2L_K_INV_R, ELL)
        self.dt_in = torch.float64 if precision == "fp64" else torch.float32
        self.levels, self.mine, self.loc, self.sh, self.ranges, self.nint = {}, {}, {}, {}, {}, {}
        self.host = {}
        for L in LEVELS:
            cells = synth.full_grid(L)
            ijk = torch.from_numpy(cells).to(device)
            off, src = m2l.m2l_build_lists(ijk, ijk)
            off, src = off.cpu().numpy(), src.cpu().numpy()
            sh = shard.shard_level(off, src, rank, world)
            t0, t1 = sh["t0"], sh["t1"]
            tgt = torch.from_numpy(np.ascontiguousarray(cells[t0:t1])).to(device)
            srcs = torch.from_numpy(np.ascontiguousarray(cells[sh["needed"]])).to(device)
            self.levels[L] = m2l.Level(2.0 / (1 << L), tgt, srcs, torch.from_numpy(sh["offsets"]).to(device),
                                       torch.from_numpy(sh["sources"]).to(device), L)
            w = synth.gaussian_vectors(len(cells), ELL ** 3, seed=seed + 100 * L)
            self.mine[L] = torch.from_numpy(np.ascontiguousarray(w[t0:t1])).to(device, self.dt_in)
            self.loc[L] = torch.zeros(t1 - t0, ELL ** 3, dtype=self.dt_in, device=device)
            self.sh[L] = sh
            self.ranges[L] = shard.target_ranges(len(cells), world)
            self.nint[L] = int(len(src))          # interactions of the whole level (all ranks)
            self.host[L] = {"mine": self.mine[L].cpu().pin_memory(),
                            "tgt": tgt.cpu().pin_memory(), "srcs": srcs.cpu().pin_memory(),
                            "off": torch.from_numpy(sh["offsets"]).pin_memory(),
                            "src": torch.from_numpy(sh["sources"]).pin_memory(),
                            "loc": torch.zeros(t1 - t0, ELL ** 3, dtype=self.dt_in).pin_memory()}
        self.total = sum(self.nint.values())
        self.local_nint = {L: self.levels[L].nnz for L in LEVELS}
        self.plans = {L: m2l.m2l_plan_create(self.ops, self.levels[L]) for L in LEVELS}
        self.streams = level_streams(device)
        torch.cuda.synchronize(device)

    def step(self, kev=None):
        import torch
        m2l = self.m2l
        cur = torch.cuda.current_stream(self.device)
        tables, ready = rebuild_on(m2l, self.ops, self.precision, cur)
        for L in sorted(LEVELS, reverse=True):
            s = self.streams[L]
            s.wait_event(tables)
            with torch.cuda.stream(s):
                halo = self.shard.exchange_multipoles(self.mine[L], self.ranges[L], self.sh[L]["needed"])
                if kev is not None:
                    kev[L][2].record(s)
                m2l.m2l_plan_classify(self.plans[L], self.levels[L], s)
                if kev is not None:
                    kev[L][3].record(s)
                s.wait_event(ready)
                if kev is not None:
                    kev[L][0].record(s)
                m2l.m2l_plan_apply(self.plans[L], halo, self.loc[L], self.precision, stream=s)
                if kev is not None:
                    kev[L][1].record(s)
            done = torch.cuda.Event()
            done.record(s)
            cur.wait_event(done)

    def e2e_step(self):
        """The sharded step from pinned host buffers: the rank's multipoles and
        shard lists in, the exchange, classification and apply, its locals out."""
        import torch
        m2l = self.m2l
        cur = torch.cuda.current_stream(self.device)
        tables, ready = rebuild_on(m2l, self.ops, self.precision, cur)
        keep = {}
        for L in sorted(LEVELS, reverse=True):
            s = self.streams[L]
            s.wait_event(tables)
            h = self.host[L]
            with torch.cuda.stream(s):
                mine = h["mine"].to(self.device, non_blocking=True)
                lv = m2l.Level(2.0 / (1 << L), h["tgt"].to(self.device, non_blocking=True),
                               h["srcs"].to(self.device, non_blocking=True), h["off"].to(self.device, non_blocking=True),
                               h["src"].to(self.device, non_blocking=True), L)
                halo = self.shard.exchange_multipoles(mine, self.ranges[L], self.sh[L]["needed"])
                loc = torch.zeros(lv.struct.ncells_tgt, ELL ** 3, dtype=self.dt_in, device=self.device)
                m2l.m2l_plan_classify(self.plans[L], lv, s)
                s.wait_event(ready)
                m2l.m2l_plan_apply(self.plans[L], halo, loc, self.precision, stream=s)
                h["loc"].copy_(loc, non_blocking=True)
            keep[L] = (lv, mine, halo, loc)
            done = torch.cuda.Event()
            done.record(s)
            cur.wait_event(done)
        return keep

    def e2e_bytes(self):
        h2d = d2h = 0
        for L in LEVELS:
            h = self.host[L]
            h2d += sum(t.numel() * t.element_size() for t in (h["mine"], h["tgt"], h["srcs"], h["off"], h["src"]))
            d2h += h["loc"].numel() * h["loc"].element_size()
        return h2d, d2h


def timed(fn, steps, flush, device, kernel_events=False, levels=LEVELS):
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    # per level: apply start/end, classification start/end
    kev = [{L: tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for L in levels}
           for _ in range(steps)] if kernel_events else None
    for i in range(steps):
        flush.zero_()   # evict L2 between timed steps (outside the event pair)
        evs[i][0].record()
        if kernel_events:
            fn(kev[i])
        else:
            fn()
        evs[i][1].record()
    torch.cuda.synchronize(device)
    total = sum(s.elapsed_time(e) for s, e in evs) / 1e3
    kt = None
    if kernel_events:
        kt = {L: [k[L][0].elapsed_time(k[L][1]) / 1e3 for k in kev] for L in levels}
        kt["classify"] = {L: [k[L][2].elapsed_time(k[L][3]) / 1e3 for k in kev] for L in levels}
    return total, kt


def traffic_for(kernel_name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    ent = d.get(kernel_name)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_1210_7292_gb300", "csrc", ent["source"])
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] if os.path.exists(src) else None
    return ent["dram_bytes_per_launch"] if h == ent.get("source_sha256_16") else None


# the level-5 launch: full levels take the target-stationary tensor-core kernel
KERNEL_FOR = {"fp64": ("simt_apply_kernel<double>", "m2l_apply_simt.cu", "alu"),
              "fp32": ("simt_apply_kernel<float>", "m2l_apply_simt.cu", "alu"),
              "tf32": ("tc_dense_kernel<tf32>", "m2l_dense.cu", "tensor"),
              "bf16x3": ("tc_dense_kernel<bf16x3>", "m2l_dense.cu", "tensor"),
              "tf32x3": ("tc_dense_kernel<tf32x3>", "m2l_dense.cu", "tensor")}


def matmul_peaks(device, n=8192):
    """Dense matrix-product throughput of this GPU, measured here with
    torch.matmul (cuBLAS) on n x n x n products, best of a few: FP64, FP32 with
    TF32 off, and TF32.  These are the roofline denominators of the FP64, FP32
    and TF32 kernels (the BF16 peaks come from MEASURED_PEAKS.json)."""
    import torch
    keep = torch.backends.cuda.matmul.allow_tf32
    out = {}
    try:
        for name, dt, tf32, reps in (("fp64", torch.float64, False, 3), ("fp32", torch.float32, False, 5),
                                     ("tf32", torch.float32, True, 10)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            g = torch.Generator(device=device).manual_seed(1)
            a = torch.randn(n, n, device=device, dtype=dt, generator=g)
            b = torch.randn(n, n, device=device, dtype=dt, generator=g)
            c = torch.matmul(a, b)
            torch.cuda.synchronize(device)
            best = float("inf")
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize(device)
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[name] = 2.0 * n ** 3 / best / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = keep
    out["how"] = "torch.matmul %d^3, best of 3 (fp64) / 5 (fp32, TF32 off) / 10 (tf32), this run" % n
    return out


def roofline(precision, achieved_tflops, peaks, src_kind, mm):
    """Roofline of the level-5 apply kernel.  The kernel is timed per launch
    inside a step of about a millisecond, so the BF16 denominator is the burst
    peak; the split precisions execute three tensor products per algorithmic
    one, so their peak is the product peak / 3."""
    kname, src, bound = KERNEL_FOR[precision]
    bf = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])
    if precision == "fp32":
        peak, how = mm["fp32"], "FP32 matmul (TF32 off) measured in this run"
    elif precision == "fp64":
        peak, how = mm["fp64"], "FP64 matmul measured in this run"
    elif precision == "tf32":
        peak, how = mm["tf32"], "TF32 matmul measured in this run"
    elif precision == "bf16x3":
        peak, how = bf / 3.0, "bf16 burst (%s, MEASURED_PEAKS.json) / 3 products" % src_kind
    else:
        peak, how = mm["tf32"] / 3.0, "TF32 matmul measured in this run / 3 products"
    nprod = 3 if precision in ("bf16x3", "tf32x3") else 1   # tensor products per algorithmic one
    return {"bound": bound, "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved_tflops / peak, "traffic": traffic_for(kname), "kernel": kname, "peak_source": how,
            "executed_tflops": achieved_tflops * nprod, "products_per_flop": nprod,
            "flops_per_launch": FLOPS_PER_INTERACTION * full_interactions(5),
            "flop_convention": "algorithmic 2*ell^6 per interaction, level-5 launch"}


def precompute_times(m2l, device, reps=3):
    """Wall time of the precompute (step a1: the 16 operators, tables and, with
    eps > 0, their low-rank factors by truncated SVD or by ACA + truncated SVD)
    at the bench's order and at the mixed-precision workload's ell = 7, 1/r^4,
    eps = 1e-7."""
    import torch
    out = {}
    svd, aca = m2l.m2l_precompute, m2l.m2l_precompute_aca
    for name, fn, kind, ell, eps in (("full_ell5_inv_r", svd, m2l.M2L_K_INV_R, ELL, 0.0),
                                     ("svd_ell5_inv_r_eps1e-5", svd, m2l.M2L_K_INV_R, ELL, 1e-5),
                                     ("aca_ell5_inv_r_eps1e-5", aca, m2l.M2L_K_INV_R, ELL, 1e-5),
                                     ("svd_ell7_inv_r4_eps1e-7", svd, m2l.M2L_K_INV_R4, 7, 1e-7),
                                     ("aca_ell7_inv_r4_eps1e-7", aca, m2l.M2L_K_INV_R4, 7, 1e-7)):
        fn(kind, ell, eps)   # first call: module load, workspace
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            ops = fn(kind, ell, eps)
            torch.cuda.synchronize(device)
            ts.append(1e3 * (time.perf_counter() - t0))
            del ops
        out[name] = round(statistics.median(ts), 3)
    out["unit"] = "ms (synchronous call, host wall time)"
    return out


def variants_compare(m2l, device, wl, flush, eps=1e-5, reps=5):
    """The level-5 apply of the workload in the paper's other variants at one
    accuracy eps (Sec. 4): SA and SArcmp (one basis for all 316 operators,
    Eqs. (17)-(19)) and the symmetry-blocked path on per-operator truncated
    SVDs (Eq. (20) with Sec. 4.2), all FP32, each with its own bucketing of the
    list; error against the FP64 full-rank result of the same level."""
    import torch
    lv = wl.levels[5]
    n3 = ELL ** 3
    mp64 = wl.mp[5].double()
    ref = torch.zeros(lv.struct.ncells_tgt, n3, dtype=torch.float64, device=device)
    m2l.m2l_apply_level(wl.ops, lv, mp64, ref, "fp64")
    mp32 = wl.mp[5].float().contiguous()
    out = {"eps": eps, "level": 5, "interactions": lv.nnz, "precision": "fp32"}

    def run(name, fn, info):
        loc = torch.zeros(lv.struct.ncells_tgt, n3, dtype=torch.float32, device=device)
        fn(loc)
        torch.cuda.synchronize(device)
        err = float(torch.linalg.norm(loc.double() - ref) / torch.linalg.norm(ref))
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(loc)
            e1.record()
            torch.cuda.synchronize(device)
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        out[name] = dict(info, ms=ms, interactions_per_s=lv.nnz / (ms / 1e3), rel_l2_vs_fp64_full=err)

    for rc in (False, True):
        t0 = time.perf_counter()
        sa = m2l.m2l_sa_create(wl.ops, eps, rc)
        setup = 1e3 * (time.perf_counter() - t0)
        r, nrc, _ = m2l.m2l_sa_info(sa)
        name = "sarcmp" if rc else "sa"
        run(name, lambda loc, sa=sa: m2l.m2l_sa_apply_level(sa, lv, mp32, loc, "fp32"),
            {"rank": r, "recompressed_cores": nrc, "setup_ms": round(setup, 1)})
        # the cores on the tensor cores (dense C_t)
        run(name + "_bf16x3", lambda loc, sa=sa: m2l.m2l_sa_apply_level(sa, lv, mp32, loc, "bf16x3"),
            {"rank": r, "core": "tcgen05 BF16x3, dense C_t"})
        del sa
    t0 = time.perf_counter()
    ops_lr = m2l.m2l_precompute(m2l.M2L_K_INV_R, ELL, eps)
    setup = 1e3 * (time.perf_counter() - t0)
    ranks = m2l.m2l_ops_query(ops_lr)[0]
    run("blocked_lowrank", lambda loc: m2l.m2l_apply_level(ops_lr, lv, mp32, loc, "fp32"),
        {"ranks_min_max": [int(ranks.min()), int(ranks.max())], "setup_ms": round(setup, 1)})
    m2l.m2l_sync_status(wl.ops)
    m2l.m2l_sync_status(ops_lr)
    return out


DFMM_PARTICLES = 168931   # the paper's sphere (Sec. 5)
DFMM_K = 32.0             # k = 1 in its box of side 64, on the unit domain of side 2
DFMM_LEVELS = (3, 4, 5, 6)


def dfmm_m2l(m2l, device, mm, reps=5):
    """The directional (Helmholtz) M2L of the paper's sphere at ell = 5 over its
    high-frequency levels 3-6: lists and plans built once (set-up, timed apart),
    then every level's complex M2L per pass, FP32 and FP64 (the FP32 error
    against FP64 over all levels)."""
    import torch

    from paper_1210_7292_gb300 import synth
    ell = ELL
    n3 = ell ** 3
    pts, _ = synth.sphere_surface(DFMM_PARTICLES, seed=21)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    plans, vecs, per_level = {}, {}, {}
    for L in DFMM_LEVELS:
        ijk = torch.from_numpy(synth.occupied_cells(pts, L)).to(device)
        C, off, src = m2l.m2l_dfmm_build_lists(L, DFMM_K, ijk)
        lv = m2l.DLevel(2.0 / (1 << L), ijk, ijk, C, off, src, L)
        plans[L] = m2l.m2l_dfmm_plan_create(ell, DFMM_K, lv)
        tsym, _, _, nnz = m2l.m2l_dfmm_plan_info(plans[L])
        g = torch.Generator(device=device).manual_seed(SEED + L)
        n = ijk.shape[0] * C * n3
        w = torch.complex(torch.randn(n, generator=g, device=device, dtype=torch.float64),
                          torch.randn(n, generator=g, device=device, dtype=torch.float64))
        vecs[L] = w
        per_level[L] = {"cells": int(ijk.shape[0]), "cones": C, "interactions": int(nnz), "T_sym": int(len(tsym))}
    setup_ms = 1e3 * (time.perf_counter() - t0)
    total = sum(v["interactions"] for v in per_level.values())
    flops = 8.0 * n3 * n3 * total
    out = {"workload": "sphere, %d particles, k w = 8, 4, 2, 1 at levels 3-6, ell = %d" % (DFMM_PARTICLES, ell),
           "levels": per_level, "interactions": total, "setup_ms": round(setup_ms, 1),
           "flop_convention": "8 ell^6 real flops per complex interaction"}
    res = {}
    for prec, dt in (("fp64", torch.complex128), ("fp32", torch.complex64), ("bf16x3", torch.complex64),
                     ("tf32x3", torch.complex64), ("tf32", torch.complex64)):
        for L in DFMM_LEVELS:   # tensor-core layouts are built ahead of the timing
            m2l.m2l_dfmm_plan_prepare(plans[L], prec)
        W = {L: vecs[L].to(dt) for L in DFMM_LEVELS}
        F = {L: torch.zeros_like(W[L]) for L in DFMM_LEVELS}

        def one():
            for L in DFMM_LEVELS:
                m2l.m2l_dfmm_plan_apply(plans[L], W[L], F[L], prec)
        one()
        torch.cuda.synchronize(device)
        res[prec] = {L: F[L].to(torch.complex128).clone() for L in DFMM_LEVELS}
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            one()
            e1.record()
            torch.cuda.synchronize(device)
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        out[prec] = {"ms": ms, "interactions_per_s": total / (ms / 1e3), "tflops": flops / (ms / 1e3) / 1e12}
        for L in DFMM_LEVELS:
            m2l.m2l_dfmm_plan_sync(plans[L])
    den = sum(float(torch.linalg.norm(res["fp64"][L]) ** 2) for L in DFMM_LEVELS)
    for prec in ("fp32", "bf16x3", "tf32x3", "tf32"):
        num = sum(float(torch.linalg.norm(res[prec][L] - res["fp64"][L]) ** 2) for L in DFMM_LEVELS)
        out[prec]["rel_l2_vs_fp64"] = (num / den) ** 0.5
    out["fp32"]["roofline"] = {"bound": "alu", "peak_tflops": round(mm["fp32"], 1),
                               "frac": out["fp32"]["tflops"] / mm["fp32"],
                               "peak_source": "FP32 matmul (TF32 off) measured in this run"}
    return out


def config3_levels(m2l, device, reps=5):
    """The mixed-precision workload (4 M points on the ellipsoid (1, 0.5, 0.25),
    ell = 7, 1/r^4, SVD at eps = 1e-7), levels 4-6: every level in the low-rank
    operators (FP64, FP32 on the CUDA cores; TF32, BF16x3, TF32x3 on the tensor
    cores, two passes) and in the full-rank ones (FP64, FP32, TF32, BF16x3,
    TF32x3), timed per level with its lists classified once, and the
    error of each against the FP64 full-rank result.  GFLOP/s counts the products
    each one performs (full: 2 ell^6; low rank: 4 r_p ell^3 per interaction)."""
    import numpy as np
    import torch

    from paper_1210_7292_gb300 import synth
    ell, eps = 7, 1e-7
    n3 = ell ** 3
    pts, _ = synth.ellipsoid_surface(4_000_000, (1.0, 0.5, 0.25), seed=3)
    ops = {"full": m2l.m2l_precompute(m2l.M2L_K_INV_R4, ell), "lowrank": m2l.m2l_precompute(m2l.M2L_K_INV_R4, ell, eps)}
    ranks = m2l.m2l_ops_query(ops["lowrank"])[0]
    out = {"workload": "4M points on the ellipsoid (1, 0.5, 0.25), ell 7, 1/r^4, SVD eps 1e-7",
           "ranks": [int(r) for r in ranks], "levels": {}}
    for L in (4, 5, 6):
        cells = synth.occupied_cells(pts, L)
        ijk = torch.from_numpy(cells).to(device)
        off, src = m2l.m2l_build_lists(ijk, ijk)
        lv = m2l.Level(2.0 / (1 << L), ijk, ijk, off, src, L)
        plans = {k: m2l.m2l_plan_create(o, lv) for k, o in ops.items()}
        counts, _ = m2l.m2l_plan_query(plans["full"])
        w64 = torch.from_numpy(synth.gaussian_vectors(len(cells), n3, seed=33 + L)).to(device)
        lr_flops = float(sum(4.0 * ranks[p] * n3 * counts[p] for p in range(16)))
        full_flops = 2.0 * n3 * n3 * lv.nnz
        res = {"cells": len(cells), "interactions": lv.nnz}
        ref = None
        for name, prec in (("full", "fp64"), ("lowrank", "fp64"), ("lowrank", "fp32"), ("full", "fp32"),
                           ("full", "tf32"), ("full", "bf16x3"), ("full", "tf32x3"),
                           ("lowrank", "tf32"), ("lowrank", "bf16x3"), ("lowrank", "tf32x3")):
            win = w64 if prec == "fp64" else w64.float()
            loc = torch.zeros(len(cells), n3, dtype=torch.float64, device=device)
            fp64_out = prec != "fp64"
            m2l.m2l_plan_apply(plans[name], win, loc, prec, out_fp64=fp64_out)
            torch.cuda.synchronize(device)
            if ref is None:
                ref = loc.clone()
            err = float(torch.linalg.norm(loc - ref) / torch.linalg.norm(ref))
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                m2l.m2l_plan_apply(plans[name], win, loc, prec, out_fp64=fp64_out)
                e1.record()
                torch.cuda.synchronize(device)
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            fl = full_flops if name == "full" else lr_flops
            res["%s_%s" % (name, prec)] = {"ms": ms, "interactions_per_s": lv.nnz / (ms / 1e3),
                                           "gflops": fl / (ms / 1e3) / 1e9, "rel_l2_vs_fp64_full": err}
        for o in ops.values():
            m2l.m2l_sync_status(o)
        out["levels"][L] = res
    return out


def fmm_matvec(m2l, device, precision, reps=5):
    """The whole bbFMM matvec of the workload's particles on the GPU
    (m2l_fmm_evaluate: P2M, M2M, M2L at levels 2-5, L2L, L2P and near field);
    set-up (tree, lists, plans) timed apart."""
    import torch

    from paper_1210_7292_gb300 import synth
    pts, q = synth.uniform_cube(N_PARTICLES, seed=SEED)
    dt = torch.float64 if precision == "fp64" else torch.float32
    xyz = torch.from_numpy(pts).to(device, dt)
    qq = torch.from_numpy(q).to(device, dt)
    ops = m2l.m2l_precompute(m2l.M2L_K_INV_R, ELL)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    fmm = m2l.m2l_fmm_create(ops, xyz, max(LEVELS))
    setup_ms = 1e3 * (time.perf_counter() - t0)
    phi = torch.zeros(N_PARTICLES, dtype=dt, device=device)
    for _ in range(2):
        m2l.m2l_fmm_evaluate(fmm, xyz, qq, phi, precision)
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        m2l.m2l_fmm_evaluate(fmm, xyz, qq, phi, precision)
        e1.record()
        torch.cuda.synchronize(device)
        ts.append(e0.elapsed_time(e1))
    _, ncells, nnz = m2l.m2l_fmm_info(fmm)
    return {"ms": statistics.median(ts), "setup_ms": setup_ms, "particles": N_PARTICLES,
            "leaf_level": max(LEVELS), "ell": ELL, "m2l_precision": precision,
            "m2l_interactions": int(nnz.sum()), "leaf_cells": int(ncells[max(LEVELS)]),
            "note": "P2M, M2M, M2L (levels 2-5), L2L, L2P and near field, particles resident on the GPU"}


def config4_batched(m2l, device, mm, peaks, reps=5):
    """The batched workload: 64 independent trees (seed 4; N log-uniform in
    [1e4, 1e6], uniform cube and sphere surface alternating, leaf levels 3-6,
    ell in {4, 5, 6}), kernel 1/sqrt(r^2 + 0.01^2), every level 2..leaf of every
    tree as one problem.  Per precision one m2l_batch (the autotuner picks its
    tile shapes), its run captured in a CUDA graph and replayed: interactions/s,
    algorithmic GFLOP/s (2 ell^6 per interaction), the roofline fraction, the
    chosen shapes, and the rel. L2 of all outputs against the FP64 batch."""
    import torch

    from paper_1210_7292_gb300 import synth
    c = 0.01
    ops_cache, probs = {}, []
    for spec in synth.batched_tree_specs(64, seed=4):
        pts, _ = synth.tree_points(spec)
        ell = spec["ell"]
        for L in range(2, spec["leaf_level"] + 1):
            cells = synth.occupied_cells(pts, L)
            width = 2.0 / (1 << L)
            if (ell, L) not in ops_cache:
                ops_cache[(ell, L)] = m2l.m2l_precompute(m2l.M2L_K_INV_SQRT_R2C2, ell, 0.0, width, c)
            ijk = torch.from_numpy(cells).to(device)
            off, src = m2l.m2l_build_lists(ijk, ijk)
            lv = m2l.Level(width, ijk, ijk, off, src, L)
            w = synth.gaussian_vectors(len(cells), ell ** 3, seed=spec["seed"] * 10 + L)
            probs.append((ops_cache[(ell, L)], lv, w, ell))
    plans = [m2l.m2l_plan_create(o, lv) for o, lv, _, _ in probs]
    nnz = sum(lv.nnz for _, lv, _, _ in probs)
    flops = sum(2.0 * (ell ** 3) ** 2 * lv.nnz for _, lv, _, ell in probs)
    bf = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])
    peak = {"fp32": mm["fp32"], "tf32x3": mm["tf32"] / 3.0, "bf16x3": bf / 3.0}
    out = {"workload": "64 trees (seed 4), N log-uniform 1e4-1e6, cube / sphere surface, leaf levels 3-6, "
                       "ell 4-6, 1/sqrt(r^2 + 0.01^2), all levels 2..leaf",
           "problems": len(probs), "interactions": nnz, "gflop": flops / 1e9}
    res = {}
    for prec in ("fp64", "fp32", "tf32x3", "bf16x3"):
        dt = torch.float64 if prec == "fp64" else torch.float32
        ins = [torch.from_numpy(w).to(device, dt) for _, _, w, _ in probs]
        outs = [torch.zeros(lv.struct.ncells_tgt, ell ** 3, dtype=dt, device=device) for _, lv, _, ell in probs]
        t0 = time.perf_counter()
        batch = m2l.m2l_batch_create(plans, ins, outs, prec)
        create_ms = 1e3 * (time.perf_counter() - t0)
        m2l.m2l_batch_run(batch)
        torch.cuda.synchronize(device)
        res[prec] = torch.cat([o.double().flatten() for o in outs])
        s = torch.cuda.Stream(device=device)
        s.wait_stream(torch.cuda.current_stream(device))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                m2l.m2l_batch_run(batch, stream=s)
        torch.cuda.current_stream(device).wait_stream(s)
        g.replay()
        torch.cuda.synchronize(device)
        n = 1 if prec == "fp64" else reps
        ts = []
        for _ in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize(device)
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        info = m2l.m2l_batch_info(batch)
        entry = {"graph_replay_ms": ms, "interactions_per_s": nnz / (ms / 1e3), "gflops": flops / (ms / 1e3) / 1e9,
                 "create_ms_incl_autotune": round(create_ms, 1), "tiles": info["tiles"],
                 "launch_groups": [{"ell3": e3, "tile_width": nt, "epilogue_groups": eg}
                                   for e3, nt, eg in m2l.m2l_batch_groups(batch)]}
        if prec in peak:
            entry["roofline"] = {"achieved_tflops": flops / (ms / 1e3) / 1e12, "peak_tflops": peak[prec],
                                 "frac": flops / (ms / 1e3) / 1e12 / peak[prec]}
        out[prec] = entry
        m2l.m2l_sync_status(probs[0][0])
        del g, batch
    for prec in ("fp32", "tf32x3", "bf16x3"):
        out[prec]["rel_l2_vs_fp64"] = float(torch.linalg.norm(res[prec] - res["fp64"]) / torch.linalg.norm(res["fp64"]))
    return out


def config5_differentiation(m2l, device, mm, peaks, reps=3):
    """The differentiation workload: full level 6 (262,144 cells), ell = 5,
    1/r, loss = sum(W * M2L(w)) with w, W ~ N(0, 1) (seeds 5, 6); one step =
    forward M2L + backward (the adjoint M2L) through torch.autograd, with plans
    classified once.  Per precision: step time, interactions/s counting both
    directions, algorithmic GFLOP/s (2 ell^6 per interaction and direction),
    the roofline fraction of the apply kernels, and the gradient's rel. L2
    against the FP64 gradient."""
    import torch

    from paper_1210_7292_gb300 import autograd, synth
    level, ell = 6, ELL
    n3 = ell ** 3
    cells = synth.full_grid(level)
    ijk = torch.from_numpy(cells).to(device)
    off, src = m2l.m2l_build_lists(ijk, ijk)
    lv = m2l.Level(2.0 / (1 << level), ijk, ijk, off, src, level)
    nnz = lv.nnz
    ops = m2l.m2l_precompute(m2l.M2L_K_INV_R, ell)
    w64 = torch.from_numpy(synth.gaussian_vectors(len(cells), n3, seed=5)).to(device)
    W64 = torch.from_numpy(synth.gaussian_vectors(len(cells), n3, seed=6)).to(device)
    flops = 2.0 * n3 * n3 * nnz * 2
    bf = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])
    peak = {"fp64": mm["fp64"], "fp32": mm["fp32"], "tf32x3": mm["tf32"] / 3.0, "bf16x3": bf / 3.0}
    out = {"workload": "full level 6 (262,144 cells), ell 5, 1/r, loss = sum(W * M2L(w)), w, W ~ N(0,1) seeds 5, 6",
           "interactions_per_direction": nnz, "flop_convention": "2 ell^6 per interaction and direction"}
    grads = {}
    for prec in ("fp64", "fp32", "tf32x3", "bf16x3"):
        op = autograd.M2LLevelOperator(ops, lv, prec)
        dt = torch.float64 if prec == "fp64" else torch.float32
        w, W = w64.to(dt), W64.to(dt)

        def step():
            x = w.clone().requires_grad_(True)
            loss = (W * op(x)).sum()
            loss.backward()
            return x.grad

        g = step()
        torch.cuda.synchronize(device)
        grads[prec] = g.double()
        n = 1 if prec == "fp64" else reps
        ts, tf, tb = [], [], []
        for _ in range(n):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record()
            step()
            e[1].record()
            op.apply_forward(w)
            e[2].record()
            op.apply_adjoint(W)
            e[3].record()
            torch.cuda.synchronize(device)
            ts.append(e[0].elapsed_time(e[1]))
            tf.append(e[1].elapsed_time(e[2]))
            tb.append(e[2].elapsed_time(e[3]))
        ms = statistics.median(ts)
        res = {"step_ms": ms, "forward_ms": statistics.median(tf), "adjoint_ms": statistics.median(tb),
               "interactions_per_s": 2 * nnz / (ms / 1e3), "gflops": flops / (ms / 1e3) / 1e9,
               "dense_kernel": m2l.m2l_plan_kernel_info(op.fwd)["dense"] and prec not in ("fp64", "fp32")}
        kern_ms = res["forward_ms"] + res["adjoint_ms"]
        res["roofline"] = {"achieved_tflops": flops / (kern_ms / 1e3) / 1e12, "peak_tflops": peak[prec],
                           "frac": flops / (kern_ms / 1e3) / 1e12 / peak[prec],
                           "peak_source": {"fp64": "FP64 matmul, this run", "fp32": "FP32 matmul, this run",
                                           "tf32x3": "TF32 matmul, this run / 3",
                                           "bf16x3": "bf16 burst (MEASURED_PEAKS.json) / 3"}[prec]}
        out[prec] = res
        m2l.m2l_sync_status(ops)
        del op
    ref = grads["fp64"]
    for prec in ("fp32", "tf32x3", "bf16x3"):
        out[prec]["grad_rel_l2_vs_fp64"] = float(torch.linalg.norm(grads[prec] - ref) / torch.linalg.norm(ref))
    return out


def direct_sum_at(pts, q, samp, device, chunk=16):
    """f_i = sum_{j != i} q_j / |x_i - x_j| at the sampled particles (Eq. (1)),
    in FP64 with torch on the GPU: the exact reference of the error figure
    below (measurement only, not the product path)."""
    import torch
    x = torch.from_numpy(pts).to(device, torch.float64)
    qq = torch.from_numpy(q).to(device, torch.float64)
    out = []
    for a in range(0, len(samp), chunk):
        idx = torch.as_tensor(samp[a:a + chunk], device=device)
        # differences taken directly (no |x|^2 + |y|^2 - 2 x.y expansion, which
        # cancels for near pairs); the particle itself is excluded by index
        d = x[idx][:, None, :] - x[None, :, :]
        r = torch.sqrt((d * d).sum(dim=2))
        inv = 1.0 / r
        inv[torch.arange(len(idx), device=device), idx] = 0.0
        out.append(inv @ qq)
    return torch.cat(out).cpu().numpy()


def fmm_equal_error(m2l, device, precisions, nsamp=1000):
    """The equal-error criterion of the metric, per M2L precision: the whole
    GPU FMM matvec of the workload's particles (m2l_fmm_evaluate; FP64
    particles and passes with the FP64 M2L, FP32 ones with the others) against
    the direct sum at 1000 sampled particles.  A precision is at equal error
    when its relative L2 error is within 10 % of the FP64 run's."""
    import numpy as np
    import torch

    from paper_1210_7292_gb300 import synth
    pts, q = synth.uniform_cube(N_PARTICLES, seed=SEED)
    samp = np.sort(np.random.default_rng(12).choice(N_PARTICLES, nsamp, replace=False))
    exact = direct_sum_at(pts, q, samp, device)
    ops = m2l.m2l_precompute(m2l.M2L_K_INV_R, ELL)
    err = {}
    for fp64 in (True, False):
        dt = torch.float64 if fp64 else torch.float32
        xyz = torch.from_numpy(pts).to(device, dt)
        qq = torch.from_numpy(q).to(device, dt)
        fmm = m2l.m2l_fmm_create(ops, xyz, max(LEVELS))
        for prec in (["fp64"] if fp64 else [p for p in precisions if p != "fp64"]):
            phi = torch.zeros(N_PARTICLES, dtype=dt, device=device)
            m2l.m2l_fmm_evaluate(fmm, xyz, qq, phi, prec)
            got = phi.double().cpu().numpy()[samp]
            err[prec] = float(np.linalg.norm(got - exact) / np.linalg.norm(exact))
        del fmm
    out = {"criterion": "rel. L2 vs the direct sum at %d sampled particles within 10 %% of the FP64 run's" % nsamp,
           "rel_l2_vs_direct_sum": err}
    out["ratio_to_fp64"] = {p: e / err["fp64"] for p, e in err.items()}
    out["at_equal_error"] = {p: bool(e <= 1.10 * err["fp64"]) for p, e in err.items()}
    return out


def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU (the product path has no CPU fallback)")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    import __graft_entry__ as g
    g.build()
    from paper_1210_7292_gb300 import m2l
    prec = args.precision
    sharded = world > 1 or args.shard
    if sharded and world == 1:
        # one rank of the sharded path (its single all-gather needs a process group)
        import socket

        import torch.distributed as dist
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1)
    if sharded:
        wl = ShardedWorkload(m2l, device, prec, SEED, rank, world)
        local5 = wl.levels[5].nnz
    else:
        wl = Workload(m2l, device, prec, SEED + rank)
        local5 = wl.nint[5]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    for _ in range(args.warmup):
        wl.step()
    torch.cuda.synchronize(device)
    m2l.m2l_sync_status(wl.ops)
    clocks = ClockSampler(gpu_selector(device))
    barrier(world)
    torch.cuda.synchronize(device)
    launches0 = m2l.m2l_launch_count()
    clocks.start()
    total, kt = timed(wl.step, args.steps, flush, device, kernel_events=True)
    clk = clocks.stop()
    launches = m2l.m2l_launch_count() - launches0
    torch.cuda.synchronize(device)
    barrier(world)
    m2l.m2l_sync_status(wl.ops)
    tmax = max_over_ranks(world, total, device)
    # replicas: every rank runs the whole workload; shards: the ranks share one
    units = wl.total if sharded else world * wl.total
    value = units * args.steps / tmax
    k5 = statistics.mean(kt[5])
    ach = FLOPS_PER_INTERACTION * local5 / k5 / 1e12
    peaks, src_kind = measured_peaks()
    mm = matmul_peaks(device)

    # end-to-end leg through host buffers
    for _ in range(2):
        wl.e2e_step()
    torch.cuda.synchronize(device)
    barrier(world)
    e2e_total, _ = timed(wl.e2e_step, max(2, args.steps // 2), flush, device)
    e2e_max = max_over_ranks(world, e2e_total, device)
    e2e_val = units * max(2, args.steps // 2) / e2e_max
    h2d, d2h = wl.e2e_bytes()

    # FP64 and the other precisions beside the headline, with their error vs FP64 at level 5
    extra = {}
    if rank == 0 and not args.quick:
        ref64 = None
        for p in ["fp64"] + [q for q in args.compare if q != "fp64"]:
            try:
                w2 = wl if p == prec else Workload(m2l, device, p, SEED)
                for _ in range(1):
                    w2.step()
                torch.cuda.synchronize(device)
                for L in LEVELS:
                    w2.loc[L].zero_()
                t2, kt2 = timed(w2.step, 2 if p == "fp64" else 5, flush, device, kernel_events=True)
                m2l.m2l_sync_status(w2.ops)
                res = {"interactions_per_s": w2.total * (2 if p == "fp64" else 5) / t2,
                       "level5_kernel_ms": 1e3 * statistics.mean(kt2[5]),
                       "level5_gflops": FLOPS_PER_INTERACTION * w2.nint[5] / statistics.mean(kt2[5]) / 1e9}
                loc5 = w2.loc[5].double() / (2 if p == "fp64" else 5)
                if p == "fp64":
                    ref64 = loc5
                    res["rel_l2_vs_fp64"] = 0.0
                elif ref64 is not None:
                    res["rel_l2_vs_fp64"] = float(torch.linalg.norm(loc5 - ref64) / torch.linalg.norm(ref64))
                extra[p] = res
            except m2l.M2LError as e:
                extra[p] = {"unavailable": str(e)}
    fmm = fmm_matvec(m2l, device, prec) if (rank == 0 and not args.quick and prec != "fp64") else None
    pre = precompute_times(m2l, device) if (rank == 0 and not args.quick) else None
    wl_full = wl if not sharded else (Workload(m2l, device, prec, SEED) if (rank == 0 and not args.quick) else None)
    variants = variants_compare(m2l, device, wl_full, flush) if (rank == 0 and not args.quick) else None
    dfmm = dfmm_m2l(m2l, device, mm) if (rank == 0 and not args.quick) else None
    cfg3 = config3_levels(m2l, device) if (rank == 0 and not args.quick) else None
    cfg5 = config5_differentiation(m2l, device, mm, peaks) if (rank == 0 and not args.quick) else None
    cfg4 = config4_batched(m2l, device, mm, peaks) if (rank == 0 and not args.quick) else None
    eqerr = (fmm_equal_error(m2l, device, ["fp64", "fp32", "tf32x3", "bf16x3", "tf32"])
             if (rank == 0 and not args.quick) else None)
    cpu = None
    if rank == 0 and world == 1 and not args.quick:
        cpu, ref_loc = cpu_oracle_sample(with_locals=True)
        cpu["host"] = host_info()
        cpu["nablk"] = cpu_nablk_sample(ref=ref_loc)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
                "scaling": "strong" if sharded else "weak", "vs_baseline": None,
                # the arithmetic of the products: BF16 (or TF32) operands, split into three
                # products for bf16x3 / tf32x3, with FP32 accumulation; FP32 vectors
                "dtype": {"fp64": "f64", "fp32": "f32"}.get(prec, prec),
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "precision": prec, "levels": list(LEVELS),
                           "interactions_per_step_per_gpu": sum(wl.local_nint.values()),
                           "l2_policy": "inputs (49 MB) fit in L2: a 256 MB buffer is written between timed steps",
                           "parallelism": ("target-range shards over %d rank(s), one multipole all-gather per level"
                                           % world) if sharded else "single GPU"},
                "gflops": value * FLOPS_PER_INTERACTION / 1e9,
                "level5_kernel_ms": 1e3 * k5,
                "per_level": {L: {"interactions": wl.local_nint[L], "apply_ms": 1e3 * statistics.mean(kt[L]),
                                  "classify_ms": 1e3 * statistics.mean(kt["classify"][L]),
                                  "interactions_per_s": wl.local_nint[L] / statistics.mean(kt[L]),
                                  "gflops": FLOPS_PER_INTERACTION * wl.local_nint[L] / statistics.mean(kt[L]) / 1e9}
                              for L in LEVELS},
                "roofline": roofline(prec, ach, peaks, src_kind, mm),
                "matmul_peaks_tflops": mm,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": "interactions/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches,
                "fmm_matvec": fmm,
                "equal_error": eqerr,
                "precompute": pre,
                "variants": variants,
                "dfmm_m2l": dfmm,
                "config3": cfg3,
                "config4": cfg4,
                "config5": cfg5,
                "clocks": clk,
                "precisions": extra}
        print(json.dumps(line), flush=True)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
    return 0


def run_apply_only(args):
    """Level-5 apply launches alone (classified once), for profiler captures of
    the dominant kernel: the same launch configuration the step times."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1210_7292_gb300 import m2l
    device = torch.device("cuda", 0)
    wl = Workload(m2l, device, args.precision, SEED)
    m2l.m2l_classify_level(wl.ops, wl.levels[5])
    for i in range(3):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        m2l.m2l_apply_classified(wl.ops, wl.mp[5], wl.loc[5], args.precision)
        e.record()
        torch.cuda.synchronize()
        log("level-5 apply (%s): %.3f ms" % (args.precision, s.elapsed_time(e)))
    m2l.m2l_sync_status(wl.ops)
    return 0


def run_dfmm_apply_only(args):
    """The directional M2L of the dFMM workload's level 5 (ell = 5) alone, three
    launches in --dfmm-precision, for profiler captures of its apply kernel."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1210_7292_gb300 import m2l, synth
    device = torch.device("cuda", 0)
    pts, _ = synth.sphere_surface(DFMM_PARTICLES, seed=21)
    L = 5
    ijk = torch.from_numpy(synth.occupied_cells(pts, L)).to(device)
    C, off, src = m2l.m2l_dfmm_build_lists(L, DFMM_K, ijk)
    plan = m2l.m2l_dfmm_plan_create(ELL, DFMM_K, m2l.DLevel(2.0 / (1 << L), ijk, ijk, C, off, src, L))
    n = ijk.shape[0] * C * ELL ** 3
    prec = args.dfmm_precision
    dt = torch.float64 if prec == "fp64" else torch.float32
    W = torch.complex(torch.randn(n, device=device, dtype=dt), torch.randn(n, device=device, dtype=dt))
    F = torch.zeros_like(W)
    m2l.m2l_dfmm_plan_prepare(plan, prec)
    for _ in range(3):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        m2l.m2l_dfmm_plan_apply(plan, W, F, prec)
        e.record()
        torch.cuda.synchronize()
        log("dFMM level-5 apply (%s, %d interactions): %.3f ms" % (prec, src.numel(), s.elapsed_time(e)))
    m2l.m2l_dfmm_plan_sync(plan)
    return 0


def run_config3_apply_only(args):
    """Level 6 of the mixed-precision workload (4M points on the ellipsoid, ell
    = 7, 1/r^4), full-rank operators (or the SVD factors at eps = 1e-7 with
    --config3-lowrank), three applies in --config3-precision: for profiler
    captures of the large-order kernel."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1210_7292_gb300 import m2l, synth
    device = torch.device("cuda", 0)
    pts, _ = synth.ellipsoid_surface(4_000_000, (1.0, 0.5, 0.25), seed=3)
    L, ell = 6, 7
    cells = synth.occupied_cells(pts, L)
    ijk = torch.from_numpy(cells).to(device)
    off, src = m2l.m2l_build_lists(ijk, ijk)
    lv = m2l.Level(2.0 / (1 << L), ijk, ijk, off, src, L)
    ops = m2l.m2l_precompute(m2l.M2L_K_INV_R4, ell, 1e-7 if args.config3_lowrank else 0.0)
    plan = m2l.m2l_plan_create(ops, lv)
    prec = args.config3_precision
    w = torch.from_numpy(synth.gaussian_vectors(len(cells), ell ** 3, seed=33 + L)).to(device, torch.float32)
    loc = torch.zeros(len(cells), ell ** 3, dtype=torch.float32, device=device)
    m2l.m2l_ops_prepare(ops, prec)
    for _ in range(3):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        m2l.m2l_plan_apply(plan, w, loc, prec)
        e.record()
        torch.cuda.synchronize()
        log("config-3 level-6 apply (%s%s, %d interactions): %.3f ms"
            % (prec, ", low rank" if args.config3_lowrank else "", lv.nnz, s.elapsed_time(e)))
    m2l.m2l_sync_status(ops)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    # BF16x3 is the fastest precision whose end-to-end FMM error equals the FP64 one on this workload
    ap.add_argument("--precision", default="bf16x3", choices=["fp64", "fp32", "tf32", "bf16x3", "tf32x3"])
    ap.add_argument("--compare", default="fp32,tf32,tf32x3,bf16x3",
                    help="comma list of extra precisions to report (FP64 is always measured)")
    ap.add_argument("--quick", action="store_true", help="skip the extra precisions and the CPU baseline")
    ap.add_argument("--shard", action="store_true",
                    help="run the target-range sharded path even on one rank (it is the default for N > 1)")
    ap.add_argument("--apply-only", action="store_true",
                    help="run three level-5 apply launches only (for profiler captures)")
    ap.add_argument("--dfmm-apply-only", action="store_true",
                    help="run three directional level-5 apply launches only (for profiler captures)")
    ap.add_argument("--config3-apply-only", action="store_true",
                    help="run three level-6 applies of the mixed-precision workload only (for profiler captures)")
    ap.add_argument("--config3-lowrank", action="store_true",
                    help="with --config3-apply-only: the per-operator SVD factors at eps = 1e-7")
    ap.add_argument("--config3-precision", default="bf16x3", choices=["fp32", "tf32", "bf16x3", "tf32x3"],
                    help="precision of --config3-apply-only")
    ap.add_argument("--dfmm-precision", default="fp32", choices=["fp64", "fp32", "tf32", "bf16x3", "tf32x3"],
                    help="precision of --dfmm-apply-only")
    args = ap.parse_args()
    args.compare = [p for p in args.compare.split(",") if p]
    if args.warmup < 3:
        log("warmup raised to 3")
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.apply_only:
        return run_apply_only(args)
    if args.dfmm_apply_only:
        return run_dfmm_apply_only(args)
    if args.config3_apply_only:
        return run_config3_apply_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
