#!/usr/bin/env python
"""Benchmark of the all-pairs UniFrac path on B300 GPUs.

One step = the whole hot path over one synthetic study, one C-ABI call: the
branch embedding (level-synchronous postorder sums), packing, and the pair
kernels of BOTH variants (unweighted on tensor cores, weighted normalized on
the CUDA cores), in mixed precision, writing both full N x N FP32 matrices
(the default workload: 50,000 samples on a 200,000-tip tree, 2 x 10 GB).  The
metric is pair-branch updates per second: each variant counts C(N,2) * B, B
the branches kept after pruning (observed below, non-zero length).

Under torchrun (N > 1) one study is split into contiguous stripe ranges of
equal pair count, one per rank (no collective in the computation; the timing
is reduced after the timed region): strong scaling of one fixed matrix.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded row sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "tips200000_samples50000"
METRIC = "UniFrac pair-branch updates/s (both variants, mixed precision)"
UNIT = "pair-branch updates/s"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-rows", type=int, default=2,
                    help="rows of the oracle's bounded sample (cpu_baseline)")
    ap.add_argument("--layout", default="full", choices=["full", "condensed"],
                    help="output layout of the timed step")
    ap.add_argument("--fp64-stripes", type=int, default=64,
                    help="stripes of the plain FP64 measurement (extrapolated to the matrix)")
    ap.add_argument("--serial-steps", type=int, default=5,
                    help="steps of the per-kernel timing loop (variants one after the other)")
    ap.add_argument("--tune-repeats", type=int, default=1,
                    help="timed runs per autotuner candidate")
    ap.add_argument("--tuned-cache", default=None,
                    help="autotuner cache file (default: the package's tuned.json)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-persistent", action="store_true",
                    help="pair kernels with one CTA per work item instead of the persistent "
                         "work queue")
    ap.add_argument("--streamed-chunk", type=int, default=0,
                    help="stripes per chunk of the streamed-output measurement (0: the "
                         "fastest of 2,048, 4,096 and 8,192)")
    ap.add_argument("--mantel-perms", type=int, default=999,
                    help="permutations of the Mantel-test measurement (0 = skip it)")
    ap.add_argument("--mantel-only", action="store_true",
                    help="run only the Mantel-test measurement on the workload (profiling)")
    ap.add_argument("--no-overlap", action="store_true",
                    help="run the two variants one after the other in the headline loop")
    ap.add_argument("--sparse-fraction", type=float, default=None,
                    help="weighted dense/sparse split as a fraction of the largest study "
                         "(instead of the autotuner)")
    ap.add_argument("--uw-sparse-fraction", type=float, default=None,
                    help="unweighted tensor-core/sparse split, same convention (0 = all "
                         "tensor core)")
    ap.add_argument("--no-per-study", action="store_true",
                    help="skip the one-launch-per-study comparison (several studies)")
    ap.add_argument("--record-traffic", default=None, metavar="CSV",
                    help="write profiles/traffic.json from an ncu --csv capture of "
                         "dram__bytes_read.sum / dram__bytes_write.sum and exit")
    ap.add_argument("--samples", type=int, default=None,
                    help="truncate the workload to this many samples (profiling runs)")
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# source files each pair kernel is built from (traffic records are void once
# any of them changes)
# (capi.cu orders the tile pairs, which shapes the L2 reuse and so the traffic)
KERNEL_SOURCES = {
    "k_pairs_tc": ("pairs_tc.cu", "epilogue.cuh", "ufb_internal.cuh"),
    "k_pairs_weighted<float>": ("pairs_simt.cu", "epilogue.cuh", "ufb_internal.cuh"),
    "k_pairs_sparse<false>": ("pairs_simt.cu", "ufb_internal.cuh"),
    "k_pairs_sparse<true>": ("pairs_simt.cu", "ufb_internal.cuh"),
    "k_pairs_list<false>": ("pairs_simt.cu", "ufb_internal.cuh"),
    "k_pairs_list<true>": ("pairs_simt.cu", "ufb_internal.cuh"),
}
# functions of capi.cu that plan the pair launches (work items, their order,
# buffer sizes): part of every pair kernel's record
PLANNING_FUNCTIONS = ("void study_items(", "static int plan_items(", "static int plan_buffers(",
                      "static int32_t sparse_parts(", "static int plan_lists(")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")


def planning_source() -> bytes:
    """The text of the launch-planning functions of capi.cu (each from its
    signature to the closing brace at column 0)."""
    text = open(os.path.join(ROOT, "paper_2107_05397_b300", "csrc", "capi.cu")).read()
    out = []
    for sig in PLANNING_FUNCTIONS:
        i = text.index(sig)
        out.append(text[i:text.index("\n}\n", i) + 3])
    return "".join(out).encode()


def code_only(text: str) -> str:
    """C++ source without // comments and blank lines (so that edits of the
    comments do not void a measurement)."""
    out = []
    for line in text.splitlines():
        i = line.find("//")
        while i >= 0 and line[:i].count('"') % 2 == 1:  # inside a string literal
            i = line.find("//", i + 2)
        if i >= 0:
            line = line[:i]
        line = line.rstrip()
        if line:
            out.append(line)
    return "\n".join(out)


def kernel_source_hash(kernel: str):
    """Hash of what a pair kernel's launches depend on: its source files (the
    shared header without the host-only context struct) and the
    launch-planning functions, comments left out."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES.get(kernel, ("pairs_simt.cu", "pairs_tc.cu", "epilogue.cuh",
                                            "ufb_internal.cuh")):
        with open(os.path.join(ROOT, "paper_2107_05397_b300", "csrc", name)) as f:
            text = f.read()
        if name == "ufb_internal.cuh" and "struct unifrac_ctx {" in text:
            i = text.index("struct unifrac_ctx {")
            text = text[:i] + text[text.index("\n};\n", i) + 4:]
        h.update(code_only(text).encode())
    h.update(code_only(planning_source().decode()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str, samples: int, thresholds: dict):
    """DRAM bytes (read + write) per launch from a committed ncu capture of the
    same workload and sample count with the same dense / sparse split, if the
    kernel's sources are unchanged since (else None).  profiles/traffic.json
    holds one record per captured split."""
    try:
        records = json.load(open(TRAFFIC_PATH)).get("records", [])
    except Exception:
        return None
    for data in records:
        rec = data.get(kernel)
        if (rec and data.get("workload") == workload and data.get("samples") == samples
                and data.get("thresholds") == thresholds
                and rec.get("source_hash") == kernel_source_hash(kernel)):
            return rec.get("bytes_per_launch")
    return None


def split_thresholds(sparse_fraction: float, uw_sparse_fraction: float, n_max: int) -> dict:
    """The option values bench.py sets for the given split fractions."""
    return {"sparse": max(1, int(round(sparse_fraction * n_max))),
            "uw_sparse": 0 if uw_sparse_fraction == 0 else max(1, int(round(uw_sparse_fraction * n_max)))}


def record_traffic(csv_path: str, workload: str, samples: int, capture: str, thresholds: dict):
    """Adds to profiles/traffic.json the record of an ncu --csv capture with the
    metrics dram__bytes_read.sum and dram__bytes_write.sum: mean bytes per
    launch of each pair kernel, with the hash of its current sources, for the
    workload, sample count and split thresholds of the captured run (replacing
    an earlier record of the same three)."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hdr]
    ki, ii, mi, vi = (h.index("Kernel Name"), h.index("ID"), h.index("Metric Name"),
                      h.index("Metric Value"))
    ui = h.index("Metric Unit") if "Metric Unit" in h else None
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    per = {}
    for r in rows[hdr + 1:]:
        if len(r) <= vi or r[mi] not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        name = r[ki].split("(")[0].split("::")[-1].replace("<1>", "<true>").replace("<0>", "<false>")
        if name not in KERNEL_SOURCES:
            continue
        unit = scale.get(r[ui], 1.0) if ui is not None else 1.0
        per.setdefault(name, {}).setdefault((r[ii], r[ki]), 0.0)
        per[name][(r[ii], r[ki])] += float(r[vi].replace(",", "")) * unit
    out = {"workload": workload, "samples": samples, "capture": capture, "thresholds": thresholds}
    for name, launches in sorted(per.items()):
        vals = list(launches.values())
        out[name] = {"bytes_per_launch": sum(vals) / len(vals), "launches": len(vals),
                     "source_hash": kernel_source_hash(name)}
    try:  # keep the records of other workloads and splits
        records = json.load(open(TRAFFIC_PATH)).get("records", [])
    except Exception:
        records = []
    records = [r for r in records if (r.get("workload"), r.get("samples"), r.get("thresholds"))
               != (workload, samples, thresholds)] + [out]
    with open(TRAFFIC_PATH, "w") as f:
        json.dump({"records": records}, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"ufb_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        finally:
            try:
                os.remove(self.path)
            except OSError:
                pass
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def oracle_sample(w, rows):
    """Time the FP64 oracle (as it stands) on `rows` x all samples, both variants."""
    import oracle
    t0 = time.perf_counter()
    out = {}
    threads = 1
    for v in (oracle.UNWEIGHTED, oracle.WEIGHTED_NORMALIZED):
        out[v], threads = oracle.unifrac_rows(w.tree, w.table, v, rows)
    dt = time.perf_counter() - t0
    return out, dt, threads


def kept_branches(w):
    """Branches with a sample below them and non-zero length (B of the metric)."""
    n = w.tree.n_nodes
    reached = np.zeros(n, dtype=bool)
    reached[w.table.feature_node[np.diff(w.table.indptr) > 0]] = True
    for k in range(n - 1):  # postorder: children first
        if reached[k]:
            reached[w.tree.parent[k]] = True
    reached[n - 1] = False
    return int(np.count_nonzero(reached & (w.tree.length > 0)))


def study_table(table, s):
    """Sub-table of study s (columns renumbered from 0)."""
    from paper_2107_05397_b300 import synth
    lo, hi = int(table.study_offsets[s]), int(table.study_offsets[s + 1])
    rows = np.repeat(np.arange(table.n_features), np.diff(table.indptr))
    m = (table.indices >= lo) & (table.indices < hi)
    return synth.coo_to_table(table.n_features, hi - lo, rows[m], table.indices[m] - lo,
                              table.counts[m], table.feature_node)


def select_studies(table, chosen):
    """Table of the chosen studies only, in the given order."""
    from paper_2107_05397_b300 import synth
    rows = np.repeat(np.arange(table.n_features), np.diff(table.indptr))
    so = table.study_offsets
    rr, cc, vv, offs = [], [], [], [0]
    for s in chosen:
        lo, hi = int(so[s]), int(so[s + 1])
        m = (table.indices >= lo) & (table.indices < hi)
        rr.append(rows[m])
        cc.append(table.indices[m] - lo + offs[-1])
        vv.append(table.counts[m])
        offs.append(offs[-1] + hi - lo)
    cat = lambda xs: np.concatenate(xs) if xs else np.empty(0, np.int64)
    return synth.coo_to_table(table.n_features, offs[-1], cat(rr), cat(cc), cat(vv),
                              table.feature_node, np.asarray(offs, np.int32))


def baseline_study(w):
    """(study index, its table, offset of its condensed block) of the study the
    CPU baseline and the error check use: the largest one."""
    so = w.table.study_offsets
    if so is None:
        return 0, w.table, 0
    sizes = np.diff(so)
    s = int(np.argmax(sizes))
    off = int(sum(int(n) * (int(n) - 1) // 2 for n in sizes[:s]))
    return s, study_table(w.table, s), off


def reference_arm(args):
    """The FP64 oracle as it stands on the host cores: each step is one seeded
    row of the workload's largest study against every column, the two
    variants alternating step by step (the oracle embeds every column each
    call, so a step is several seconds at 50,000 samples)."""
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from paper_2107_05397_b300 import synth
    w0 = synth.make_workload(args.workload)
    _, sub, _ = baseline_study(w0)
    w = synth.Workload(w0.name, w0.tree, sub, w0.description)
    N = w.table.n_samples
    B = kept_branches(w)
    import oracle
    rng = np.random.default_rng(7)
    rows = rng.choice(N, size=max(1, args.steps + min(args.warmup, 1)), replace=True)
    variants = (oracle.UNWEIGHTED, oracle.WEIGHTED_NORMALIZED)
    k = 0
    for _ in range(min(args.warmup, 1)):
        oracle.unifrac_rows(w.tree, w.table, variants[k % 2], rows[k:k + 1])
        k += 1
    times = []
    threads = 1
    for step in range(args.steps):
        t0 = time.perf_counter()
        _, threads = oracle.unifrac_rows(w.tree, w.table, variants[step % 2], rows[k:k + 1])
        times.append(time.perf_counter() - t0)
        k += 1
    units = 1.0 * (N - 1) * B  # one row, one variant per step
    value = units * len(times) / sum(times)
    sample = (f"1 seeded row x {N} columns per step, variants alternating "
              f"(unweighted, weighted normalized)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "samples": N, "branches": B, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def mantel_leg(args, w, stream, tuned_opts, peaks):
    """The Mantel test (Pearson and Spearman, args.mantel_perms permutations)
    between the unweighted and weighted matrices of workload `w` (full
    layout, FP32): the downstream comparison of two distance matrices.
    Wall time of the synchronous calls; roofline of the whole Pearson call
    against the HBM peak."""
    import torch
    from paper_2107_05397_b300 import binding as ub
    N = w.table.n_samples
    with ub.Context(w.tree, w.table, stream=stream) as mctx:
        for k_, v_ in tuned_opts.items():
            mctx.set_option(k_, v_)
        Xu = mctx.run(ub.UNWEIGHTED, ub.MIXED, ub.OUT_FULL)
        Xw = mctx.run(ub.WEIGHTED_NORMALIZED, ub.MIXED, ub.OUT_FULL)
        torch.cuda.synchronize()
    m_perm = args.mantel_perms
    perms = np.random.default_rng(5).permuted(
        np.tile(np.arange(N, dtype=np.int32), (m_perm, 1)), axis=1)
    mres = {}
    for method in ("pearson", "spearman"):
        ub.unifrac_mantel(Xu, Xw, perms[:8], method)  # warm-up
        tm_ = []
        for rep in range(2):
            t0 = time.perf_counter()
            r_m, _, p_m = ub.unifrac_mantel(Xu, Xw, perms, method)
            tm_.append(time.perf_counter() - t0)
        mres[method] = {"s_per_call": float(np.median(tm_)), "r": r_m, "p": p_m}
    P_ = N * (N - 1) // 2
    # per permutation every pair of x is read once (HBM); rows of y are staged
    # once per batch of 16 permutations and are not counted
    alg = (m_perm + 1) * P_ * 4.0
    t_pear = mres["pearson"]["s_per_call"]
    hbm = (peaks or {}).get("hbm_gbs") or 6400.0
    ach = alg / t_pear / 1e9
    out = {"n": N, "permutations": m_perm, **mres,
           "roofline": {"kernel": "k_mantel_cross", "bound": "hbm", "achieved": ach, "peak": hbm,
                        "unit": "GB/s", "frac": ach / hbm,
                        "work": "every pair of x once per permutation (4 bytes x P pairs)",
                        "timed": "whole synchronous Pearson call (moments, permutation "
                                 "upload, cross sums, reduction)"}}
    if not args.no_cpu_baseline:
        from oracle import mantel as om
        n_c, m_c = min(1500, N), 4
        rng_c = np.random.default_rng(6)
        iu = np.triu_indices(n_c, 1)
        xc = Xu.view(N, N)[:n_c, :n_c].double().cpu().numpy()[iu]
        yc = Xw.view(N, N)[:n_c, :n_c].double().cpu().numpy()[iu]
        pc = np.array([rng_c.permutation(n_c) for _ in range(m_c)])
        t0 = time.perf_counter()
        om.mantel(xc, yc, n_c, pc, "pearson")
        t_c = time.perf_counter() - t0
        per = t_c / ((m_c + 1) * (n_c * (n_c - 1) // 2))
        out["cpu_baseline"] = {
            "kind": "oracle", "cores": 1, "sample": f"Pearson, n = {n_c}, {m_c} permutations",
            "s_per_pair_permutation": per, "est_s_per_call": per * (m_perm + 1) * P_}
    del Xu, Xw
    return out


def pipe_peaks():
    """Measured FP32 and FP64 FMA rates of this GPU (ops/s), the ALU ceilings."""
    from paper_2107_05397_b300 import binding as ub
    return (ub.unifrac_measure_peak(ub.PEAK_FP32_FMA), ub.unifrac_measure_peak(ub.PEAK_FP64_FMA))


def row_values(out, v, layout, N, rows):
    """Rows `rows` of variant v's matrix (FP64 numpy [len(rows), N]) from the
    device output of a BOTH run (full: contiguous rows; condensed: gathered)."""
    import torch
    if layout == "full":
        M = out[v * N * N:(v + 1) * N * N].view(N, N)
        return M.index_select(0, torch.as_tensor(rows, device=out.device)).double().cpu().numpy()
    P = N * (N - 1) // 2
    vec = out[v * P:(v + 1) * P]
    res = np.zeros((len(rows), N))
    for r, i in enumerate(rows):
        j = np.arange(N)
        a, b = np.minimum(i, j), np.maximum(i, j)
        idx = a * N - a * (a + 1) // 2 + (b - a - 1)
        g = vec[torch.as_tensor(np.where(i == j, 0, idx), device=out.device)].double().cpu().numpy()
        res[r] = np.where(i == j, 0.0, g)
    return res


def fp64_leg(args, w, stream, flush, units_full, rows_check=16):
    """The plain FP64 path (bit-packed lookup unweighted, FP64 min-sum
    weighted) on the same GPU, over a seeded range of args.fp64_stripes
    stripes, both variants one after the other (CUDA events), extrapolated to
    the whole matrix by the ratio of 128 x 128 tile pairs; per-kernel
    fractions against the measured FP64 rate; the range's values checked on
    seeded pairs against the oracle."""
    import torch
    import oracle
    from paper_2107_05397_b300 import binding as ub
    from paper_2107_05397_b300 import replicas
    N = w.table.n_samples
    S = replicas.n_stripes(N)
    width = max(1, min(args.fp64_stripes, S))
    s0 = int(np.random.default_rng(8).integers(0, S - width + 1))
    s1 = s0 + width
    T = -(-N // 128)
    res = {"stripes": [s0, s1], "extrapolated": True}
    with ub.Context(w.tree, w.table, stream=stream) as c:
        c.set_option(ub.OPT_OVERLAP_VARIANTS, 0)
        out = c.run(ub.BOTH, ub.FP64, ub.OUT_STRIPES, s0, s1)  # warm-up (allocates)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.run(ub.BOTH, ub.FP64, ub.OUT_STRIPES, s0, s1, out=out)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        tiles = c.stat(ub.STAT_TILE_PAIRS)
        uw_ms = c.stat(ub.STAT_PAIR_MS_UNWEIGHTED)
        wn_ms = c.stat(ub.STAT_PAIR_MS_WEIGHTED)
        sel_uw = c.stat(ub.STAT_SELECTED_UNWEIGHTED)
        sel_wn = c.stat(ub.STAT_SELECTED_WEIGHTED)
        got = out.view(2, s1 - s0, N).cpu().numpy()
        dev_err = c.stat(ub.STAT_DEVICE_ERROR)
        del out
    torch.cuda.empty_cache()
    full_tiles = T * (T + 1) / 2
    ms_full = ms * full_tiles / max(tiles, 1.0)
    res.update({"ms_range": ms, "tile_pairs_range": tiles, "tile_pairs_full": full_tiles,
                "ms_per_step": ms_full, "value": units_full / (ms_full / 1e3),
                "device_error": dev_err,
                "extrapolation": "range time x (tile pairs of the matrix / tile pairs of the "
                                 "range); embedding and packing counted once per range"})
    rng = np.random.default_rng(9)
    ss = rng.integers(0, s1 - s0, size=rows_check)
    kk = rng.integers(0, N, size=rows_check)
    jj = (kk + s0 + ss + 1) % N
    errs = {}
    for name, v in (("unweighted", 0), ("weighted_normalized", 1)):
        ref = oracle.unifrac_pairs(w.tree, w.table, v, kk, jj)
        errs[name] = float(np.max(np.abs(got[v][ss, kk] - ref)))
    res["max_abs_err_vs_oracle"] = errs
    res["kernel_ms"] = {"k_pairs_lookup": uw_ms, "k_pairs_weighted<double>": wn_ms}
    res["_work"] = {"lookup_group_adds": sel_uw / 8.0, "weighted_fp64_updates": sel_wn}
    return res


def main():
    args = parse()
    if args.record_traffic:
        if args.sparse_fraction is None or args.uw_sparse_fraction is None:
            raise SystemExit("--record-traffic needs the captured run's --sparse-fraction and "
                             "--uw-sparse-fraction")
        from paper_2107_05397_b300 import synth
        tb = synth.make_workload(args.workload, n_samples=args.samples).table
        n_max = (int(max(np.diff(tb.study_offsets))) if tb.study_offsets is not None
                 else tb.n_samples)
        return record_traffic(args.record_traffic, args.workload, tb.n_samples,
                              "one ncu call per pair-kernel family <k> (k_pairs_sparse, "
                              "k_pairs_weighted, k_pairs_tc, k_pairs_list): ncu --metrics "
                              "dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                              "--clock-control none -k regex:<k> -c 6 --csv python bench.py "
                              f"--workload {args.workload} --steps 1 --warmup 1 --no-e2e "
                              "--no-fp64 --no-cpu-baseline --mantel-perms 0 --no-graph "
                              "--no-overlap (settings from the package's tuned cache: split "
                              f"fractions {args.sparse_fraction} weighted, "
                              f"{args.uw_sparse_fraction} unweighted)",
                              split_thresholds(args.sparse_fraction, args.uw_sparse_fraction, n_max))
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    from paper_2107_05397_b300 import binding as ub
    from paper_2107_05397_b300 import replicas
    from paper_2107_05397_b300 import synth

    rank, world, local_rank = env_rank()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = synth.make_workload(args.workload, n_samples=args.samples)
    batched = w.table.study_offsets is not None
    if batched and world > 1:
        # independent studies: each rank takes its share (no data-path collective)
        sizes = [int(x) for x in np.diff(w.table.study_offsets)]
        w = synth.Workload(w.name, w.tree,
                           select_studies(w.table, replicas.shard_studies(sizes, rank, world)),
                           w.description)
    N = w.table.n_samples
    stream = torch.cuda.current_stream()
    if args.mantel_only:
        print(json.dumps({"workload": w.name, "samples": N,
                          "mantel": mantel_leg(args, w, stream, {}, measured_peaks())}))
        return
    layout = ub.OUT_FULL if (args.layout == "full") else ub.OUT_CONDENSED
    # one study on several ranks: contiguous stripe ranges of equal pair count
    s0, s1 = (0, -1)
    if not batched and world > 1:
        s0, s1 = replicas.shard_stripes(N, rank, world)
    ctx = ub.Context(w.tree, w.table, stream=stream)
    nb_out = ctx.output_bytes(ub.MIXED, layout)
    out_both = torch.empty(2 * nb_out // 4, dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    pair_branch = ctx.stat(ub.STAT_PAIR_BRANCH)
    if s1 >= 0:  # this rank's share of the pairs
        mine = sum(replicas.stripe_pairs(N, s) for s in range(s0, s1))
        units_per_step = 2.0 * pair_branch * mine / max(N * (N - 1) // 2, 1)
    else:
        units_per_step = 2.0 * pair_branch  # both variants

    def step(precision=ub.MIXED, out=out_both):
        # both variants from one embedding pass, one C-ABI call
        ctx.run(ub.BOTH, precision, layout, s0, s1, out=out)
        return ctx.stat(ub.STAT_KERNEL_LAUNCHES)

    tuned = {}
    if not args.no_autotune:  # the library's own tuner (cached per shape), before timing
        from paper_2107_05397_b300 import autotune
        cache = args.tuned_cache or autotune.DEFAULT_CACHE
        for v in (ub.UNWEIGHTED, ub.WEIGHTED_NORMALIZED):
            rec = autotune.tune(ctx, v, ub.MIXED, cache_path=cache, repeats=args.tune_repeats)
            tuned.update(rec)
    n_max = int(max(np.diff(w.table.study_offsets))) if batched else N
    if args.sparse_fraction is not None:
        ctx.set_option(ub.OPT_SPARSE_THRESHOLD, max(1, int(round(args.sparse_fraction * n_max))))
        tuned["sparse_fraction"] = args.sparse_fraction
    if args.uw_sparse_fraction is not None:
        f = args.uw_sparse_fraction
        ctx.set_option(ub.OPT_UNWEIGHTED_SPARSE_THRESHOLD, 0 if f == 0 else max(1, int(round(f * n_max))))
        tuned["uw_sparse_fraction"] = f
    if not args.no_graph:
        ctx.set_option(ub.OPT_USE_GRAPH, 1)
    ctx.set_option(ub.OPT_PERSISTENT, 0 if args.no_persistent else 1)
    for _ in range(args.warmup):
        step()
    barrier()

    ctx.set_option(ub.OPT_OVERLAP_VARIANTS, 0 if args.no_overlap else 1)
    for _ in range(args.warmup):  # (re-)capture with the headline setting
        step()
    step_ms, pair_wn_ms, pair_uw_ms, sel_wn, sel_uw = [], [], [], [], []
    sp_uw_ms, sp_wn_ms, sp_uw_n, sp_wn_n, serial_ms = [], [], [], [], []
    li_uw_ms, li_wn_ms, li_uw_n, li_wn_n = [], [], [], []
    launches = 0
    peaks = measured_peaks()

    def timed_step():
        flush.zero_()  # L2 flush, outside the event pair
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n = step()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), n

    with ClockSampler(torch.cuda.current_device()) as clocks:
        # headline: the whole step as a user runs it (variants overlapped on two
        # streams unless --no-overlap)
        barrier()
        t_wall0 = time.perf_counter()
        for _ in range(args.steps):
            ms, n = timed_step()
            step_ms.append(ms)
            launches += n
        barrier()
        t_wall = time.perf_counter() - t_wall0
        # per-kernel times for the rooflines: steps with the variants one after
        # the other, so that no kernel shares the GPU with another
        ctx.set_option(ub.OPT_OVERLAP_VARIANTS, 0)
        step()
        for _ in range(max(1, min(args.steps, args.serial_steps))):
            ms, _n = timed_step()
            serial_ms.append(ms)
            pair_uw_ms.append(ctx.stat(ub.STAT_PAIR_MS_UNWEIGHTED))
            pair_wn_ms.append(ctx.stat(ub.STAT_PAIR_MS_WEIGHTED))
            sel_wn.append(ctx.stat(ub.STAT_SELECTED_WEIGHTED))
            sel_uw.append(ctx.stat(ub.STAT_SELECTED_UNWEIGHTED))
            sp_uw_ms.append(ctx.stat(ub.STAT_SPARSE_MS_UNWEIGHTED))
            sp_wn_ms.append(ctx.stat(ub.STAT_SPARSE_MS_WEIGHTED))
            sp_uw_n.append(ctx.stat(ub.STAT_SPARSE_UPDATES_UNWEIGHTED))
            sp_wn_n.append(ctx.stat(ub.STAT_SPARSE_UPDATES_WEIGHTED))
            li_uw_ms.append(ctx.stat(ub.STAT_LIST_MS_UNWEIGHTED))
            li_wn_ms.append(ctx.stat(ub.STAT_LIST_MS_WEIGHTED))
            li_uw_n.append(ctx.stat(ub.STAT_LIST_UPDATES_UNWEIGHTED))
            li_wn_n.append(ctx.stat(ub.STAT_LIST_UPDATES_WEIGHTED))
        ctx.set_option(ub.OPT_OVERLAP_VARIANTS, 0 if args.no_overlap else 1)
    clk = clocks.summary()
    dev_err = ctx.stat(ub.STAT_DEVICE_ERROR)
    total_ms, units_all = replicas.reduce_timing(float(sum(step_ms)), units_per_step * args.steps,
                                                 dist, device="cuda")
    ms_per_step = total_ms / args.steps
    value = units_all / (total_ms / 1e3)

    # live per-kernel times (CUDA events recorded by the library on its
    # stream) and the algorithmic work of each launch, against measured pipe
    # rates: the FP32 FMA rate for the CUDA-core kernels (one FP32 operation
    # per lane and cycle), the cuBLAS BF16 rate for the tensor-core kernel
    fp32_rate, fp64_rate = pipe_peaks()
    alu_peak = fp32_rate / 1e12
    alu_src = ("measured FP32 FMA issue rate (unifrac_measure_peak: full-occupancy FFMA chains, "
               "CUDA events)")
    long_step = ms_per_step >= 100.0
    tc_peak = (peaks or {}).get("bf16_tflops_sustained" if long_step else "bf16_tflops",
                                1401.4 if long_step else 1791.5)
    tc_src = ("measured cuBLAS bf16 " + ("sustained (kernel timed inside a step of "
                                         f"{ms_per_step:.0f} ms)" if long_step else "burst")
              + " (MEASURED_PEAKS.json)")
    sm_max = (peaks or {}).get("sm_max_mhz", 2032.0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mean = lambda xs: float(np.mean(xs)) if xs else 0.0
    uw_ms, wn_ms = mean(pair_uw_ms), mean(pair_wn_ms)
    kernels = []
    thresholds_now = {"sparse": ctx.get_option(ub.OPT_SPARSE_THRESHOLD),
                      "uw_sparse": ctx.get_option(ub.OPT_UNWEIGHTED_SPARSE_THRESHOLD)}

    def entry(kernel, ms, work, bound, peak, unit, work_note, peak_note, **extra):
        if ms <= 0:
            return
        ach = work / (ms / 1e3) / 1e12
        kernels.append({"kernel": kernel, "ms": ms, "bound": bound, "achieved": ach,
                        "peak": peak, "unit": unit, "frac": ach / peak,
                        "traffic": recorded_traffic(kernel, w.name, N, thresholds_now),
                        "work": work_note, "peak_source": peak_note, **extra})

    entry("k_pairs_tc", uw_ms - mean(sp_uw_ms) - mean(li_uw_ms), 6.0 * mean(sel_uw), "tensor",
          tc_peak, "TFLOP/s",
          "3 BF16 digit planes x 2 flops per selected pair-branch (64-branch K-tiles)", tc_src)
    # the shared-memory atomic unit (one 32-lane wavefront per cycle per SM):
    # a secondary ceiling of the sparse kernels' implementation
    atom = sms * 32 * sm_max * 1e6
    entry("k_pairs_sparse<true>", mean(sp_uw_ms), mean(sp_uw_n), "alu", alu_peak, "T ops/s",
          "1 add of len_b per co-present pair-branch (the unweighted update)", alu_src,
          smem_atomic_frac=(2.0 * mean(sp_uw_n) / (mean(sp_uw_ms) / 1e3) / atom
                            if mean(sp_uw_ms) > 0 else None))
    entry("k_pairs_weighted<float>", wn_ms - mean(sp_wn_ms) - mean(li_wn_ms), 2.0 * mean(sel_wn),
          "alu", alu_peak,
          "T ops/s", "2 FP32 ops (min, add) per selected pair-branch", alu_src)
    entry("k_pairs_sparse<false>", mean(sp_wn_ms), 2.0 * mean(sp_wn_n), "alu", alu_peak,
          "T ops/s", "2 ops (min, add) per co-present pair-branch (the weighted update)", alu_src,
          smem_atomic_frac=(mean(sp_wn_n) / (mean(sp_wn_ms) / 1e3) / atom
                            if mean(sp_wn_ms) > 0 else None))
    # per-branch lists of the very rarely present branches: each pair update is
    # a read-modify-write of one partial sum in device memory (4 bytes each
    # way weighted, 8 unweighted), the branches' entries read once besides
    hbm = (peaks or {}).get("hbm_gbs") or 6400.0
    for kern, ms_l, n_l, b_upd in (("k_pairs_list<true>", mean(li_uw_ms), mean(li_uw_n), 16.0),
                                   ("k_pairs_list<false>", mean(li_wn_ms), mean(li_wn_n), 8.0)):
        entry(kern, ms_l, n_l * b_upd * 1e3, "hbm", hbm, "GB/s",  # entry() divides by 1e12
              f"{b_upd:g} bytes per co-present pair-branch update (a read and a write of one "
              "partial sum, global atomics)", "measured copy bandwidth (MEASURED_PEAKS.json)")
    roofline = max(kernels, key=lambda k: k["ms"])
    layout_name = "full" if layout == ub.OUT_FULL else "condensed"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "strong" if (world > 1 and not batched) else "weak",
        "vs_baseline": None,
        "dtype": "f32+bf16(int digits), integer sums", "data": "synthetic",
        "config": {"workload": args.workload if args.samples is None
                   else f"{args.workload} truncated to {N} samples", "samples": N,
                   "studies": 1 if not batched else int(len(w.table.study_offsets) - 1),
                   "branches_kept": ctx.stat(ub.STAT_BRANCHES_KEPT),
                   "levels": ctx.stat(ub.STAT_LEVELS), "layout": layout_name,
                   "output_bytes": 2 * nb_out,
                   "stripes": ("all stripes in one call (the device holds the whole matrix)"
                               if s1 < 0 else f"stripes [{s0}, {s1}) of this rank"),
                   "parallelism": (f"studies sharded over {world} GPUs" if batched and world > 1
                                   else f"stripe ranges over {world} GPUs" if world > 1
                                   else "1 GPU"),
                   "l2": "flushed (512 MB write) before every timed step; inputs and outputs "
                         "are far larger than L2",
                   "description": w.description},
        "roofline": roofline,
        "kernels": kernels,
        "gpu_launches": int(launches),
        "clocks": clk,
        "breakdown_ms": {"serial_step": mean(serial_ms), "pair_unweighted": uw_ms,
                         "pair_weighted": wn_ms,
                         "embedding_packing_other": mean(serial_ms) - uw_ms - wn_ms,
                         "note": "per-kernel and breakdown times from a second timed loop "
                                 "with the variants one after the other (no kernel shares "
                                 "the GPU); ms_per_step is the headline loop, variants "
                                 "overlapped on two streams" if not args.no_overlap else
                                 "variants one after the other in both loops"},
        "measured_pipes": {"fp32_fma_tops": fp32_rate / 1e12, "fp64_fma_tops": fp64_rate / 1e12,
                           "sm_mhz_median": clk.get("sm_mhz")},
        "tuned_options": tuned, "graph_replay": not args.no_graph,
        "persistent_work_queue": not args.no_persistent,
        "useful_fraction": ctx.stat(ub.STAT_USEFUL) / max(pair_branch, 1.0),
        "device_gb_held": round(ctx.stat(ub.STAT_DEVICE_BYTES) / 1e9, 2),
        "wall_s_timed_loop": t_wall,
        "device_error": dev_err,
    }

    if rank == 0 and not args.no_cpu_baseline:
        s_idx, sub, block0 = baseline_study(w)
        ws = synth.Workload(w.name, w.tree, sub, w.description)
        Ns = sub.n_samples
        rng = np.random.default_rng(7)
        rows = np.sort(rng.choice(Ns, size=min(args.cpu_rows, Ns), replace=False))
        ref, dt, threads = oracle_sample(ws, rows)
        B = kept_branches(ws)
        units = 2.0 * len(rows) * (Ns - 1) * B
        line["cpu_baseline"] = {"value": units / dt, "unit": UNIT, "cores": threads,
                                "kind": "oracle",
                                "sample": f"{len(rows)} seeded rows x {Ns} columns of study "
                                          f"{s_idx}, both variants ({dt:.1f} s)"}
        if not batched and s1 < 0:
            # error of this run's outputs on the same rows
            line["max_abs_err_vs_oracle"] = {
                name: float(np.max(np.abs(row_values(out_both, v, layout_name, N, rows)
                                          - ref[v])))
                for name, v in (("unweighted", 0), ("weighted_normalized", 1))}

    # the device memory of the timed context is released before the FP64,
    # end-to-end and downstream legs create contexts of their own
    tuned_opts = {o: ctx.get_option(o) for o in (ub.OPT_SPARSE_THRESHOLD,
                                                 ub.OPT_UNWEIGHTED_SPARSE_THRESHOLD,
                                                 ub.OPT_SPARSE_LANE_PAIRS,
                                                 ub.OPT_UNWEIGHTED_SPARSE_LANE_PAIRS,
                                                 ub.OPT_WEIGHTED_FLUSH, ub.OPT_RARE_LIST,
                                                 ub.OPT_UNWEIGHTED_RARE_LIST)}
    ctx.close()
    del out_both
    torch.cuda.empty_cache()

    if rank == 0 and not args.no_fp64 and not batched:
        try:
            f64 = fp64_leg(args, w, stream, flush, 2.0 * pair_branch)
            work = f64.pop("_work")
            km = f64["kernel_ms"]
            f64["mixed_speedup"] = f64["ms_per_step"] / ms_per_step
            f64_peak = fp64_rate / 1e12
            f64_src = ("measured FP64 FMA issue rate (unifrac_measure_peak: full-occupancy DFMA "
                       "chains, CUDA events)")
            for kern, ms_k, ops, note in (
                    ("k_pairs_lookup", km["k_pairs_lookup"], work["lookup_group_adds"],
                     "1 FP64 add of a table entry per pair and selected 8-branch group"),
                    ("k_pairs_weighted<double>", km["k_pairs_weighted<double>"],
                     2.0 * work["weighted_fp64_updates"],
                     "2 FP64 ops (min, add) per selected pair-branch")):
                if ms_k > 0:
                    ach = ops / (ms_k / 1e3) / 1e12
                    kernels.append({"kernel": kern, "ms": ms_k, "bound": "alu", "achieved": ach,
                                    "peak": f64_peak, "unit": "T ops/s", "frac": ach / f64_peak,
                                    "traffic": None, "work": note, "peak_source": f64_src,
                                    "timed": f"FP64 run over stripes {f64['stripes']}"})
            line["fp64_plain"] = f64
        except (ub.UniFracError, torch.OutOfMemoryError) as exc:
            line["fp64_plain"] = {"skipped": str(exc)}
            torch.cuda.empty_cache()
    nb_cond = None
    # end to end through the public API with host buffers
    if rank == 0 and not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        host_in = [pin(w.tree.parent), pin(w.tree.length), pin(w.table.feature_node),
                   pin(w.table.indptr), pin(w.table.indices), pin(w.table.counts)]
        h2d = int(sum(a.nbytes for a in host_in))
        res = torch.empty(2 * nb_out // 4, dtype=torch.float32).pin_memory().numpy()
        e2e_t, parts, create_parts = [], [], []
        for rep in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = ub.unifrac_create(*host_in, n_samples=N, stream=stream,
                                  study_offsets=w.table.study_offsets)
            for k_, v_ in tuned_opts.items():
                ub.unifrac_set_option(h, k_, v_)
            t1 = time.perf_counter()
            ub.unifrac_run(h, ub.BOTH, ub.MIXED, 0, -1, layout, res)
            t2 = time.perf_counter()
            # the create breakdown (host-side values, read outside the timing)
            create_parts.append((ub.unifrac_get_stat(h, ub.STAT_CREATE_HOST_MS),
                                 ub.unifrac_get_stat(h, ub.STAT_CREATE_DEVICE_MS)))
            t2b = time.perf_counter()
            ub.unifrac_destroy(h)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            e2e_t.append(t3 - t0 - (t2b - t2))
            parts.append((t1 - t0, t2 - t1, t3 - t2b))
        t_e2e = float(np.median(e2e_t))
        med = np.median(np.array(parts), axis=0)
        cmed = np.median(np.array(create_parts), axis=0)
        line["e2e"] = {"value": 2.0 * pair_branch / t_e2e, "unit": UNIT,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(2 * nb_out),
                       "s_per_step": t_e2e,
                       "s_create_run_destroy": [round(float(x), 5) for x in med],
                       "create_ms_host_device": [round(float(x), 2) for x in cmed],
                       "s_first_step": round(float(e2e_t[0]), 5),
                       "includes": f"create (validation, host prep, upload) + one run of both "
                                   f"variants into pinned host memory ({layout_name} layout, "
                                   f"D2H inside) + destroy; median of 3 steps, the later two "
                                   f"taking the device blocks the step before freed from the "
                                   f"library's block cache (s_first_step: the first, which "
                                   f"allocates them)"}

        # streamed output: both matrices into host memory, computed in chunks
        # of stripes (only two chunks on the device), copies and merge
        # overlapped; the chunk width is the faster of two candidates
        if not batched:
            nst = replicas.n_stripes(N)
            cands = ([args.streamed_chunk] if args.streamed_chunk > 0
                     else sorted({min(nst, 2048), min(nst, 4096), min(nst, 8192)}))
            with ub.Context(w.tree, w.table, stream=stream) as sctx:
                for k_, v_ in tuned_opts.items():
                    sctx.set_option(k_, v_)
                # warm-up with the widest chunk: its buffers serve every candidate
                sctx.run_streamed(ub.BOTH, ub.MIXED, layout, cands[-1], out=res)
                trial = {}
                for c_ in cands:
                    t0 = time.perf_counter()
                    sctx.run_streamed(ub.BOTH, ub.MIXED, layout, c_, out=res)
                    trial[c_] = time.perf_counter() - t0
                chunk = min(trial, key=trial.get)
                ts_ = []
                for rep in range(2):
                    t0 = time.perf_counter()
                    sctx.run_streamed(ub.BOTH, ub.MIXED, layout, chunk, out=res)
                    ts_.append(time.perf_counter() - t0)
            t_s = float(np.median(ts_))
            line["streamed"] = {"value": 2.0 * pair_branch / t_s, "unit": UNIT, "s_per_call": t_s,
                                "chunk_stripes": chunk, "chunks": -(-nst // chunk),
                                "candidates_s": {str(k_): round(v_, 4) for k_, v_ in trial.items()},
                                "includes": f"both variants into host memory ({layout_name}), "
                                            "stripes computed chunk by chunk, D2H and host merge "
                                            "overlapped with the next chunk"}
        del res
        # the freed contexts' blocks back to the driver before the framework
        # allocations of the legs below
        ub.unifrac_release_cached_memory(-1)

    # PCoA of the weighted matrix (full layout, FP32) on the device: the
    # ordination the distance matrix feeds
    if rank == 0 and not args.no_e2e and not batched:
        k_pc, it_pc = 10, 12
        with ub.Context(w.tree, w.table, stream=stream) as pctx:
            for k_, v_ in tuned_opts.items():
                pctx.set_option(k_, v_)
            Dfull = pctx.run(ub.WEIGHTED_NORMALIZED, ub.MIXED, ub.OUT_FULL)
            torch.cuda.synchronize()
        ub.unifrac_pcoa(Dfull, k=k_pc, iters=it_pc, seed=1)  # warm-up
        tp_ = []
        for rep in range(3):
            t0 = time.perf_counter()
            lam_pc, _ = ub.unifrac_pcoa(Dfull, k=k_pc, iters=it_pc, seed=1)
            tp_.append(time.perf_counter() - t0)
        t_p = float(np.median(tp_))
        # device traffic: D read and A written once, A read once per product
        dev_bytes = (2 + it_pc + 1) * 4.0 * N * N
        line["pcoa"] = {"s_per_call": t_p, "n": N, "k": k_pc, "iters": it_pc,
                        "eigenvalues_top3": [float(x) for x in lam_pc[:3]],
                        "device_stream_gbs": dev_bytes / t_p / 1e9,
                        "includes": "A = -1/2 D o D on the device, subspace iteration (products "
                                    "with A and the orthonormalisation on the device), wall time "
                                    "of the synchronous call"}
        del Dfull
        torch.cuda.empty_cache()

    # Mantel test, Pearson and Spearman, between the unweighted and weighted
    # matrices of this workload
    if rank == 0 and not args.no_e2e and not batched and args.mantel_perms > 0:
        line["mantel"] = mantel_leg(args, w, stream, tuned_opts, peaks)
        torch.cuda.empty_cache()

    if rank == 0 and batched and not args.no_per_study:
        # the same studies with one context and one launch sequence per study,
        # one study at a time (device memory), each run timed with events
        per = 0.0
        for s_ in range(len(w.table.study_offsets) - 1):
            t_ = study_table(w.table, s_)
            if t_.n_samples < 2:
                continue
            with ub.Context(w.tree, t_, stream=stream) as c:
                if not args.no_autotune:
                    from paper_2107_05397_b300 import autotune
                    for v in (ub.UNWEIGHTED, ub.WEIGHTED_NORMALIZED):
                        autotune.tune(c, v, ub.MIXED, repeats=args.tune_repeats)
                o_ = torch.empty(2 * c.output_bytes(ub.MIXED, layout) // 4, device="cuda")
                c.run(ub.BOTH, ub.MIXED, layout, out=o_)
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                c.run(ub.BOTH, ub.MIXED, layout, out=o_)
                e1.record(stream)
                e1.synchronize()
                per += e0.elapsed_time(e1)
                del o_
        line["one_launch_sequence_per_study"] = {
            "ms_per_step": per, "value": units_per_step / (per / 1e3),
            "batched_speedup": per / ms_per_step,
            "note": "sum of per-study runs (each its own context, tuned, warm)"}

    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
