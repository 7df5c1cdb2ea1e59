#!/usr/bin/env python
"""Benchmark of the center-star MSA hot path on one GB300 (or N, one process
each, independent sequence sets = weak scaling).

A step is one pass of the whole path over the 10,000-protein batched uneven
workload (lognormal lengths, median 350, sigma 0.6, clipped 50-2000, 5
families, BLOSUM62, gap 11/1): encode, exact center (all pairs), alignment of
every sequence to the center with traceback, merge of the inserted spaces,
MSA rows, sum-of-pairs cost.  Metric: GCUPS = DP cells of the step (center
selection + alignment, real cells only) / step time.

`value` times the step with inputs already in HBM (letters as a device
buffer, outputs left in HBM); `e2e` times the same step through the C ABI
with pinned host letters in and the MSA rows copied back to host memory.
L2 is flushed (a 512 MB write) before every timed step, outside its events.

--impl reference times the CPU oracle (plain C, all host cores) on bounded
samples of the same workload's pairs, the same metric and unit.
"""
import argparse
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

WORKLOAD = "batched_uneven_10k"
METRIC = "GCUPS and % of integer/DPX roofline; end-to-end MSA sec (learned vs exact center)"
UNIT = "GCUPS"
# ALU roofline of the packed DP: 152 SMs x 64 integer (DPX) lanes per clock x
# 2.07 GHz maximum SM clock / 3 integer instructions per cell (the Gotoh
# update is 6 DPX instructions per packed pair of int16 cells).  64 lanes per
# SM per clock is the issue rate msa_probe_int_rate measures for the DPX
# instructions on GB300 (half the 128 FP32 lanes).
SMS, INT_LANES, MAX_GHZ, OPS_PER_CELL = 152, 64, 2.07, 3.0
ALU_PEAK_GCUPS = SMS * INT_LANES * MAX_GHZ / OPS_PER_CELL
# Alignment with traceback codes: the same 3 DPX instructions per cell plus 4
# two-operand integer instructions for the 4-bit code (two source flags, two
# gap-extension flags), which issue at twice the DPX rate (128 lanes per clock
# per SM): 3 x 2 + 4 = 10 lane-slots per cell at 128 lanes per clock per SM.
CODES_SLOTS_PER_CELL = 3 * 2 + 4
CODES_PEAK_GCUPS = SMS * 2 * INT_LANES * MAX_GHZ / CODES_SLOTS_PER_CELL
CODES_BYTES_PER_CELL = 0.5   # 4-bit traceback code per cell written to HBM
# DRAM bytes read + written per cell by the codes kernel, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum = 10.6 + 528.5 MB for 1.007e9
# cells of 20,000 peptides against the 500-residue center, 8-lane groups); the
# traffic grows with the cells, so a launch's traffic is this times its cells
CODES_TRAFFIC_PER_CELL = (10.6e6 + 528.5e6) / 1.006925e9
ALIGN_WORKLOAD, ALIGN_N = "short_peptides_1m", 200_000
# distance kernel of the tree: 9 integer instructions per 32-bit word of both
# rows (4 columns: xor, nonzero test, residue mask, two counter updates)
TREE_PEAK_TCPS = 152 * 128 * 2.07e9 / (9 / 4) / 1e12
# the library's center kernel variants, in msa_autotune's column order:
# (two queries per int16x2 register?, lanes per group, query rows per lane, packed)
CENTER_VARIANTS = [(1, 8, 12, 1), (1, 8, 20, 1), (1, 8, 28, 1), (1, 16, 12, 1), (1, 16, 20, 1),
                   (1, 16, 28, 1), (1, 32, 12, 1), (1, 32, 20, 1), (1, 32, 28, 1), (0, 32, 16, 1),
                   (0, 32, 24, 1), (0, 8, 16, 0), (0, 16, 16, 0), (0, 32, 16, 0)]
BUCKET_EDGES = [1, 48, 80, 112, 144, 176, 208, 256, 320, 384, 448, 512, 640, 768, 896, 1024, 1280,
                1536, 2048, 3072, 4096, 8193]


def tuner_choices(rates):
    """Per timed length bucket: the fastest center variant and its rate."""
    out = {}
    for bk in range(rates.shape[0]):
        if not (rates[bk] > 0).any():
            continue
        v = int(np.argmax(rates[bk]))
        paired, G, R, packed = CENTER_VARIANTS[v]
        out["%d-%d" % (BUCKET_EDGES[bk], BUCKET_EDGES[bk + 1] - 1)] = {
            "variant": "%s G%d R%d %s" % ("query pair" if paired else "single query", G, R,
                                          "int16x2" if packed else "int32"),
            "gcups": float(rates[bk, v]) / 1e9}
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--n", type=int, default=None, help="override the sequence count")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--length", default=None,
                    help="override lengths, e.g. uniform:340:360 (profiling cases)")
    ap.add_argument("--only-center", action="store_true",
                    help="time the exact-center selection alone (profiling cases)")
    ap.add_argument("--align-group", type=int, default=0,
                    help="lanes per subject group of the alignment kernels (0 = modelled)")
    ap.add_argument("--only-align", action="store_true",
                    help="time the alignment to one center alone (profiling cases): the "
                         "workload's own center if it has one, else the median-length sequence")
    ap.add_argument("--only-embed", action="store_true",
                    help="time the selector's embedding of every sequence alone, random "
                         "network (profiling cases)")
    ap.add_argument("--only-train", action="store_true",
                    help="time selector training steps alone (256 pairs per step; profiling cases)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-center comparison")
    ap.add_argument("--center", default="exact", choices=["exact", "sampled", "first"],
                    help="exact all-pairs center, the sampled exact center over 1,000 "
                         "seeded references (the larger workloads), or the first sequence "
                         "(the paper's center for similar nucleotides)")
    ap.add_argument("--anchored", type=int, default=0, metavar="K",
                    help="with --only-align: time the anchored path for similar sequences "
                         "(K-residue center segments) beside the Smith-Waterman path")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuners (center variants per length bucket; alignment "
                         "group width and int16x2 / int32 cells) and use the cost models")
    ap.add_argument("--align-mode", default="full", choices=["full", "box", "both"],
                    help="with --only-align: the full alignment (codes of every cell), the "
                         "traceback-light one (score pass, reverse pass, codes of each box), "
                         "or both, checked equal")
    ap.add_argument("--align-threads", type=int, default=0,
                    help="threads per CTA of the packed alignment kernel (256 or 384)")
    ap.add_argument("--only-tree", action="store_true",
                    help="time the neighbour-joining tree of the workload's MSA only")
    ap.add_argument("--tree-sample", type=float, default=0.0,
                    help="with --only-tree: the clustered tree over a seeded sample of this "
                         "fraction of the rows (else one NJ over all rows)")
    ap.add_argument("--tree-cap", type=int, default=0,
                    help="with --tree-sample: sample rows per cluster at most (default: a "
                         "tenth of the sample)")
    ap.add_argument("--no-tree-record", action="store_true",
                    help="skip the neighbour-joining tree of the step's MSA")
    ap.add_argument("--no-align-record", action="store_true",
                    help="skip the alignment-kernel record (peptides against their 500-residue "
                         "ancestor)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    """The generated peaks of the GB300s (empty if absent)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(letters, offsets, alph, M, o, e, seconds, seed=7):
    """The oracle, as it stands, on random pairs of the workload for ~`seconds`."""
    import oracle
    prob = oracle.Problem(letters, offsets, alph, M, o, e)
    lens = np.diff(offsets).astype(np.int64)
    rng = np.random.default_rng(seed)
    threads = oracle.default_threads()
    probe = rng.integers(0, prob.n, size=(max(64, threads * 8), 2))
    t0 = time.perf_counter()
    oracle.pair_scores(prob, probe, threads)
    dt = time.perf_counter() - t0
    rate = float((lens[probe[:, 0]] * lens[probe[:, 1]]).sum()) / max(dt, 1e-6)
    count = int(max(threads, min(2_000_000, rate * seconds / float((lens ** 2).mean()))))
    pairs = rng.integers(0, prob.n, size=(count, 2))
    cells = float((lens[pairs[:, 0]] * lens[pairs[:, 1]]).sum())
    t0 = time.perf_counter()
    oracle.pair_scores(prob, pairs, threads)
    dt = time.perf_counter() - t0
    return {"value": cells / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d uniformly drawn pairs of the %d-sequence set (%.3g DP cells), "
                      "scalar C full-matrix Gotoh, %.1f s" % (count, prob.n, cells, dt)}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    from seqgen import generate, scoring
    letters, offsets, w, _ = generate(args.workload, n=args.n)
    alph, M, _, _ = scoring(w.kind)
    prob = oracle.Problem(letters, offsets, alph, M, w.gap_open, w.gap_extend)
    lens = np.diff(offsets).astype(np.int64)
    threads = oracle.default_threads()
    rng = np.random.default_rng(11)
    # size one step at a few seconds of CPU work
    probe = rng.integers(0, prob.n, size=(threads * 8, 2))
    t0 = time.perf_counter()
    oracle.pair_scores(prob, probe, threads)
    rate = float((lens[probe[:, 0]] * lens[probe[:, 1]]).sum()) / max(time.perf_counter() - t0, 1e-6)
    per_step = int(max(threads, rate * 4.0 / float((lens ** 2).mean())))
    times, cells_all = [], []
    for s in range(args.warmup + args.steps):
        pairs = rng.integers(0, prob.n, size=(per_step, 2))
        cells = float((lens[pairs[:, 0]] * lens[pairs[:, 1]]).sum())
        t0 = time.perf_counter()
        oracle.pair_scores(prob, pairs, threads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            cells_all.append(cells)
    value = sum(cells_all) / sum(times) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "%s: %d proteins, lognormal lengths median 350 sigma 0.6 "
                                   "clipped 50-2000, 5 families, BLOSUM62 11/1" % (w.name, prob.n),
                       "step": "oracle pair scores on %d random pairs of the set" % per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d random pairs per step (%.3g cells)" %
                                       (per_step, float(np.mean(cells_all)))},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_text(w, n, center, length=None):
    """The workload of a bench line, from its generator parameters."""
    ln = length or w.length
    if ln[0] == "lognormal":
        lens = "lognormal lengths median %d sigma %.1f clipped %d-%d" % ln[1:]
    else:
        lens = "lengths uniform %d-%d" % ln[1:]
    kind = "proteins (BLOSUM62)" if w.kind == "protein" else "DNA sequences (+2/-3)"
    return ("%s: %d %s per GPU, %s, %d families at %.0f%% substitutions, %.1f%% indels, gap "
            "open %d / extend %d, %s center" % (w.name, n, kind, lens, w.families, 100 * w.p_sub,
                                                100 * w.p_indel, w.gap_open, w.gap_extend,
                                                "the named ancestor as" if w.center_seq else
                                                "exact all-pairs" if center == "exact"
                                                else "sampled exact (1,000 references)"))


def time_alignment(b, h, center, mode, flush, stream, n, reps=3):
    """msa_align_to_center in one mode (MSA_ALIGN_FULL / MSA_ALIGN_BOX), L2
    flushed before each of `reps` timed calls: the call (CUDA events on the
    context stream, host round trips included), the kernels' own time from the
    library's stage events, and for the box mode its passes and the cells its
    codes covered."""
    import torch
    b.msa_set_align_mode(h, mode)
    for _ in range(2):
        b.msa_align_to_center(h, center)
    call, kern, tb, passes = [], [], [], {"light_score": [], "light_corner": [], "light_box": []}
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        b.msa_align_to_center(h, center)
        ev1.record(stream)
        torch.cuda.synchronize()
        call.append(ev0.elapsed_time(ev1))
        ms, cnt = b.msa_stage_times(h)
        kern.append(ms["align_kernels"])
        tb.append(ms["traceback"])
        for k in passes:
            passes[k].append(ms[k])
    cells = cnt["align_cells"]
    k = float(np.mean(kern))
    rec = {"kernel_ms": k, "traceback_ms": float(np.mean(tb)), "call_ms": float(np.mean(call)),
           "cells": cells, "gcups": cells / (k * 1e-3) / 1e9}
    seg = b.msa_alignment_info(h)[0]
    if mode == b.MSA_ALIGN_BOX:
        boxes = b.msa_align_boxes(h, n)
        box_cells = int(((boxes[:, 2] - boxes[:, 0]).astype(np.int64) *
                         (boxes[:, 3] - boxes[:, 1])).sum())
        rec.update({"pass_ms": {k2[6:]: float(np.mean(v)) for k2, v in passes.items()},
                    "box_cells": box_cells, "box_fraction": box_cells / cells,
                    "code_bytes": box_cells * CODES_BYTES_PER_CELL})
    else:
        rec["code_bytes"] = cells * CODES_BYTES_PER_CELL
    b.msa_set_align_mode(h, b.MSA_ALIGN_FULL)
    return rec, seg


def align_record(flush, stream, peak_gbs, no_tune=False):
    """The alignment to the center with traceback codes (the batched DP), on
    its own: 200,000 short peptides (the 1e6-peptide workload's generator and
    lengths) against their 500-residue common ancestor, the center the
    workload names.  Inputs in HBM, L2 flushed before each timed call; CUDA
    events around msa_align_to_center on the context stream, and the codes
    kernels' own time from the library's stage events."""
    import torch
    from seqgen import generate, scoring
    from paper_1704_00878_gb300 import binding as b
    letters, offsets, w, _ = generate(ALIGN_WORKLOAD, n=ALIGN_N)
    alph, M, _, _ = scoring(w.kind)
    lens = np.diff(offsets)
    dlet = torch.from_numpy(letters).cuda()
    with b.Context(M, alph, w.gap_open, w.gap_extend, stream=stream) as h:
        b.msa_load(h, dlet, offsets)
        tune = None if no_tune else b.msa_align_autotune(h, 0)
        for _ in range(2):
            b.msa_align_to_center(h, 0)
        call_ms, kern_ms, tb_ms = [], [], []
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            b.msa_align_to_center(h, 0)
            ev1.record(stream)
            torch.cuda.synchronize()
            call_ms.append(ev0.elapsed_time(ev1))
            ms, cnt = b.msa_stage_times(h)
            kern_ms.append(ms["align_kernels"])
            tb_ms.append(ms["traceback"])
        cells = cnt["align_cells"]
        full_seg = b.msa_alignment_info(h)[0]
        light, light_seg = time_alignment(b, h, 0, b.MSA_ALIGN_BOX, flush, stream, ALIGN_N)
    k = float(np.mean(kern_ms))
    gcups = cells / (k * 1e-3) / 1e9
    light.update(same_as_full=bool((light_seg == full_seg).all()),
                 kernel_vs_full=light["kernel_ms"] / k,
                 note="traceback-light: score pass to the best cell, reverse pass to the corner, "
                      "codes of each segment's box only; gcups over the full matrices' cells")
    tuned = None
    if tune is not None:
        rates, (lanes, packed, cta) = tune
        tuned = {"choice": {"lanes": lanes, "cells": "int16x2" if packed else "int32",
                            "threads": cta},
                 "gcups": {"%s_G%d" % (p, G): float(rates[i, g]) / 1e9
                           for i, p in enumerate(("int16x2", "int32", "int16x2_t384"))
                           for g, G in enumerate(b.ALIGN_LANES)
                           if rates[i, g] > 0}}
    return {"autotune": tuned, "workload": "%d short peptides (lognormal lengths median 90 sigma 0.6 clipped 30-200, "
                        "one family at 30%% substitutions, 3%% indels) against their %d-residue "
                        "ancestor, BLOSUM62 11/1, packed int16x2 cells" % (ALIGN_N - 1, lens[0]),
            "cells": cells, "kernel_ms": k, "traceback_ms": float(np.mean(tb_ms)),
            "call_ms": float(np.mean(call_ms)), "gcups": gcups, "light": light,
            "gcups_with_traceback": cells / (float(np.mean(call_ms)) * 1e-3) / 1e9,
            "roofline": {"bound": "alu", "kernel": "k_codes2 (Gotoh fill + 4-bit traceback codes, "
                                                  "two subjects per int16x2 register)",
                         "achieved": gcups, "peak": CODES_PEAK_GCUPS, "unit": UNIT,
                         "frac": gcups / CODES_PEAK_GCUPS,
                         "traffic": cells * CODES_TRAFFIC_PER_CELL,
                         "traffic_note": "bytes per launch, the ncu per-cell DRAM traffic of "
                                         "20,000 peptides scaled to this launch's cells",
                         "peak_source": "152 SMs x 128 integer lanes/clk x 2.07 GHz / (3 DPX "
                                        "instructions at half rate + 4 two-operand ops) per cell",
                         "hbm_bound_gcups": peak_gbs / CODES_BYTES_PER_CELL,
                         "hbm_gbs_of_codes": gcups * CODES_BYTES_PER_CELL}}


def tree_record(b, h, n, W, stream, peak_gbs, cpu_n=600):
    """The neighbour-joining tree of the step's MSA (already merged on the
    device): the distance kernel (column pairs per second against its integer
    issue bound) and the joins (bytes of the matrix the Q minimum reads, per
    second), CUDA events on the context stream; the oracle's NJ on the first
    `cpu_n` rows' distances beside it."""
    import torch
    from oracle import nj as T
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    d = torch.empty((n, n), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    ev[0].record(stream)
    b.msa_tree_distances(h, d)
    ev[1].record(stream)
    joins, lengths = b.msa_nj(h, d)
    ev[2].record(stream)
    torch.cuda.synchronize()
    dist_ms, nj_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    col_pairs = n * (n + 1) / 2 * W  # tiles on and above the diagonal
    # matrix bytes the Q minimum reads: the active pairs of every join
    nj_bytes = sum(m * (m - 1) / 2 for m in range(3, n + 1)) * 8
    sub = d[:cpu_n, :cpu_n].cpu().numpy()
    t0 = time.perf_counter()
    T.nj(sub)
    cpu_s = time.perf_counter() - t0
    return {"workload": "NJ tree of the step's %d-row MSA (%d columns), fixed-point p-distances"
                        % (n, W),
            "distances_ms": dist_ms, "nj_ms": nj_ms, "joins": int(len(joins)),
            "column_pairs_per_s": col_pairs / (dist_ms * 1e-3),
            "distances_roofline": {"bound": "alu", "kernel": "k_pdist",
                                   "achieved": col_pairs / (dist_ms * 1e-3) / 1e12,
                                   "peak": TREE_PEAK_TCPS, "unit": "T column pairs/s",
                                   "frac": col_pairs / (dist_ms * 1e-3) / 1e12 / TREE_PEAK_TCPS,
                                   "peak_source": "152 SMs x 128 integer lanes/clk x 2.07 GHz / "
                                                  "9 instructions per 4 column pairs"},
            "nj_matrix_gbs": nj_bytes / (nj_ms * 1e-3) / 1e9, "hbm_peak_gbs": peak_gbs,
            "cpu_oracle_nj": {"rows": int(sub.shape[0]), "seconds": cpu_s,
                              "kind": "oracle", "cores": 1}}


def learned_vs_exact(b, h, dlet, offsets, fam, n, flush, stream, exact_ms, exact_sp, refs,
                     exact_center, exact_rowsum):
    """Train the selector on exact-kernel distances (untimed), then time the
    whole step with the learned center (network embedding + exact row sums of
    its best candidates, over every sequence when the exact center is the
    all-pairs one, else over the same reference sample) against the exact
    center's step.  Also: where the network's own pick (top 1) and the
    methods without it (first sequence, shortest, longest, the best of as many
    random candidates refined the same way) rank among the exact row sums,
    and the avg SP of their MSAs."""
    import torch
    from seqgen import training_pairs
    pairs = training_pairs(n, 60000, fam, seed=8)
    t0 = time.perf_counter()
    b.msa_selector_init(h, seed=1)
    losses = b.msa_selector_train(h, pairs, steps=6000, batch_pairs=256, lr=3e-4, seed=3)
    train_s = time.perf_counter() - t0

    # candidates checked exactly: as many as ~2e10 DP cells of row sums
    # allow (short sequences: more of them), at least 128, at most 4096
    lens = np.diff(offsets).astype(np.float64)
    nj = n if refs is None else len(refs)
    cand = int(np.clip(2e10 / (nj * float(lens.mean()) ** 2), 128, 4096))

    def step_learned():
        b.msa_load(h, dlet, offsets)
        c, _ = b.msa_select_center_refined(h, candidates=cand, refs=refs)
        b.msa_align_to_center(h, c)
        b.msa_merge_gaps(h, want_rows=False)
        return c, b.msa_sp_score(h)

    step_learned()
    ms = []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        c, sp = step_learned()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    stages = b.msa_stage_times(h)[0]
    pairs_n = n * (n - 1) / 2

    def avg_sp_of(center):
        b.msa_align_to_center(h, int(center))
        b.msa_merge_gaps(h, want_rows=False)
        return b.msa_sp_score(h) / pairs_n

    top1, _ = b.msa_select_center(h, b.MSA_CENTER_LEARNED)
    rank = lambda i: 100.0 * float((exact_rowsum < exact_rowsum[int(i)]).mean())
    rng = np.random.default_rng(0)
    rand_rank = float(np.mean([100.0 * float((exact_rowsum < exact_rowsum[
        rng.choice(n, min(cand, n), replace=False)].min()).mean()) for _ in range(100)]))
    picks = {"exact": exact_center, "learned_refined": c, "learned_top1": top1, "first": 0,
             "shortest": int(np.argmin(lens)), "longest": int(np.argmax(lens))}
    compare = {name: {"center": int(i), "length": int(lens[int(i)]), "rowsum_rank_pct": rank(i),
                      "avg_sp": (sp / pairs_n if name == "learned_refined" else
                                 exact_sp / pairs_n if name == "exact" else avg_sp_of(i))}
               for name, i in picks.items()}
    # the same training from two more seeds (network, pair sample, batches):
    # the spread of what the learned center gives
    seeds = [{"seed": 1, "refined_rank_pct": rank(c), "top1_rank_pct": rank(top1),
              "sp_loss_pct": 100.0 * (sp - exact_sp) / exact_sp}]
    for sd in (2, 3):
        b.msa_selector_init(h, seed=sd)
        b.msa_selector_train(h, training_pairs(n, 60000, fam, seed=8 + sd), steps=6000,
                             batch_pairs=256, lr=3e-4, seed=3 + sd)
        c_s, _ = b.msa_select_center_refined(h, candidates=cand, refs=refs)
        t_s, _ = b.msa_select_center(h, b.MSA_CENTER_LEARNED)
        seeds.append({"seed": sd, "refined_rank_pct": rank(c_s), "top1_rank_pct": rank(t_s),
                      "sp_loss_pct": 100.0 * (avg_sp_of(c_s) * pairs_n - exact_sp) / exact_sp})
    spread = {k: [min(x[k] for x in seeds), max(x[k] for x in seeds)]
              for k in ("refined_rank_pct", "top1_rank_pct", "sp_loss_pct")}
    return {"exact_step_ms": exact_ms, "learned_step_ms": float(np.mean(ms)),
            "speedup": exact_ms / float(np.mean(ms)),
            "avg_sp_exact": exact_sp / pairs_n, "avg_sp_learned": sp / pairs_n,
            "sp_loss_pct": 100.0 * (sp - exact_sp) / exact_sp, "learned_center": c,
            "sp_loss_top1_pct": 100.0 * (compare["learned_top1"]["avg_sp"] * pairs_n - exact_sp)
                                / exact_sp,
            "compare": compare,
            "seeds": seeds, "spread_over_seeds": spread,
            "random_candidates_refined_mean_rank_pct": rand_rank,
            "selector": "4-layer conv, width 128, k 9, 64-d, bf16 on tcgen05 tensor cores",
            "train": {"pairs": int(pairs.shape[0]), "steps": 6000, "batch_pairs": 256,
                      "seconds": train_s, "loss_first": float(losses[:10].mean()),
                      "loss_last": float(losses[-50:].mean())},
            "candidates_refined_exactly": min(cand, n),
            "refined_over": "every sequence" if refs is None else "the %d references" % len(refs),
            "stages_ms": {k: round(stages[k], 3) for k in
                          ("encode", "selector", "center", "align_dp", "traceback", "merge", "sp")}}


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from seqgen import generate, scoring
    from paper_1704_00878_gb300 import binding as b

    # weak scaling: every rank aligns its own independent set of the same shape
    base_seed = generate.__globals__["WORKLOADS"][args.workload].seed
    length = None
    if args.length:
        kind, lo, hi = args.length.split(":")
        length = (kind, int(lo), int(hi))
    letters, offsets, w, fam = generate(args.workload, n=args.n, seed=base_seed + 1000 * rank,
                                        length=length)
    alph, M, _, _ = scoring(w.kind)
    n = offsets.size - 1
    stream = torch.cuda.current_stream()
    dlet = torch.from_numpy(letters).cuda()
    hlet = torch.from_numpy(letters).pin_memory()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ctx = b.Context(M, alph, w.gap_open, w.gap_extend, stream=stream)
    h = ctx.h

    from seqgen import reference_sample
    refs = reference_sample(n, 1000, 8) if args.center == "sampled" else None
    center_mode = b.MSA_CENTER_EXACT_SAMPLED if refs is not None else b.MSA_CENTER_EXACT

    def select_exact():
        if w.center_seq or args.center == "first":  # a named center, or the first sequence
            return 0, 0
        return b.msa_select_center(h, center_mode, refs)

    def step_device():
        b.msa_load(h, dlet, offsets)
        c, _ = select_exact()
        b.msa_align_to_center(h, c)
        _, W = b.msa_merge_gaps(h, want_rows=False)
        sp = b.msa_sp_score(h)
        return c, W, sp

    host_rows = {}

    def step_e2e():
        b.msa_load(h, hlet, offsets)
        c, _ = select_exact()
        b.msa_align_to_center(h, c)
        _, W = b.msa_merge_gaps(h, want_rows=False)
        buf = host_rows.get(W)
        if buf is None:
            host_rows.clear()
            buf = host_rows[W] = torch.empty((n, W), dtype=torch.uint8).pin_memory()
        b.msa_merge_gaps(h, out=buf)
        sp = b.msa_sp_score(h)
        return c, W, sp

    align_kern = [0.0, 0]  # codes kernels' ms and cells over the timed steps

    def timed(fn, steps):
        total_ms, cells, center_ms, center_cells, launches0 = 0.0, 0, 0.0, 0, None
        align_kern[:] = [0.0, 0]
        out = None
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            if launches0 is None:
                launches0 = b.msa_stage_times(h)[1]["launches"]
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            out = fn()
            ev1.record(stream)
            torch.cuda.synchronize()
            total_ms += ev0.elapsed_time(ev1)
            ms, cnt = b.msa_stage_times(h)
            cells += cnt["center_cells"] + cnt["align_cells"]
            center_ms += ms["center_kernels"]
            center_cells += cnt["center_cells"]
            align_kern[0] += ms["align_kernels"]
            align_kern[1] += cnt["align_cells"]
        launches = b.msa_stage_times(h)[1]["launches"] - launches0
        return total_ms, cells, center_ms, center_cells, launches, out

    if args.only_center:
        for _ in range(args.warmup):
            b.msa_load(h, dlet, offsets)
            b.msa_select_center(h, b.MSA_CENTER_EXACT)
        b.msa_load(h, dlet, offsets)
        t0 = time.perf_counter()
        c, _ = b.msa_select_center(h, b.MSA_CENTER_EXACT)
        dt = time.perf_counter() - t0
        ms, cnt = b.msa_stage_times(h)
        print(json.dumps({"only_center": True, "n": n, "center": c, "wall_s": dt,
                          "center_kernel_ms": ms["center_kernels"], "cells": cnt["center_cells"],
                          "gcups": cnt["center_cells"] / (ms["center_kernels"] * 1e-3) / 1e9}))
        ctx.close()
        return

    if args.align_group:
        b.msa_set_align_group(h, args.align_group)
    if args.align_threads:
        b.msa_set_align_threads(h, args.align_threads)
    if args.only_tree:
        lens = np.diff(offsets)
        center = 0 if (w.center_seq or args.center == "first") else \
            int(np.argsort(lens, kind="stable")[len(lens) // 2])
        b.msa_load(h, dlet, offsets)
        b.msa_align_to_center(h, center)
        _, Wt = b.msa_merge_gaps(h, want_rows=False)
        if args.tree_sample > 0:
            m = max(2, int(round(args.tree_sample * n)))
            sample = np.sort(np.random.default_rng(12).choice(n, m, replace=False))
            cap = args.tree_cap or max(1, m // 10)
            for _ in range(max(1, args.warmup)):
                t0 = time.perf_counter()
                joins, lengths, cluster = b.msa_nj_cluster_tree(h, sample, cap)
                wall = time.perf_counter() - t0
            sizes = np.bincount(cluster)
            print(json.dumps({"only_tree": True, "clustered": True, "n": n, "msa_width": Wt,
                              "sample": m, "cap": cap, "clusters": int(sizes.size),
                              "largest_cluster": int(sizes.max()), "seconds": wall,
                              "tree_stage_ms": b.msa_stage_times(h)[0]["tree"],
                              "joins": int(len(joins))}))
            ctx.close()
            return
        for _ in range(max(1, args.warmup)):
            rec = tree_record(b, h, n, Wt, stream, measured_peaks().get("hbm_gbs", 6800.0),
                              cpu_n=min(n, 300))
        print(json.dumps(dict(rec, only_tree=True)))
        ctx.close()
        return
    if args.only_align:
        lens = np.diff(offsets)
        center = 0 if (w.center_seq or args.center == "first") else \
            int(np.argsort(lens, kind="stable")[len(lens) // 2])
        b.msa_load(h, dlet, offsets)
        if args.anchored:
            # the anchored path against the Smith-Waterman path, same center: the
            # alignment alone, and the whole MSA (alignment + merged rows + SP)
            rows = {}

            def run(align_fn):
                out = {}
                for _ in range(max(1, args.warmup)):
                    align_fn()
                    _, W = b.msa_merge_gaps(h, want_rows=False)
                    if rows.get("W") != W:
                        rows.clear()
                        rows.update(W=W, buf=torch.empty((n, W), dtype=torch.uint8,
                                                         device="cuda"))
                t_al, t_msa = [], []
                for _ in range(3):
                    flush.zero_()
                    torch.cuda.synchronize()
                    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                    ev[0].record(stream)
                    r = align_fn()
                    ev[1].record(stream)
                    _, W = b.msa_merge_gaps(h, want_rows=False)
                    if rows["W"] != W:
                        raise SystemExit("alignment width changed between runs")
                    b.msa_merge_gaps(h, out=rows["buf"])
                    sp = b.msa_sp_score(h)
                    ev[2].record(stream)
                    torch.cuda.synchronize()
                    t_al.append(ev[0].elapsed_time(ev[1]))
                    t_msa.append(ev[0].elapsed_time(ev[2]))
                out.update(align_ms=float(np.median(t_al)), msa_ms=float(np.median(t_msa)),
                           msa_width=W, avg_sp=sp / (n * (n - 1) / 2))
                return r, out

            nf, rec_a = run(lambda: b.msa_align_anchored(h, center, args.anchored))
            _, rec_s = run(lambda: b.msa_align_to_center(h, center))
            print(json.dumps({"only_align": True, "n": n, "center": center,
                              "Lc": int(lens[center]), "k": args.anchored,
                              "residues": int(lens.sum()),
                              "full_matrix_cells": int(lens[center]) * int(lens.sum()),
                              "anchored": dict(rec_a, local_path_sequences=nf),
                              "smith_waterman": rec_s}))
            ctx.close()
            return
        if args.align_mode != "full":
            rec = {"only_align": True, "n": n, "center": center, "Lc": int(lens[center])}
            segs = {}
            for name, mode in (("full", b.MSA_ALIGN_FULL), ("box", b.MSA_ALIGN_BOX)):
                if args.align_mode in (name, "both"):
                    rec[name], segs[name] = time_alignment(b, h, center, mode, flush, stream, n)
            if len(segs) == 2:
                rec["same"] = bool((segs["full"] == segs["box"]).all())
                rec["box_kernel_vs_full"] = rec["box"]["kernel_ms"] / rec["full"]["kernel_ms"]
            print(json.dumps(rec))
            ctx.close()
            return
        for _ in range(max(1, args.warmup)):
            b.msa_align_to_center(h, center)
        ms, cnt = b.msa_stage_times(h)
        print(json.dumps({"only_align": True, "n": n, "center": center, "Lc": int(lens[center]),
                          "align_kernel_ms": ms["align_kernels"], "traceback_ms": ms["traceback"],
                          "cells": cnt["align_cells"],
                          "gcups": cnt["align_cells"] / (ms["align_kernels"] * 1e-3) / 1e9}))
        ctx.close()
        return
    if args.only_embed:
        lens = np.diff(offsets)
        b.msa_load(h, dlet, offsets)
        b.msa_selector_init(h, seed=1)
        for _ in range(max(1, args.warmup)):
            b.msa_select_center(h, b.MSA_CENTER_LEARNED)
        ms = b.msa_stage_times(h)[0]["selector"]
        # convolution flops: 2 x 9 taps x (32x128 + 128x128 + 128x128) per row,
        # and the output layer (128x64) on the nine window sums per sequence
        rows = int(lens.sum()) + 4 * (n + 1)
        flops = 2 * 9 * (32 * 128 + 2 * 128 * 128) * rows + 2 * 9 * 128 * 64 * 9 * n
        print(json.dumps({"only_embed": True, "n": n, "rows": rows, "selector_ms": ms,
                          "tflops": flops / (ms * 1e-3) / 1e12}))
        ctx.close()
        return

    if args.only_train:
        from seqgen import training_pairs
        lens = np.diff(offsets)
        b.msa_load(h, dlet, offsets)
        b.msa_selector_init(h, seed=1)
        pairs = training_pairs(n, 4096, fam, seed=3)
        targets = b.msa_selector_targets(h, pairs, scale=1e-3)
        steps = 20
        b.msa_selector_train(h, pairs, targets, steps=max(1, args.warmup), batch_pairs=256)
        b.msa_selector_train(h, pairs, targets, steps=steps, batch_pairs=256)
        ms = b.msa_stage_times(h)[0]["selector"] / steps
        # 512 sequences of the set's mean length (+ 4 zero rows each): forward
        # (output layer on nine window sums per sequence), data gradients of
        # layers 4-2, weight gradients of all four layers
        rows = 512 * (float(lens.mean()) + 4)
        fwd = 2 * 9 * (32 * 128 + 2 * 128 * 128) * rows + 2 * 9 * 128 * 64 * 9 * 512
        dgrad = 2 * 9 * (64 * 128 + 2 * 128 * 128) * rows
        wgrad = 2 * 9 * (32 * 128 + 2 * 128 * 128 + 128 * 64) * rows
        flops = fwd + dgrad + wgrad
        print(json.dumps({"only_train": True, "n": n, "ms_per_step": ms,
                          "tflops": flops / (ms * 1e-3) / 1e12}))
        ctx.close()
        return

    rate, per_clk = b.msa_probe_int_rate(b.MSA_PROBE_VIADDMAX_S16X2)
    b.msa_load(h, dlet, offsets)
    t0 = time.perf_counter()
    # untimed: the center kernel variant per length bucket, then (with the
    # center of a first step) the alignment's group width and cell precision
    tune = b.msa_autotune(h) if not args.no_autotune else np.zeros((0, 0))
    align_tune = None
    if not args.no_autotune:
        c0, _, _ = step_device()
        rates_a, (lanes_a, packed_a, cta_a) = b.msa_align_autotune(h, c0)
        align_tune = {"choice": {"lanes": lanes_a, "cells": "int16x2" if packed_a else "int32",
                                 "threads": cta_a},
                      "gcups": {"%s_G%d" % (p, G): float(rates_a[i, g]) / 1e9
                                for i, p in enumerate(("int16x2", "int32", "int16x2_t384"))
                                for g, G in enumerate(b.ALIGN_LANES)
                                if rates_a[i, g] > 0}}
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    total_ms, cells, center_ms, center_cells, launches, (c, W, sp) = timed(step_device, args.steps)
    clocks = sampler.stop()
    align_ms_t, align_cells_t = align_kern
    stage_ms = b.msa_stage_times(h)[0]
    # one untimed pass first: the pinned host buffer for the rows is allocated
    # (and reused) outside the timed steps, as the input buffer is
    step_e2e()
    torch.cuda.synchronize()
    e2e_ms, e2e_cells, *_ = timed(step_e2e, max(1, args.steps))

    def reduce_max(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    def reduce_sum(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t)
        return float(t.item())

    learned = None
    if not args.no_learned:
        b.msa_load(h, dlet, offsets)
        ex_c, _ = b.msa_select_center(h, center_mode, refs)
        ex_rows = b.msa_center_rowsums(h).astype(np.float64)
        ex_ms, ex_sp = total_ms / args.steps, sp
        if w.center_seq:  # the timed step used the named center: time the selecting one
            b.msa_align_to_center(h, ex_c)
            b.msa_merge_gaps(h, want_rows=False)
            ex_sp = b.msa_sp_score(h)
            ex_ms = b.msa_stage_times(h)[0]["center"] + (total_ms / args.steps)
        learned = learned_vs_exact(b, h, dlet, offsets, fam, n, flush, stream, ex_ms, ex_sp,
                                   refs, ex_c, ex_rows)
        if w.center_seq:
            learned["named_center_rowsum_rank_pct"] = 100.0 * float((ex_rows < ex_rows[0]).mean())
    tree = None
    if not args.no_tree_record and rank == 0:
        b.msa_load(h, dlet, offsets)
        b.msa_align_to_center(h, c)
        _, Wt = b.msa_merge_gaps(h, want_rows=False)
        if n <= 20000:  # one NJ over all rows (an n x n matrix)
            tree = tree_record(b, h, n, Wt, stream, measured_peaks().get("hbm_gbs", 6800.0))
        elif n <= 200000:  # the clustered tree over a 10 % sample
            m = n // 10
            sample = np.sort(np.random.default_rng(12).choice(n, m, replace=False))
            t0 = time.perf_counter()
            joins, _, cluster = b.msa_nj_cluster_tree(h, sample, max(1, m // 10))
            sizes = np.bincount(cluster)
            tree = {"workload": "clustered NJ tree of the step's %d-row MSA (%d columns): 10 %% "
                                "sample, at most %d sample rows per cluster" % (n, Wt, max(1, m // 10)),
                    "seconds": time.perf_counter() - t0, "clusters": int(sizes.size),
                    "largest_cluster": int(sizes.max()), "joins": int(len(joins))}
        else:
            tree = {"skipped": "%d rows: a cluster of a 10 %% sample would pass the 65,536-row "
                               "limit of one NJ" % n}
    align = None
    if not args.no_align_record and rank == 0:
        align = align_record(flush, stream, measured_peaks().get("hbm_gbs", 6800.0),
                             args.no_autotune)

    t_max = reduce_max(total_ms)
    all_cells = reduce_sum(float(cells))
    e2e_max = reduce_max(e2e_ms)
    e2e_all = reduce_sum(float(e2e_cells))
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    value = all_cells / (t_max * 1e-3) / 1e9
    achieved = center_cells / (center_ms * 1e-3) / 1e9 if center_ms > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int16x2", "data": "synthetic",
        "config": {"workload": workload_text(w, n, args.center, length),
                   "step": "encode + %s center + align with traceback + merge + rows + SP"
                           % ("the named (500-residue ancestor)" if w.center_seq else
                              "exact all-pairs" if refs is None else "sampled exact"),
                   "l2": "flushed (512 MB write) before every timed step",
                   "cells_per_step": cells / args.steps, "center": c, "msa_width": W,
                   "avg_sp": sp / (n * (n - 1) / 2)},
        "roofline": ({"bound": "alu", "kernel": "k_center (exact-center DP, packed int16x2)",
                      "achieved": achieved, "peak": ALU_PEAK_GCUPS, "unit": UNIT,
                      "frac": achieved / ALU_PEAK_GCUPS if achieved else None, "traffic": None,
                      "traffic_note": "not scaled: the center kernels' DRAM traffic is the "
                                      "residues and profiles, which does not grow with the "
                                      "cells (0.28 MB for one 1.57 ms launch on 2,000 "
                                      "proteins, profiles/k_center2_batched_uneven_10k.md)",
                      "peak_source": "152 SMs x 64 DPX lanes/clk x 2.07 GHz / 3 DPX ops per cell",
                      "peak_measured": rate / OPS_PER_CELL / 1e9,
                      "dpx_ops_per_clk_sm_measured": per_clk}
                     if center_cells else
                     # a named center: the step's DP is the alignment with codes
                     {"bound": "alu", "kernel": "k_codes2 (Gotoh fill + 4-bit traceback codes)",
                      "achieved": align_cells_t / (align_ms_t * 1e-3) / 1e9, "peak": CODES_PEAK_GCUPS,
                      "unit": UNIT,
                      "frac": align_cells_t / (align_ms_t * 1e-3) / 1e9 / CODES_PEAK_GCUPS,
                      "traffic": align_cells_t / args.steps * CODES_TRAFFIC_PER_CELL,
                      "peak_source": "152 SMs x 128 integer lanes/clk x 2.07 GHz / (3 DPX "
                                     "instructions at half rate + 4 two-operand ops) per cell"}),
        "stages_ms": {k: round(v, 3) for k, v in stage_ms.items()},
        "clocks": clocks,
        "e2e": {"value": e2e_all / (e2e_max * 1e-3) / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": int(letters.nbytes + offsets.nbytes),
                "d2h_bytes_per_step": int(n * W + 8 * 4)},
        "gpu_launches": launches,
        "device_mem_gb": b.msa_memory(h)[1] / 1e9,
        "autotune": {"seconds": tune_s, "buckets_timed": int((tune > 0).any(axis=1).sum()),
                     "variants_timed": int((tune > 0).sum()),
                     "center_choice_per_bucket": tuner_choices(tune) if tune.size else {},
                     "align": align_tune},
    }
    if learned is not None:
        line["learned_vs_exact"] = learned
    if align is not None:
        line["align"] = align
    if tree is not None:
        line["tree"] = tree
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(letters, offsets, alph, M, w.gap_open, w.gap_extend,
                                            args.cpu_seconds)
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
