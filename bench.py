#!/usr/bin/env python3
"""Benchmark: exact selectivity computation and selection push-down.

Headline workload (the largest single-GPU configuration): the 1.2B-row,
6-column synthetic table of config 5 (24 B/row, 28.8 GB resident in HBM) with
its 256 seeded probe predicates (OR of 1-3 ANDs of 1-3 clauses; selectivities
log-spaced in [1e-6, 0.9]).  One step is one optimiser pass of the method over
that table (Ch3; Algorithm 1 Execute for the relation, with every probe):
  a1  compile the 256 probe predicates;
  a5  their exact counts in one batched scan (the column-bucket kernel, one
      graph launch, autotuned shape) -- a2 is the single-probe count;
  a3  maxSize = floor(n * 0.05): probes above it are not pushed down;
  a4  push-down (fused count + stable compaction) of 3 projected columns for
      every probe at or under maxSize;
  a6-a9  the learned estimator on config 4's table (config 2's 300M-row
      table): features and the tensor-core forward pass of 4096 held-out
      probes, the uncertainty gate, and one training minibatch (the model is
      trained before the timed region on exact counts from the count kernel,
      tau is chosen on a validation split; the gate's exact fallback is the
      batched scan, timed separately as exact_ms_per_estimate).
value = algorithmic bytes of all scans of a step / device time of the step.

Other configurations are reported beside it: config 2's probes (batched vs
one launch per probe, single counts, push-downs at every selectivity),
config 3's star schema, config 1's latency.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --estimator-curve     (config 4's learning curve: 20k / 200k / 2M pairs)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import datagen as dg  # noqa: E402

METRIC = "exact-count scan GB/s (% HBM peak), ms/estimate; surrogate p95 q-error"
MAX_SELECTIVITY = 0.05          # PUSH_DOWN_MAX_SELECTIVITY of Algorithm 1 (ratio form)
WIDTH = {"i32": 4, "i64": 8, "f32": 4, "date": 4, "dict": 4}
CFG5_ROWS = 1_200_000_000
CFG2_ROWS = 300_000_000


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    """SM clock and clock-event reasons sampled through NVML (read only) while
    the timed region runs, every interval_s seconds (NVML queries take driver
    locks that also serve this process's CUDA calls: sampling much faster
    slows the host side of the step)."""
    REASONS = [("hw_slowdown", "nvmlClocksEventReasonHwSlowdown"),
               ("hw_thermal_slowdown", "nvmlClocksEventReasonHwThermalSlowdown"),
               ("sw_thermal_slowdown", "nvmlClocksEventReasonSwThermalSlowdown"),
               ("sw_power_cap", "nvmlClocksEventReasonSwPowerCap"),
               ("hw_power_brake_slowdown", "nvmlClocksEventReasonHwPowerBrakeSlowdown")]

    def __init__(self, index: int, interval_s: float = 0.05):
        self.index = index
        self.interval_s = interval_s
        self.samples = []
        self.reasons = set()
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None

    def start(self):
        self.error = None
        try:
            import pynvml as nv
            nv.nvmlInit()
            h = nv.nvmlDeviceGetHandleByIndex(self.index)
            self.max_mhz = float(nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM))
        except Exception as e:   # fall back to nvidia-smi
            self.error = f"nvml: {type(e).__name__}: {e}"
            self._start_smi()
            return

        def run():
            while not self._stop.is_set():
                try:
                    self.samples.append(float(nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)))
                    r = nv.nvmlDeviceGetCurrentClocksEventReasons(h)
                    for name, const in self.REASONS:
                        if r & getattr(nv, const, 0):
                            self.reasons.add(name)
                except Exception:
                    pass
                time.sleep(self.interval_s)
        self._thread = threading.Thread(target=run, daemon=True)
        self._thread.start()

    def _start_smi(self):
        def run():
            try:
                p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,"
                                      "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                                      "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                                      "--format=csv,noheader,nounits", "-lms", "100"],
                                     stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except OSError as e:
                self.error = (self.error or "") + f"; nvidia-smi: {e}"
                return
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for line in p.stdout:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) == 6:
                    try:
                        self.samples.append(float(parts[0]))
                        self.max_mhz = float(parts[1])
                    except ValueError:
                        pass
                    for k, v in zip(names, parts[2:]):
                        if v.lower() == "active":
                            self.reasons.add(k)
                if self._stop.is_set():
                    break
            p.terminate()
        self._thread = threading.Thread(target=run, daemon=True)
        self._thread.start()
        time.sleep(0.3)   # let nvidia-smi start before the timed region

    def stop(self):
        self._stop.set()
        if self._thread:
            self._thread.join(timeout=2)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unsampled"], "error": self.error}
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples)}


# ----------------------------------------------------------------------------
# the workload
# ----------------------------------------------------------------------------

def algorithmic_bytes(types, n, trees, counts, accepted, proj):
    """Bytes a step must move at least: each predicate column of the batched
    scan once, and for each push-down its predicate columns, the projected
    values of the selected rows that are not predicate columns, and the
    written rows (projected values + int64 row id)."""
    union = sorted({c for t in trees for c in dg.tree_columns(t)})
    batch = sum(WIDTH[types[c]] for c in union) * n
    pds = []
    for i in accepted:
        pc = set(dg.tree_columns(trees[i]))
        rd = sum(WIDTH[types[c]] for c in pc) * n + counts[i] * sum(WIDTH[types[c]] for c in proj if c not in pc)
        wr = counts[i] * (sum(WIDTH[types[c]] for c in proj) + 8)
        pds.append(rd + wr)
    return batch, pds


def pushdown_pass_bytes(types, n, trees, counts, accepted, proj):
    """Per push-down, the algorithmic bytes of its two passes: the count pass
    reads the predicate columns; the scatter reads every projected value of
    the selected rows (predicate columns included: the count pass keeps only
    the row masks) and writes them with their int64 row ids."""
    out = []
    for i in accepted:
        pc = dg.tree_columns(trees[i])
        pw = sum(WIDTH[types[c]] for c in proj)
        out.append((sum(WIDTH[types[c]] for c in set(pc)) * n, counts[i] * (2 * pw + 8)))
    return out


class Workload:
    """Config 5: 1.2B rows x 6 columns, 256 probes, push-down of 3 columns."""

    def __init__(self, n_rows: int, device, seed_offset: int = 0):
        label = "cfg5" if seed_offset == 0 else f"cfg5_r{seed_offset}"
        self.table = dg.gen_table(label, dg.config5_specs(), n_rows, device,
                                  cfg_label="cfg5" if seed_offset == 0 else None)
        self.n = n_rows
        self.types = [c.type for c in self.table.columns]
        self.trees = dg.config5_predicates()
        self.proj = [self.table.index(c) for c in dg.CONFIG5_PROJECTION]
        self.max_rows = int(math.floor(n_rows * MAX_SELECTIVITY))


class DeviceRing:
    """Output regions for the end-to-end push-downs: consecutive slices of one
    device buffer, each reused only after the copy that read it (its event)
    has run, so that the copy-backs of large push-downs never hold up the
    push-downs after them."""

    def __init__(self, nbytes: int, device):
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.head = 0
        self.live = []          # [start, end, event or None] of regions still to be read
        self.pending = []       # regions of the current take, until release_on

    def take(self, counts, dtypes, stream):
        sizes = [(n * torch.empty(0, dtype=d).element_size() + 255) // 256 * 256 for n, d in zip(counts, dtypes)]
        need = max(256, sum(sizes))
        assert need <= self.buf.numel(), "push-down output larger than the ring"
        if self.head + need > self.buf.numel():
            self.head = 0
        a, b = self.head, self.head + need
        keep = []
        for r in self.live:
            if r[0] < b and a < r[1]:
                stream.wait_event(r[2])         # its copy has read it
            else:
                keep.append(r)
        self.live = keep
        self.head = b
        self.pending = [a, b]
        out, off = [], a
        for n, d, sz in zip(counts, dtypes, sizes):
            out.append(self.buf[off:off + sz].view(d)[:n])
            off += sz
        return out[:-1], out[-1]

    def release_on(self, event):
        self.live.append([self.pending[0], self.pending[1], event])


class OurStep:
    def __init__(self, w: Workload, sel):
        self.w, self.sel = w, sel
        self.ctx = sel.Context()
        self.T = sel.Table(w.table.columns)
        dev = w.table.columns[0].data.device
        P = len(w.trees)
        self.counts_dev = torch.zeros(P, dtype=torch.int64, device=dev)
        self.pd_counts = torch.zeros(P, dtype=torch.int64, device=dev)
        cap = max(1, w.max_rows)
        self.out_cols = [torch.empty(cap, dtype=w.table.columns[c].data.dtype, device=dev) for c in w.proj]
        self.out_ids = torch.empty(cap, dtype=torch.int64, device=dev)
        self.events = []            # (kind, start, end[, split]) of the timed steps
        self.host_out = None
        self.next_preds = None
        # the batch plan (autotuned, graph-captured) is created and cached by the first call
        preds = [sel.Predicate(self.T, t) for t in w.trees]
        t0 = time.perf_counter()
        self.ctx.count_batch_async(preds, [self.T] * len(preds), self.counts_dev)
        self.ctx.synchronize()
        self.plan_s = time.perf_counter() - t0

    def run(self, record=False, e2e=False, T=None, rows_back=False):
        w, sel, ctx = self.w, self.sel, self.ctx
        T = T or self.T                                                          # the table's device copy
        # a1: this step's predicates, compiled while the previous step's batched
        # count ran (a predicate fits every table of the same columns)
        preds = self.next_preds or [sel.Predicate(T, t) for t in w.trees]
        self.next_preds = None
        ev = lambda: torch.cuda.Event(enable_timing=True) if record else None
        e0, e1 = ev(), ev()
        if record:
            e0.record()
        torch.cuda.nvtx.range_push("a5_count_batch")
        ctx.count_batch_async(preds, [T] * len(preds), self.counts_dev)         # a5 (a2)
        torch.cuda.nvtx.range_pop()
        if record:
            e1.record()
            self.events.append(("count", e0, e1))
        self.next_preds = [sel.Predicate(T, t) for t in w.trees]               # a1 of the next step
        counts = self.counts_dev.tolist()                                       # exact counts on the host
        accepted = [i for i, c in enumerate(counts) if c <= w.max_rows]         # a3
        d2h = 8 * len(counts)
        for k, i in enumerate(accepted):                                        # a4
            a, b = ev(), ev()
            mr = w.max_rows
            if e2e and rows_back:
                # end to end: each push-down writes into its own region of a device
                # ring, sized by its exact count (known from the batched count, so
                # max_rows = the count bounds the writes to the region), and its rows
                # go back to the host on a copy stream while the next ones run
                outs, ids = self.e2e_ring.take([counts[i]] * len(w.proj) + [counts[i]],
                                               [o.dtype for o in self.out_cols] + [torch.int64], ctx.stream)
                mr = counts[i]
            else:
                outs, ids = self.out_cols, self.out_ids
            if record:
                a.record()
                # the library records `mid` between the push-down's count pass and its scatter
                mid = ev()
                mid.record()
                ctx.set_pushdown_split_event(mid)
            torch.cuda.nvtx.range_push("a4_pushdown")
            ctx.pushdown_async(preds[i], T, w.proj, mr, outs, ids, self.pd_counts[i:i + 1])
            torch.cuda.nvtx.range_pop()
            if record:
                ctx.set_pushdown_split_event(None)
                b.record()
                self.events.append(("pushdown", a, b, mid))
            if e2e and rows_back:
                done = torch.cuda.Event()
                done.record(ctx.stream)
                self.copy_stream.wait_event(done)
                with torch.cuda.stream(self.copy_stream):
                    for o, h in zip(outs + [ids], self.host_out):
                        h[:counts[i]].copy_(o[:counts[i]], non_blocking=True)
                    copied = torch.cuda.Event()
                    copied.record(self.copy_stream)
                self.e2e_ring.release_on(copied)
                d2h += counts[i] * (sum(o.element_size() for o in self.out_cols) + 8)
        if e2e:
            # the step's result on the host: the exact counts (above) and the
            # push-downs' counts; the materialised rows stay on the device for
            # the rest of the query unless rows_back
            self.pd_counts_host = self.pd_counts.cpu()
            d2h += 8 * len(counts)
        ctx.synchronize()
        if e2e and rows_back:
            self.copy_stream.synchronize()
        return counts, accepted, d2h


def q_error(est, true):
    e = np.maximum(np.asarray(est, np.float64), 1.0)
    t = np.maximum(np.asarray(true, np.float64), 1.0)
    return np.maximum(e / t, t / e)


def estimator_workload(n, seed_label="bench_estimator"):
    rng = np.random.default_rng(dg.mix_seed(seed_label))
    specs = dg.config2_specs()
    return [dg.random_dnf_predicate(specs, rng) for _ in range(n)]


def train_and_gate(sel, ctx, T, preds, counts, n_train, n_val, n_test, sample_rows=4096):
    """Config 4: train on n_train labelled probes, choose tau on the next
    n_val (the largest tau whose accepted estimates keep the 95th-percentile
    q-error <= 2), score the n_test after them."""
    model = sel.Estimator(ctx, T, sample_rows=sample_rows, seed=dg.MASTER_SEED)
    epochs = max(4, min(40, 800_000 // max(1, n_train)))
    cfg = sel.train_cfg(epochs=epochs, batch=256, lr=1e-3, seed=1)
    t0 = time.perf_counter()
    loss = model.train(preds[:n_train], counts[:n_train], cfg)
    train_s = time.perf_counter() - t0

    def outputs(lo, hi):
        pl = sel.PredicateList(preds[lo:hi])
        feat, ok = model.featurize(pl)
        out = model.forward(feat).cpu().numpy().astype(np.float64)
        okm = ok.cpu().numpy().astype(bool)
        est = np.maximum(np.expm1(out[:, 0]), 0.0)
        sig = np.where(okm, np.exp(0.5 * np.clip(out[:, 1], -8, 8)), np.inf)
        return pl, feat, okm, est, sig
    _, _, okv, est_v, sig_v = outputs(n_train, n_train + n_val)
    tau, answered_val = sel.choose_tau(sig_v, est_v, counts[n_train:n_train + n_val])
    pl, feat, okt, est_t, sig_t = outputs(n_train + n_val, n_train + n_val + n_test)
    exact_t = counts[n_train + n_val:n_train + n_val + n_test]
    q = q_error(est_t, exact_t)
    acc = okt & (sig_t <= tau)
    from paper_1806_08384_b300 import baselines
    ind = baselines.independence_selectivity(feat.float().cpu().numpy()) * T.n_rows
    qi = q_error(ind, exact_t)
    gated = np.where(acc, est_t, exact_t.astype(np.float64))
    qg = q_error(gated, exact_t)
    quality = {
        "n_train": n_train, "n_val": n_val, "n_test": n_test, "epochs": epochs,
        "train_seconds": round(train_s, 2), "final_train_loss": round(loss, 4),
        "q_error_p50": round(float(np.median(q[okt])), 3), "q_error_p95": round(float(np.percentile(q[okt], 95)), 3),
        "tau": round(float(tau), 4), "tau_rule": "largest tau with 95th-percentile q-error <= 2 on the validation split",
        "answered_fraction_validation": round(answered_val, 3),
        "gated_answered_fraction": round(float(acc.mean()), 3),
        "gated_accepted_q_error_p50": round(float(np.median(q[acc])), 3) if acc.any() else None,
        "gated_accepted_q_error_p95": round(float(np.percentile(q[acc], 95)), 3) if acc.any() else None,
        "gated_all_q_error_p95": round(float(np.percentile(qg, 95)), 3),
        "independence_q_error_p50": round(float(np.median(qi[okt])), 3),
        "independence_q_error_p95": round(float(np.percentile(qi[okt], 95)), 3)}
    return model, tau, pl, quality, okt


class Surrogate:
    """a6-a9 on config 4's table: the learned estimator, trained before the
    timed region on exact counts from the count kernel (a5), tau chosen on a
    validation split; inside every timed step: featurize + forward of the
    held-out test probes, the gate decision, and one training minibatch.  The
    gate's exact fallback is the batched scan; its cost per estimate is timed
    separately."""

    def __init__(self, sel, ctx, table, n_train=200_000, n_val=20_000, n_test=4096, sample_rows=4096):
        self.sel, self.ctx = sel, ctx
        T = sel.Table(table.columns)
        self.T = T
        trees = estimator_workload(n_train + n_val + n_test)
        preds = [sel.Predicate(T, t) for t in trees]
        t0 = time.perf_counter()
        counts = np.array(sel.count_many(ctx, preds, T), dtype=np.uint64)
        self.label_s = time.perf_counter() - t0
        self.n_labels = len(preds)
        self.model, self.tau, self.eval_preds, self.quality, okt = train_and_gate(
            sel, ctx, T, preds, counts, n_train, n_val, n_test, sample_rows)
        self.eval_counts = counts[n_train + n_val:]
        self.traditional = self.traditional_baselines(table, trees[n_train + n_val:], okt)
        self.train_feat, _ = self.model.featurize(preds[:256])
        self.train_y = torch.from_numpy(np.log1p(counts[:256].astype(np.float64)).astype(np.float32)).cuda()
        self.step_cfg = sel.train_cfg(batch=256, lr=1e-4, apply_update=1)
        # exact fallback cost: one batched scan of 128 of the held-out probes
        self.exact_plan = sel.BatchPlan(ctx, self.eval_preds[:128], [T] * 128, autotune=False)
        self.events = []
        self.accepted = 0

    def traditional_baselines(self, table, eval_trees, okm, sample_rows=65_536):
        """Ch2's estimators on the same held-out probes: the textbook heuristics
        (1/V, 1/3) with exact distinct counts, equi-depth histograms (64 buckets)
        built from a row sample, and the sampling estimator (the library's count
        on that sample, scaled by |R| / |R'|)."""
        from paper_1806_08384_b300 import baselines
        sel, T = self.sel, self.T
        cols = table.columns
        n = T.n_rows
        distinct = [int(torch.unique(c.data).numel()) for c in cols]
        dicts = [c.dictionary for c in cols]
        sample = baselines.row_sample(cols, sample_rows, dg.mix_seed("bench_row_sample"))
        hists = [baselines.EquiDepthHistogram.build(c.data.cpu().numpy(), n, buckets=64) for c in sample]
        TS = sel.Table(sample)
        sp = [sel.Predicate(TS, t) for t in eval_trees]
        t0 = time.perf_counter()
        sc = np.array(sel.count_many(self.ctx, sp, TS), dtype=np.float64)
        samp_ms = (time.perf_counter() - t0) * 1e3 / len(sp)
        est = {"textbook": np.array([baselines.textbook_selectivity(t, distinct, dicts) for t in eval_trees]) * n,
               "histogram": np.array([baselines.histogram_selectivity(t, hists, dicts) for t in eval_trees]) * n,
               "sampling": np.array([baselines.sampling_estimate(c, sample_rows, n) for c in sc])}
        out = {}
        for name, e in est.items():
            q = q_error(e, self.eval_counts)[okm]
            out[name + "_q_error_p50"] = round(float(np.median(q)), 3)
            out[name + "_q_error_p95"] = round(float(np.percentile(q, 95)), 3)
        out["sampling_rows"] = sample_rows
        out["sampling_ms_per_estimate"] = round(samp_ms, 4)
        return out

    def run(self, record=False):
        ev = lambda: torch.cuda.Event(enable_timing=True)
        a, a2, b, c = ev(), ev(), ev(), ev()
        if record:
            a.record()
        torch.cuda.nvtx.range_push("a6_featurize")
        feat, ok = self.model.featurize(self.eval_preds)              # a6
        torch.cuda.nvtx.range_pop()
        if record:
            a2.record()
        torch.cuda.nvtx.range_push("a7_forward")
        out = self.model.forward(feat)                                # a7
        torch.cuda.nvtx.range_pop()
        if record:
            b.record()
        o = out.cpu().numpy()                                         # a9: gate decision on the host
        self.accepted = int(((np.exp(0.5 * np.clip(o[:, 1], -8, 8)) <= self.tau) & ok.cpu().numpy().astype(bool)).sum())
        torch.cuda.nvtx.range_push("a8_train_step")
        self.model.train_step(self.train_feat, self.train_y, self.step_cfg)   # a8
        torch.cuda.nvtx.range_pop()
        if record:
            c.record()
            self.events.append((a, a2, b, c))

    def summary(self):
        inf = [x.elapsed_time(y) for x, _, y, _ in self.events]
        fz = [x.elapsed_time(y) for x, y, _, _ in self.events]
        fw = [x.elapsed_time(y) for _, x, y, _ in self.events]
        trn = [y.elapsed_time(z) for _, _, y, z in self.events]
        reps = 5
        self.exact_plan.run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            self.exact_plan.run()
        e1.record()
        torch.cuda.synchronize()
        exact_ms = e0.elapsed_time(e1) / reps
        n = len(self.eval_preds)
        return dict(self.quality, **self.traditional, **{
            "workload": f"config 4: {n} held-out OR-of-AND probes (<= 6 leaves) on config 2's 300M-row table; "
                        f"trained on {self.quality['n_train']} probes labelled by the count kernel, tau chosen on "
                        f"{self.quality['n_val']} validation probes",
            "label_seconds": round(self.label_s, 2), "labels": self.n_labels,
            "ms_per_label": round(self.label_s * 1e3 / self.n_labels, 4),
            "ms_per_batch_featurize_forward": round(statistics.mean(inf), 3),
            "ms_featurize": round(statistics.mean(fz), 3), "ms_forward": round(statistics.mean(fw), 3),
            "ms_per_estimate": round(statistics.mean(inf) / n, 6),
            "exact_ms_per_estimate": round(exact_ms / 128, 4),
            "train_step_ms": round(statistics.mean(trn), 3),
            "answered_without_scan_per_step": self.accepted})


# ----------------------------------------------------------------------------
# config 2: batched vs separate, single counts, push-downs at every selectivity
# ----------------------------------------------------------------------------

def config2_measurements(sel, table, peak: float, reps=5):
    """Config 2's five probes (OR of 3 ANDs; s = 1e-4 .. 0.5) on the 300M-row
    table: one batched launch (the bucket kernel and the interpreter) vs one
    launch per probe; each probe's count alone; and each probe's push-down of
    4 columns with maxSize = n (every selection materialised, up to 150M rows),
    with its algorithmic bytes (predicate columns read, projected values of
    the selected rows read, rows + row ids written) and GB/s."""
    T = sel.Table(table.columns)
    trees = [dg.config2_predicate(s) for s in dg.CONFIG2_TARGETS]
    preds = [sel.Predicate(T, t) for t in trees]
    types = [c.type for c in table.columns]
    n = T.n_rows
    dev = table.columns[0].data.device
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn, r=reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record()
        for _ in range(r):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / r
    outs = torch.zeros(len(preds), dtype=torch.int64, device=dev)
    res = {}
    union = sorted({c for t in trees for c in dg.tree_columns(t)})
    shared = sum(WIDTH[types[c]] for c in union) * n
    for kernel, mode in (("bucket", 0), ("interpreter", 1)):
        ctx = sel.Context()
        ctx.set_batch_kernel(mode)
        plan = sel.BatchPlan(ctx, preds, [T] * len(preds), autotune=True)
        ms = timed(lambda: plan.run(outs))
        res[f"batched_{kernel}_ms"] = round(ms, 4)
        res[f"batched_{kernel}_frac"] = round(shared / ms / 1e6 / peak, 4)
        res[f"batched_{kernel}_pick"] = plan.info()
        counts = outs.cpu().tolist()
    ctx = sel.Context()
    res["separate_ms"] = round(timed(lambda: [ctx.count_async(p, T, outs[i:i + 1]) for i, p in enumerate(preds)]), 4)
    res["speedup"] = round(res["separate_ms"] / min(res["batched_bucket_ms"], res["batched_interpreter_ms"]), 3)
    res["batched_shared_pass_bytes"] = shared
    single = []
    one = torch.zeros(1, dtype=torch.int64, device=dev)
    for t, p in zip(trees, preds):
        nb = sum(WIDTH[types[c]] for c in dg.tree_columns(t)) * n
        ms = timed(lambda: ctx.count_async(p, T, one))
        single.append({"bytes": nb, "ms": round(ms, 4), "gbs": round(nb / ms / 1e6, 1),
                       "frac": round(nb / ms / 1e6 / peak, 4)})
    res["count_single"] = single
    res["count_single_frac_mean"] = round(statistics.mean(x["frac"] for x in single), 4)
    proj = [table.index(c) for c in dg.CONFIG2_PROJECTION]
    mr = max(counts)
    cols_out = [torch.empty(mr, dtype=table.columns[c].data.dtype, device=dev) for c in proj]
    ids = torch.empty(mr, dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    pds = []
    for s, t, p, c in zip(dg.CONFIG2_TARGETS, trees, preds, counts):
        ms = timed(lambda: ctx.pushdown_async(p, T, proj, mr, cols_out, ids, cnt), 3)
        assert int(cnt.item()) == c
        _, (b,) = algorithmic_bytes(types, n, [t], [c], [0], proj)
        written = c * (sum(WIDTH[types[k]] for k in proj) + 8)
        pds.append({"target_s": s, "count": c, "ms": round(ms, 3), "bytes": int(b), "written_bytes": int(written),
                    "gbs": round(b / ms / 1e6, 1), "frac": round(b / ms / 1e6 / peak, 4)})
    res["pushdown"] = pds
    del cols_out, ids
    res["distinct_and_join"] = distinct_and_join(sel, ctx, T, table, preds[2])
    res["workload"] = ("config2: 300M rows x 8 cols (2 i32 U, i64 Zipf1.1, f32 U, f32 LogN, date, dict-25, "
                       "dict-10k); 5 probes OR of 3 ANDs, s = 1e-4 .. 0.5; push-down of k0, k2, f0, d")
    return res


def distinct_and_join(sel, ctx, T, table, pred, reps=3):
    """f3: V(R, k2) and V(sigma_P(R), k2) of the int64 key (exact, GPU hash set)
    and the join-size estimate of sigma_P(R) with R on that key."""
    k = table.index("k2")
    out = {}
    for name, p in (("all_rows", None), ("selected_rows", pred)):
        ctx.count_distinct(T, k, p)
        t0 = time.perf_counter()
        for _ in range(reps):
            d, r = ctx.count_distinct(T, k, p)
        out[name] = {"distinct": d, "rows": r, "ms": round((time.perf_counter() - t0) * 1e3 / reps, 3)}
    a, b_ = out["selected_rows"], out["all_rows"]
    out["join_size_estimate"] = round(sel.join_size_estimate(a["rows"], b_["rows"], a["distinct"], b_["distinct"]), 1)
    out["note"] = "host-timed synchronous calls; with a predicate the time includes the push-down of k2"
    return out


def config5_gated(step: "OurStep", n_train=100_000, n_val=10_000, reps=3):
    """Config 5's gated mode: an estimator trained on config 5's own table
    (random OR-of-AND probes labelled by the batched count, 256 a launch), tau
    chosen on a validation split, then the step's 256 probes answered through
    the library's gated call (sel_mlp_estimate: features, forward, the gate,
    and one batched exact count of every probe the network does not answer).
    The fallbacks' counts are checked against the step's exact counts."""
    sel, w, T = step.sel, step.w, step.T
    ctx = sel.Context()
    rng = np.random.default_rng(dg.mix_seed("bench_cfg5_estimator"))
    specs = dg.config5_specs()
    trees = [dg.random_dnf_predicate(specs, rng) for _ in range(n_train + n_val)]
    preds = [sel.Predicate(T, t) for t in trees]
    t0 = time.perf_counter()
    counts = np.array(sel.count_many(ctx, preds, T), dtype=np.uint64)
    label_s = time.perf_counter() - t0
    wl = [sel.Predicate(T, t) for t in w.trees]
    exact = np.array(step.counts_dev.tolist(), dtype=np.uint64)
    model, tau, _, quality, okt = train_and_gate(sel, ctx, T, preds + wl, np.concatenate([counts, exact]),
                                                 n_train, n_val, len(wl))
    model.estimate(wl, T, tau)          # the first call builds and caches the fallback's batch plan
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        est, sig, used = model.estimate(wl, T, tau)
    gated_ms = (time.perf_counter() - t0) * 1e3 / reps
    assert all(int(e) == int(c) for e, c, u in zip(est, exact, used) if u), "an exact fallback differs"
    q = q_error(est, exact)
    acc = ~used
    return {
        "workload": "config 5's 256 probes on the 1.2B-row table; estimator trained on %d random OR-of-AND "
                    "probes of the same table (labelled by the batched count), tau on %d more" % (n_train, n_val),
        "labels": len(preds), "label_seconds": round(label_s, 1), "ms_per_label": round(label_s * 1e3 / len(preds), 4),
        "tau": quality["tau"], "train_seconds": quality["train_seconds"],
        "featurizable_fraction": round(float(okt.mean()), 3),
        "answered_by_network": int(acc.sum()), "exact_fallbacks": int(used.sum()),
        "gated_ms": round(gated_ms, 3), "gated_ms_per_estimate": round(gated_ms / len(wl), 4),
        "exact_batched_ms_per_estimate": round(statistics.mean(e[1].elapsed_time(e[2]) for e in step.events
                                                               if e[0] == "count") / len(wl), 4),
        "q_error_p50": round(float(np.median(q)), 3), "q_error_p95": round(float(np.percentile(q, 95)), 3),
        "accepted_q_error_p95": round(float(np.percentile(q[acc], 95)), 3) if acc.any() else None,
        "network_q_error_p50_featurizable": quality["q_error_p50"],
        "network_q_error_p95_featurizable": quality["q_error_p95"]}


def config5_extras(step: "OurStep", peak: float, reps=3):
    """On the headline table: three single-probe counts and the push-down of
    the s = 0.9 probe (about 1.08B rows written; its own maxSize = n)."""
    sel, w, ctx, T = step.sel, step.w, step.ctx, step.T
    counts = step.counts_dev.tolist()
    dev = step.counts_dev.device
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn, r):
        fn()
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record()
        for _ in range(r):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / r
    targets = np.logspace(-6, np.log10(0.9), len(w.trees))
    res = {"count_single": []}
    one = torch.zeros(1, dtype=torch.int64, device=dev)
    for i in (0, len(w.trees) // 2, len(w.trees) - 1):
        p = sel.Predicate(T, w.trees[i])
        ms = timed(lambda: ctx.count_async(p, T, one), reps)
        assert int(one.item()) == counts[i]
        b = sum(WIDTH[w.types[c]] for c in dg.tree_columns(w.trees[i])) * w.n
        res["count_single"].append({"target_s": float(f"{targets[i]:.3g}"), "count": counts[i], "ms": round(ms, 3),
                                    "gbs": round(b / ms / 1e6, 1), "frac": round(b / ms / 1e6 / peak, 4)})
    i = len(w.trees) - 1
    p = sel.Predicate(T, w.trees[i])
    c = counts[i]
    cols_out = [torch.empty(c, dtype=w.table.columns[k].data.dtype, device=dev) for k in w.proj]
    ids = torch.empty(c, dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ms = timed(lambda: ctx.pushdown_async(p, T, w.proj, c, cols_out, ids, cnt), 2)
    assert int(cnt.item()) == c
    _, (b,) = algorithmic_bytes(w.types, w.n, [w.trees[i]], [c], [0], w.proj)
    res["pushdown_s09"] = {"target_s": 0.9, "count": c, "ms": round(ms, 3), "bytes": int(b),
                           "gbs": round(b / ms / 1e6, 1), "frac": round(b / ms / 1e6 / peak, 4)}
    del cols_out, ids
    torch.cuda.empty_cache()
    return res


# ----------------------------------------------------------------------------
# config 3 and config 1
# ----------------------------------------------------------------------------

def star_batch(sel, peak: float, device, reps=5):
    """a5 on the star schema: 64 probes over a 480M-row fact table and four
    dimension tables (2k, 200k, 2.4M, 16M rows) as one autotuned, graph-captured
    launch sequence vs one count launch per probe on the same stream."""
    tabs = dg.config3_tables(device=device)
    T = [sel.Table(t.columns) for t in tabs]
    probes = dg.config3_predicates()
    preds = [sel.Predicate(T[ti], tr) for ti, tr in probes]
    ptabs = [T[ti] for ti, _ in probes]
    ctx = sel.Context()
    t0 = time.perf_counter()
    plan = sel.BatchPlan(ctx, preds, ptabs)
    plan_s = time.perf_counter() - t0
    out = torch.zeros(len(preds), dtype=torch.int64, device=device)
    # bytes: each referenced column of each table once (shared pass) vs per probe
    shared = 0
    for ti, t in enumerate(tabs):
        cols = sorted({c for tj, tr in probes if tj == ti for c in dg.tree_columns(tr)})
        shared += sum(t.columns[c].spec.width for c in cols) * t.n_rows
    separate_bytes = sum(sum(tabs[ti].columns[c].spec.width for c in dg.tree_columns(tr)) * tabs[ti].n_rows
                         for ti, tr in probes)
    res = {}
    for mode in ("batched", "separate"):
        def run():
            if mode == "batched":
                plan.run(out)
            else:
                for i, (p, tb) in enumerate(zip(preds, ptabs)):
                    ctx.count_async(p, tb, out[i:i + 1])
        for _ in range(2):
            run()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            run()
        b.record()
        torch.cuda.synchronize()
        res[mode + "_ms"] = round(a.elapsed_time(b) / reps, 4)
        res[mode + "_counts"] = out.cpu().tolist()
    assert res["batched_counts"] == res["separate_counts"]
    counts = res["batched_counts"]
    del res["batched_counts"], res["separate_counts"]
    # f3 / f4 on the star: the exact COUNT of sigma(fact) join sigma(dim) on a fact column whose
    # domain is the dimension key's (a1: 1000 Zipf values for the 2k-row dimension, a2: uniform
    # below 1M for the 200k- and 2.4M-row ones) next to the join-size estimate from exact
    # selectivities and distinct counts; the fact probe with the most rows under 10 % of the
    # fact table, each dimension's probe with the most rows
    joins = []
    fact_idx = [i for i, (ti, _) in enumerate(probes) if ti == 0]
    fact_i = max((i for i in fact_idx if counts[i] <= 0.1 * tabs[0].n_rows), key=lambda i: counts[i])
    fact_p = preds[fact_i]
    for k, fk in ((1, tabs[0].index("a1")), (2, tabs[0].index("a2")), (3, tabs[0].index("a2"))):
        dim_i = max((i for i, (ti, _) in enumerate(probes) if ti == k), key=lambda i: counts[i])
        t0 = time.perf_counter()
        exact, nr, ns = ctx.join_count(T[0], fk, fact_p, T[k], 0, preds[dim_i])
        join_ms = (time.perf_counter() - t0) * 1e3
        vr, _ = ctx.count_distinct(T[0], fk, fact_p)
        vs, _ = ctx.count_distinct(T[k], 0, preds[dim_i])
        est = sel.join_size_estimate(nr, ns, vr, vs)
        joins.append({"dimension_rows": tabs[k].n_rows, "fact_column": tabs[0].columns[fk].name,
                      "fact_selected": nr, "dim_selected": ns, "fact_distinct": vr, "dim_distinct": vs,
                      "join_count": exact, "join_count_ms": round(join_ms, 3), "estimate": round(est, 1),
                      "estimate_q_error": round(max(est, 1.0, exact) / max(min(est, exact), 1.0), 3)})
    info = plan.info()
    res.update({
        "join_counts": joins,
        "workload": "config3 star: fact 480M x 6 cols (i32 U/Zipf/U, f32 U/N/U) + dims 2k/200k/2.4M/16M x 4 cols; "
                    "32 fact probes + 8 per dimension, OR of 1-3 ANDs, s log-uniform in [1e-4, 0.5]",
        "speedup": round(res["separate_ms"] / res["batched_ms"], 3),
        "batched_gbs_shared_pass": round(shared / res["batched_ms"] / 1e6, 1),
        "batched_frac_shared_pass": round(shared / res["batched_ms"] / 1e6 / peak, 4),
        "shared_pass_bytes": shared, "separate_bytes": separate_bytes,
        "ms_per_estimate_batched": round(res["batched_ms"] / len(preds), 4),
        "autotune_pick": info, "plan_create_s": round(plan_s, 2)})
    del plan, T, tabs
    torch.cuda.empty_cache()
    return res


def config1_latency(sel, device, reps=200):
    """Config 1: one exact count over a 1M-row table (12 B/row of referenced
    columns, 12 MB: it fits in L2), so the time is launch latency and is
    reported per estimate.  Plain launch (sel_count_async) and graph replay (a
    one-probe batch plan), each with L2 warm (back-to-back launches) and L2
    flushed (a 512 MB buffer overwritten before each timed launch), and the
    synchronous host call an optimiser waiting for the answer sees."""
    tab = dg.config1_table(device=device)
    T = sel.Table(tab.columns)
    p = sel.Predicate(T, dg.config1_predicate(0))
    ctx = sel.Context()
    out = torch.zeros(1, dtype=torch.int64, device=device)
    plan = sel.BatchPlan(ctx, [p], [T], autotune=False)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=device)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    res = {}
    for name, fn in (("plain", lambda: ctx.count_async(p, T, out)), ("graph", lambda: plan.run(out))):
        for _ in range(10):
            fn()
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        res[name + "_l2_warm_us"] = round(a.elapsed_time(b) * 1e3 / reps, 2)
        pairs = []
        for i in range(reps // 4):
            flush.fill_(i & 0xFF)
            a, b = ev(), ev()
            a.record()
            fn()
            b.record()
            pairs.append((a, b))
        torch.cuda.synchronize()
        res[name + "_l2_flushed_us"] = round(statistics.median(x.elapsed_time(y) for x, y in pairs) * 1e3, 2)
    n = ctx.count(p, T)
    t0 = time.perf_counter()
    for _ in range(reps):
        n = ctx.count(p, T)
    res["sync_call_us"] = round((time.perf_counter() - t0) * 1e6 / reps, 2)
    assert int(out.item()) == n
    cols = dg.tree_columns(dg.config1_predicate(0))
    nbytes = sum(tab.columns[c].spec.width for c in set(cols)) * tab.n_rows
    res.update({"count": n, "bytes": nbytes,
                "workload": "config1: 1M rows x 4 cols (i32 U, i32 Zipf1.2/1000, f32 N(0,1), date); "
                            "c0 BETWEEN a AND b AND c1 IN {5} AND c2 < t",
                "note": "device time per launch from CUDA events; flushed = 512 MB written before each launch"})
    del plan, flush
    torch.cuda.empty_cache()
    return res



# ----------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------

def oracle_step(ot, trees, max_rows_ratio, threads):
    import oracle
    counts = [oracle.count(ot, t, threads=threads) for t in trees]
    mr = int(math.floor(ot.n_rows * max_rows_ratio))
    accepted = [i for i, c in enumerate(counts) if c <= mr]
    for i in accepted:
        oracle.select(ot, trees[i], threads=threads)
    return counts, accepted


def oracle_sample(table, trees, target_s: float, threads: int):
    """A prefix of the table sized so that one oracle step takes about target_s."""
    import oracle
    n = table.n_rows
    m0 = min(n, 200_000)
    ot = oracle.OTable([c.data[:m0].cpu().numpy() for c in table.columns], [c.type for c in table.columns],
                       [c.dictionary for c in table.columns])
    t0 = time.perf_counter()
    oracle_step(ot, trees, MAX_SELECTIVITY, threads)
    dt = time.perf_counter() - t0
    m = int(min(n, max(m0, m0 * target_s / max(dt, 1e-6))))
    return oracle.OTable([c.data[:m].cpu().numpy() for c in table.columns], [c.type for c in table.columns],
                         [c.dictionary for c in table.columns])


def cpu_rate(ot, types, trees, proj, threads, reps=1):
    best = 1e30
    for _ in range(reps):
        t0 = time.perf_counter()
        counts, accepted = oracle_step(ot, trees, MAX_SELECTIVITY, threads)
        best = min(best, time.perf_counter() - t0)
    b, pds = algorithmic_bytes(types, ot.n_rows, trees, counts, accepted, proj)
    return (b + sum(pds)) / best / 1e9, best


# ----------------------------------------------------------------------------
# traffic and instruction counts from the committed ncu summaries
# (null if the kernel changed since)
# ----------------------------------------------------------------------------

KERNEL_SOURCES = {
    "bucket_count_kernel": ("scan.cuh", "program.h", "kernels.h", "bucket.h", "bucket_count.cu"),
    "scan_count_kernel": ("scan.cuh", "program.h", "kernels.h", "count.cu"),
    "pushdown_persistent_kernel": ("scan.cuh", "program.h", "kernels.h", "lookback.cuh", "rowmask.cuh", "pushdown.cu"),
    "scan_count_kernel_mask": ("scan.cuh", "program.h", "kernels.h", "count.cu"),
    "pushdown_scatter_kernel": ("program.h", "kernels.h", "rowmask.cuh", "scatter.cu"),
}


def kernel_source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1806_08384_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_entry(kernel):
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        e = json.load(f).get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e


def traffic_for(kernel: str, algorithmic_bytes: float):
    """DRAM bytes of one launch: the DRAM-to-algorithmic byte ratio measured by
    ncu on a smaller case of the same kernel (profiles/traffic.json) times this
    launch's algorithmic bytes; None when the kernel source changed since."""
    e = _traffic_entry(kernel)
    return int(e["traffic_per_algorithmic_byte"] * algorithmic_bytes) if e else None


def issue_roofline(kernel: str, n_rows: int, launch_ms: float, sm_mhz: float):
    """A count scan's instruction-issue roofline, for launches bound by the
    instruction stream rather than by HBM.  Achieved: the warp instructions per
    row that ncu measured on a smaller case of the same kernel and probe set
    (profiles/traffic.json) times this launch's rows, over the launch time.
    Peak: 148 SMs x 4 schedulers x 1 warp instruction per cycle x the SM
    clock.  None when the kernel source changed since the capture."""
    e = _traffic_entry(kernel)
    if not e or "warp_instructions_per_row" not in e or launch_ms <= 0:
        return None
    achieved = e["warp_instructions_per_row"] * n_rows / (launch_ms / 1e3) / 1e9
    peak = 148 * 4 * sm_mhz / 1e3
    return {"bound": "alu", "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G warp instructions/s", "frac": round(achieved / peak, 4), "kernel": kernel,
            "warp_instructions_per_row": e["warp_instructions_per_row"],
            "peak_source": f"148 SMs x 4 schedulers x 1 warp instruction/cycle x {sm_mhz:.0f} MHz"}


def smem_roofline(kernel: str, n_rows: int, launch_ms: float, sm_mhz: float):
    """A kernel bound by its shared-memory accesses (the column-bucket batch
    kernel's gathers): achieved = the shared-memory wavefronts per row that ncu
    measured on a smaller case of the same kernel and probe set
    (profiles/traffic.json) times this launch's rows, over the launch time;
    peak = 148 SMs x 1 wavefront (128 bytes) per cycle x the SM clock.  None
    when the kernel source changed since the capture."""
    e = _traffic_entry(kernel)
    if not e or "smem_wavefronts_per_row" not in e or launch_ms <= 0:
        return None
    achieved = e["smem_wavefronts_per_row"] * n_rows / (launch_ms / 1e3) / 1e9
    peak = 148 * sm_mhz / 1e3
    return {"bound": "smem", "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G shared-memory wavefronts/s", "frac": round(achieved / peak, 4), "kernel": kernel,
            "smem_wavefronts_per_row": e["smem_wavefronts_per_row"],
            "peak_source": f"148 SMs x 1 wavefront/cycle x {sm_mhz:.0f} MHz"}


# ----------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rows", type=int, default=CFG5_ROWS, help="rows of the headline (config 5) table")
    ap.add_argument("--cfg2-rows", type=int, default=CFG2_ROWS, help="rows of the config 2 / 4 table")
    ap.add_argument("--train", type=int, default=200_000, help="labelled training probes of the estimator")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the config 1/2/3 and extra config 5 measurements")
    ap.add_argument("--estimator-curve", action="store_true",
                    help="config 4's learning curve (20k / 200k / 2M labelled pairs); prints its own JSON")
    ap.add_argument("--kernel-case", choices=["batch-cfg5", "batch-cfg2", "pushdown-cfg5", "mlp-forward"],
                    help="run one kernel case twice (for an ncu capture) and exit: the batched count of config 5's "
                         "256 probes or of config 2's 5 probes, or the push-down of the config 5 probe nearest "
                         "selectivity --case-s, over a --rows-row table; or the estimator's inference pass over "
                         "4096 random OR-of-AND probes of a 1M-row config 2 table")
    ap.add_argument("--case-s", type=float, default=1e-3)
    ap.add_argument("--clock-interval-ms", type=float, default=50.0, help="NVML clock sampling interval")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    assert args.warmup >= 3 or args.steps <= 2, "at least 3 warm-up steps"

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    threads = os.cpu_count() or 1

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, threads)
        return

    import paper_1806_08384_b300 as sel
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.estimator_curve:
        estimator_curve(sel, dev, args)
        return
    if args.kernel_case:
        kernel_case(sel, dev, args)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    w = Workload(args.rows, dev, seed_offset=rank)
    step = OurStep(w, sel)
    sur = None
    cfg2_table = None
    if not args.no_surrogate or (rank == 0 and not args.no_extras):
        cfg2_table = dg.gen_table("cfg2", dg.config2_specs(), args.cfg2_rows, dev)
    if not args.no_surrogate:
        n_val = max(2_000, args.train // 10)
        sur = Surrogate(sel, sel.Context(), cfg2_table, n_train=args.train, n_val=n_val)
    for _ in range(args.warmup):
        step.run()
        if sur:
            sur.run()
    # per-step bytes are fixed (same probes, same data)
    counts, accepted, _ = step.run()
    b_batch, b_pds = algorithmic_bytes(w.types, w.n, w.trees, counts, accepted, w.proj)
    step_bytes = b_batch + sum(b_pds)

    clocks = ClockSampler(local, args.clock_interval_ms / 1e3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = step.ctx.launches + (sur.ctx.launches if sur else 0)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    torch.cuda.nvtx.range_push("timed_steps")
    for _ in range(args.steps):
        step.run(record=True)
        if sur:
            sur.run(record=True)
    torch.cuda.nvtx.range_pop()
    t1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = step.ctx.launches + (sur.ctx.launches if sur else 0) - launches0
    elapsed_ms, value = replica_throughput(t0.elapsed_time(t1), step_bytes, args.steps, world, dev)

    # per-kernel durations inside the timed region: the batched count, and each
    # push-down's count pass (start -> the library's split event) and the rest
    # (segment sums, group offsets, scatter)
    dur = {"count": [], "pushdown": [], "pass1": [], "scatter": []}
    for e in step.events:
        if e[0] == "count":
            dur["count"].append(e[1].elapsed_time(e[2]))
        else:
            _, a, b, m = e
            dur["pushdown"].append(a.elapsed_time(b))
            dur["pass1"].append(a.elapsed_time(m))
            dur["scatter"].append(m.elapsed_time(b))
    count_ms = statistics.mean(dur["count"])
    mean = lambda xs: statistics.mean(xs) if xs else 0.0
    split = pushdown_pass_bytes(w.types, w.n, w.trees, counts, accepted, w.proj)
    peak, peak_kind = load_peaks()
    count_kernel = "bucket_count_kernel"
    kernels = {
        "count": {"name": count_kernel, "ms": count_ms, "bytes": b_batch, "launches": len(dur["count"]),
                  "total_ms": sum(dur["count"])},
        "pass1": {"name": "scan_count_kernel_mask", "ms": mean(dur["pass1"]), "bytes": mean([p for p, _ in split]),
                  "launches": len(dur["pass1"]), "total_ms": sum(dur["pass1"])},
        "scatter": {"name": "pushdown_scatter_kernel", "ms": mean(dur["scatter"]),
                    "bytes": mean([q for _, q in split]), "launches": len(dur["scatter"]),
                    "total_ms": sum(dur["scatter"])},
        "pushdown": {"name": "push-down (all its kernels)", "ms": mean(dur["pushdown"]), "bytes": mean(b_pds),
                     "launches": len(dur["pushdown"]), "total_ms": sum(dur["pushdown"])},
    }

    def roof(k):
        kk = kernels[k]
        ach = kk["bytes"] / (kk["ms"] / 1e3) / 1e9 if kk["ms"] > 0 else 0.0
        return {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": traffic_for(kk["name"], kk["bytes"]), "kernel": kk["name"],
                "algorithmic_bytes_per_launch": int(kk["bytes"]), "avg_launch_ms": round(kk["ms"], 4),
                "launches_timed": kk["launches"], "total_ms_timed": round(kk["total_ms"], 3)}
    dominant = max(("count", "pass1", "scatter"), key=lambda k: kernels[k]["total_ms"])
    other = "count" if dominant != "count" else "pass1"

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32/f32 compares, u64 counts",
        "data": "synthetic, seeded (datagen; shapes of the paper's fact tables), resident in HBM",
        "config": workload_config(w.n, len(w.trees), len(accepted), world),
        "ms_per_estimate": round(count_ms / len(w.trees), 4),
        "ms_per_estimate_note": "the batched count's device time over its 256 probes",
        "roofline": roof(dominant),
        "roofline_other": roof(other),
        "roofline_scatter": dict(roof("scatter"), note="the events between the count pass and the call's end also "
                                 "hold the segment-sum and group-scan kernels (about 20 us a push-down)"),
        "pushdown_call": dict(roof("pushdown"), note="the whole push-down call (its count pass, offsets and "
                              "scatter) against the step's algorithmic bytes of that push-down: predicate columns, "
                              "projected values of the selected rows that are not predicate columns, written rows"),
        "roofline_issue": issue_roofline(count_kernel, w.n, count_ms, float((clk or {}).get("sm_max_mhz") or 2032.0)),
        "roofline_smem": smem_roofline(count_kernel, w.n, count_ms, float((clk or {}).get("sm_max_mhz") or 2032.0)),
        "gpu_launches": int(launches),
        "clocks": clk,
        "batch_plan_create_s": round(step.plan_s, 2),
    }
    if sur:
        out["surrogate"] = sur.summary()
    if rank == 0 and not args.no_extras:
        out["config5_extras"] = config5_extras(step, peak)
        out["config5_gated"] = config5_gated(step)
        out["config2"] = config2_measurements(sel, cfg2_table, peak)
        out["star_batch"] = star_batch(sel, peak, dev)
        out["config1_latency"] = config1_latency(sel, dev)
    if rank == 0 and not args.no_e2e:
        out["e2e"] = run_e2e(step, args, step_bytes)
        out["e2e_rows_to_host"] = run_e2e(step, args, step_bytes, rows_back=True)
    if rank == 0 and not args.no_cpu:
        ot = oracle_sample(w.table, w.trees, args.cpu_seconds, threads)
        gbs, secs = cpu_rate(ot, w.types, w.trees, w.proj, threads)
        out["cpu_baseline"] = {"value": round(gbs, 3), "unit": "GB/s", "cores": threads, "kind": "oracle",
                               "sample": f"first {ot.n_rows} rows of the same table, the same step "
                                         f"({len(w.trees)} counts + push-down row ids), {secs:.1f} s"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def kernel_case(sel, dev, args):
    """One kernel case launched twice (the profiles' captures take the second)."""
    if args.kernel_case == "mlp-forward":
        t = dg.gen_table("cfg2", dg.config2_specs(), 1_000_000, dev)
        T = sel.Table(t.columns)
        ctx = sel.Context()
        est = sel.Estimator(ctx, T, sample_rows=4096, seed=dg.MASTER_SEED)
        rng = np.random.default_rng(5)
        preds = [sel.Predicate(T, dg.random_dnf_predicate(dg.config2_specs(), rng)) for _ in range(4096)]
        feat, _ = est.featurize(preds)
        for _ in range(2):
            out = est.forward(feat)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.kernel_case, "probes": len(preds), "out": out[:2].tolist()}))
        return
    if args.kernel_case == "batch-cfg2":
        t = dg.gen_table("cfg2", dg.config2_specs(), args.rows, dev)
        trees = [dg.config2_predicate(s) for s in dg.CONFIG2_TARGETS]
    else:
        t = dg.gen_table("cfg5", dg.config5_specs(), args.rows, dev)
        trees = dg.config5_predicates()
    T = sel.Table(t.columns)
    ctx = sel.Context()
    if args.kernel_case.startswith("batch"):
        preds = [sel.Predicate(T, tr) for tr in trees]
        ctx.set_batch_kernel(2)
        plan = sel.BatchPlan(ctx, preds, [T] * len(preds), autotune=False)
        out = torch.zeros(len(preds), dtype=torch.int64, device=dev)
        for _ in range(2):
            plan.run(out)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.kernel_case, "rows": args.rows, "plan": plan.info(),
                          "counts": out[:8].tolist()}))
        return
    targets = np.logspace(-6, np.log10(0.9), len(trees))
    i = int(np.argmin(np.abs(np.log(targets) - np.log(args.case_s))))
    proj = [t.index(c) for c in dg.CONFIG5_PROJECTION]
    # the step's maxSize, or every row for a case above it (the write-heavy path)
    mr = int(math.floor(args.rows * MAX_SELECTIVITY)) if args.case_s <= MAX_SELECTIVITY else args.rows
    outs = [torch.empty(mr, dtype=t.columns[c].data.dtype, device=dev) for c in proj]
    ids = torch.empty(mr, dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    p = sel.Predicate(T, trees[i])
    for _ in range(2):
        ctx.pushdown_async(p, T, proj, mr, outs, ids, cnt)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.kernel_case, "rows": args.rows, "probe": i, "count": int(cnt.item()),
                      "predicate_columns": len(dg.tree_columns(trees[i]))}))


def estimator_curve(sel, dev, args):
    """Config 4 at its stated size: 2.2M probes labelled once by the count
    kernel on config 2's 300M-row table; networks trained from scratch on the
    first 20k, 200k and 2M, tau chosen on the same 100k validation probes,
    all scored on the same 100k test probes."""
    table = dg.gen_table("cfg2", dg.config2_specs(), args.cfg2_rows, dev)
    T = sel.Table(table.columns)
    ctx = sel.Context()
    n_train, n_val, n_test = 2_000_000, 100_000, 100_000
    trees = estimator_workload(n_train + n_val + n_test, "bench_estimator_curve")
    preds = [sel.Predicate(T, t) for t in trees]
    t0 = time.perf_counter()
    counts = np.array(sel.count_many(ctx, preds, T), dtype=np.uint64)
    label_s = time.perf_counter() - t0
    val = slice(n_train, n_train + n_val)
    curve = []
    for m in (20_000, 200_000, 2_000_000):
        sub_p = preds[:m] + preds[val] + preds[n_train + n_val:]
        sub_c = np.concatenate([counts[:m], counts[val], counts[n_train + n_val:]])
        _, _, _, quality, _ = train_and_gate(sel, ctx, T, sub_p, sub_c, m, n_val, n_test)
        curve.append(quality)
        print(json.dumps({"n_train": m, **quality}), flush=True)
    print(json.dumps({"estimator_curve": curve, "labels": len(preds), "label_seconds": round(label_s, 1),
                      "ms_per_label": round(label_s * 1e3 / len(preds), 4),
                      "workload": "config 4: random OR-of-AND probes (<= 6 leaves, <= 3 groups) on config 2's "
                                  f"{args.cfg2_rows}-row table, labels from the count kernel"}))


def run_e2e(step: OurStep, args, step_bytes, rows_back=False):
    """The same step through the C ABI with the table in pinned HOST memory:
    every step copies the columns host->device and its result (the exact
    counts and the push-downs' counts) back; with rows_back, every
    push-down's rows too.  Two device copies of the table: step k + 1's upload
    (on its own stream) runs while step k computes, and starts only after the
    step that last read that copy (k - 1) has finished; push-down rows go back
    on a copy stream while the next push-down runs (OurStep.run)."""
    w, sel = step.w, step.sel
    host_cols = [torch.empty_like(c.data, device="cpu").pin_memory() for c in w.table.columns]
    for h, c in zip(host_cols, w.table.columns):
        h.copy_(c.data)
    # host sinks for the rows (each push-down's rows land at their start) and a
    # copy stream: the rows of push-down k are copied back while the next ones
    # run, out of a 16 GB device ring of output regions
    if rows_back:
        step.host_out = [torch.empty(o.numel(), dtype=o.dtype).pin_memory() for o in step.out_cols + [step.out_ids]]
        step.e2e_ring = DeviceRing(16 << 30, w.table.columns[0].data.device)
        step.copy_stream = torch.cuda.Stream()
    dev_cols = [[c.data for c in w.table.columns], [torch.empty_like(c.data) for c in w.table.columns]]
    tabs = [step.T, sel.Table([dg.Column(c.spec, d, c.dictionary) for c, d in zip(w.table.columns, dev_cols[1])])]
    up = torch.cuda.Stream()
    uploaded, released = [None, None], [None, None]

    def upload(b):
        with torch.cuda.stream(up):
            if released[b] is not None:
                up.wait_event(released[b])
            for h, c in zip(host_cols, dev_cols[b]):
                c.copy_(h, non_blocking=True)
            uploaded[b] = torch.cuda.Event()
            uploaded[b].record(up)

    def one_step(k):
        b = k % 2
        cur = torch.cuda.current_stream()
        cur.wait_event(uploaded[b])
        _, _, d2h = step.run(e2e=True, T=tabs[b], rows_back=rows_back)
        released[b] = torch.cuda.Event()
        released[b].record(cur)
        return d2h

    h2d = sum(h.numel() * h.element_size() for h in host_cols)
    for b in (0, 1):                    # untimed: each copy's batch plan is built on its first step
        upload(b)
        one_step(b)
    torch.cuda.synchronize()
    k = max(1, args.steps)              # as many steps as the device-timed region
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    d2h = 0
    upload(0)
    for i in range(k):
        if i + 1 < k:
            upload((i + 1) % 2)
        d2h = one_step(i)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / k
    del host_cols, dev_cols, tabs
    step.host_out = None
    step.e2e_ring = None
    torch.cuda.empty_cache()
    return {"value": round(step_bytes / (ms / 1e3) / 1e9, 2), "unit": "GB/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": round(ms, 3), "steps": k,
            "result_to_host": ("the exact counts, the push-downs' counts and every push-down's rows" if rows_back else
                               "the exact counts and the push-downs' counts; the materialised rows stay on the device "
                               "for the rest of the query (Algorithm 1 materialises while R is on the GPU)"),
            "overlap": ("step k + 1's table upload" + (" and each push-down's copy-back" if rows_back else "") +
                        " run during step k's kernels (two device copies of the table" +
                        ("; push-down outputs in a 16 GB device ring)" if rows_back else ")"))}


def replica_throughput(elapsed_ms: float, step_bytes: int, steps: int, world: int, device) -> tuple:
    """Replicas (one per GPU, each over its own table): the job's time is the
    slowest rank's (all-reduce MAX), its throughput all ranks' bytes over it."""
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed_ms = float(tt.item())
        dist.barrier()
    return elapsed_ms, step_bytes * steps * world / (elapsed_ms / 1e3) / 1e9


def workload_config(n: int, probes: int, pushed: int, world: int = 1) -> dict:
    """The bench's config object (both arms)."""
    return {"workload": f"config5 table: {n} rows x 6 cols (3 i32 U/Zipf1.1/U, 2 f32 N/U, dict-1000 Zipf), "
                        f"24 B/row; {probes} probes OR of 1-3 ANDs, s log-spaced in [1e-6, 0.9]; push-down of "
                        f"{list(dg.CONFIG5_PROJECTION)} when count <= floor(n*{MAX_SELECTIVITY})",
            "n_rows": n, "table_bytes": n * 24, "probes": probes, "pushed_down": pushed,
            "max_rows": int(math.floor(n * MAX_SELECTIVITY)),
            "l2": "inputs larger than L2 (table 28.8 GB vs 126 MB L2), no flush needed",
            "parallelism": f"replicas{world}" if world > 1 else "single"}


def run_reference(args, threads):
    """The oracle as it stands, on the host cores, on a bounded sample per step."""
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    n = args.rows
    w_tab = dg.gen_table("cfg5", dg.config5_specs(), min(n, 50_000_000), dev)
    trees = dg.config5_predicates()
    types = [c.type for c in w_tab.columns]
    proj = [w_tab.index(c) for c in dg.CONFIG5_PROJECTION]
    per_step = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    ot = oracle_sample(w_tab, trees, per_step, threads)
    del w_tab
    for _ in range(args.warmup):
        oracle_step(ot, trees, MAX_SELECTIVITY, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        counts, accepted = oracle_step(ot, trees, MAX_SELECTIVITY, threads)
    dt = (time.perf_counter() - t0) / args.steps
    b, pds = algorithmic_bytes(types, ot.n_rows, trees, counts, accepted, proj)
    gbs = (b + sum(pds)) / dt / 1e9
    sample = (f"first {ot.n_rows} of {n} rows of the config 5 table per step, {len(trees)} counts + push-down "
              f"row ids")
    out = {"impl": "reference", "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "i32/f32 compares, u64 counts",
           "data": "synthetic, seeded (datagen)",
           "config": workload_config(n, len(trees), len(accepted), args.gpus),
           "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
