#!/usr/bin/env python3
"""Benchmark of the FuseFSS online hot path on one B300.

Workload (default): all nonlinearities of one BERT-base layer at batch 1,
seq 128 (GeLU on 128x3072, softmax nExp on 12x128x128, reciprocal on 12x128,
LayerNorm rsqrt on 128), one plain fused-gate launch per operator, both
parties on this GPU.  A step evaluates every operator once on fresh one-time
keys (generated by the GPU dealer before the timed region; dealer throughput
is reported separately).  Metric: FSS-evaluated elements/s (both parties,
open + packed comparison + interval lookup + Horner/Beaver).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank runs an independent replica of the workload
on its own GPU (weak scaling, no data-path collective); the timed region is
bracketed by barriers and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Per AES-128 block of the shared-memory T-table code with byte-permute +
# multiply-add addressing, measured by ncu on the AES-only micro-kernel
# (smsp__inst_executed_pipe_alu.sum and shared wavefronts x 32 / blocks):
ALU_OPS_PER_AES = 240
LDS_PER_AES = 160
SMS = 148


def _measured_peaks():
    """The measured peaks of the B300s this runs on (MEASURED_PEAKS.json at
    the repository root: STREAM-style copy bandwidth and the maximum SM
    clock), else the recorded fallback figures."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2032.0)), "measured"
    except (OSError, ValueError, KeyError):
        return 6400.0, 2032.0, "fallback"


HBM_GBS, SM_MAX_MHZ, PEAKS_BASIS = _measured_peaks()
# gate_kernel DRAM bytes (read + write) per element by spec, from ncu
# captures of small launches of the same spec and layout
# (profiles/gate_kernel_nexp16_gelu8_a64.md); retaken whenever the kernel
# changes
# The AES form of every walk, per spec: the measured forms are the T-table
# addressing variants and the bitsliced code (roofline.aes_microkernel_blocks_per_s);
# the interleaved T-table form is the fastest on every pipe, and the bitsliced
# form (32 independent blocks per thread) cannot run a walk, which chains one
# block per tree level.
AES_FORM = {"walks": "t_table_interleaved", "chosen_by": "micro-kernel rates measured in this run",
            "alternatives": ["t_table_shift_mask", "t_table_permute_mad", "bitsliced_lop3 (not a walk form)"]}
# spec -> (DRAM bytes read + written per element, elements of the ncu capture),
# for the kernel as it stands; a spec without a capture of this kernel
# reports traffic null.  (The last capture, 38,367 B per nExp arity-64
# element pair, was of the walks that branched around their predicated
# correction-word loads; the branch-free form reads the same lines but has
# not been captured.)
GATE_DRAM_BYTES_PER_ELEM = {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["bert_layer", "gelu4", "exp_small", "gelu_small", "bert_rescale"],
                    default="bert_layer")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--served-requests", type=int, default=16)
    ap.add_argument("--served-layers", type=int, default=1)
    ap.add_argument("--no-served-plain", action="store_true",
                    help="skip the plain per-operator run of the served trace")
    ap.add_argument("--no-large", action="store_true", help="skip the streamed large-layer run")
    ap.add_argument("--gpt2-layers", type=int, default=1, help="layers per request in the 32-request batch")
    ap.add_argument("--no-gpt2", action="store_true", help="skip the 32-request GPT-2 batch run")
    ap.add_argument("--no-xhat", action="store_true", help="skip the x^-basis variant run")
    ap.add_argument("--no-serial", action="store_true",
                    help="skip the streamed forms' second pass that times the dealer and the evaluation apart")
    ap.add_argument("--no-rescale", action="store_true", help="skip the layer-rescale (ARS) run")
    ap.add_argument("--no-blocks", action="store_true", help="skip the softmax / LayerNorm block runs")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the cost model's work split (no measured tuning before the timed region)")
    ap.add_argument("--slots", type=int, default=0,
                    help="force the gate's work split (slots per element) for every call (profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-work budget per op sample")
    ap.add_argument("--elements", type=int, default=0,
                    help="elements of the exp_small / gelu_small profiling workloads (default 65536)")
    ap.add_argument("--tuning-from", default="",
                    help="replay the DCF arity, key layout and tuning record of each operator from the JSON "
                         "line of an earlier run of the same workload (for a run under a profiler, whose "
                         "serialised launches distort the tuner's timings)")
    ap.add_argument("--records", action="store_true",
                    help="with --dcf-bits N: lay the lookup keys out as per-child records")
    ap.add_argument("--dcf-bits", type=int, default=0, choices=[0, 1, 2, 3, 4, 5, 6],
                    help="DCF input bits per tree level of every gate; 0: the library measures each "
                         "spec at arities 2 to 64 and keeps the fastest for its form")
    return ap.parse_args()


def workload(name, elements=0):
    from paper_2606_09551_b300 import inputs as I
    if name == "exp_small":
        # profiling case: the BERT-layer softmax nExp spec on 65,536 elements
        # (6.6 GB of keys at arity 4, 8.8 GB at arity 8), or the first `elements`
        n = elements or 65536
        c = I.bert_layer()[1]
        c.x = c.x[:n]
        return [c], {"workload": "nexp16_%d" % n, "spec": "nExp-16 k=24 f=12 d=3", "elements": n,
                     "form": "plain"}
    if name == "gelu_small":
        # profiling case: the BERT-layer GeLU-8 spec on the first 65,536 elements (or `elements`)
        n = elements or 65536
        c = I.bert_layer()[0]
        c.x = c.x[:n]
        return [c], {"workload": "gelu8_%d" % n, "spec": "GeLU-8 k=16 f=12 d=2", "elements": n, "form": "plain"}
    if name == "bert_rescale":
        # the shift gates of one BERT-base layer alone (each matrix product's
        # output shifted right by 12 on a 32-bit signed view)
        calls = I.bert_layer_rescales()
        return calls, {"workload": "bert_base_layer_rescales", "spec": "ARS k=32 s=12",
                       "ops": {c.name: c.n for c in calls}, "elements": sum(c.n for c in calls),
                       "form": "plain per-product launches"}
    if name == "gelu4":
        return I.single_gelu4(), {"workload": "gelu4_single_op", "spec": "GeLU-4 k=16 f=12 d=2",
                                  "elements": 65536, "form": "plain"}
    calls = I.bert_layer()
    return calls, {"workload": "bert_base_layer_nonlinearities", "seq_len": 128, "hidden": 768,
                   "heads": 12, "mlp": 3072, "batch": 1,
                   "ops": {c.name: {"elements": c.n, "spec": c.spec.name, "k": c.spec.k, "m": c.spec.m,
                                    "degree": c.spec.degree} for c in calls},
                   "elements": sum(c.n for c in calls), "form": "plain per-operator launches",
                   "ring": "Z_2^64", "frac_bits": 12}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    """Samples the SM clock and the clock-event reasons of one GPU every
    10 ms while the timed region runs (NVML reads only; nothing is set).
    Falls back to `nvidia-smi -lms 200` when NVML cannot be used."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.thread = None
        self.rows = []
        self.nvml_error = None

    def _nvml_handle(self):
        """NVML through the driver's libnvidia-ml (read-only queries); the
        device is matched by PCI bus id, which survives device masking."""
        import ctypes
        import torch
        L = ctypes.CDLL("libnvidia-ml.so.1")
        if L.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit_v2 failed")
        h = ctypes.c_void_p()
        rc = -1
        try:
            pr = torch.cuda.get_device_properties(self.gpu)
            bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
            rc = L.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h))
        except AttributeError:
            pass
        if rc != 0 and L.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(h)) != 0:
            raise RuntimeError("no NVML handle for GPU %d" % self.gpu)
        return L, h

    def _loop(self, L, h, first):
        import ctypes
        NVML_CLOCK_SM = 1
        # clock-event reason bits of the NVML API
        bits = (0x8, 0x40, 0x20, 0x4)   # hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
        reasons_fn = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            L.nvmlDeviceGetCurrentClocksThrottleReasons
        mx, sm, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        L.nvmlDeviceGetMaxClockInfo(h, NVML_CLOCK_SM, ctypes.byref(mx))
        while not self.stop.is_set():
            if L.nvmlDeviceGetClockInfo(h, NVML_CLOCK_SM, ctypes.byref(sm)) != 0 or \
                    reasons_fn(h, ctypes.byref(rs)) != 0:
                return
            self.rows.append((float(sm.value), float(mx.value),
                              [n for n, b in zip(self.NAMES, bits) if rs.value & b]))
            first.set()
            self.stop.wait(0.010)

    def __enter__(self):
        import threading
        try:
            lib, h = self._nvml_handle()
            self.stop, first = threading.Event(), threading.Event()
            self.thread = threading.Thread(target=self._loop, args=(lib, h, first), daemon=True)
            self.thread.start()
            if first.wait(2.0):
                return self
            self.stop.set()
            self.thread.join(2.0)
            raise RuntimeError("no NVML sample within 2 s")
        except Exception as ex:
            self.nvml_error = "%s: %s" % (type(ex).__name__, ex)
            self.thread = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.thread is not None:
            self.stop.set()
            self.thread.join(2.0)
            return
        out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
        for r in csv.reader(io.StringIO(out or "")):
            if len(r) < 9:
                continue
            try:
                self.rows.append((float(r[1]), float(r[2]),
                                  [n for n, v in zip(self.NAMES, r[5:9]) if v.strip().lower() == "active"]))
            except ValueError:
                continue

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = sorted({n for _, _, rs in self.rows for n in rs})
        return {"sm_mhz": statistics.median(r[0] for r in self.rows), "sm_max_mhz": self.rows[-1][1],
                "reasons": reasons, "samples": len(self.rows),
                "source": "nvml 10 ms" if self.thread is not None else "nvidia-smi 200 ms (nvml: %s)" % self.nvml_error}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, threads over element chunks
# ---------------------------------------------------------------------------

def oracle_rates(calls, cpu_seconds, threads=None):
    """Per-op oracle eval seconds per element (wall, all threads), on a
    bounded sample of each op's elements.  Keys for the sample come from the
    oracle dealer before timing."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    import oracle as O
    from paper_2606_09551_b300 import inputs as I
    threads = threads or os.cpu_count() or 1
    out, desc = {}, {}
    for c in calls:
        o = O.Spec(**c.spec.descriptor())
        # single-core cost estimate: 0.45 us per AES block, both parties
        per_elem = 0.45e-6 * 2 * (sum(f for f, _, _ in o.queries())
                                  + (o.M - 1) * (o.k * (1 + (o.p + 1) // 2) + (o.p + 1) // 2))
        ns = int(min(c.n, max(threads, cpu_seconds / max(per_elem, 1e-9))))
        chunks = [(i * ns // threads, (i + 1) * ns // threads) for i in range(threads)]
        chunks = [ch for ch in chunks if ch[1] > ch[0]]

        def deal(ch):
            return O.dealer(o, I.KEY_SEED, c.call_id, ch[0], ch[1] - ch[0], c.x[ch[0]:ch[1]])

        with ThreadPoolExecutor(len(chunks)) as ex:
            dealt = list(ex.map(deal, chunks))

        def ev(d):
            k0, k1, x0, x1 = d
            return O.eval_pair(o, k0, k1, x0, x1)

        t0 = time.perf_counter()
        with ThreadPoolExecutor(len(chunks)) as ex:
            list(ex.map(ev, dealt))
        dt = time.perf_counter() - t0
        out[c.name] = dt / ns
        desc[c.name] = ns
    return out, desc, threads


def cpu_baseline(calls, cpu_seconds):
    rates, sample, threads = oracle_rates(calls, cpu_seconds)
    total = sum(c.n for c in calls)
    t = sum(c.n * rates[c.name] for c in calls)
    ar = {c.name: 1 << c.spec.dcf_bits for c in calls}
    return {"value": total / t, "unit": "elements/s", "cores": threads, "kind": "oracle",
            "sample": "oracle eval_pair (both parties) on the first " +
                      ", ".join(f"{sample[k]} {k} (DCF arity {ar[k]})" for k in sample) +
                      " elements; per-op s/element combined with the full layer's op mix"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2606_09551_b300 import build as B
    from paper_2606_09551_b300 import fusefss as F
    from paper_2606_09551_b300 import inputs as I

    B.build()
    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    ctx = F.Context(local_rank)
    calls, config = workload(args.workload, args.elements)
    # the DCF arity per spec (resident keys: form 0), then the measured launch
    # shape, before any timing: the library times the gate under every work
    # split (and, with --dcf-bits 0, every arity) on throw-away samples
    replay = load_tuning(args.tuning_from) if args.tuning_from else None
    css = compile_specs(ctx, calls, args, form=0, replay=replay)
    tuning = None
    if not args.no_autotune:
        tuning = {}
        for c in calls:
            cs = css[c.name]
            t0 = time.perf_counter()
            if replay and c.name in replay:
                tune = {k: replay[c.name][k] for k in ("slots", "tile_us", "fixed_us", "sample_elems", "dealer_ms")}
            else:
                tune = cs.autotune()
            tuning[c.name] = dict(tune, elements=c.n, slots_tuned=cs.gate_slots(c.n), tune_s=time.perf_counter() - t0,
                                  aes_form=AES_FORM, dcf_bits=cs.spec.dcf_bits, lookup_records=cs.records,
                                  dcf_bits_chosen_by=cs.arity_choice)
    if args.slots:
        ctx.set_slots(args.slots)
        config = dict(config, forced_slots=args.slots)
    xp = {c.name: torch.from_numpy(c.x).to(dev) for c in calls}
    total = sum(c.n for c in calls)
    stream = torch.cuda.current_stream()

    class KeySet:
        def __init__(self):
            self.k = {}
            for c in calls:
                cs = css[c.name]
                x0 = torch.empty(c.n, dtype=torch.uint64, device=dev)
                self.k[c.name] = (F.Keys(cs, c.n, 0), F.Keys(cs, c.n, 1), x0, torch.empty_like(x0))

        def generate(self, tag):
            for c in calls:
                k0, k1, x0, x1 = self.k[c.name]
                F.keygen(ctx, css[c.name], I.KEY_SEED, c.call_id + 16 * tag, c.n, k0, k1, xp[c.name], x0, x1)

    outs = {}
    for c in calls:
        y0 = torch.empty(c.n * c.spec.n_out, dtype=torch.uint64, device=dev)
        z0 = torch.empty(c.n, dtype=torch.uint32, device=dev)
        outs[c.name] = (y0, torch.empty_like(y0), z0, torch.empty_like(z0))
    comm = torch.zeros(2, dtype=torch.uint64, device=dev)

    def step(ks, evs=None):
        for i, c in enumerate(calls):
            k0, k1, x0, x1 = ks.k[c.name]
            y0, y1, z0, z1 = outs[c.name]
            if evs is not None:
                evs[i][0].record(stream)
            F.eval_pair(ctx, css[c.name], k0, k1, x0, x1, y0, y1, z0, z1, comm)
            if evs is not None:
                evs[i][1].record(stream)

    # warm-up: fresh keys before every warm-up step (keys are one-time)
    warm = KeySet()
    for w in range(args.warmup):
        warm.generate(1000 + w)
        step(warm)
    torch.cuda.synchronize()
    del warm
    # dealer: as many key sets as HBM holds (one-time keys: one set per step),
    # timed separately
    set_bytes = sum(2 * css[c.name].key_bytes(c.n) for c in calls)
    G = sets_that_fit(set_bytes, args.steps)
    sets = [KeySet() for _ in range(G)]
    kg0, kg1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kg0.record(stream)
    for s, ks in enumerate(sets):
        ks.generate(s)
    kg1.record(stream)
    torch.cuda.synchronize()
    keygen_ms = kg0.elapsed_time(kg1) / G

    # timed region: K steps on fresh keys, inputs resident in HBM (keys > L2
    # every step); when K sets do not fit, the K steps run in groups of G
    # sets, the dealer refilling them between groups outside the timing
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
            for _ in calls] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_ms = 0.0
    with ClockSampler(local_rank) as clk:
        for g0 in range(0, args.steps, G):
            gs = min(G, args.steps - g0)
            if g0 > 0:
                for s in range(gs):
                    sets[s].generate(g0 + s)
            torch.cuda.synchronize()
            barrier(world)
            torch.cuda.synchronize()
            t0.record(stream)
            for s in range(gs):
                step(sets[s], evs[g0 + s])
            t1.record(stream)
            torch.cuda.synchronize()
            barrier(world)
            total_ms += t0.elapsed_time(t1)
    ms = total_ms / args.steps
    ms = max_over_ranks(ms, world, dev)
    per_op_ms = {c.name: statistics.mean(evs[s][i][0].elapsed_time(evs[s][i][1]) for s in range(args.steps))
                 for i, c in enumerate(calls)}
    comm_b = [int(v) for v in comm.cpu().tolist()]

    # end to end through the public API: each step's input shares come from
    # page-locked host memory and its output shares go back there, through
    # ffss_eval_pair_host (copy in, gate, copy out, queued on a stream); the
    # calls alternate between two streams so one's copies overlap another's
    # gate
    e2e = None
    if not args.no_e2e:
        ne = len(sets)                         # steps on resident fresh key sets
        for s, ks in enumerate(sets):
            ks.generate(100 + s)
        torch.cuda.synchronize()
        host_in = [{c.name: (ks.k[c.name][2].cpu().pin_memory(), ks.k[c.name][3].cpu().pin_memory()) for c in calls}
                   for ks in sets]
        host_out = {}
        for c in calls:
            y0, y1, z0, z1 = outs[c.name]
            host_out[c.name] = tuple(torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (y0, y1, z0, z1))
        h2d = sum(2 * 8 * c.n for c in calls)
        d2h = sum(2 * 8 * c.n * c.spec.n_out + 2 * 4 * c.n for c in calls)
        lanes = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]
        # calls alternate between the two streams in issue order; an
        # operator's host output buffers are used by every other step on
        # each stream, so each stream keeps its own (allocated before timing)
        host_out2 = [host_out, {c.name: tuple(torch.empty(t.shape, dtype=t.dtype).pin_memory()
                                              for t in host_out[c.name]) for c in calls}]
        # untimed warm-up: the library's staging slots grow to their size here
        for q in range(2):
            c = calls[q % len(calls)]
            k0, k1, _, _ = sets[0].k[c.name]
            F.eval_pair_host(ctx, css[c.name], k0, k1, *host_in[0][c.name], *host_out2[q][c.name],
                             stream=lanes[q])
            torch.cuda.synchronize()
            sets[0].generate(100)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for ln in lanes:
            ln.wait_event(e0)
        q = 0
        for s in range(ne):
            for i, c in enumerate(calls):
                k0, k1, _, _ = sets[s].k[c.name]
                F.eval_pair_host(ctx, css[c.name], k0, k1, *host_in[s][c.name], *host_out2[q % 2][c.name],
                                 stream=lanes[q % 2])
                q += 1
        for ln in lanes:
            stream.wait_stream(ln)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ems = max_over_ranks(e0.elapsed_time(e1) / ne, world, dev)
        e2e = {"value": total * world / (ems * 1e-3), "unit": "elements/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": ems, "steps": ne,
               "api": "ffss_eval_pair_host per operator call (page-locked host buffers), calls alternating "
                      "between two streams"}
        del host_in

    # batched form: the same layer as ONE persistent launch per step (graph replay)
    batched = None
    if not args.no_batch:
        bt = F.Batch(ctx, max(len(calls), 1))

        def batch_step(ks):
            bt.eval([(css[c.name],) + ks.k[c.name] + outs[c.name] for c in calls], comm=None)

        # warm-up on the first resident set (a second set may not fit beside
        # them), which is dealt fresh again below before it is timed
        for w in range(2):                       # captures both plan slots' graphs
            sets[0].generate(2000 + w)
            batch_step(sets[0])
        for s, ks in enumerate(sets):
            ks.generate(300 + s)
        torch.cuda.synchronize()
        bev = [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(len(sets))]
        barrier(world)
        torch.cuda.synchronize()
        for s in range(len(sets)):
            bev[s][0].record(stream)
            batch_step(sets[s])
            bev[s][1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        steps_ms = sorted(b0.elapsed_time(b1) for b0, b1 in bev)
        bms = max_over_ranks(statistics.mean(steps_ms), world, dev)
        batched = {"value": total * world / (bms * 1e-3), "unit": "elements/s", "ms_per_step": bms,
                   "step_ms_p50": statistics.median(steps_ms), "step_ms_max": steps_ms[-1],
                   "vs_plain": ms / bms, "launches_per_step": 1,
                   "form": "one persistent work-queue launch per layer, CUDA graph replay"}
        bt.close()

    ks = k0 = k1 = None                          # the loops' last references to a key set
    del sets
    torch.cuda.empty_cache()

    # x^-basis payload variant: the same layer, local evaluation on the public
    # x^ (no Beaver rounds, no triples); plain per-operator launches
    xhat = None
    if not args.no_xhat:
        vcss = {c.name: F.CompiledSpec(c.spec.variant(True), ctx, records=css[c.name].records) for c in calls}
        if not args.no_autotune:
            for cs in vcss.values():
                cs.autotune()
        # as many timed key sets as fit beside one warm-up set; when only one
        # set fits, the warm-up set is dealt again (untimed) and timed once
        nfit = sets_that_fit(sum(2 * vcss[c.name].key_bytes(c.n) for c in calls), args.steps + 1)
        nx = max(1, nfit - 1)

        def vdeal(s_):
            ks = {}
            for c in calls:
                x0 = torch.empty(c.n, dtype=torch.uint64, device=dev)
                x1 = torch.empty_like(x0)
                k0, k1 = F.Keys(vcss[c.name], c.n, 0), F.Keys(vcss[c.name], c.n, 1)
                F.keygen(ctx, vcss[c.name], I.KEY_SEED, c.call_id + 16 * (400 + s_), c.n, k0, k1, xp[c.name], x0, x1)
                ks[c.name] = (k0, k1, x0, x1)
            return ks

        vcomm = torch.zeros(2, dtype=torch.uint64, device=dev)

        def vstep(ks, cm=None):
            for c in calls:
                F.eval_pair(ctx, vcss[c.name], *ks[c.name], *outs[c.name], cm)

        if nfit >= 2:
            vsets = [vdeal(s_) for s_ in range(nx + 1)]
            vstep(vsets[-1])                  # warm-up
        else:
            vsets = [vdeal(nx)]
            vstep(vsets[0])                   # warm-up
            del vsets
            torch.cuda.empty_cache()
            vsets = [vdeal(0)]
        torch.cuda.synchronize()
        barrier(world)
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        for s_ in range(nx):
            vstep(vsets[s_], vcomm)
        v1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        vms = max_over_ranks(v0.elapsed_time(v1) / nx, world, dev)
        xhat = {"value": aggregate(total, vms, world), "unit": "elements/s", "ms_per_step": vms,
                "vs_standard": ms / vms,
                "comm_bytes_per_party_per_step": int(vcomm.cpu().tolist()[0]) // nx, "steps": nx,
                "comm_bytes_per_party_per_step_standard": comm_b[0] // (args.steps + args.warmup),
                "key_bytes_per_step": sum(2 * vcss[c.name].shape.key_bytes_per_elem * c.n for c in calls),
                "online_rounds": 1,
                "form": "dealer re-expands P(x^ - r) in the public x^; lookup returns shares of those "
                        "coefficients; Horner on x^ is local (no triples, one opening round)"}
        del vsets
        torch.cuda.empty_cache()

    rescale = None
    if not args.no_rescale:
        rescale = run_rescales(ctx, args, dev, stream, world)
    blocks = None
    if not args.no_blocks:
        blocks = run_blocks(ctx, args, dev, stream, world)

    served = large = gpt2 = None
    if not args.no_served:
        served = run_served(ctx, args, dev)
    if not args.no_large:
        large = run_large_layer(ctx, dev, args, no_serial=args.no_serial)
    if not args.no_gpt2:
        gpt2 = run_gpt2_batch(ctx, args, dev)

    # roofline of the dominant kernel (the op with the largest launch time)
    dom = max(calls, key=lambda c: per_op_ms[c.name])
    sh = css[dom.name].shape
    aes_launch = 2 * sh.aes_per_elem * dom.n
    key_bytes_launch = 2 * sh.key_bytes_per_elem * dom.n
    lop3_rate, _ = F.microbench(ctx, 0, 4096)
    aes_rates = {name: F.microbench(ctx, v + 1, 2048)[0]
                 for v, name in enumerate(("shift_mask", "permute_mad", "permute_mad_ptx", "permute_interleaved",
                                           "dealer_4block_calls"))}
    # the integer-ALU alternative: bitsliced AES (Boyar-Peralta S-box), 32
    # sliced chains per thread, checked against the T-table AES by the call
    aes_rates["bitsliced_lop3"] = F.microbench(ctx, 6, 256)[0]
    dom_s = per_op_ms[dom.name] * 1e-3
    roof = {
        # the AES that binds is the shared-memory T-table lookups: the LSU pipe
        # (on-chip; neither HBM nor a tensor pipe)
        "bound": "lsu", "kernel": f"gate_kernel ({dom.name}: {dom.spec.name}, {dom.n} elements)",
        "unit": "Gop/s",
        "aes_blocks_per_launch": aes_launch,
        "aes_blocks_per_s": aes_launch / dom_s,
        "aes_microkernel_blocks_per_s": aes_rates,
        "lop3_peak_gops_measured": lop3_rate / 1e9,
        # the key bytes the launch holds; a walk reads one child's correction
        # words of each level's 2^r, so DRAM moves far fewer (traffic, below)
        "key_bytes_per_launch": key_bytes_launch,
        "traffic": None,
    }
    # AES roofline: per SM a T-table block needs ALU_OPS_PER_AES integer-ALU
    # ops at 64/clock and LDS_PER_AES shared-memory lookups at 32/clock; the
    # slower pipe sets the block rate (148 SMs at the 2,032 MHz maximum clock).
    cyc = max(ALU_OPS_PER_AES / 64.0, LDS_PER_AES / 32.0)
    roof["achieved"] = aes_launch / dom_s / 1e9
    roof["peak"] = SMS * SM_MAX_MHZ * 1e6 / cyc / 1e9
    roof["unit"] = "G AES blocks/s"
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["peak_basis"] = ("derived: 148 SMs x 2032 MHz / max(%d ALU ops / 64 lanes, %d shared lookups / 32 banks) "
                          "per block; ops per block measured by ncu on the AES micro-kernel" % (ALU_OPS_PER_AES, LDS_PER_AES))
    # the same work against the integer-ALU pipe alone: the T-table block's
    # ALU ops at 64 per clock per SM (what the block would cost were the
    # lookups free), and the fastest AES measured on the ALU pipe only
    alu_peak = SMS * SM_MAX_MHZ * 1e6 / (ALU_OPS_PER_AES / 64.0) / 1e9
    roof["alu_only"] = {"peak": alu_peak, "frac": roof["achieved"] / alu_peak,
                        "basis": "148 SMs x 2032 MHz x 64 ALU ops per clock / %d ALU ops per T-table block" %
                                 ALU_OPS_PER_AES,
                        "bitsliced_measured": aes_rates["bitsliced_lop3"] / 1e9,
                        "frac_of_bitsliced": roof["achieved"] / (aes_rates["bitsliced_lop3"] / 1e9)}
    roof["hbm_peak_gbs"] = HBM_GBS
    roof["hbm_peak_basis"] = PEAKS_BASIS
    # DRAM traffic of this kernel per element, from an ncu capture of a
    # smaller launch of the same spec, scaled by elements (traffic grows in
    # proportion: one-time keys are read once, outputs written once)
    cap = GATE_DRAM_BYTES_PER_ELEM.get(dom.spec.name + ("_rec" if css[dom.name].records else ""))
    if cap is not None:
        per_elem, cap_n = cap
        roof["traffic"] = per_elem * dom.n
        roof["traffic_basis"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of gate_kernel on %s, "
                                 "%d elements, scaled to %d elements" % (dom.spec.name, cap_n, dom.n))
        roof["hbm_traffic_gbs"] = roof["traffic"] / dom_s / 1e9
        roof["hbm_traffic_frac_of_measured"] = roof["hbm_traffic_gbs"] / HBM_GBS

    res = {
        "metric": "FSS-evaluated elements/s per nonlinear op (both parties, online phase)",
        "value": aggregate(total, ms, world),
        "unit": "elements/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic (seeded activations; random masks, keys and triples from the GPU dealer)",
        "config": full_config(config, calls, world, args),
        "timing": {"key_sets_resident": G, "timed_groups": -(-args.steps // G)},
        "per_op_ms": per_op_ms,
        "autotune": tuning,
        "keygen": {"ms_per_step": keygen_ms, "elements_per_s": total / (keygen_ms * 1e-3)},
        "comm_bytes_per_party": comm_b,
        "network_projection": network_projection(calls, css, ms, comm_b, args.steps + args.warmup),
        "gpu_launches": args.steps * len(calls),
        "clocks": clk.summary(),
        "roofline": roof,
        "e2e": e2e,
        "batched": batched,
        "served": served,
        "large_layer": large,
        "gpt2_batch": gpt2,
        "xhat_variant": xhat,
        "rescale": rescale,
        "blocks": blocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        res["cpu_baseline"] = cpu_baseline(calls, args.cpu_seconds)
    return res


# ---------------------------------------------------------------------------
# served form: BERT-large-shaped requests, Poisson arrivals, key streaming
# ---------------------------------------------------------------------------

def _stream_aes(pending_ops, nlay):
    """Algorithmic AES blocks of a streamed run: (dealer, both parties online)."""
    deal = online = 0
    for ops in pending_ops:
        for cs, x, *_ in ops:
            deal += x.numel() * nlay * cs.shape.keygen_aes_per_elem
            online += x.numel() * nlay * 2 * cs.shape.aes_per_elem
    return deal, online


def load_tuning(path):
    """The per-operator autotune records of an earlier bench JSON line."""
    with open(path) as fh:
        line = [ln for ln in fh if ln.lstrip().startswith("{")][-1]
    return json.loads(line)["autotune"]


def compile_specs(ctx, calls, args, form, n_of=None, replay=None):
    """One compiled spec per call.  With --dcf-bits 0 (and tuning on) the
    library compiles each at DCF arities 2 to 64, tunes each and keeps the
    one with the least predicted time for the call's size (form 0: resident
    keys; form 1: keys dealt as they are used, so the dealer's time counts);
    every call's spec is replaced by the kept one.  Otherwise the given (or
    forced) arity, tuned unless --no-autotune.  replay: saved records by call
    name (load_tuning), installed instead of measuring."""
    from paper_2606_09551_b300 import fusefss as F
    css = {}
    for c in calls:
        n = n_of(c) if n_of else c.n
        if replay and c.name in replay:
            rec = replay[c.name]
            cs = F.CompiledSpec(c.spec.arity(rec["dcf_bits"]), ctx, records=bool(rec["lookup_records"]))
            cs.set_tune(rec)
            cs.arity_choice = "replayed (%s)" % rec.get("dcf_bits_chosen_by", "saved")
        elif args.dcf_bits == 0 and not args.no_autotune:
            cs = F.CompiledSpec(c.spec, ctx, best_for=(n, form))
            cs.arity_choice = "measured, form %d at %d elements" % (form, n)
        else:
            cs = F.CompiledSpec(c.spec.arity(args.dcf_bits) if args.dcf_bits else c.spec, ctx,
                                records=bool(args.dcf_bits and args.records))
            cs.arity_choice = "forced" if args.dcf_bits else "default"
            if not args.no_autotune:
                cs.autotune()
        c.spec = cs.spec
        css[c.name] = cs
    return css


def _compile_requests(ctx, reqs, args, n):
    """One compiled spec per operator of the requests (the served and streamed
    forms: keys dealt as they are used), its arity chosen for calls of n
    elements; every request's op takes the kept spec."""
    css = compile_specs(ctx, list(reqs[0].ops), args, form=1, n_of=lambda c: n)
    for rq in reqs:
        for op in rq.ops:
            op.spec = css[op.name].spec
    return css


def _request_ops(css, rq, dev):
    """The server's op tuples of one request: its seeded inputs on the device
    and output share buffers."""
    import torch
    ops = []
    for op in rq.ops:
        x = torch.from_numpy(op.x).to(dev)
        y = torch.empty(op.n * op.spec.n_out, dtype=torch.uint64, device=dev)
        z = torch.empty(op.n, dtype=torch.uint32, device=dev)
        ops.append((css[op.name], x, y, torch.empty_like(y), z, torch.empty_like(z)))
    return ops


def run_rescales(ctx, args, dev, stream, world):
    """The shift gates of one BERT-base layer (every matrix product's output
    shifted right by 12 on a 32-bit signed view): K steps of fresh keys dealt
    before the timed region, one fused launch per product."""
    import numpy as np
    import torch

    from paper_2606_09551_b300 import fusefss as F
    from paper_2606_09551_b300 import inputs as I
    calls = I.bert_layer_rescales()
    # one spec for every product, its arity chosen for the largest call
    cs = compile_specs(ctx, [calls[0]], args, form=0, n_of=lambda c: max(d.n for d in calls))[calls[0].name]
    for c in calls:
        c.spec = cs.spec
    total = sum(c.n for c in calls)
    xp = {c.name: torch.from_numpy(c.x).to(dev) for c in calls}
    outs = {}
    for c in calls:
        y0 = torch.empty(c.n, dtype=torch.uint64, device=dev)
        z0 = torch.empty(c.n, dtype=torch.uint32, device=dev)
        outs[c.name] = (y0, torch.empty_like(y0), z0, torch.empty_like(z0))
    sets = []
    for s_ in range(args.steps + 1):
        ks = {}
        for c in calls:
            x0 = torch.empty(c.n, dtype=torch.uint64, device=dev)
            x1 = torch.empty_like(x0)
            k0, k1 = F.Keys(cs, c.n, 0), F.Keys(cs, c.n, 1)
            F.keygen(ctx, cs, I.KEY_SEED, c.call_id + 16 * (600 + s_), c.n, k0, k1, xp[c.name], x0, x1)
            ks[c.name] = (k0, k1, x0, x1)
        sets.append(ks)
    comm = torch.zeros(2, dtype=torch.uint64, device=dev)

    def step(ks, cm=None):
        for c in calls:
            F.eval_pair(ctx, cs, *ks[c.name], *outs[c.name], cm)

    step(sets[-1])                            # warm-up
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s_ in range(args.steps):
        step(sets[s_], comm)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    # the last step's reconstruction against numpy's arithmetic shift (in-range inputs)
    ok = True
    for c in calls:
        y = (outs[c.name][0].cpu().numpy() + outs[c.name][1].cpu().numpy()).view(np.int64)
        ok &= bool(np.array_equal(y, np.right_shift(c.x.view(np.int64), 12)))
    sh = cs.shape
    aes = 2 * sh.aes_per_elem * total
    res = {"value": aggregate(total, ms, world), "unit": "elements/s", "ms_per_step": ms,
           "elements": total, "spec": "ARS k=32 s=12 (signed)",
           "ops": {c.name: c.n for c in calls},
           "aes_per_elem_per_party": sh.aes_per_elem,
           "aes_roofline_frac": aes / (ms * 1e-3) / _aes_roofline(),
           "key_bytes_per_elem_per_party": sh.key_bytes_per_elem,
           "comm_bytes_per_party_per_step": int(comm.cpu().tolist()[0]) // args.steps,
           "reconstruction_equals_numpy_right_shift": ok,
           "form": "plain per-product launches; keys dealt on the GPU before the timed region"}
    del sets
    torch.cuda.empty_cache()
    return res


def run_blocks(ctx, args, dev, stream, world):
    """The composed blocks of one BERT-base layer at seq 128: attention
    softmax over 12 x 128 rows of 128 scores, and one LayerNorm over 128
    rows of 768.  Fresh keys are dealt (untimed) before each evaluation;
    CUDA events bracket the evaluations only."""
    import numpy as np
    import torch

    from paper_2606_09551_b300 import fusefss as F
    from paper_2606_09551_b300 import inputs as I
    from paper_2606_09551_b300 import specs as S
    rng = np.random.default_rng(I.MASTER_SEED + 7)
    out = {}

    def timed(plan, x, n, call_base):
        x0 = rng.integers(0, 2 ** 64, size=x.size, dtype=np.uint64)
        X0 = torch.from_numpy(x0).to(dev)
        X1 = torch.from_numpy(x.reshape(-1) - x0).to(dev)
        Y0 = torch.empty(n, dtype=torch.uint64, device=dev)
        Y1 = torch.empty_like(Y0)
        comm = torch.zeros(2, dtype=torch.uint64, device=dev)
        plan.keygen(I.KEY_SEED, call_base)
        plan.eval(X0, X1, Y0, Y1)                       # warm-up
        total = 0.0
        for s_ in range(args.steps):
            plan.keygen(I.KEY_SEED, call_base + 64 * (s_ + 1))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            plan.eval(X0, X1, Y0, Y1, comm)
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        ms = max_over_ranks(total / args.steps, world, dev)
        y = (Y0.cpu().numpy() + Y1.cpu().numpy()).view(np.int64) / 2.0 ** 12
        return ms, y, int(comm.cpu().tolist()[0]) // args.steps

    def aes_of(gates, counts):
        return sum(2 * g.shape.aes_per_elem * c for g, c in zip(gates, counts))

    def gates_for(specs, sizes):
        """The block's gates, each with its arity chosen for its call size."""
        calls = [I.OpCall(f"g{i}", sp_, np.zeros(1, np.uint64), 0) for i, sp_ in enumerate(specs)]
        css = compile_specs(ctx, calls, args, form=0, n_of=lambda c: sizes[int(c.name[1:])])
        return [css[c.name] for c in calls]

    # softmax
    rows, L = 12 * 128, 128
    sp = S.softmax_specs()
    names = ["relu", "exp", "shift_e", "recip", "shift_t", "shift_p"]
    gates = gates_for([sp[k] for k in names], [rows * L // 2, rows * L, rows * L, rows, rows, rows * L])
    sm = F.Softmax(ctx, gates, rows, L)
    scores = 2.0 * rng.standard_normal((rows, L))
    ms, y, cb = timed(sm, S.encode(scores.reshape(-1), 12), rows * L, 2000)
    ref = np.exp(scores - scores.max(axis=1, keepdims=True))
    ref /= ref.sum(axis=1, keepdims=True)
    tree = 0
    n = L
    while n > 1:
        tree += rows * (n // 2)
        n = n // 2 + n % 2
    aes = aes_of(gates, [tree, rows * L, rows * L, rows, rows, rows * L])
    info = sm.info()
    out["softmax"] = {"value": aggregate(rows * L, ms, world), "unit": "elements/s", "ms_per_block": ms,
                      "shape": [rows, L], "tree_rounds": info["rounds"], "gate_elements": info["gate_elements"],
                      "key_bytes": info["key_bytes"], "comm_bytes_per_party": cb,
                      "comm_bytes_per_elem_per_party": cb / (rows * L),
                      "aes_blocks": aes, "aes_roofline_frac": aes / (ms * 1e-3) / _aes_roofline(),
                      "max_abs_err_vs_float64": float(np.abs(y.reshape(rows, L) - ref).max()),
                      "form": "comparison-tree max (ReLU gates), nExp, row sums, Recip, Beaver product, "
                              "rounding shift gates; one plan, keys dealt before each evaluation"}
    sm.close()
    # the same block with one Newton step refining the reciprocal
    ngates = gates_for([sp[k] for k in ("shift_n1", "shift_n2")], [rows, rows])
    smn = F.Softmax(ctx, gates, rows, L, newton_gates=ngates, newton=1)
    ms_n, y_n, cb_n = timed(smn, S.encode(scores.reshape(-1), 12), rows * L, 2500)
    aes_n = aes + aes_of(ngates, [rows, rows])
    out["softmax_newton"] = {"value": aggregate(rows * L, ms_n, world), "unit": "elements/s", "ms_per_block": ms_n,
                             "newton_steps": 1, "comm_bytes_per_party": cb_n,
                             "aes_blocks": aes_n, "aes_roofline_frac": aes_n / (ms_n * 1e-3) / _aes_roofline(),
                             "max_abs_err_vs_float64": float(np.abs(y_n.reshape(rows, L) - ref).max())}
    smn.close()
    # LayerNorm
    rows, H = 128, 768
    lsp, cH = S.layernorm_specs(H)
    names = ["shift_mu", "shift_var", "rsqrt", "shift_r", "shift_y"]
    gates = gates_for([lsp[k] for k in names], [rows, rows, rows, rows, rows * H])
    ln = F.LayerNorm(ctx, gates, rows, H, cH)
    hid = rng.standard_normal((rows, H)) * 1.2 + 0.3
    ms, y, cb = timed(ln, S.encode(hid.reshape(-1), 12), rows * H, 3000)
    ref = (hid - hid.mean(axis=1, keepdims=True)) / np.sqrt(hid.var(axis=1, keepdims=True) + 1e-5)
    aes = aes_of(gates, [rows, rows, rows, rows, rows * H])
    info = ln.info()
    out["layernorm"] = {"value": aggregate(rows * H, ms, world), "unit": "elements/s", "ms_per_block": ms,
                        "shape": [rows, H], "gate_elements": info["gate_elements"], "key_bytes": info["key_bytes"],
                        "comm_bytes_per_party": cb, "comm_bytes_per_elem_per_party": cb / (rows * H),
                        "aes_blocks": aes, "aes_roofline_frac": aes / (ms * 1e-3) / _aes_roofline(),
                        "max_abs_err_vs_float64": float(np.abs(y.reshape(rows, H) - ref).max()),
                        "form": "row mean and variance by local sums, Beaver square, Rsqrt, Beaver product, "
                                "rounding shift gates (no affine weights)"}
    ln.close()
    # the same block with one Newton step refining 1/sqrt
    ngates = gates_for([lsp[k] for k in ("shift_n1", "shift_n2", "shift_n3")], [rows, rows, rows])
    lnn = F.LayerNorm(ctx, gates, rows, H, cH, newton_gates=ngates, newton=1)
    ms_n, y_n, cb_n = timed(lnn, S.encode(hid.reshape(-1), 12), rows * H, 3500)
    aes_n = aes + aes_of(ngates, [rows, rows, rows])
    out["layernorm_newton"] = {"value": aggregate(rows * H, ms_n, world), "unit": "elements/s",
                               "ms_per_block": ms_n, "newton_steps": 1, "comm_bytes_per_party": cb_n,
                               "aes_blocks": aes_n, "aes_roofline_frac": aes_n / (ms_n * 1e-3) / _aes_roofline(),
                               "max_abs_err_vs_float64": float(np.abs(y_n.reshape(rows, H) - ref).max())}
    lnn.close()
    torch.cuda.empty_cache()
    return out


def op_rounds(shape) -> int:
    """Interactive rounds of one fused gate call: the masked opening, then the
    Horner steps' Beaver openings (none in the x^ basis), then the piecewise
    outputs' AND rounds; a shift gate's byte travels with the first of those,
    or takes a round of its own when there is none."""
    r = 1 + (shape.degree if shape.n_mults else 0) + (shape.bx_rounds if shape.n_piecewise else 0)
    if shape.trunc_shift and r == 1:
        r += 1
    return r


def network_projection(calls, css, ms, comm_b, counted_steps):
    """Projected online time of one layer step with one party per machine
    (the paper's Eq. for T_proj): T_comp + 2 B_comm / BW + R RTT, on its LAN
    (1 GB/s, 0.5 ms) and WAN (400 MB/s, 4 ms) models.  B_comm is one party's
    bytes per step (the closed form per element, checked against the counted
    bytes), R the rounds of the operator calls run one after another, and
    T_comp the measured step time with both parties on this one GPU."""
    b = sum(c.n * css[c.name].shape.comm_bytes_per_elem for c in calls)
    rounds = sum(op_rounds(css[c.name].shape) for c in calls)
    out = {"t_comp_ms": ms, "comm_bytes_per_party": b, "rounds": rounds,
           "counted_bytes_match": all(v == b * counted_steps for v in comm_b),
           "note": "T_comp is both parties' time on one GPU; one party per GPU would halve it at most"}
    for name, bw, rtt in (("lan", 1e9, 0.5), ("wan", 400e6, 4.0)):
        out[name] = {"bw_bytes_per_s": bw, "rtt_ms": rtt,
                     "t_proj_ms": ms + 2e3 * b / bw + rounds * rtt}
    return out


def sets_that_fit(set_bytes: int, want: int, margin: float = 12e9) -> int:
    """How many key sets of set_bytes fit in free HBM (at least 1, at most want)."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    return max(1, min(want, int((free - margin) // max(set_bytes, 1))))


def _aes_roofline():
    return SMS * SM_MAX_MHZ * 1e6 / max(ALU_OPS_PER_AES / 64.0, LDS_PER_AES / 32.0)


def _pct(sorted_vals, q):
    """Nearest-rank percentile of an ascending list."""
    i = max(0, min(len(sorted_vals) - 1, -(-q * len(sorted_vals) // 100) - 1))
    return sorted_vals[i]


def run_plain_fifo(ctx, dev, trace, pool_bytes, seed):
    """The plain per-operator form on a served trace: requests one at a time
    in arrival order, and within a request every layer's operator calls one
    after another; each call's keys are dealt into a key pool of pool_bytes
    (both parties) chunk by chunk, each chunk by its own dealer launch and
    then its own fused-gate launch.  Returns elements/s and per-request
    latency (arrival to last share written) on the GPU event timeline."""
    import torch

    from paper_2606_09551_b300 import fusefss as F
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device=dev)
    cap = 1 << 22
    xs0 = torch.empty(cap, dtype=torch.uint64, device=dev)
    xs1 = torch.empty_like(xs0)
    order = sorted(range(len(trace)), key=lambda i: trace[i][1])
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t0.record()
    host0 = time.perf_counter()
    done, layer_ev, elements, launches, call_id = {}, [], 0, 0, 3_000_000
    for i in order:
        layers, arrival_s, _ = trace[i]
        # a request cannot start before it arrives
        wait = arrival_s - (time.perf_counter() - host0)
        if wait > 0:
            time.sleep(wait)
        for ops in layers:
            a = torch.cuda.Event(enable_timing=True)
            a.record()
            for cs, x, y0, y1, z0, z1 in ops:
                n = x.numel()
                per = 2 * cs.shape.key_bytes_per_elem
                chunk = max(1, min(cap, (pool_bytes - 4096) // per))
                for s0 in range(0, n, chunk):
                    c = min(chunk, n - s0)
                    nb = cs.key_bytes(c)
                    off = -(-nb // 256) * 256
                    k0 = F.Keys(cs, c, 0, buf=pool[:nb])
                    k1 = F.Keys(cs, c, 1, buf=pool[off:off + nb])
                    F.keygen(ctx, cs, seed, call_id, c, k0, k1, x[s0:s0 + c], xs0[:c], xs1[:c])
                    F.eval_pair(ctx, cs, k0, k1, xs0[:c], xs1[:c], y0[s0:s0 + c], y1[s0:s0 + c],
                                z0[s0:s0 + c], z1[s0:s0 + c])
                    k0.close()
                    k1.close()
                    call_id += 1
                    launches += 2
                elements += n
            b = torch.cuda.Event(enable_timing=True)
            b.record()
            layer_ev.append((a, b))
        done[i] = layer_ev[-1][1]
    torch.cuda.synchronize()
    # trace clock: 0 at t0, request i arrives at arrival_s; the first request
    # starts on an idle GPU at its arrival
    req = sorted(t0.elapsed_time(done[i]) - 1e3 * trace[i][1] for i in order)
    span_s = t0.elapsed_time(layer_ev[-1][1]) * 1e-3 - trace[order[0]][1]
    lay = sorted(a.elapsed_time(b) for a, b in layer_ev)
    del pool
    return {"value": elements / span_s, "unit": "elements/s", "elements": elements, "launches": launches,
            "span_s": span_s, "request_ms_p50": _pct(req, 50), "request_ms_p99": _pct(req, 99),
            "layer_service_ms_p50": _pct(lay, 50), "layer_service_ms_p99": _pct(lay, 99),
            "form": "plain per-operator launches, requests first-come first-served, keys dealt per chunk "
                    "into a %d GB pool just before each chunk's gate launch" % (pool_bytes >> 30)}


def _serial_rates(ctx, pending, max_active, aes_blocks):
    """The same requests once more through a server that never overlaps the
    dealer with an evaluation (FFSS_SERVER_SERIAL): the evaluation launches'
    GPU time alone gives the online (keygen-excluded) rate, the dealer
    launches' the dealer rate.  Same call ids, so the same keys and shares."""
    from paper_2606_09551_b300 import fusefss as F
    from paper_2606_09551_b300 import inputs as I
    sv = F.Server(ctx, 64 << 30, max_active, 1 << 22, I.KEY_SEED, serial=True)
    for layers, _, cid in pending:
        sv.submit(layers, 0.0, call_id_base=cid)
    sv.run()
    st = sv.summary()
    sv.close()
    ev_s, gen_s = st["eval_ms"] * 1e-3, st["gen_ms"] * 1e-3
    return {"elements_per_s": st["elements"] / ev_s, "eval_s": ev_s,
            "aes_roofline_frac": aes_blocks[1] / ev_s / _aes_roofline(),
            "dealer_elements_per_s": st["elements"] / gen_s, "dealer_s": gen_s,
            "dealer_aes_roofline_frac": aes_blocks[0] / gen_s / _aes_roofline(),
            "serial_span_s": (st["last_done_ms"] - st["first_admit_ms"]) * 1e-3,
            "basis": "keygen excluded: GPU time of the batched evaluation launches of a second pass in "
                     "which the dealer never overlaps an evaluation (same keys and shares)"}


def _server_result(sv, nreq, clk, wall, aes_blocks):
    st = sv.summary()
    infos = [sv.request_info(i) for i in range(nreq)]
    queue = sorted(max(0.0, r["admitted_ms"] - r["arrival_ms"]) for r in infos)
    req = sorted(r["done_ms"] - r["arrival_ms"] for r in infos)
    span_s = (st["last_done_ms"] - st["first_admit_ms"]) * 1e-3
    return st, {"value": st["elements"] / span_s, "unit": "elements/s",
                "aes_blocks": aes_blocks[0] + aes_blocks[1],
                "aes_roofline_frac": (aes_blocks[0] + aes_blocks[1]) / span_s / _aes_roofline(),
                "note": "includes the on-device dealer: keys are streamed through the key pool, not preloaded; "
                        "aes_roofline_frac counts dealer + online AES blocks against the AES roofline",
                "requests": nreq, "elements": int(st["elements"]), "steps": int(st["steps"]),
                "chunks": int(st["chunks"]), "batched_launches": int(st["steps"]),
                "layer_ms_p50": st["layer_ms_p50"], "layer_ms_p99": st["layer_ms_p99"],
                "layer_ms_max": st["layer_ms_max"],
                "queue_ms_p50": queue[len(queue) // 2], "queue_ms_max": queue[-1],
                "request_ms_p50": _pct(req, 50), "request_ms_p99": _pct(req, 99),
                "span_s": span_s, "wall_s": wall, "clocks": clk.summary()}


def run_served(ctx, args, dev):
    """A finite trace of secure-inference requests through the library's
    continuous-batching server: BERT-large layer shapes (hidden 1024, 16 heads,
    MLP 4096), sequence lengths log-uniform in [16, 2048], Poisson arrivals
    at 20 requests/s, a 64 GB key budget; keys are made on the device chunk by
    chunk just before use.  Every layer of a request reuses its inputs and gets
    fresh masks and keys."""
    import torch

    from paper_2606_09551_b300 import fusefss as F
    from paper_2606_09551_b300 import inputs as I
    nreq, nlay = args.served_requests, args.served_layers
    reqs = I.bert_large_trace(nreq)
    lens = [rq.L for rq in reqs]
    css = _compile_requests(ctx, reqs, args, 1 << 22)
    total = 0
    pending = []
    for rq in reqs:
        ops = _request_ops(css, rq, dev)
        total += sum(o[1].numel() for o in ops) * nlay
        pending.append(([ops] * nlay, rq.arrival_s, rq.call_base))
    del reqs
    torch.cuda.synchronize()
    # the server clock starts here: arrivals are offsets from its creation
    sv = F.Server(ctx, 64 << 30, 8, 1 << 22, I.KEY_SEED)
    for layers, arr, cid in pending:
        sv.submit(layers, arr, call_id_base=cid)
    t0 = time.perf_counter()
    with ClockSampler(int(dev.split(":")[1])) as clk:
        sv.run()
    wall = time.perf_counter() - t0
    st, res = _server_result(sv, nreq, clk, wall, _stream_aes([p_[0][0] for p_ in pending], nlay))
    assert st["elements"] == total
    res["dcf_bits"] = {name: cs.spec.dcf_bits for name, cs in css.items()}
    res["lookup_records"] = {name: cs.records for name, cs in css.items()}
    res.update({"layers_per_request": nlay, "seq_lens": [int(v) for v in lens],
                "offered_requests_per_s": 20.0,
                "sustainable_requests_per_s": nreq / res["span_s"],
                "config": "BERT-large shapes (hidden 1024, 16 heads, MLP 4096), L log-uniform [16, 2048], "
                          "Poisson 20 req/s, 64 GB key budget, max 8 admitted, chunks <= 4M elements"})
    sv.close()
    if not args.no_serial:
        res["online"] = _serial_rates(ctx, pending, 8, _stream_aes([p_[0][0] for p_ in pending], nlay))
    if not args.no_served_plain:
        # the same trace in the plain per-operator form; the server keeps half
        # of its 64 GB key pool for the chunks it evaluates (the other half is
        # filled meanwhile), so the plain form gets the same 32 GB per chunk set
        trace = [(layers, arr, cid) for layers, arr, cid in pending]
        plain = run_plain_fifo(ctx, dev, trace, 32 << 30, I.KEY_SEED)
        plain["vs_served"] = {"elements_per_s": res["value"] / plain["value"],
                              "request_ms_p50": plain["request_ms_p50"] / res["request_ms_p50"],
                              "request_ms_p99": plain["request_ms_p99"] / res["request_ms_p99"]}
        res["plain_fifo"] = plain
    return res


def run_gpt2_batch(ctx, args, dev):
    """Config 3: 32 GPT-2-small-shaped requests (hidden 768, 12 heads, MLP
    3072), sequence lengths uniform in [32, 1024], all present at once; every
    step evaluates chunks of all admitted requests' GeLU / exp / reciprocal /
    rsqrt calls in one batched launch, keys streamed through a 64 GB pool."""
    import torch

    from paper_2606_09551_b300 import fusefss as F
    from paper_2606_09551_b300 import inputs as I
    nreq, nlay = 32, args.gpt2_layers
    reqs = I.gpt2_batch(nreq)
    lens = [rq.L for rq in reqs]
    css = _compile_requests(ctx, reqs, args, 1 << 22)
    total = 0
    pending = []
    for rq in reqs:
        ops = _request_ops(css, rq, dev)
        total += sum(o[1].numel() for o in ops) * nlay
        pending.append(([ops] * nlay, 0.0, rq.call_base))
    del reqs
    torch.cuda.synchronize()
    sv = F.Server(ctx, 64 << 30, 32, 1 << 22, I.KEY_SEED)
    for layers, arr, cid in pending:
        sv.submit(layers, arr, call_id_base=cid)
    t0 = time.perf_counter()
    with ClockSampler(int(dev.split(":")[1])) as clk:
        sv.run()
    wall = time.perf_counter() - t0
    st, res = _server_result(sv, nreq, clk, wall, _stream_aes([p_[0][0] for p_ in pending], nlay))
    assert st["elements"] == total
    res["dcf_bits"] = {name: cs.spec.dcf_bits for name, cs in css.items()}
    res["lookup_records"] = {name: cs.records for name, cs in css.items()}
    res.update({"layers_per_request": nlay, "seq_lens": [int(v) for v in lens],
                "config": "32 GPT-2-small requests (hidden 768, 12 heads, MLP 3072, 2 LayerNorms), "
                          "L uniform [32, 1024], %d of 12 layers each, 64 GB key budget" % nlay})
    sv.close()
    if not args.no_serial:
        res["online"] = _serial_rates(ctx, pending, 32, _stream_aes([p_[0][0] for p_ in pending], nlay))
    return res


def run_large_layer(ctx, dev, args, no_serial=False):
    """One GPT-style 2.7B layer (hidden 2560, 32 heads, MLP 10240 with SiLU,
    seq 1024): SiLU on 1024 x 10240, softmax nExp on 32 x 1024 x 1024, the
    reciprocal of the 32 x 1024 row sums and rsqrt for two LayerNorms (2 x
    1024); 16-interval degree-3 specs, k = 24, 16 fractional bits.  The keys
    (2.3 TB for the layer) cannot be resident: the server generates them on
    the device chunk by chunk into a 64 GB pool and evaluates each chunk set
    in one batched launch."""
    import torch

    from paper_2606_09551_b300 import fusefss as F
    from paper_2606_09551_b300 import inputs as I
    reqs = I.large_layer()
    css = _compile_requests(ctx, reqs, args, 1 << 22)
    ops = _request_ops(css, reqs[0], dev)
    xs = {name: o[1] for name, o in zip(css, ops)}
    call_base = reqs[0].call_base
    del reqs
    total = sum(x.numel() for x in xs.values())
    torch.cuda.synchronize()
    sv = F.Server(ctx, 64 << 30, 1, 1 << 22, I.KEY_SEED)
    sv.submit([ops], 0.0, call_id_base=call_base)
    t0 = time.perf_counter()
    with ClockSampler(int(dev.split(":")[1])) as clk:
        sv.run()
    wall = time.perf_counter() - t0
    st = sv.summary()
    assert st["elements"] == total
    span_s = (st["last_done_ms"] - st["first_admit_ms"]) * 1e-3
    key_tb = sum(2 * css[n].shape.key_bytes_per_elem * xs[n].numel() for n in xs) / 1e12
    sv.close()
    deal, online = _stream_aes([ops], 1)
    return {"value": total / span_s, "unit": "elements/s", "elements": int(total), "layer_ms": st["layer_ms_max"],
            "dcf_bits": {name: cs.spec.dcf_bits for name, cs in css.items()},
            "lookup_records": {name: cs.records for name, cs in css.items()},
            "online": None if no_serial else _serial_rates(ctx, [([ops], 0.0, call_base)], 1, (deal, online)),
            "aes_blocks": deal + online, "aes_roofline_frac": (deal + online) / span_s / _aes_roofline(),
            "steps": int(st["steps"]), "chunks": int(st["chunks"]), "keys_tb_streamed": key_tb,
            "wall_s": wall, "clocks": clk.summary(),
            "note": "includes the on-device dealer: keys are streamed through a 64 GB pool, not preloaded",
            "config": "GPT-style 2.7B layer, seq 1024: SiLU 1024x10240, nExp 32x1024x1024, recip 32x1024, "
                      "rsqrt 2x1024; k=24, f=16, m=16, d=3"}


# ---------------------------------------------------------------------------
# reference arm: the oracle (the paper ships no code), on the host cores
# ---------------------------------------------------------------------------

# The DCF arity the reference arm's oracle runs for the plain form (resident
# keys): the one the layer's gates measure fastest at on this GPU (arity 64
# with lookup keys in records, within 2 % of arity 32 for the nExp gate;
# the measured choice per spec is in the GPU arm's autotune record).  The
# reference arm has no GPU to measure with.
PLAIN_DCF_BITS = 6


def reference_calls(calls, args):
    """The calls at the arity the reference arm (and the printed config) uses."""
    from paper_2606_09551_b300 import inputs as I
    return I.with_arity(calls, args.dcf_bits or PLAIN_DCF_BITS)


def full_config(config, calls, world, args):
    """The workload's config as both arms print it: the workload, how L2 is
    kept out of the measurement, and the process layout."""
    from paper_2606_09551_b300 import fusefss as F
    key_gb = sum(2 * F.CompiledSpec(c.spec, records=c.spec.m > 1 and c.spec.p in (3, 4)).shape.key_bytes_per_elem * c.n
                 for c in reference_calls(calls, args)) / 1e9
    return dict(config, l2="inputs > L2: every step reads %.1f GB of fresh one-time keys" % key_gb,
                parallelism="replicas x %d" % world if world > 1 else "one process; both parties in it")


def run_reference(args, world):
    """The oracle on the host cores.  A step evaluates (both parties, online
    phase) a fixed sample of every operator of the workload, the same
    fraction of each, sized so that all warm-up and timed steps take about
    two minutes; ms_per_step is that step's measured wall time.  The sample's
    keys are dealt once by the oracle dealer before timing (the evaluation's
    cost does not depend on the key values)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle as O
    from paper_2606_09551_b300 import inputs as I
    calls, config = workload(args.workload, args.elements)
    calls = reference_calls(calls, args)
    from paper_2606_09551_b300 import fusefss as F
    threads = os.cpu_count() or 1
    step_s = min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup))
    # per-element oracle time estimate: 0.2 us per AES block per core, both
    # parties, at the keys' arity; the sample's keys stay in host memory, so
    # they also get a budget: a quarter of the available memory, at most 32 GB
    per_elem, key_elem = {}, {}
    ospec = {}
    for c in calls:
        o = O.Spec(**c.spec.descriptor())
        ospec[c.name] = o
        r = c.spec.dcf_bits
        lv = lambda f: -(-f // r)
        per_elem[c.name] = 0.2e-6 * 2 * (sum(lv(f) for f, _, _ in o.queries())
                                        + (o.M - 1) * (lv(o.k) * (1 + (o.p + 1) // 2) + (o.p + 1) // 2))
        key_elem[c.name] = 2 * F.CompiledSpec(c.spec).shape.key_bytes_per_elem
    est = sum(c.n * per_elem[c.name] for c in calls) / threads
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = 16 << 30
    mem_budget = min(avail / 4, 32e9)
    frac = min(1.0, step_s / est, mem_budget / sum(c.n * key_elem[c.name] for c in calls))
    sample = {c.name: max(1, int(round(c.n * frac))) for c in calls}
    work = []
    for c in calls:
        ns = sample[c.name]
        for i in range(threads):
            a, b = i * ns // threads, (i + 1) * ns // threads
            if b > a:
                work.append((c, a, b))

    def deal(w):
        c, a, b = w
        return O.dealer(ospec[c.name], I.KEY_SEED, c.call_id, a, b - a, c.x[a:b])

    with ThreadPoolExecutor(threads) as ex:
        dealt = list(ex.map(deal, work))

    def ev(i):
        c = work[i][0]
        k0, k1, x0, x1 = dealt[i]
        O.eval_pair(ospec[c.name], k0, k1, x0, x1)

    times = []
    with ThreadPoolExecutor(threads) as ex:
        for s_ in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            list(ex.map(ev, range(len(work))))
            if s_ >= args.warmup:
                times.append(time.perf_counter() - t0)
    per_step_s = statistics.mean(times)
    total = sum(sample.values())
    value = total / per_step_s
    ar = {c.name: 1 << c.spec.dcf_bits for c in calls}
    desc = ("oracle eval_pair (both parties) per step on %s elements (%.4f of each operator: %s), "
            "%d threads; the sample bounded by %.0f s of estimated work per step and %.1f GB of host "
            "memory for its keys" % (total, frac, ", ".join(f"{sample[k]} {k} (DCF arity {ar[k]})" for k in sample),
                                     threads, step_s, mem_budget / 1e9))
    return {
        "impl": "reference",
        "metric": "FSS-evaluated elements/s per nonlinear op (both parties, online phase)",
        "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic", "config": full_config(config, calls, world, args),
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ---------------------------------------------------------------------------
# process group helpers (N > 1 under torchrun)
# ---------------------------------------------------------------------------

def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, dev):
    """The slowest rank's time (the job finishes when the last replica does)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(per_rank_elements, ms, world):
    """Whole-job throughput: the elements all ranks processed over the max time."""
    return per_rank_elements * world / (ms * 1e-3)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, world)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
