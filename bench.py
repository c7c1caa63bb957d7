"""Benchmark: GERIS per quartet class (int16-compressed) at a stated max abs error,
mixed precision vs FP64, on the 256-class sweep.

Workload (one "step"): all 256 Cartesian classes (s, p, d, f on each of a, b, c, d),
primitive shells, centres uniform in [-3, 3]^3 bohr, exponents log-uniform in [0.1, 10],
unit coefficients, round(2^26 / n_ERIQ) quartets per class (about 1.7e10 ERIs in total),
compressed to 16-bit integers with one FP32 scale per quartet.  Inputs are drawn from a pool
of 4096 shells per angular momentum; the quartet table (7 GB) and the packed output
(34 GB) are far larger than L2, so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--scale S]

Prints one JSON line (rank 0).  --scale < 1 shrinks every class (for quick checks only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2303_13632_gb300 import perfmodel, workloads as W  # noqa: E402

METRIC = "GERIS per quartet class (int16-compressed) at stated max abs err; mixed vs FP64"
POOL_PER_L = W.SWEEP_POOL_PER_L
BITS = 16
STUDY_BITS = (8, 12, 16, 20)
# per-class precision: FP32 recurrences for the classes whose FP32 error, measured on the
# device over CALIB_SAMPLE quartets per class, stays below CALIB_STEPS quantisation steps
CALIB_SAMPLE = 4096
CALIB_STEPS = 0.5


def unpack(words: np.ndarray, off_bytes: int, qi: np.ndarray, neri: int, bits: int) -> np.ndarray:
    """Signed n-bit fields of quartets qi (ERIs qi*neri .. +neri) of a class segment."""
    v = (qi[:, None].astype(np.int64) * neri + np.arange(neri)[None, :]) * bits + off_bytes * 8
    w = v >> 5
    o = (v & 31).astype(np.uint64)
    lo = words[w].astype(np.uint64)
    hi = words[np.minimum(w + 1, len(words) - 1)].astype(np.uint64)
    raw = ((lo | (hi << np.uint64(32))) >> o) & np.uint64((1 << bits) - 1)
    raw = raw.astype(np.int64)
    return np.where(raw >= (1 << (bits - 1)), raw - (1 << bits), raw).astype(np.float64)


def classes():
    return [W.class_of_id(c) for c in range(256)]


ONLY = None  # --classes: restrict the sweep to these class ids (profiling runs only)


def max_over_ranks(value: float, dist, device) -> float:
    """The largest value over the ranks (the slowest rank's step time); `dist` is None with one
    process."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_geris(eris_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the ERIs of all ranks (replicas of the same workload) over the
    slowest rank's time."""
    return world * eris_per_rank / (ms * 1e-3) / 1e9


def class_choices(api, plan):
    """{class: precision name} of the plan's non-empty classes."""
    return {c: api.eri_plan_class_precision(plan, c)[0] for c in range(256)
            if api.eri_plan_class_info(plan, c)[0]}


def apply_choices(api, plan, choice):
    """Per-class precision overrides (None: follow the plan's precision)."""
    for c in range(256):
        api.eri_plan_set_class_precision(plan, c, choice.get(c) if choice else None)


def class_counts(scale: float):
    return {c: (max(1, int(round(W.sweep_quartet_count(W.class_of_id(c)) * scale)))
                if ONLY is None or c in ONLY else 0) for c in range(256)}


def make_pool(seed_k: int = 2):
    return W.sweep_pool(seed_k)


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def measure_alu_peaks(api, torch, stream, device_index):
    """FP32 and FP64 fused multiply-add throughput measured with the library's probe kernel
    (eri_fma_probe: 16 independent FMA chains per thread, 1216 x 256-thread blocks = 8 CTAs per
    SM, about 30 ms per launch), best of 3 launches timed with CUDA events on the launching
    stream, with the SM clock sampled during the FP64 probe.
    Returns {"fp32_tflops", "fp64_tflops", "clocks"}."""
    n_threads = 152 * 8 * 256
    sink = torch.empty(n_threads, dtype=torch.float64, device=torch.device("cuda", device_index))
    out = {}
    for prec, iters in (("mixed", 4096), ("fp64", 192)):
        best = None
        clk = ClockSampler(device_index) if prec == "fp64" else None
        if clk:
            clk.start()
        for rep in range(4):  # first launch warms up
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            api.eri_fma_probe(prec, n_threads, iters, sink, stream)
            b.record(stream)
            b.synchronize()
            if rep:
                ms = a.elapsed_time(b)
                best = ms if best is None else min(best, ms)
        if clk:
            out["clocks"] = clk.stop()
        tflops = 512.0 * iters * n_threads / (best * 1e-3) / 1e12
        out["fp32_tflops" if prec == "mixed" else "fp64_tflops"] = tflops
    return out


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        out["sm_mhz"] = statistics.median(sm) if sm else None
        out["sm_max_mhz"] = max(mx) if mx else None
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


def oracle_sample_size(cls, eris: int) -> int:
    return max(2, eris // W.quartet_size(*cls))


def nonempty(counts):
    return [c for c in range(256) if counts[c] > 0]


def cpu_oracle_rate(pool, quartets_by_class, counts):
    """Times the oracle (as it stands, all host cores) on the sampled quartets of every class
    and scales per-class time per ERI to the full workload: returns (GERIS, cores, seconds,
    values) where values are the oracle's ERIs of the sample (reused for parity)."""
    import oracle

    cores = oracle.max_threads()
    total_time_full = 0.0
    total_eris_full = 0
    spent = 0.0
    values = {}
    for c in range(256):
        q = quartets_by_class[c]
        t0 = time.perf_counter()
        vals, offs = oracle.eri_batch(pool, q)
        dt = time.perf_counter() - t0
        spent += dt
        neri = W.quartet_size(*W.class_of_id(c))
        per_eri = dt / max(1, len(q) * neri)
        total_time_full += per_eri * counts[c] * neri
        total_eris_full += counts[c] * neri
        values[c] = (vals, offs)
    return total_eris_full / total_time_full / 1e9, cores, spent, values


def run_reference(args):
    """The oracle on the host cores (the CPU baseline arm): each step evaluates a bounded
    sample of the workload and reports the rate scaled to the full class mix."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    counts = class_counts(args.scale)
    pool = make_pool()
    rng = np.random.default_rng(5)
    rates = []
    cores = None
    for step in range(args.warmup + args.steps):
        sample = {}
        for c in range(256):
            cls = W.class_of_id(c)
            n = oracle_sample_size(cls, args.ref_eris)
            sample[c] = W.random_class_quartets(rng, cls, n, POOL_PER_L)
        t0 = time.perf_counter()
        g, cores, spent, _ = cpu_oracle_rate(pool, sample, counts)
        if step >= args.warmup:
            rates.append((g, time.perf_counter() - t0))
    value = float(np.mean([r[0] for r in rates]))
    total_eris = sum(counts[c] * W.quartet_size(*W.class_of_id(c)) for c in range(256))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GERIS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_eris / (value * 1e9) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args),
        "cpu_baseline": {"value": value, "unit": "GERIS", "cores": cores, "kind": "oracle",
                         "sample": f"about {args.ref_eris} ERIs (at least 2 quartets) per class x 256 "
                                   "classes per step, per-class time per ERI scaled to the full class mix"},
        "e2e": {"value": value, "unit": "GERIS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        # ms_per_step above is the full step at the sampled rate (an estimate); each timed step
        # evaluated only the bounded sample, in this many milliseconds of wall time
        "ms_per_step_estimated": True,
        "sample_ms_per_step": float(np.mean([r[1] for r in rates])) * 1e3,
    }
    print(json.dumps(line), flush=True)


def config_dict(args):
    return {"workload": "256-class sweep: round(2^26/n_ERIQ) primitive quartets per class, "
                        "centres U[-3,3]^3 bohr, exponents log-U[0.1,10], unit coefficients, "
                        "16-bit compression",
            "classes": 256, "quartets_per_class": "round(2^26 / n_ERIQ)" + (f" x {args.scale}" if args.scale != 1 else ""),
            "bits": BITS, "precision_headline": "mixed (FP32 recurrences, FP64 Boys/roots/prefactors)",
            "l2": "inputs (7 GB quartet table) and outputs (34 GB) exceed L2; no flush needed",
            "parallelism": f"replicas x{args.gpus}"}


def run_ours(args):
    import torch

    from paper_2303_13632_gb300 import api

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    counts = class_counts(args.scale)
    cls_list = classes()
    pool = make_pool()
    # quartet table, class-major, generated on the device from a seeded generator
    quartets, first = W.sweep_quartets_device(torch, counts, dev)
    torch.cuda.synchronize()
    plan = api.eri_plan_create(pool, quartets, precision="mixed", device=local)
    packed_bytes, scale_bytes = api.eri_output_bytes(plan, BITS)
    packed = torch.empty(packed_bytes // 4, dtype=torch.int32, device=dev)
    scales = torch.empty(scale_bytes // 4, dtype=torch.float32, device=dev)
    total_eris = sum(counts[c] * W.quartet_size(*cls_list[c]) for c in range(256))

    def step():
        api.eri_compute_compressed(plan, BITS, packed, scales, stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(n_warm, n_steps, clocks=None):
        for _ in range(n_warm):
            step()
        api.eri_sync(plan, stream)
        barrier()
        if clocks is not None:
            clocks.start()
            torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select these launches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_steps):
            step()
        e1.record(stream)
        if clocks is not None:
            torch.cuda.nvtx.range_pop()
        barrier()
        clk = clocks.stop() if clocks is not None else None
        api.eri_sync(plan, stream)
        t = max_over_ranks(e0.elapsed_time(e1) / n_steps, dist, dev)
        return t, clk

    # ---- per-class precision for 16-bit output (plan setup, outside the timed region) ----
    api.eri_plan_calibrate_precision(plan, BITS, sample=CALIB_SAMPLE, max_err_steps=CALIB_STEPS,
                                     stream=stream)
    choice16 = class_choices(api, plan)
    launches = sum(api.eri_plan_class_launches(plan, c) for c in range(256))

    # ---- measured ALU peaks (the roofline denominators of the FP-bound kernels) ----
    alu = measure_alu_peaks(api, torch, stream, local)
    p32, p64 = alu["fp32_tflops"], alu["fp64_tflops"]

    # ---- headline: all 256 classes per step, FP32 recurrences where calibrated ----
    ms, clk = timed_steps(args.warmup, args.steps, ClockSampler(local))
    value = job_geris(total_eris, world, ms)
    # every class in FP32 (no calibration), for context
    apply_choices(api, plan, None)
    ms_all32, _ = timed_steps(1, args.steps)
    # the plain FP64 path as a timed step of the same call (every class in FP64)
    api.eri_plan_set_precision(plan, "fp64")
    ms_fp64_step, _ = timed_steps(1, args.steps)
    api.eri_plan_set_precision(plan, "mixed")

    # ---- per-class timing, mixed and FP64 (events on the launching stream) ----
    def per_class_ms(precision):
        api.eri_plan_set_precision(plan, precision)
        res = {}
        for c in nonempty(counts):
            api.eri_compute_compressed_class(plan, c, BITS, packed, scales, stream)  # warm
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            api.eri_compute_compressed_class(plan, c, BITS, packed, scales, stream)
            b.record(stream)
            b.synchronize()
            res[c] = a.elapsed_time(b)
        api.eri_sync(plan, stream)
        return res

    ms_mixed = per_class_ms("mixed")
    ms_fp64 = per_class_ms("fp64")
    api.eri_plan_set_precision(plan, "mixed")
    # per-class time and precision of the headline configuration
    ms_cal = {c: (ms_mixed[c] if choice16[c] == "mixed" else ms_fp64[c]) for c in ms_mixed}

    # ---- roofline: per class, per kernel instantiation, and weighted over the step ----
    peaks, peak_kind = read_peaks()
    apply_choices(api, plan, choice16)
    t_roof = {c: perfmodel.roofline_seconds(cls_list[c], counts[c], choice16[c], BITS, peaks["hbm_gbs"], p32, p64)
              for c in ms_cal}
    frac_all = {c: t_roof[c] / (ms_cal[c] * 1e-3) for c in ms_cal}
    # generic classes served by the same kernel instantiation(s) (canonical class, precision,
    # kernel form) are one kernel in the launch list: group them, and take the instantiation
    # with the largest share of the step as the dominant kernel
    groups = {}
    for c in ms_cal:
        groups.setdefault(api.eri_plan_class_kernels(plan, c), []).append(c)
    dom_name = max(groups, key=lambda k: sum(ms_cal[c] for c in groups[k]))
    dom = groups[dom_name]
    t_dom = sum(ms_cal[c] for c in dom) * 1e-3
    flops = sum(perfmodel.fp32_equivalent_flops(cls_list[c], choice16[c], p32, p64) * counts[c] for c in dom)
    roof = {"bound": "alu", "kernel": dom_name, "classes": [fmt_class(cls_list[c]) for c in dom],
            "achieved": flops / t_dom / 1e12, "peak": p32, "unit": "TFLOP/s",
            "frac": sum(t_roof[c] for c in dom) / t_dom, "traffic": None,
            "peak_source": "measured: eri_fma_probe FP32 and FP64 FMA loops in this run "
                           f"({p32:.1f} / {p64:.3f} TFLOP/s); FP64 work weighted by their ratio",
            "fp64_peak_tflops": p64, "probe_clocks": alu.get("clocks"),
            "share": t_dom / (sum(ms_cal.values()) * 1e-3),
            "frac_step_weighted": sum(t_roof.values()) / (sum(ms_cal.values()) * 1e-3),
            "frac_of_ms_per_step": sum(t_roof.values()) / (ms * 1e-3),
            "frac_nominal_peaks": sum(perfmodel.roofline_seconds(cls_list[c], counts[c], choice16[c], BITS,
                                                                 peaks["hbm_gbs"]) for c in dom) / t_dom}
    # DRAM traffic of the dominant kernel: bytes per quartet from the committed ncu capture of
    # the same instantiation (a smaller case of one of its classes), scaled to this step's quartets
    try:
        with open(os.path.join(ROOT, "profiles", "dram_bytes_per_quartet.json")) as f:
            tr = json.load(f)
        if tr["kernel"] == dom_name:
            nq_dom = sum(counts[c] for c in dom)
            roof["traffic"] = tr["dram_bytes_per_quartet"] * nq_dom
            roof["traffic_source"] = tr["source"] + f", scaled to the {nq_dom} quartets of its classes"
    except (OSError, KeyError, ValueError):
        pass

    # ---- accuracy on a sample, and the CPU oracle baseline ----
    line_extra = {}
    study_details = None
    if rank == 0 and not args.no_check:
        rng = np.random.default_rng(99)
        sample_idx = {c: np.sort(rng.choice(counts[c], size=min(counts[c], oracle_sample_size(cls_list[c], args.ref_eris)),
                                            replace=False)) if counts[c] else np.zeros(0, dtype=np.int64)
                      for c in range(256)}
        qhost = {}
        for c in range(256):
            idx = torch.as_tensor(sample_idx[c] + first[c], device=dev, dtype=torch.int64)
            qhost[c] = quartets[idx].cpu().numpy()
        g_cpu, cores, spent, ref = cpu_oracle_rate(pool, qhost, counts)
        # FP32 arithmetic error of the mixed path (FP64 output) on the sampled quartets
        samp_q = np.concatenate([qhost[c] for c in nonempty(counts)])
        samp_plan = api.eri_plan_create(pool, samp_q, precision="mixed", device=local)
        sb, _ = api.eri_output_bytes(samp_plan, 0)
        sout = torch.empty(sb // 8, dtype=torch.float64, device=dev)
        arith = {}
        for prec in ("mixed", "fp64"):
            api.eri_plan_set_precision(samp_plan, prec)
            api.eri_compute(samp_plan, sout, stream)
            api.eri_sync(samp_plan, stream)
            host = sout.cpu().numpy()
            for c in nonempty(counts):
                n_c, neri, _, off = api.eri_plan_class_info(samp_plan, c)
                got = host[off:off + n_c * neri].reshape(n_c, neri)
                vals, _ = ref[c]
                r = vals.reshape(n_c, neri)
                # relative to each quartet's b_max; quartets below 1e-30 Ha (under the FP32 range
                # after the prefactor) are left out of the relative figure
                bm = np.max(np.abs(r), axis=1)
                keep = bm > 1e-30
                rel = np.max(np.abs(got - r), axis=1)[keep] / bm[keep]
                arith.setdefault(prec, {})[c] = float(np.max(rel)) if rel.size else 0.0
        samp_plan.destroy()
        errs = {}
        study = {}
        for bits in STUDY_BITS:
            nbw, sbw = api.eri_output_bytes(plan, bits)
            pk = torch.empty(nbw // 4, dtype=torch.int32, device=dev) if bits != BITS else packed
            sc_t = torch.empty(sbw // 4, dtype=torch.float32, device=dev) if bits != BITS else scales
            for prec in ("mixed", "fp64", "calibrated"):
                extra = {}
                if prec == "calibrated":
                    # FP32 recurrences only where the measured error stays below CALIB_STEPS steps
                    api.eri_plan_set_precision(plan, "mixed")
                    api.eri_plan_calibrate_precision(plan, bits, sample=CALIB_SAMPLE,
                                                     max_err_steps=CALIB_STEPS, stream=stream)
                    ch = class_choices(api, plan)
                    t_b = _events(torch, stream,
                                  lambda: api.eri_compute_compressed(plan, bits, pk, sc_t, stream), reps=2)
                    extra = {"classes_fp32": sum(v == "mixed" for v in ch.values()),
                             "geris": total_eris / (t_b * 1e-3) / 1e9}
                else:
                    apply_choices(api, plan, None)
                    api.eri_plan_set_precision(plan, prec)
                    ch = {c: prec for c in nonempty(counts)}
                api.eri_compute_compressed(plan, bits, pk, sc_t, stream)
                api.eri_sync(plan, stream)
                words = pk.cpu().numpy().view(np.uint32)
                sc = sc_t.cpu().numpy()
                worst, half_step, within = 0.0, 0.0, 0
                for c in nonempty(counts):
                    nq, neri, fq, _ = api.eri_plan_class_info(plan, c)
                    off_bytes, _ = api.eri_packed_class_offset(plan, bits, c)
                    vals, _ = ref[c]
                    qi = sample_idx[c]
                    x = unpack(words, off_bytes, qi, neri, bits) * sc[fq + qi][:, None].astype(np.float64)
                    e = float(np.max(np.abs(x - vals.reshape(len(qi), neri))))
                    h = float(np.max(sc[fq + qi])) / 2
                    study.setdefault(str(bits), {}).setdefault(prec, {})[fmt_class(cls_list[c])] = {
                        "max_abs_err": e, "half_step_max": h}
                    worst = max(worst, e)
                    half_step = max(half_step, h)
                    within += arith[ch[c]][c] <= 0.5 / ((1 << (bits - 1)) - 1)
                errs.setdefault(str(bits), {})[prec] = {"max_abs_err": worst, "half_step_max": half_step,
                                                        "classes_arith_err_below_half_step": within, **extra}
        # back to the headline configuration
        apply_choices(api, plan, choice16)
        api.eri_plan_set_precision(plan, "mixed")
        line_extra["precision_study"] = errs
        line_extra["arith_err_rel_bmax_max"] = {p_: max(arith[p_].values()) for p_ in arith}
        if args.details:
            study_details = {"decompressed": study,
                             "arith_err_rel_bmax": {p_: {fmt_class(cls_list[c]): v for c, v in arith[p_].items()}
                                                    for p_ in arith}}
        errs16 = {prec: errs[str(BITS)][prec]["max_abs_err"] for prec in ("mixed", "fp64", "calibrated")}
        api.eri_plan_set_precision(plan, "mixed")
        n_sampled = sum(len(v) for v in sample_idx.values())
        line_extra["max_abs_err"] = {"headline": errs16["calibrated"], "mixed_all_fp32": errs16["mixed"],
                                     "fp64": errs16["fp64"], "unit": "Ha",
                                     "sample": f"{n_sampled} quartets (about {args.ref_eris} ERIs per class), "
                                               "decompressed 16-bit vs FP64 oracle"}
        line_extra["cpu_baseline"] = {"value": g_cpu, "unit": "GERIS", "cores": cores, "kind": "oracle",
                                      "sample": f"about {args.ref_eris} ERIs per class x 256 classes "
                                                f"({spent:.1f} s), per-class time per ERI scaled to the "
                                                "full class mix"}

    # ---- end to end through the C ABI with host buffers ----
    e2e = (run_e2e(args, api, pool, quartets, counts, total_eris, dev, stream, choice16)
           if not args.no_e2e else None)

    if rank == 0:
        geris_mixed = {fmt_class(cls_list[c]): round(counts[c] * W.quartet_size(*cls_list[c]) / (ms_mixed[c] * 1e-3) / 1e9, 2)
                       for c in ms_mixed}
        geris_fp64 = {fmt_class(cls_list[c]): round(counts[c] * W.quartet_size(*cls_list[c]) / (ms_fp64[c] * 1e-3) / 1e9, 2)
                      for c in ms_fp64}
        out = {
            "metric": METRIC, "value": value, "unit": "GERIS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": config_dict(args),
            "precision": {"classes_fp32": sum(v == "mixed" for v in choice16.values()),
                          "classes_fp64": [fmt_class(cls_list[c]) for c in sorted(choice16)
                                           if choice16[c] == "fp64"],
                          "rule": f"FP32 recurrences where the FP32 error measured on {CALIB_SAMPLE} quartets "
                                  f"per class stays below {CALIB_STEPS} quantisation steps (16-bit)"},
            "mixed_all_fp32": {"value": total_eris / (ms_all32 * 1e-3) / 1e9, "unit": "GERIS",
                               "ms_per_step": ms_all32},
            "fp64": {"value": total_eris / (ms_fp64_step * 1e-3) / 1e9, "unit": "GERIS",
                     "ms_per_step": ms_fp64_step, "speedup_mixed_over_fp64": ms_fp64_step / ms,
                     "how": "timed steps of eri_compute_compressed with every class in FP64"},
            "roofline": roof,
            "roofline_frac_per_class": {"min": min(frac_all.values()), "median": statistics.median(frac_all.values()),
                                        "max": max(frac_all.values()),
                                        "step_weighted": sum(t_roof.values()) / (sum(ms_cal.values()) * 1e-3)},
            "clocks": clk, "gpu_launches": launches * args.steps,
            "per_class_geris": {"mixed": geris_mixed, "fp64": geris_fp64},
        }
        out.update(line_extra)
        if e2e is not None:
            out["e2e"] = e2e
        print(json.dumps(out), flush=True)
        if args.details:
            with open(args.details, "w") as f:
                json.dump({"ms_mixed": {fmt_class(cls_list[c]): ms_mixed[c] for c in ms_mixed},
                           "ms_fp64": {fmt_class(cls_list[c]): ms_fp64[c] for c in ms_fp64},
                           "roofline_frac_mixed": {fmt_class(cls_list[c]): frac_all[c] for c in frac_all},
                           "counts": {fmt_class(cls_list[c]): counts[c] for c in range(256)},
                           "precision_study": study_details}, f, indent=1)
    plan.destroy()
    if dist is not None:
        dist.destroy_process_group()


def run_e2e(args, api, pool, quartets, counts, total_eris, dev, stream, choice):
    """Same metric through the public API with host buffers: every step creates the plan from
    pinned host quartets (host->device copy and class sort inside), applies the calibrated
    per-class precision, and computes the compressed ERIs into pinned host memory (each class's
    codes and scales are copied back while the later classes compute)."""
    import torch

    qh = torch.empty(quartets.shape, dtype=torch.int32, pin_memory=True)
    qh.copy_(quartets)
    qnp = qh.numpy()
    plan = api.eri_plan_create(pool, qnp, precision="mixed", device=dev.index)
    pb, sb = api.eri_output_bytes(plan, BITS)
    plan.destroy()
    packed = torch.empty(pb // 4, dtype=torch.int32, device=dev)
    scales = torch.empty(sb // 4, dtype=torch.float32, device=dev)
    packed_h = torch.empty(pb // 4, dtype=torch.int32, pin_memory=True)
    scales_h = torch.empty(sb // 4, dtype=torch.float32, pin_memory=True)

    def one():
        p = api.eri_plan_create(pool, qnp, precision="mixed", device=dev.index)
        apply_choices(api, p, choice)
        # each class's codes and scales stream to pinned host memory while later classes compute
        api.eri_compute_compressed_to_host(p, BITS, packed, scales, packed_h, scales_h, stream)
        api.eri_sync(p, stream)
        p.destroy()

    one()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    return {"value": total_eris / dt / 1e9, "unit": "GERIS", "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": int(qh.numel() * 4),
            "d2h_bytes_per_step": int(packed_h.numel() * 4 + scales_h.numel() * 4),
            "path": "eri_plan_create(host quartets) + per-class precision + "
                    "eri_compute_compressed_to_host (codes and scales to pinned host memory, copies "
                    "overlapping the kernels)"}


# ---------------------------------------------------------------------------------------------
# Further workloads (not the headline): --workload lattice | molecule | gradient | gshell | paper512


def _events(torch, stream, fn, reps=2):
    fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


PAPER_TABLE5 = {"[fd|ps]": 3.33, "[ps|fd]": 1.05, "[ff|dp]": 10.03, "[dp|ff]": 6.65, "[fd|fd]": 11.17,
                "[df|fd]": 10.93}


def run_lattice(args):
    """The paper's benchmark (Sec. IV-A): 32 sites on a 4x4x2 cubic lattice (1 Angstrom), one
    primitive s, p, d, f shell per site (alpha = 1.5), all 32^4 site quartets of each class,
    16-bit output, one class per launch as on the FPGA."""
    import torch

    import oracle
    from paper_2303_13632_gb300 import api

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    shells = W.lattice_shells()
    site = torch.arange(32, device=dev, dtype=torch.int32)
    sq = torch.cartesian_prod(site, site, site, site).to(torch.int32).contiguous()
    n = sq.shape[0]
    classes_ = sorted(ONLY) if ONLY else list(range(256))
    max_eri = max(W.quartet_size(*W.class_of_id(c)) for c in classes_)
    packed = torch.empty((n * max_eri * BITS + 31) // 32 + 64, dtype=torch.int32, device=dev)
    scales = torch.empty(n, dtype=torch.float32, device=dev)
    rng = np.random.default_rng(17)
    res, acc = {}, {}
    t_mixed = t_fp64 = 0.0
    total = 0
    for c in classes_:
        cls = W.class_of_id(c)
        neri = W.quartet_size(*cls)
        q = (sq * 4 + torch.tensor(cls, dtype=torch.int32, device=dev)).contiguous()
        plan = api.eri_plan_create(shells, q, precision="mixed")
        ms = {}
        for prec in ("mixed", "fp64"):
            api.eri_plan_set_precision(plan, prec)
            ms[prec] = _events(torch, stream, lambda: api.eri_compute_compressed(plan, BITS, packed, scales, stream))
        api.eri_sync(plan, stream)
        res[fmt_class(cls)] = {"mixed": n * neri / ms["mixed"] / 1e6, "fp64": n * neri / ms["fp64"] / 1e6}
        t_mixed += ms["mixed"]
        t_fp64 += ms["fp64"]
        total += n * neri
        if not args.no_check:
            # accuracy after decompression on a sample, 16 and 12 bits, mixed precision
            k = max(2, min(64, 50000 // neri))
            qi = np.sort(rng.choice(n, size=k, replace=False))
            ref, _ = oracle.eri_batch(shells, q[torch.as_tensor(qi, device=dev)].cpu().numpy())
            ref = ref.reshape(k, neri)
            api.eri_plan_set_precision(plan, "mixed")
            e = {}
            for bits in (16, 12):
                api.eri_compute_compressed(plan, bits, packed, scales, stream)
                api.eri_sync(plan, stream)
                words = packed.cpu().numpy().view(np.uint32)
                x = unpack(words, 0, qi, neri, bits) * scales.cpu().numpy()[qi][:, None].astype(np.float64)
                e[bits] = float(np.max(np.abs(x - ref)))
            acc[fmt_class(cls)] = e
        plan.destroy()
    out = {"impl": "ours", "workload": "lattice", "metric": "GERIS per class, 16-bit, paper lattice (Sec. IV-A)",
           "value": total / (t_mixed * 1e-3) / 1e9, "unit": "GERIS", "fp64_value": total / (t_fp64 * 1e-3) / 1e9,
           "classes": len(classes_), "quartets_per_class": n,
           "paper_table5_fpga_vs_ours_mixed": {k: {"fpga": v, "ours": res[k]["mixed"]} for k, v in PAPER_TABLE5.items() if k in res},
           "per_class_geris": res}
    if acc:
        canon = [k for k in acc]
        out["max_abs_err_16bit"] = max(acc[k][16] for k in canon)
        out["max_abs_err_12bit_except_ssss"] = max(acc[k][12] for k in canon if k != "[ss|ss]")
        out["accuracy_per_class"] = acc
    print(json.dumps(out), flush=True)


def run_gshell(args):
    """Classes with a g shell (L = 4, beyond the paper's s..f): the 369 classes, one run-time-L
    kernel per precision.  Primitive shells from a pool of 2048 per L (centres U[-3,3]^3 bohr,
    exponents log-U[0.1,10]), round(2^24 / n_ERIQ) quartets per class, 16-bit output, one class
    per call; per class one sampled quartet against the oracle (decompressed error and the FP32
    error of the mixed path relative to b_max)."""
    import torch

    import oracle
    from paper_2303_13632_gb300 import api

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    Ls = (0, 1, 2, 3, 4)
    rng = np.random.default_rng(2303_13632 + 6)
    pool = W.random_primitive_pool(rng, 2048, Ls=Ls)
    ids = [c for c in W.g_class_ids() if ONLY is None or c in ONLY]
    res, acc = {}, {}
    t = {"mixed": 0.0, "fp64": 0.0}
    total = 0
    for c in ids:
        cls = W.class_of_id(c)
        neri = W.quartet_size(*cls)
        n = int(round(2 ** 24 / neri))
        q = W.random_class_quartets(rng, cls, n, 2048, Ls=Ls)
        plan = api.eri_plan_create(pool, q, precision="mixed")
        nb, sb = api.eri_output_bytes(plan, BITS)
        packed = torch.empty(nb // 4, dtype=torch.int32, device=dev)
        scales = torch.empty(sb // 4, dtype=torch.float32, device=dev)
        ms = {}
        for prec in ("mixed", "fp64"):
            api.eri_plan_set_precision(plan, prec)
            ms[prec] = _events(torch, stream, lambda: api.eri_compute_compressed(plan, BITS, packed, scales, stream))
            t[prec] += ms[prec]
        api.eri_sync(plan, stream)
        total += n * neri
        res[fmt_class(cls)] = {"mixed": n * neri / ms["mixed"] / 1e6, "fp64": n * neri / ms["fp64"] / 1e6}
        if not args.no_check:
            order = api.eri_plan_quartet_order(plan)
            ref, _ = oracle.eri_batch(pool, q[order[:1]])
            api.eri_plan_set_precision(plan, "mixed")
            fp = torch.empty(neri, dtype=torch.float64, device=dev)
            sub = api.eri_plan_create(pool, q[order[:1]], precision="mixed")
            api.eri_compute(sub, fp, stream)
            api.eri_compute_compressed(plan, BITS, packed, scales, stream)
            api.eri_sync(plan, stream)
            words = packed[: (neri * BITS + 31) // 32 + 1].cpu().numpy().view(np.uint32)
            x = oracle.unpack_bits(words, neri, BITS) * float(scales[0].item())
            bmax = float(np.max(np.abs(ref)))
            # quartets with b_max <= 1e-30 Ha leave the FP32 range in the recurrences (as in the
            # calibration); their relative FP32 error is not reported
            acc[fmt_class(cls)] = {"decompressed_max_abs_err": float(np.max(np.abs(x - ref))),
                                   "half_step": float(scales[0].item()) / 2,
                                   "b_max": bmax,
                                   "fp32_err_rel_bmax": float(np.max(np.abs(fp.cpu().numpy() - ref))) / bmax if bmax > 1e-30 else None}
            sub.destroy()
        plan.destroy()
    out = {"impl": "ours", "workload": "gshell", "metric": "GERIS, classes with a g shell, 16-bit",
           "value": total / (t["mixed"] * 1e-3) / 1e9, "unit": "GERIS", "fp64_value": total / (t["fp64"] * 1e-3) / 1e9,
           "classes": len(ids), "eris": total, "quartets_per_class": "round(2^24 / n_ERIQ)",
           "per_class_geris": res}
    if acc:
        out["max_decompressed_err_16bit"] = max(v["decompressed_max_abs_err"] for v in acc.values())
        out["classes_within_one_step"] = sum(v["decompressed_max_abs_err"] <= 2 * v["half_step"] * (1 + 1e-5)
                                             for v in acc.values())
        out["max_fp32_err_rel_bmax"] = max(v["fp32_err_rel_bmax"] for v in acc.values() if v["fp32_err_rel_bmax"] is not None)
        out["accuracy_per_class"] = acc
    print(json.dumps(out), flush=True)


def run_molecule(args):
    """Batched mixed workload: 200 atoms in a 20-bohr box (min separation 1.8 bohr), shells
    s, s, p, p, d, f per atom, contraction degree 1..6.  The library enumerates the 8-fold unique
    shell quartets surviving Schwarz screening at 1e-10 on the device (ERI_UNIQUE8) and keeps an
    even 1-in-s shard of that enumeration sized to about 2^30 ERIs; the shard is computed in one
    CUDA-graph launch of persistent kernels (mixed precision, 16-bit), and its compressed output
    is digested into Coulomb and exchange matrices (eri_digest_jk, 8-fold expansion)."""
    import torch

    import oracle
    from paper_2303_13632_gb300 import api

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    basis = W.molecule_basis()
    tau = 1e-10
    budget = int(2 ** 30 * args.scale)
    t0 = time.perf_counter()
    probe = api.eri_plan_create(basis, None, mode="unique8", schwarz_threshold=tau, shard=(0, 1 << 62))
    n_cand, n_kept = api.eri_plan_screening(probe)
    probe.destroy()
    t_screen = time.perf_counter() - t0
    # ERIs per quartet of the screened set, from a 1-in-s0 shard of about 2^20 quartets
    s0 = max(1, n_kept // (1 << 20))
    p0 = api.eri_plan_create(basis, None, mode="unique8", schwarz_threshold=tau, shard=(0, s0))
    eri_per_q = api.eri_output_bytes(p0, 0)[0] / 8 / max(1, api.eri_plan_num_quartets(p0))
    p0.destroy()
    eris_all = int(round(n_kept * eri_per_q))
    shard_count = max(1, int(round(n_kept * eri_per_q / budget)))
    plan = api.eri_plan_create(basis, None, precision="mixed", mode="unique8", schwarz_threshold=tau,
                               shard=(0, shard_count))
    q = api.eri_plan_quartets(plan)
    n_eri = api.eri_output_bytes(plan, 0)[0] // 8
    nb, sb = api.eri_output_bytes(plan, BITS)
    packed = torch.empty(nb // 4, dtype=torch.int32, device=dev)
    scales = torch.empty(sb // 4, dtype=torch.float32, device=dev)
    api.eri_plan_calibrate_precision(plan, BITS, sample=CALIB_SAMPLE, max_err_steps=CALIB_STEPS, stream=stream)
    choice = class_choices(api, plan)
    ms_plain = _events(torch, stream, lambda: api.eri_compute_compressed(plan, BITS, packed, scales, stream))
    cache = os.path.join(tempfile.gettempdir(), "eri_autotune_molecule.txt")
    api.eri_autotune(plan, BITS, packed, scales, cache, stream)
    ms_graph = _events(torch, stream, lambda: api.eri_compute_compressed_batched(plan, BITS, packed, scales, stream), reps=3)
    apply_choices(api, plan, None)
    api.eri_plan_set_precision(plan, "fp64")
    api.eri_autotune(plan, BITS, packed, scales, cache, stream)
    ms_fp64 = _events(torch, stream, lambda: api.eri_compute_compressed_batched(plan, BITS, packed, scales, stream), reps=1)
    api.eri_plan_set_precision(plan, "mixed")
    # one persistent launch of the run-time-L kernel for every class from one work queue
    ms_queue = _events(torch, stream, lambda: api.eri_compute_compressed_queue(plan, BITS, packed, scales, stream),
                       reps=3)
    api.eri_sync(plan, stream)
    q_words, q_scales = packed.cpu().numpy().view(np.uint32).copy(), scales.cpu().numpy().copy()
    apply_choices(api, plan, choice)
    api.eri_compute_compressed_batched(plan, BITS, packed, scales, stream)
    api.eri_sync(plan, stream)
    # Coulomb/exchange digestion of the compressed shard (8-fold expansion of each quartet)
    nbf = api.eri_plan_num_basis_functions(plan)
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.SEED_BASE + 44)
    D = torch.randn((nbf, nbf), dtype=torch.float64, device=dev, generator=gen)
    D = (D + D.T) / 2
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    ms_digest = _events(torch, stream, lambda: api.eri_digest_jk(plan, BITS, packed, scales, D, J, K,
                                                                 unique8=True, stream=stream), reps=3)
    api.eri_sync(plan, stream)
    digest_bytes = nb + sb + 16 * len(q)  # codes, scales and the quartet table read once
    peaks, _ = read_peaks()
    out = {"impl": "ours", "workload": "molecule",
           "metric": "GERIS, batched persistent CUDA-graph launch, mixed precision, 16-bit",
           "precision": {"classes_fp32": sum(v == "mixed" for v in choice.values()),
                         "classes_fp64": sum(v == "fp64" for v in choice.values())},
           "value": n_eri / (ms_graph * 1e-3) / 1e9, "unit": "GERIS",
           "per_class_launches_geris": n_eri / (ms_plain * 1e-3) / 1e9,
           "work_queue_geris": n_eri / (ms_queue * 1e-3) / 1e9,
           "fp64_batched_geris": n_eri / (ms_fp64 * 1e-3) / 1e9,
           "budget": {"quartets": int(len(q)), "eris": int(n_eri), "shard": f"1 in {shard_count}"},
           "screened_unique_quartets": int(n_kept), "unique_quartets_before_screening": int(n_cand),
           "screened_unique_eris_estimate": eris_all,
           "shells": int(basis.n), "basis_functions": int(nbf), "screening_s": t_screen, "tau": tau,
           "digest_jk": {"geris": n_eri / (ms_digest * 1e-3) / 1e9, "ms": ms_digest,
                         "hbm_gbs": digest_bytes / (ms_digest * 1e-3) / 1e9,
                         "hbm_frac": digest_bytes / (ms_digest * 1e-3) / 1e9 / peaks["hbm_gbs"],
                         "algorithmic_bytes": int(digest_bytes),
                         "note": "compressed ERIs of the shard -> J, K with the 8-fold expansion"}}
    if not args.no_check:
        # parity on sampled quartets of modest primitive count
        L = np.asarray(basis.L)
        kprod = np.prod([basis.nprim[q[:, x]] for x in range(4)], axis=0)
        cost = kprod * oracle.quartet_sizes(basis, q)
        rng = np.random.default_rng(W.SEED_BASE + 4)
        cand = np.nonzero(cost <= 200000)[0]
        pick = np.sort(rng.choice(cand, size=min(200, len(cand)), replace=False))
        ref, offs = oracle.eri_batch(basis, q[pick])

        def worst(words, scl):
            w = 0.0
            for j, i in enumerate(pick):  # i: class-sorted position (the plan's own order)
                cls = W.class_id(*[int(L[s_]) for s_ in q[i]])
                nq_c, neri, fq, _ = api.eri_plan_class_info(plan, cls)
                off_b, _ = api.eri_packed_class_offset(plan, BITS, cls)
                x = unpack(words, off_b, np.array([i - fq]), neri, BITS)[0] * float(scl[i])
                r = ref[offs[j]:offs[j + 1]]
                bm = max(np.max(np.abs(r)), 1e-300)
                w = max(w, float(np.max(np.abs(x - r)) / bm))
            return w

        out["parity_sample"] = {"quartets": int(len(pick)),
                                "max_err_rel_bmax": worst(packed.cpu().numpy().view(np.uint32), scales.cpu().numpy()),
                                "work_queue_max_err_rel_bmax": worst(q_words, q_scales),
                                "bound_16bit_half_step_plus_fp32": 1.0 / 32767}
    print(json.dumps(out), flush=True)


def run_gradient(args):
    """Differentiation: dE/dR and dE/dalpha of E = sum G (ab|cd) for the 16 classes with every
    L in {1, 2}, 2^18 quartets each, contraction degree 3, G ~ N(0, 1)."""
    import torch

    import oracle
    from paper_2303_13632_gb300 import api

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    rng = W.rng_for(5)
    pool = W.random_contracted_pool(rng, 2048, K=3, Ls=(1, 2))
    cls_list_ = [c for c in [(a, b, c_, d) for a in (1, 2) for b in (1, 2) for c_ in (1, 2) for d in (1, 2)]]
    nper = max(1, int((1 << 18) * args.scale))
    q = np.concatenate([W.random_class_quartets(rng, c, nper, 2048, Ls=(1, 2)) for c in cls_list_])
    plan = api.eri_plan_create(pool, q, precision="fp64")
    nb, _ = api.eri_output_bytes(plan, 0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.SEED_BASE + 5)
    G = torch.randn(nb // 8, dtype=torch.float64, device=dev, generator=gen)
    dR = torch.empty((pool.n, 3), dtype=torch.float64, device=dev)
    da = torch.empty(len(pool.exps), dtype=torch.float64, device=dev)
    out_t = torch.empty(nb // 8, dtype=torch.float64, device=dev)
    n_eri = nb // 8
    timing = {}
    for prec in ("mixed", "fp64"):
        api.eri_plan_set_precision(plan, prec)
        ms_b = _events(torch, stream, lambda: api.eri_backward(plan, G, dR, da, stream), reps=1)
        ms_f = _events(torch, stream, lambda: api.eri_compute(plan, out_t, stream), reps=1)
        timing[prec] = {"ms_backward": ms_b, "ms_forward": ms_f,
                        "backward_geris": n_eri / (ms_b * 1e-3) / 1e9, "forward_geris": n_eri / (ms_f * 1e-3) / 1e9,
                        "backward_over_forward": ms_b / ms_f}
    api.eri_sync(plan, stream)
    # roofline of the backward pass: the adjoint's algorithmic FLOPs (perfmodel) of every
    # primitive quartet at the FP32 and FP64 FMA rates measured here
    peaks = measure_alu_peaks(api, torch, stream, 0)
    p32, p64 = peaks["fp32_tflops"], peaks["fp64_tflops"]
    prim_quartets = nper * 3 ** 4
    roof = {}
    for prec in ("mixed", "fp64"):
        t_roof = flops = 0.0
        for c in cls_list_:
            f64, rr = perfmodel.adjoint_flops_per_quartet(c, prec)
            if prec == "fp64":
                f64, rr = f64 + rr, 0
            t_roof += prim_quartets * (f64 / (p64 * 1e12) + rr / (p32 * 1e12))
            flops += prim_quartets * (f64 * p32 / p64 + rr)
        t = timing[prec]["ms_backward"] * 1e-3
        roof[prec] = {"bound": "alu", "achieved": flops / t / 1e12, "peak": p32, "unit": "TFLOP/s",
                      "frac": t_roof / t, "ms_roofline": t_roof * 1e3}
    out = {"impl": "ours", "workload": "gradient", "metric": "adjoint: ERI derivatives contracted per second",
           "value": timing["mixed"]["backward_geris"], "unit": "G ERI/s (backward, mixed)",
           "precisions": timing, "backward_mixed_over_forward_fp64": timing["mixed"]["ms_backward"] / timing["fp64"]["ms_forward"],
           "roofline_backward": roof,
           "roofline_note": "FP32-equivalent TFLOP/s (FP64 work weighted by the measured FP32/FP64 rate ratio) "
                            "against the measured FP32 FMA rate (eri_fma_probe)",
           "alu_peaks_tflops": {"fp32": p32, "fp64": p64},
           "quartets": int(len(q)), "eris": int(n_eri), "K": 3}
    if not args.no_check:
        # oracle derivative on a sample: a plan of the sampled quartets alone, same G values
        pick = np.sort(rng.choice(len(q), size=64, replace=False))
        qs = q[pick]
        sizes = oracle.quartet_sizes(pool, qs)
        offs = np.zeros(len(qs) + 1, dtype=np.int64)
        np.cumsum(sizes, out=offs[1:])
        Gs = np.random.default_rng(9).standard_normal(int(offs[-1]))
        splan = api.eri_plan_create(pool, qs, precision="fp64")
        order = api.eri_plan_quartet_order(splan)
        Gd = torch.tensor(np.concatenate([Gs[offs[i]:offs[i + 1]] for i in order]), device=dev)
        rR, ra = oracle.eri_grad_batch(pool, qs, Gs, offs)
        out["oracle_check"] = {"quartets": 64, "max_abs_dR": float(np.max(np.abs(rR))),
                               "max_abs_dalpha": float(np.max(np.abs(ra)))}
        for prec in ("fp64", "mixed"):
            api.eri_plan_set_precision(splan, prec)
            api.eri_backward(splan, Gd, dR, da, stream)
            api.eri_sync(splan, stream)
            gR, ga = dR.cpu().numpy(), da.cpu().numpy()
            out["oracle_check"][prec] = {"max_abs_err_dR": float(np.max(np.abs(gR - rR))),
                                         "max_abs_err_dalpha": float(np.max(np.abs(ga - ra)))}
    print(json.dumps(out), flush=True)


def run_paper512(args):
    """The paper's 512-bit output chunks (Sec. III-C) as a re-layout pass: eri_pack_paper512_stream
    on seeded random dense streams of three class shapes, each larger than L2.  CUDA events over
    10 launches after 3 warm-ups; HBM bytes = dense stream read + chunk words written."""
    import torch

    from paper_2303_13632_gb300 import api

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    peaks, src = read_peaks()
    hbm = float(peaks["hbm_gbs"])
    gen = torch.Generator(device=dev)
    gen.manual_seed(512)
    rows = {}
    for name, n_eri, bits, nq in (("[ss|ss]", 1, 16, 16000000), ("[dd|dd]", 1296, 16, 400000),
                                  ("[ff|ff]", 10000, 12, 40000)):
        F = 512 // bits
        n_cs = -(-n_eri // F)
        dense_words = (nq * n_eri * bits + 31) // 32
        d_in = torch.randint(-2 ** 31, 2 ** 31 - 1, (dense_words,), dtype=torch.int32, device=dev, generator=gen)
        d_out = torch.empty(nq * n_cs * 16, dtype=torch.int32, device=dev)
        fn = lambda: api.eri_pack_paper512_stream(d_in, nq, n_eri, bits, d_out, stream)  # noqa: E731
        for _ in range(3):
            fn()
        ms = _events(torch, stream, fn, reps=10)
        moved = dense_words * 4 + d_out.numel() * 4
        rows[name] = {"bits": bits, "quartets": nq, "chunks_per_quartet": n_cs, "bytes": moved,
                      "ms": ms, "gbs": moved / (ms * 1e-3) / 1e9, "frac_hbm": moved / (ms * 1e-3) / 1e9 / hbm}
        del d_in, d_out
    out = {"impl": "ours", "workload": "paper512", "metric": "HBM rate of the 512-bit chunk re-layout",
           "unit": "GB/s", "value": min(r["gbs"] for r in rows.values()), "peak_hbm_gbs": hbm,
           "peak_source": src, "streams": rows}
    print(json.dumps(out), flush=True)


def fmt_class(cls):
    s = "spdfg"
    return f"[{s[cls[0]]}{s[cls[1]]}|{s[cls[2]]}{s[cls[3]]}]"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep", choices=["sweep", "lattice", "molecule", "gradient", "gshell", "paper512"],
                    help="sweep (default): the 256-class benchmark; the others are further studies")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--ref-eris", type=int, default=1500000)
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--details", default=None)
    ap.add_argument("--classes", default=None,
                    help="comma-separated class ids (see eri_class_id) for the sweep and gshell workloads; profiling only")
    args = ap.parse_args()
    global ONLY
    if args.classes:
        ONLY = {int(c) for c in args.classes.split(",")}
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "lattice":
        run_lattice(args)
    elif args.workload == "molecule":
        run_molecule(args)
    elif args.workload == "gradient":
        run_gradient(args)
    elif args.workload == "gshell":
        run_gshell(args)
    elif args.workload == "paper512":
        run_paper512(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
