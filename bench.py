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
POOL_PER_L = 4096
BITS = 16


def classes():
    return [W.class_of_id(c) for c in range(256)]


ONLY = None  # --classes: restrict the sweep to these class ids (profiling runs only)


def class_counts(scale: float):
    return {c: (max(1, int(round(W.sweep_quartet_count(W.class_of_id(c)) * scale)))
                if ONLY is None or c in ONLY else 0) for c in range(256)}


def make_pool(seed_k: int = 2):
    return W.random_primitive_pool(W.rng_for(seed_k), POOL_PER_L)


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


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
    n_total = sum(counts.values())
    quartets = torch.empty((n_total, 4), dtype=torch.int32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(W.SEED_BASE + 2)
    first = {}
    pos = 0
    for c in range(256):
        cls = cls_list[c]
        n = counts[c]
        first[c] = pos
        for x in range(4):
            quartets[pos:pos + n, x] = (torch.randint(0, POOL_PER_L, (n,), generator=gen, device=dev,
                                                      dtype=torch.int32) + cls[x] * POOL_PER_L)
        pos += n
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

    # ---- headline: mixed precision, all 256 classes per step ----
    for _ in range(args.warmup):
        step()
    api.eri_sync(plan, stream)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    api.eri_sync(plan, stream)
    ms = e0.elapsed_time(e1) / args.steps
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * total_eris / (ms * 1e-3) / 1e9

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
    fp64_total_ms = sum(ms_fp64.values())

    # ---- roofline of the dominant kernel (largest share of the mixed step) ----
    peaks, peak_kind = read_peaks()
    dom = max(ms_mixed, key=lambda c: ms_mixed[c])
    dcls = cls_list[dom]
    flops = perfmodel.fp32_equivalent_flops(dcls, "mixed") * counts[dom]
    achieved = flops / (ms_mixed[dom] * 1e-3) / 1e12
    t_roof = perfmodel.roofline_seconds(dcls, counts[dom], "mixed", BITS, peaks["hbm_gbs"])
    roof = {"bound": "alu", "kernel": f"eri_class_kernel {W.class_id(*dcls)} {fmt_class(dcls)} mixed",
            "achieved": achieved, "peak": perfmodel.PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
            "frac": t_roof / (ms_mixed[dom] * 1e-3), "traffic": None,
            "peak_kind": "nominal FP32 (152 SMs x 128 lanes x 2 x 2.07 GHz); FP64 work weighted "
                         "by the FP32/FP64 peak ratio (1.25 TFLOP/s FP64)",
            "share": ms_mixed[dom] / sum(ms_mixed.values())}
    frac_all = {c: perfmodel.roofline_seconds(cls_list[c], counts[c], "mixed", BITS, peaks["hbm_gbs"])
                / (ms_mixed[c] * 1e-3) for c in ms_mixed}

    # ---- accuracy on a sample, and the CPU oracle baseline ----
    line_extra = {}
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
        errs = {}
        for prec in ("mixed", "fp64"):
            api.eri_plan_set_precision(plan, prec)
            step()
            api.eri_sync(plan, stream)
            words = packed.cpu().numpy().view(np.int16)
            sc = scales.cpu().numpy()
            worst = 0.0
            for c in nonempty(counts):
                nq, neri, fq, _ = api.eri_plan_class_info(plan, c)
                off_bytes, _ = api.eri_packed_class_offset(plan, BITS, c)
                vals, _ = ref[c]
                qi = sample_idx[c]
                pos = off_bytes // 2 + qi[:, None] * neri + np.arange(neri)[None, :]
                x = words[pos].astype(np.float64) * sc[fq + qi][:, None].astype(np.float64)
                worst = max(worst, float(np.max(np.abs(x - vals.reshape(len(qi), neri)))))
            errs[prec] = worst
        api.eri_plan_set_precision(plan, "mixed")
        n_sampled = sum(len(v) for v in sample_idx.values())
        line_extra["max_abs_err"] = {"mixed": errs["mixed"], "fp64": errs["fp64"], "unit": "Ha",
                                     "sample": f"{n_sampled} quartets (about {args.ref_eris} ERIs per class), "
                                               "decompressed 16-bit vs FP64 oracle"}
        line_extra["cpu_baseline"] = {"value": g_cpu, "unit": "GERIS", "cores": cores, "kind": "oracle",
                                      "sample": f"about {args.ref_eris} ERIs per class x 256 classes "
                                                f"({spent:.1f} s), per-class time per ERI scaled to the "
                                                "full class mix"}

    # ---- end to end through the C ABI with host buffers ----
    e2e = run_e2e(args, api, pool, quartets, counts, total_eris, dev, stream) if not args.no_e2e else None

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
            "fp64": {"value": total_eris / (fp64_total_ms * 1e-3) / 1e9, "unit": "GERIS",
                     "ms_per_step": fp64_total_ms, "speedup_mixed_over_fp64": fp64_total_ms / ms},
            "roofline": roof,
            "roofline_frac_per_class": {"min": min(frac_all.values()), "median": statistics.median(frac_all.values()),
                                        "max": max(frac_all.values())},
            "clocks": clk, "gpu_launches": len(nonempty(counts)) * args.steps,
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
                           "counts": {fmt_class(cls_list[c]): counts[c] for c in range(256)}}, f, indent=1)
    plan.destroy()
    if dist is not None:
        dist.destroy_process_group()


def run_e2e(args, api, pool, quartets, counts, total_eris, dev, stream):
    """Same metric through the public API with host buffers: every step creates the plan from
    pinned host quartets (host->device copy and class sort inside), computes the compressed
    ERIs and copies packed codes and scales back to pinned host memory."""
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
        api.eri_compute_compressed(p, BITS, packed, scales, stream)
        packed_h.copy_(packed, non_blocking=True)
        scales_h.copy_(scales, non_blocking=True)
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
            "path": "eri_plan_create(host quartets) + eri_compute_compressed + D2H of codes and scales"}


def fmt_class(cls):
    s = "spdf"
    return f"[{s[cls[0]]}{s[cls[1]]}|{s[cls[2]]}{s[cls[3]]}]"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--ref-eris", type=int, default=1500000)
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--details", default=None)
    ap.add_argument("--classes", default=None,
                    help="comma-separated class ids ((La*4+Lb)*4+Lc)*4+Ld; profiling only")
    args = ap.parse_args()
    global ONLY
    if args.classes:
        ONLY = {int(c) for c in args.classes.split(",")}
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
