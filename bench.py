#!/usr/bin/env python
"""Benchmark: periodic KIFMM targets/s on the Stokes triply periodic workload.

Workload (default): Stokes velocity kernel, triply periodic unit cube,
N = 1,048,576 uniform points (sources = targets), forces N(0,1) per component
with the net force removed, p = 8, leaf <= 64, one density vector; the MIXED
path (binary32 kernel sums, M2L on the tensor cores, binary64 root operator).
A step is one pkifmm_evaluate: Morton sort, octree, lists, upward pass, root
periodic operator, M2L, downward pass, leaves.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 oracle
(Ewald sum) instead, on a bounded sample of the same workload's targets.
Multi-GPU (torchrun): each rank evaluates its own independent problem of the
same size (independent problems shard with no data-path collective); the
value is the sum over ranks, the time the max over ranks.
"""

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "periodic KIFMM targets/sec at rel L2 err ≤1e-5 vs FP64 Ewald (mixed+batched vs FP64)"
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, gpu):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={SMI_FIELDS}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu), "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].strip().replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


def workload(n, seed):
    from paper_1705_02043_gb300 import workloads as w
    x, f = w.stokes_uniform(n, seed=seed, nrhs=1)
    return x, f


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on a bounded target sample per step."""
    if rank != 0:
        return
    import oracle
    x, f = workload(args.n, 0)
    rng = np.random.default_rng(123)
    per_step = args.ref_sample
    times = []
    for s in range(args.warmup + args.steps):
        idx = rng.choice(args.n, per_step, replace=False)
        t = time.perf_counter()
        oracle.stokes_tp(x, f[0], x[idx])
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
    v = per_step / float(np.mean(times))
    sample = f"{per_step} of {args.n} targets per step (seeded), all {args.n} sources"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "targets/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"stokes_tp_uniform_N{args.n}_p8_leaf64", "oracle": "Hasimoto Ewald, FP64, CPU"},
        "cpu_baseline": {"value": v, "unit": "targets/s", "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "targets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--sample", type=int, default=256, help="oracle targets for accuracy / cpu_baseline")
    ap.add_argument("--ref-sample", type=int, default=64, help="oracle targets per reference step")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison step")
    args = ap.parse_args()

    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1705_02043_gb300 as pk
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    x, f = workload(args.n, rank)
    cache = os.path.join(ROOT, "_build_cache")
    plan = pk.PeriodicKIFMM(pk.STOKES, 7, p=args.p, leaf_max=args.leaf, depth_max=10, precision=pk.MIXED,
                            nrhs=1, cache_dir=cache)
    tx, tf = torch.tensor(x, device=dev), torch.tensor(f, device=dev)
    out = torch.empty((1, args.n, 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MiB > L2
    for _ in range(args.warmup):
        plan.evaluate(tx, tf, tx, out)
    barrier()
    clk = ClockSampler(local)
    l0 = pk.pkifmm_launch_count()
    step_ms, m2l_ms = [], []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.add_(1.0)  # write a buffer larger than L2 between timed steps
        ev[k][0].record(stream)
        plan.evaluate(tx, tf, tx, out)
        ev[k][1].record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev[k][0].elapsed_time(ev[k][1]))
        m2l_ms.append(float(plan.stage_times()[4]))
    barrier()
    launches = pk.pkifmm_launch_count() - l0
    clocks = clk.stop()
    stages = plan.stage_times().tolist()
    stats = plan.tree_stats().tolist()
    t_step = float(np.mean(step_ms))
    if dist is not None:
        t = torch.tensor([t_step], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_step = float(t.item())
    value = world * args.n / (t_step / 1e3)

    # end to end through the host-buffer entry point (pinned host memory)
    hx = torch.tensor(x).pin_memory()
    hf = torch.tensor(f).pin_memory()
    hp = torch.empty((1, args.n, 3), dtype=torch.float64).pin_memory()
    plan.evaluate_host(hx, hf, hx, hp)
    barrier()
    e2e_t = []
    for _ in range(max(3, min(args.steps, 5))):
        flush.add_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.evaluate_host(hx, hf, hx, hp)
        e2e_t.append(time.perf_counter() - t0)
    e2e_v = world * args.n / float(np.mean(e2e_t))
    h2d = 3 * 8 * args.n * 3  # sources, forces, targets
    d2h = 3 * 8 * args.n

    result = None
    if rank == 0:
        u = out.cpu().numpy()[0]
        pk_, src = peaks()
        nV = stats[4]
        kn = 3 * (6 * (args.p - 1) ** 2 + 2)
        flops = 2.0 * kn * kn * nV  # per M2L launch, nrhs = 1
        m2l_avg = float(np.mean(m2l_ms))
        achieved = flops / (m2l_avg / 1e3) / 1e12
        tc = plan_uses_tensor_cores()
        if tc:
            peak = pk_.get("bf16_tflops_sustained", 1700.0)
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": "M2L (V list), split-fp16 x3 tcgen05", "peak_source": f"bf16_tflops_sustained ({src})"}
        else:
            mhz = (clocks or {}).get("sm_mhz") or pk_.get("sm_max_mhz", 2070.0)
            peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": None, "kernel": "M2L (V list), FP32 FMA",
                    "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz"}
        roof["algorithmic_flops_per_launch"] = flops
        roof["avg_launch_ms"] = m2l_avg
        # accuracy and the CPU baseline: the FP64 oracle on a seeded target sample
        import oracle
        rng = np.random.default_rng(123)
        idx = np.sort(rng.choice(args.n, args.sample, replace=False))
        t0 = time.perf_counter()
        ref = oracle.stokes_tp(x, f[0], x[idx])
        t_cpu = time.perf_counter() - t0
        err = oracle.error_metrics(u[idx], ref)
        fp64 = None
        if not args.no_fp64:
            p64 = pk.PeriodicKIFMM(pk.STOKES, 7, p=args.p, leaf_max=args.leaf, depth_max=10, precision=pk.FP64,
                                   nrhs=1, cache_dir=cache)
            o64 = torch.empty_like(out)
            p64.evaluate(tx, tf, tx, o64)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.add_(1.0)
            e0.record(stream)
            p64.evaluate(tx, tf, tx, o64)
            e1.record(stream)
            torch.cuda.synchronize()
            t64 = e0.elapsed_time(e1)
            fp64 = {"value": args.n / (t64 / 1e3), "unit": "targets/s", "ms_per_step": t64,
                    "rel_l2": oracle.error_metrics(o64.cpu().numpy()[0][idx], ref)["rel_l2"],
                    "stage_ms": p64.stage_times().tolist()}
            p64.close()
        result = {
            "metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "mixed: f32 sums, fp16x3 tensor M2L, f64 root" if tc else "f32",
            "data": "synthetic (seeded uniform points, N(0,1) forces, net force removed)",
            "config": {"workload": f"stokes_tp_uniform_N{args.n}_p{args.p}_leaf{args.leaf}", "kernel": "stokes",
                       "periodic": "xyz", "N": args.n, "p": args.p, "leaf_max": args.leaf, "nrhs": 1,
                       "precision": "mixed", "parallelism": f"{world} independent problems",
                       "l2": "256 MiB buffer written between timed steps"},
            "e2e": {"value": e2e_v, "unit": "targets/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": 1e3 * float(np.mean(e2e_t))},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": {"value": args.sample / t_cpu, "unit": "targets/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{args.sample} of {args.n} targets (seeded), all {args.n} sources"},
            "accuracy": {"vs": "FP64 Ewald oracle", "targets": args.sample, **err},
            "fp64_path": fp64,
            "stage_ms": dict(zip(["sort", "tree_lists", "upward", "root", "m2l", "downward", "leaves", "total"],
                                 stages)),
            "tree": dict(zip(["boxes", "leaves", "depth", "U", "V", "W", "X", "p2p_pairs"], stats)),
            "clocks": clocks,
        }
    plan.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if result is not None:
        print(json.dumps(result), flush=True)


def plan_uses_tensor_cores():
    """True when the library's M2L runs on the tensor cores (tcgen05)."""
    import paper_1705_02043_gb300 as pk
    return hasattr(pk.load_library(), "pkifmm_m2l_tensor_core_enabled") and \
        bool(pk.load_library().pkifmm_m2l_tensor_core_enabled())


if __name__ == "__main__":
    main()
