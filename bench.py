#!/usr/bin/env python
"""Benchmark: periodic KIFMM targets/s.

Workloads (``--workload``; the default is the first):

* ``stokes_tp``: Stokes velocity kernel, triply periodic unit cube,
  N = 1,048,576 uniform points (sources = targets), forces N(0,1) per
  component with the net force removed, p = 8, leaf <= 64, one density
  vector.
* ``stokes_dp_slab``: Stokes, periodic in x and y, N = 4,194,304 points in 64
  Gaussian clusters (sigma 0.02) inside the slab z in [0, 0.2], zero net
  force, p = 10, adaptive tree to depth 12.
* ``stokes_tp_batch16``: Stokes TP, N = 2,097,152 uniform points, 16 force
  vectors on one geometry, p = 8.
* ``laplace_tp_multi``: 256 independent triply periodic Laplace problems,
  N log-uniform in [1024, 65536], neutral charges U[-1,1], p = 6, one batched
  evaluation; the leaf size is picked by the library's autotuner first.
* ``stokes_chebyshev`` / ``stokes_lognormal``: the paper's Stokes timing point
  sets (97^3 Chebyshev grid; 912,673 lognormal(0.2, 0.5) points), any
  periodicity (``--periodic``).
* ``stokes_tp_pressure``: the ``stokes_tp`` problem with velocity and pressure
  at every target (the Stokes evaluation plus a Laplace field evaluation of
  the three force components).

All run the MIXED path (binary32 kernel sums, M2L on the tensor cores,
binary64 root operator).  A step is one evaluation: Morton sort, octree,
lists, upward pass, root periodic operator, M2L, downward pass, leaves.
Targets/s counts targets x density vectors.

Prints one JSON line (rank 0): throughput, the device-timed step and the
end-to-end one through the host entry point, the M2L roofline, accuracy
against the FP64 oracle on sampled targets, the FP64 path beside the MIXED
one, and two CPU baselines: the oracle on the sampled targets
(``cpu_baseline``) and the plain binary64 KIFMM of ``baseline/cpu_kifmm`` on a
2^17-point instance of the workload with the library timed on the same
instance (``cpu_kifmm``; ``--cpu-kifmm-n 0`` skips it).  `--impl reference`
times the FP64 oracle (Ewald sum) instead, on a bounded sample of the same
workload's targets.
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


WORKLOADS = {
    "stokes_tp": dict(kernel=1, periodic=7, n=1 << 20, p=8, leaf=64, depth=10, nrhs=1, sample=1024),
    "stokes_dp_slab": dict(kernel=1, periodic=3, n=1 << 22, p=10, leaf=64, depth=12, nrhs=1, sample=128),
    "stokes_tp_batch16": dict(kernel=1, periodic=7, n=1 << 21, p=8, leaf=64, depth=10, nrhs=16, sample=128),
    "laplace_tp_multi": dict(kernel=0, periodic=7, n=256, p=6, leaf=32, depth=10, nrhs=1, sample=32),
    "stokes_chebyshev": dict(kernel=1, periodic=7, n=97, p=8, leaf=64, depth=12, nrhs=1, sample=128),
    "stokes_lognormal": dict(kernel=1, periodic=7, n=97 ** 3, p=8, leaf=64, depth=12, nrhs=1, sample=128),
    # velocity and pressure (kernel 3): the Stokes evaluation plus a Laplace field
    # evaluation on the three force components
    "stokes_tp_pressure": dict(kernel=3, periodic=7, n=1 << 20, p=8, leaf=64, depth=10, nrhs=1, sample=128),
}


def workload(name, n, seed):
    """(points, densities [nrhs][N][k], problem offsets or None, description)."""
    from paper_1705_02043_gb300 import workloads as w
    if name in ("stokes_tp", "stokes_tp_pressure"):
        x, f = w.stokes_uniform(n, seed=seed, nrhs=1)
        return x, f, None, "seeded uniform points, N(0,1) forces, net force removed"
    if name == "stokes_dp_slab":
        x, f = w.clustered_slab(n, seed=seed, nclusters=64, sigma=0.02, zlo=0.0, zhi=0.2, kdim=3)
        return x, f[None], None, "64 Gaussian clusters (sigma 0.02) in the slab z in [0, 0.2], N(0,1) forces, zero net"
    if name == "stokes_tp_batch16":
        x, f = w.stokes_uniform(n, seed=seed, nrhs=16)
        return x, f, None, "seeded uniform points, 16 N(0,1) force vectors, each with zero net force"
    if name == "laplace_tp_multi":
        x, q, off = w.multi_laplace_tp(n, seed=seed)
        return x, q[None, :, None], off, f"{n} problems, N log-uniform in [1024, 65536], neutral U[-1,1] charges"
    if name in ("stokes_chebyshev", "stokes_lognormal"):
        # the point sets of the paper's Stokes timing tests, forces U[-0.5, 0.5)^3 with zero net
        if name == "stokes_chebyshev":
            x = w.chebyshev_grid(n)
            desc = f"{n}^3 Chebyshev grid (both ends; on free axes scaled by 1 - 2^-20 into [0, 1))"
            if PERIODIC_OVERRIDE is not None and PERIODIC_OVERRIDE != 7:
                x = x * (1.0 - 2.0 ** -20)
        else:
            x = w.lognormal_points(n, seed=seed)
            desc = f"{n} points, each coordinate lognormal(0.2, 0.5) wrapped mod 1"
        f = w.make_neutral(np.random.default_rng(seed).uniform(-0.5, 0.5, size=(len(x), 3)))
        return x, f[None], None, desc + ", U[-0.5, 0.5)^3 forces, zero net"
    raise ValueError(name)


PERIODIC_OVERRIDE = None  # --periodic for the paper-shaped workloads


def oracle_sum(kernel, periodic, x, d, xt):
    import oracle
    if kernel == 3:  # velocity and pressure
        return np.concatenate([oracle.periodic_sum(1, periodic, x, d, xt),
                               oracle.stokes_pressure(periodic, x, d, xt)[:, None]], axis=1)
    out = oracle.periodic_sum(kernel, periodic, x, d, xt)
    return out if kernel == 1 else out[:, None]


def oracle_sample(wl, x, d, off, nsample, rng):
    """Seeded target sample and the oracle's values there (first density vector)."""
    kernel, periodic = wl["kernel"], wl["periodic"]
    if off is None:
        idx = np.sort(rng.choice(len(x), nsample, replace=False))
        return idx, oracle_sum(kernel, periodic, x, d[0], x[idx])
    # independent problems: 8 seeded problems, nsample targets each
    probs = np.sort(rng.choice(len(off) - 1, min(8, len(off) - 1), replace=False))
    idx, ref = [], []
    for j in probs:
        a, b = off[j], off[j + 1]
        t = np.sort(rng.choice(b - a, min(nsample, b - a), replace=False)) + a
        idx.append(t)
        ref.append(oracle_sum(kernel, periodic, x[a:b], d[0, a:b], x[t]))
    return np.concatenate(idx), np.concatenate(ref)


def oracle_sample_cached(cache_dir, wl, x, d, off, nsample, rng):
    """oracle_sample, kept on disk under cache_dir (when given) by a digest of
    the kernel, periodicity, points, first density vector and sample size, with
    the oracle's own time for it.  Returns (idx, ref, seconds, cached)."""
    key = None
    if cache_dir:
        import hashlib
        h = hashlib.sha1()
        h.update(repr((wl["kernel"], wl["periodic"], nsample)).encode())
        h.update(np.ascontiguousarray(x).tobytes())
        h.update(np.ascontiguousarray(d[0]).tobytes())
        if off is not None:
            h.update(np.asarray(off).tobytes())
        key = os.path.join(cache_dir, f"oracle_{h.hexdigest()}.npz")
        if os.path.exists(key):
            z = np.load(key)
            return z["idx"], z["ref"], float(z["seconds"]), True
    t0 = time.perf_counter()
    idx, ref = oracle_sample(wl, x, d, off, nsample, rng)
    t_cpu = time.perf_counter() - t0
    if key:
        os.makedirs(cache_dir, exist_ok=True)
        np.savez(key, idx=idx, ref=ref, seconds=t_cpu)
    return idx, ref, t_cpu, False


def workload_name(name, wl, n, p, leaf):
    if name == "laplace_tp_multi":
        return f"laplace_tp_multi_{n}problems_p{p}"
    if name in ("stokes_chebyshev", "stokes_lognormal"):
        per = {0: "free", 1: "spx", 2: "spy", 4: "spz", 3: "dpxy", 7: "tp"}[wl["periodic"]]
        return f"{name}_{per}_N{n ** 3 if name == 'stokes_chebyshev' else n}_p{p}_leaf{leaf}"
    return f"{name}_N{n}_p{p}_leaf{leaf}" + (f"_nrhs{wl['nrhs']}" if wl["nrhs"] > 1 else "")


def run_reference(args, rank, world, wl):
    """Reference arm: the FP64 oracle on a bounded target sample per step."""
    if rank != 0:
        return
    x, d, off, desc = workload(args.workload, args.n, 0)
    rng = np.random.default_rng(123)
    times, ntg = [], 0
    for s in range(args.warmup + args.steps):
        t = time.perf_counter()
        idx, _ = oracle_sample(wl, x, d, off, args.ref_sample, rng)
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
            ntg = len(idx)
    v = ntg / float(np.mean(times))
    sample = (f"{ntg} targets per step (seeded) of the workload, all sources of their problem; "
              f"first density vector")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "targets/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.workload, wl, args.n, args.p, args.leaf),
                   "oracle": "Ewald sums (Hasimoto for Stokes), FP64, CPU"},
        "cpu_baseline": {"value": v, "unit": "targets/s", "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "targets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_precompute(args, wl, pk):
    """Stage 1 timing (the precompute of Algorithm 2; Sec. 3.7 tabulates it on CPUs)."""
    from paper_1705_02043_gb300 import _binding as pkb
    import torch
    kernel, periodic = wl["kernel"], wl["periodic"]
    kop = 0 if kernel in (0, 2) else 1  # the translation kernel
    torch.cuda.init()
    dev = pkb.pkifmm_precompute_operators(kop, periodic, args.p, args.ell, pk.MIXED, 1, want_ops=False)
    dev_s, ph = dev[4], dev[5]
    host_s = (pkb.pkifmm_precompute_operators(kop, periodic, args.p, args.ell, pk.MIXED, 0, want_ops=False)[4]
              if args.precompute_host else None)
    t0 = time.perf_counter()
    plan = pk.PeriodicKIFMM(kernel, periodic, p=args.p, ell=args.ell, leaf_max=args.leaf, depth_max=wl["depth"],
                            precision=pk.MIXED, nrhs=wl["nrhs"], cache_dir=None)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    plan.close()
    kn = (6 * (args.p - 1) ** 2 + 2) * (1 if kop == 0 else 3)
    print(json.dumps({
        "metric": "Stage 1 precompute time (surface SVD, M2M/L2L, root far-field table), device build",
        "value": dev_s, "unit": "s", "n_gpus": 1, "higher_is_better": False, "dtype": "f64",
        "data": "none (operators depend only on kernel, periodicity, p, ell)",
        "config": {"workload": f"precompute_{'stokes' if kernel else 'laplace'}_per{periodic}_p{args.p}_ell{args.ell}",
                   "kernel": "stokes" if kernel else "laplace", "periodic": periodic, "p": args.p, "ell": args.ell,
                   "kn": kn},
        "device_phases_s": {"svd": ph[0], "m2m_l2l": ph[1], "root_table": ph[2]}, "jacobi_sweeps": int(ph[3]),
        "host_s": host_s, "host_threads": os.cpu_count() if host_s is not None else None,
        "plan_create_s": plan_s,
        "plan_create_covers": "device Stage 1 + the 316 M2L operators + uploads, no cache",
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stokes_tp", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=None, help="points (problems for laplace_tp_multi)")
    ap.add_argument("--p", type=int, default=None)
    ap.add_argument("--ell", type=int, default=2, choices=[1, 2, 3],
                    help="image layers summed directly in the root operator (Sec. 3.6 varies 1..3)")
    ap.add_argument("--leaf", type=int, default=None)
    ap.add_argument("--sample", type=int, default=None, help="oracle targets for accuracy / cpu_baseline")
    ap.add_argument("--cpu-kifmm-n", type=int, default=1 << 17,
                    help="points of the instance the plain CPU KIFMM baseline runs on (0: skip it)")
    ap.add_argument("--oracle-cache", default=None,
                    help="directory keeping the oracle's sampled values between runs on the same inputs")
    ap.add_argument("--ref-sample", type=int, default=64, help="oracle targets per reference step")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison step")
    ap.add_argument("--precompute-host", action="store_true", help="also time Stage 1 built on the host")
    ap.add_argument("--precompute-only", action="store_true",
                    help="time Stage 1 alone for the workload's kernel, periodicity, p and ell (one JSON line)")
    ap.add_argument("--periodic", type=int, default=None, choices=[0, 1, 2, 4, 3, 7],
                    help="periodic axes for stokes_chebyshev / stokes_lognormal (bit 0 = x)")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.periodic is not None:
        if not args.workload.startswith("stokes_chebyshev") and not args.workload.startswith("stokes_lognormal"):
            ap.error("--periodic applies to the paper-shaped workloads only")
        wl["periodic"] = args.periodic
        global PERIODIC_OVERRIDE
        PERIODIC_OVERRIDE = args.periodic
    args.n = args.n or wl["n"]
    args.p = args.p or wl["p"]
    args.leaf = args.leaf or wl["leaf"]
    args.sample = args.sample or wl["sample"]
    kernel, periodic, nrhs = wl["kernel"], wl["periodic"], wl["nrhs"]
    ks = 1 if kernel in (0, 2) else 3  # source density components
    k = {0: 1, 1: 3, 2: 4, 3: 4}[kernel]  # target components

    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        run_reference(args, rank, world, wl)
        return

    import torch
    import paper_1705_02043_gb300 as pk
    from paper_1705_02043_gb300 import multi
    if args.precompute_only:
        if rank == 0:
            run_precompute(args, wl, pk)
        return
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

    x, d, off, desc = workload(args.workload, args.n, rank)
    ntrg = len(x)
    cache = os.path.join(ROOT, "_build_cache")
    plan = pk.PeriodicKIFMM(kernel, periodic, p=args.p, ell=args.ell, leaf_max=args.leaf, depth_max=wl["depth"],
                            precision=pk.MIXED, nrhs=nrhs, cache_dir=cache)
    tx, td = torch.tensor(x, device=dev), torch.tensor(np.ascontiguousarray(d), device=dev)
    out = torch.empty((nrhs, ntrg, k), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    tuned = None
    if off is not None:
        best, ms = plan.autotune_leaf(off, off, tx, td, tx, candidates=(16, 24, 32, 48, 64, 96), reps=1)
        tuned = {"candidates": [16, 24, 32, 48, 64, 96], "ms": [round(float(v), 3) for v in ms], "best": best}
        args.leaf = best

    def evaluate(o):
        if off is None:
            plan.evaluate(tx, td, tx, o)
        else:
            plan.evaluate_batched(off, off, tx, td, tx, o)

    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MiB > L2
    for _ in range(args.warmup):
        evaluate(out)
    barrier()
    clk = ClockSampler(local)
    l0 = pk.pkifmm_launch_count()
    step_ms, m2l_ms = [], []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.add_(1.0)  # write a buffer larger than L2 between timed steps
        ev[i][0].record(stream)
        evaluate(out)
        ev[i][1].record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev[i][0].elapsed_time(ev[i][1]))
        m2l_ms.append(float(plan.stage_times()[8]))
    barrier()
    launches = pk.pkifmm_launch_count() - l0
    clocks = clk.stop()
    stages = plan.stage_times().tolist()
    stats = plan.tree_stats().tolist()
    m2l_rank = plan.m2l_rank()
    m2l_rank_p = None
    if kernel == 3:  # the pressure plan's Laplace M2L works in its own dimension
        lp = pk.PeriodicKIFMM(0, periodic, p=args.p, ell=args.ell, leaf_max=args.leaf, depth_max=wl["depth"],
                              precision=pk.MIXED, nrhs=nrhs, cache_dir=cache)
        m2l_rank_p = lp.m2l_rank()
        lp.close()
    t_step = multi.max_over_ranks(float(np.mean(step_ms)), dist, dev)
    value = world * ntrg * nrhs / (t_step / 1e3)

    # end to end through the public API with host buffers (pinned host memory):
    # host->device copies of points and densities, the evaluation, device->host result
    hx = torch.tensor(x).pin_memory()
    hd = torch.tensor(np.ascontiguousarray(d)).pin_memory()
    hp = torch.empty((nrhs, ntrg, k), dtype=torch.float64).pin_memory()

    def e2e_step():
        if off is None:
            plan.evaluate_host(hx, hd, hx, hp)
        else:
            gx, gd = hx.to(dev, non_blocking=True), hd.to(dev, non_blocking=True)
            go = plan.evaluate_batched(off, off, gx, gd, gx)
            hp.copy_(go, non_blocking=True)
            torch.cuda.synchronize()

    e2e_step()
    barrier()
    e2e_t = []
    for _ in range(max(3, min(args.steps, 5))):
        flush.add_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_v = world * ntrg * nrhs / multi.max_over_ranks(float(np.mean(e2e_t)), dist, dev)
    h2d = 8 * (3 * ntrg + nrhs * ntrg * ks) if off is not None else 8 * (3 * ntrg + nrhs * ntrg * ks + 3 * ntrg)
    d2h = 8 * nrhs * ntrg * k

    result = None
    if rank == 0:
        u = out.cpu().numpy()
        pk_, src = peaks()
        nV = stats[4]
        nsurf = 6 * (args.p - 1) ** 2 + 2
        kn = ks * nsurf
        rk = m2l_rank  # kn, or r of the shared M2L basis
        flops = 2.0 * rk * rk * nV * nrhs  # per M2L (all launches of one evaluation)
        if kernel == 3:  # plus the pressure evaluation's M2L (Laplace translations, one vector)
            flops += 2.0 * m2l_rank_p * m2l_rank_p * nV * nrhs
        m2l_avg = float(np.mean(m2l_ms))
        achieved = flops / (m2l_avg / 1e3) / 1e12
        peak = pk_.get("bf16_tflops_sustained", 1700.0)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": m2l_traffic(workload_name(args.workload, wl, args.n, args.p, args.leaf)),
                "kernel": "k_m2l_tc / k_m2l_tcw: M2L (V list), split-fp16 x3 tcgen05",
                "m2l_dimension": m2l_rank, "kn": kn,
                "flops_counted": "2 r^2 per V pair and vector, r the dimension the M2L works in "
                                 "(the shared basis's rank, or kn for dense operators)",
                "peak_source": f"bf16_tflops_sustained ({src}), same rate as fp16",
                "algorithmic_flops_per_launch": flops, "avg_launch_ms": m2l_avg,
                "issued_tensor_frac": achieved * 3 / peak}
        # accuracy and the CPU baseline: the FP64 oracle on a seeded target sample
        rng = np.random.default_rng(123)
        idx, ref, t_cpu, cached = oracle_sample_cached(args.oracle_cache, wl, x, d, off, args.sample, rng)
        err = __import__("oracle").error_metrics(u[0][idx], ref)
        kifmm_cpu = cpu_kifmm_block(args, wl, pk, dev, cache) if args.cpu_kifmm_n > 0 else None
        fp64 = None
        if not args.no_fp64:
            p64 = pk.PeriodicKIFMM(kernel, periodic, p=args.p, ell=args.ell, leaf_max=args.leaf,
                                   depth_max=wl["depth"], precision=pk.FP64, nrhs=nrhs, cache_dir=cache)
            o64 = torch.empty_like(out)

            def ev64():
                if off is None:
                    p64.evaluate(tx, td, tx, o64)
                else:
                    p64.evaluate_batched(off, off, tx, td, tx, o64)
            ev64()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.add_(1.0)
            e0.record(stream)
            ev64()
            e1.record(stream)
            torch.cuda.synchronize()
            t64 = e0.elapsed_time(e1)
            fp64 = {"value": ntrg * nrhs / (t64 / 1e3), "unit": "targets/s", "ms_per_step": t64,
                    "rel_l2": __import__("oracle").error_metrics(o64.cpu().numpy()[0][idx], ref)["rel_l2"],
                    "stage_ms": p64.stage_times().tolist()}
            p64.close()
        # Stage 1 (precompute) timed on its own, device build and optionally host build
        from paper_1705_02043_gb300 import _binding as pkb
        kop = 0 if kernel in (0, 2) else 1  # the translation kernel
        dev_pre = pkb.pkifmm_precompute_operators(kop, periodic, args.p, args.ell, pk.MIXED, 1, want_ops=False)
        pre = {"device_s": dev_pre[4],
               "device_phases_s": {"svd": dev_pre[5][0], "m2m_l2l": dev_pre[5][1], "root_table": dev_pre[5][2]},
               "jacobi_sweeps": int(dev_pre[5][3]),
               "host_s": (pkb.pkifmm_precompute_operators(kop, periodic, args.p, args.ell, pk.MIXED, 0,
                                                          want_ops=False)[4] if args.precompute_host else None),
               "host_threads": os.cpu_count() if args.precompute_host else None,
               "covers": "surface SVD, M2M/L2L, root far-field table (the M2L operators are formed on the "
                         "device at plan creation in both builds)"}
        result = {
            "metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "mixed: f32 kernel sums, fp16x3 tensor-core M2L and translations, f64 root",
            "data": f"synthetic ({desc})",
            "config": {"workload": workload_name(args.workload, wl, args.n, args.p, args.leaf),
                       "kernel": {0: "laplace", 1: "stokes", 2: "laplace_field", 3: "stokes_velocity_pressure"}[kernel],
                       "periodic": {7: "xyz", 3: "xy", 0: "none"}.get(periodic, str(periodic)),
                       "N": ntrg, "p": args.p, "ell": args.ell, "leaf_max": args.leaf, "depth_max": wl["depth"], "nrhs": nrhs,
                       "problems": 1 if off is None else len(off) - 1,
                       "precision": "mixed", "parallelism": f"{world} independent problems",
                       "l2": "256 MiB buffer written between timed steps"},
            "e2e": {"value": e2e_v, "unit": "targets/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": 1e3 * float(np.mean(e2e_t))},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": {"value": len(idx) / t_cpu, "unit": "targets/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{len(idx)} seeded targets of the workload, all sources of their problem, "
                                       f"first density vector" + (" (time of the cached oracle run)" if cached else "")},
            "cpu_kifmm": kifmm_cpu,
            "accuracy": {"vs": "FP64 Ewald oracle", "targets": int(len(idx)), "density_vector": 0, **err},
            "fp64_path": fp64,
            "precompute": pre,
            "stage_ms": dict(zip(["sort", "tree_lists", "upward", "root", "m2l", "downward", "leaves", "total"],
                                 stages)),
            "tree": dict(zip(["boxes", "leaves", "depth", "U", "V", "W", "X", "p2p_pairs"], stats)),
            "autotune": tuned,
            "p2p": p2p_block(kernel, args.p, ntrg, nrhs, stats, stages[6], clocks, pk_,
                             torch.cuda.get_device_properties(dev).multi_processor_count) if kernel in (0, 1) else None,
            "clocks": clocks,
        }
    plan.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if result is not None:
        print(json.dumps(result), flush=True)


def cpu_kifmm_block(args, wl, pk, dev, cache):
    """The plain binary64 KIFMM on the host cores (baseline/cpu_kifmm, C++/OpenMP,
    sharing no code with the library or the oracle) on a smaller instance of the
    same workload (same point and density distribution, p and leaf size), with
    the GPU library timed on that same instance and both checked against the
    oracle on a target sample.  Kernels Laplace/Stokes, free or triply periodic,
    one density vector, one problem; else None."""
    kernel, periodic = wl["kernel"], wl["periodic"]
    if kernel not in (0, 1) or periodic not in (0, 7) or wl["nrhs"] != 1 or args.workload == "laplace_tp_multi":
        return None
    import torch
    from baseline import cpu_kifmm
    n = min(args.n, args.cpu_kifmm_n)
    x, d, _, _ = workload(args.workload, n, 0)
    u, t, depth = cpu_kifmm.evaluate(kernel, periodic, args.p, args.leaf, x, d[0].reshape(n, -1))
    idx = np.sort(np.random.default_rng(7).choice(n, min(64, n), replace=False))
    ref = oracle_sum(kernel, periodic, x, d[0], x[idx]).reshape(len(idx), -1)
    rel = lambda a: float(np.linalg.norm(a - ref) / np.linalg.norm(ref))
    # the GPU library (MIXED) on the same instance, device time per evaluation
    plan = pk.PeriodicKIFMM(kernel, periodic, p=args.p, ell=args.ell, leaf_max=args.leaf, depth_max=wl["depth"],
                            precision=pk.MIXED, nrhs=1, cache_dir=cache)
    tx, td = torch.tensor(x, device=dev), torch.tensor(np.ascontiguousarray(d), device=dev)
    out = torch.empty((1, n, 1 if kernel == 0 else 3), dtype=torch.float64, device=dev)
    for _ in range(3):
        plan.evaluate(tx, td, tx, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        plan.evaluate(tx, td, tx, out)
    e1.record()
    torch.cuda.synchronize()
    gpu_ms = e0.elapsed_time(e1) / 5
    ug = out[0].cpu().numpy()[idx]
    plan.close()
    return {"value": n / (t[1] + t[2]), "unit": "targets/s", "cores": cpu_kifmm.threads(),
            "kind": "plain FP64 KIFMM, C++/OpenMP (uniform octree, dense operators)",
            "N": n, "p": args.p, "leaf_max": args.leaf, "depth": depth,
            "tree_s": float(t[1]), "eval_s": float(t[2]), "operator_setup_s": float(t[0]),
            "rel_l2": rel(u[idx].reshape(len(idx), -1)), "targets_checked": int(len(idx)),
            "gpu_same_instance": {"value": n / (gpu_ms / 1e3), "ms": gpu_ms, "precision": "mixed",
                                  "rel_l2": rel(ug.reshape(len(idx), -1))}}


def p2p_block(kernel, p, ntrg, nrhs, stats, leaves_ms, clocks, pk_, sms):
    """Leaf stage as kernel-sum throughput: U-list source-target pairs plus the L2T
    pairs (n surface points per target), per density vector; FMA-pipe operations
    per pair as the leaf kernel issues them (Stokes 17, Laplace 8, plus one rsqrt);
    fraction of the FP32 FMA-pipe issue peak (the device's SMs x 128 lanes per
    clock).  W-list pairs are not counted (a lower bound)."""
    n = 6 * (p - 1) ** 2 + 2
    pairs = (stats[7] + ntrg * n) * nrhs
    ops = 8 if kernel == 0 else 17
    mhz = (clocks or {}).get("sm_mhz") or pk_.get("sm_max_mhz", 2070.0)
    peak = sms * 128 * mhz * 1e6
    rate = pairs / (leaves_ms / 1e3) if leaves_ms > 0 else 0.0
    return {"pairs": pairs, "leaves_ms": leaves_ms, "pairs_per_s": rate, "fma_pipe_ops_per_pair": ops, "sms": sms,
            "fma_pipe_peak_ops_per_s": peak, "frac": rate * ops / peak}


def m2l_traffic(workload_name):
    """DRAM bytes (read + write) of one evaluation's M2L launches from the committed
    ncu note for this workload, or None when there is none or the kernel source has
    changed since it was taken (the note records the source's SHA-256)."""
    import hashlib
    note = os.path.join(ROOT, "profiles", f"m2l_tc_traffic_{workload_name}.md")
    src = os.path.join(ROOT, "paper_1705_02043_gb300", "csrc", "m2l_tc.cu")
    try:
        fields = dict(l.split(":", 1) for l in open(note).read().splitlines() if l.startswith(("source_sha256:", "dram_bytes_per_evaluation:")))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if fields["source_sha256"].strip() != sha:
            return None
        return float(fields["dram_bytes_per_evaluation"].strip())
    except Exception:
        return None


def plan_uses_tensor_cores():
    """True when the library's M2L runs on the tensor cores (tcgen05)."""
    import paper_1705_02043_gb300 as pk
    return hasattr(pk.load_library(), "pkifmm_m2l_tensor_core_enabled") and \
        bool(pk.load_library().pkifmm_m2l_tensor_core_enabled())


if __name__ == "__main__":
    main()
