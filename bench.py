#!/usr/bin/env python3
"""Throughput of the FP64-accurate Ozaki-scheme NTT FFT on GB300.

Workload (one step): 64 complex128 signals of length n = 2^18, real and
imaginary parts i.i.d. U[-1, 1) (seeded), forward transforms with K = 3 split
levels, two primes and no NTT-domain accumulation (L = 1: up to 96 32-bit NTTs
per transform, 84 at run time).  `value` is FFTs per second over all ranks,
one ozfft_execute per step on the whole batch, inputs resident in HBM (the 256
MiB of inputs per step exceed the 129 MB L2, so no flush is needed).  The plain
per-transform pipeline (64 executions of a batch-1 plan per step) is reported
beside it, and `e2e` repeats the batched measurement through
ozfft_execute_host with pinned host buffers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 run under torchrun: every rank transforms its own batch on its
own GPU (independent replicas, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64-accurate Ozaki-NTT FFTs/s at n=2^18 (batched); NTT GB/s; rel err"
BUTTERFLY_INSTR = 7.17   # lane instructions per radix-2 butterfly of the NTT kernels (profiles/)
UNIT = "FFT/s"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=1 << 18)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--K", type=int, default=3)
    ap.add_argument("--L", type=int, default=1)
    ap.add_argument("--nprimes", type=int, default=2)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-signals", type=int, default=0,
                    help="oracle transforms timed for cpu_baseline (default: one per host core)")
    ap.add_argument("--cpu-runs", type=int, default=5,
                    help="timed runs of the oracle sample for cpu_baseline (median reported, after one warm-up)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default NTT column/row split instead of timing the candidates at plan time")
    ap.add_argument("--merge", action="store_true", help="merged schedules across the convolutions of a part")
    ap.add_argument("--row-log", type=int, default=0,
                    help="force the NTT row pass to 2^row_log residues (profiling runs without plan-time tuning)")
    ap.add_argument("--ts", action="store_true", help="the TS (triple-single) variant of the method")
    ap.add_argument("--inv-vecs", type=int, default=0,
                    help="force 1 or 2 vectors per CTA in the inverse row pass (0: default or autotuned)")
    ap.add_argument("--crt-fuse", type=int, default=0,
                    help="force the inverse column pass fused with the CRT (1) or apart (2); 0: default or autotuned")
    ap.add_argument("--split-fuse", type=int, default=0,
                    help="force the Ozaki split fused with the forward column pass (1) or apart (2); "
                         "0: default or autotuned")
    ap.add_argument("--uneven-count", type=int, default=4096, help="signals of the uneven workload")
    ap.add_argument("--plain-sample", type=int, default=256,
                    help="signals of the uneven workload timed through per-signal plans")
    ap.add_argument("--workload", choices=("batch", "autograd", "stress", "uneven"), default="batch",
                    help="batch: the headline batched forward FFT; autograd: forward + backward of "
                         "sum |FFT(x) w|^2 over 256 Gaussian signals of n = 2^16; stress: n = 2^20 and "
                         "2^22, batch 8, 1%% spikes of 1e12, L = 1 (96 NTTs) vs L = 3 (64 NTTs); uneven: "
                         "4096 signals of log-uniform lengths in [1000, 300000] in one plan")
    a = ap.parse_args(argv)
    given = sys.argv if argv is None else argv
    if a.workload == "autograd":
        if "--n" not in given:
            a.n = 1 << 16
        if "--batch" not in given:
            a.batch = 256
        if "--seed" not in given:
            a.seed = 5
    return a


def workload(a):
    return {"workload": f"complex128 n=2^{a.n.bit_length() - 1} x {a.batch} signals, uniform[-1,1) parts, "
                        f"forward, K={a.K}, L={a.L}, {a.nprimes} primes",
            "n": a.n, "batch_per_gpu": a.batch, "K": a.K, "L": a.L, "nprimes": a.nprimes, "seed": a.seed,
            "autotune": a.autotune, "merge": a.merge, "ts": a.ts, "row_log": a.row_log,
            "inv_vecs": a.inv_vecs, "crt_fuse": a.crt_fuse, "split_fuse": a.split_fuse,
            "l2": "inputs (batch x n x 16 B) exceed L2 each step; no flush"}


# ----------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("ntt_impl.cuh", "k_ntt.cu", "k_ntt_row_inv.cu", "k_ntt_row_fwd.cu", "k_ntt_col.cu", "oz_common.cuh",
              "oz_kernels.h"):
        h.update(open(os.path.join(ROOT, "paper_2603_29129_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------- ranks
def init_dist(world):
    """One process per GPU under torchrun (NCCL), gloo when no GPU is present."""
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return dist


def max_over_ranks(dist, v, device):
    """The slowest rank's time (the job's time); v unchanged on one process."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps, per_rank_units, world, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return steps * per_rank_units * world / (ms / 1e3)


# ----------------------------------------------------------------- host-core oracle runs
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo; Arm parts by implementer/part id)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return None
    for line in info.splitlines():
        if line.lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    impl = [l.split(":", 1)[1].strip() for l in info.splitlines() if l.startswith("CPU implementer")]
    part = [l.split(":", 1)[1].strip() for l in info.splitlines() if l.startswith("CPU part")]
    return f"implementer {impl[0]} part {part[0]}" if impl and part else None


def _parse_cpulist(text):
    cpus = set()
    for tok in text.strip().split(","):
        if "-" in tok:
            a, b = tok.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif tok:
            cpus.add(int(tok))
    return cpus


def gpu_host_locality(local):
    """NUMA node and local CPUs of GPU `local` from sysfs (None where unknown)."""
    info = {"gpu_numa_node": None, "gpu_local_cpus": None}
    try:
        import torch
        props = torch.cuda.get_device_properties(local)
        bus = "%04x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except Exception:   # noqa: BLE001 - older torch without PCI ids
        return info
    base = os.path.join("/sys/bus/pci/devices", bus)
    try:
        node = int(open(os.path.join(base, "numa_node")).read())
        info["gpu_numa_node"] = node if node >= 0 else None
    except (OSError, ValueError):
        pass
    try:
        cpus = _parse_cpulist(open(os.path.join(base, "local_cpulist")).read())
        info["gpu_local_cpus"] = sorted(cpus) if cpus else None
    except (OSError, ValueError):
        pass
    return info


def numa_nodes_of(addr):
    """Pages per NUMA node of the host mapping that holds `addr` (/proc/self/numa_maps)."""
    try:
        start = None
        for line in open("/proc/self/maps"):
            lo, hi = (int(v, 16) for v in line.split()[0].split("-"))
            if lo <= addr < hi:
                start = lo
                break
        if start is None:
            return None
        for line in open("/proc/self/numa_maps"):
            f = line.split()
            if int(f[0], 16) == start:
                return {k[1:]: int(v) for k, v in (t.split("=") for t in f[1:] if t[0] == "N" and "=" in t)}
    except (OSError, ValueError):
        pass
    return None


def _oracle_one(job):
    """One oracle transform (worker of the spawned pool; the oracle is single-threaded C)."""
    import oracle
    x, K, L, P, ts = job
    y, _ = oracle.ozfft_ts(x, K=K, L=L) if ts else oracle.ozfft(x, K=K, L=L, nprimes=P)
    return y


class OraclePool:
    """A spawned process pool on the host cores (spawned, not forked, so that it
    is safe whatever the CUDA state of the parent)."""

    def __init__(self, workers):
        import multiprocessing as mp
        import oracle
        oracle.build()
        self.workers = max(1, workers)
        self.pool = mp.get_context("spawn").Pool(self.workers)
        self.pool.map(_oracle_one, [(np_signal(8), 3, 1, 2, False)] * self.workers)   # start-up and import

    def run(self, xs, K, L, P, ts=False):
        return self.pool.map(_oracle_one, [(x, K, L, P, ts) for x in xs], chunksize=1)

    def close(self):
        self.pool.close()
        self.pool.join()


def np_signal(n):
    from paper_2603_29129_gb300 import synth
    return synth.complex_signal("uniform", n, 0)[0]


# ----------------------------------------------------------------- reference arm
def run_reference(a, rank, world):
    """The oracle, as it stands, timed on the host cores: each step transforms one
    signal per core (a spawned process per core, the oracle itself single-threaded)."""
    if rank != 0:
        return
    from paper_2603_29129_gb300 import synth
    cores = min(host_cores(), a.batch)
    xs = list(synth.complex_signal("uniform", a.n, a.seed, batch=cores))
    pool = OraclePool(cores)
    for _ in range(a.warmup):
        pool.run(xs, a.K, a.L, a.nprimes, a.ts)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        pool.run(xs, a.K, a.L, a.nprimes, a.ts)
    dt = time.perf_counter() - t0
    pool.close()
    v = a.steps * cores / dt
    cfg = workload(a)
    cfg["reference_sample"] = f"{cores} signals per step, one per host core"
    print(json.dumps({"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                      "warmup": a.warmup, "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": cfg, "impl": "reference",
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                       "cpu_model": cpu_model(),
                                       "build": "gcc -O3 -ffp-contract=off (no -march=native: portable host code)",
                                       "sample": f"{cores} transforms of n={a.n} per step, one single-threaded C "
                                                 f"oracle process per core"},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


# ----------------------------------------------------------------- autograd workload
def run_autograd(a, rank, world, local):
    """Forward + backward of loss = sum |FFT(x) . w|^2 (per-signal complex
    Gaussian weights) through torch.autograd; the backward pass is the adjoint
    transform F^H through the same kernels.  Compared with the plain pipeline:
    per signal, one batch-1 forward execution and one batch-1 adjoint execution."""
    import numpy as np
    import torch
    dist = init_dist(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2603_29129_gb300 import build as bld
    if rank == 0:
        bld.build()
    if dist:
        dist.barrier()
    from paper_2603_29129_gb300 import autograd as ad
    from paper_2603_29129_gb300 import ozfft, synth
    B, n = a.batch, a.n
    xh = synth.complex_signal("gaussian", n, a.seed + 1000 * rank, batch=B)
    x = torch.from_numpy(xh).to(dev).requires_grad_()
    w = torch.from_numpy(synth.complex_signal("gaussian", n, a.seed + 1 + 1000 * rank, batch=B)).to(dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        x.grad = None
        loss = (ad.fft(x, K=a.K, L=a.L, nprimes=a.nprimes) * w).abs().square().sum()
        loss.backward()
        return loss

    def timed(fn, steps):
        for _ in range(a.warmup):
            fn()
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        return max_over_ranks(dist, e0.elapsed_time(e1), dev)

    clocks = ClockSampler(local)
    time.sleep(0.25)
    ms = timed(step, a.steps)
    clk = clocks.stop()
    fw = ozfft._plans[(n, B, ozfft.FORWARD, a.K, a.L, a.nprimes, dev.index)]
    bw = ozfft._plans[(n, B, ozfft.ADJOINT, a.K, a.L, a.nprimes, dev.index)]
    launches = fw.stats()["kernel_launches"] + bw.stats()["kernel_launches"]
    value = job_value(a.steps, B, world, ms)

    # plain: per signal one batch-1 forward and one batch-1 adjoint execution
    p_f = ozfft.Plan(n, 1, ozfft.FORWARD, K=a.K, L=a.L, nprimes=a.nprimes)
    p_b = ozfft.Plan(n, 1, ozfft.ADJOINT, K=a.K, L=a.L, nprimes=a.nprimes)
    xd = x.detach()
    yb = torch.empty_like(xd)
    gb = torch.empty_like(xd)

    def plain_step():
        for i in range(B):
            p_f.execute(xd[i:i + 1], yb[i:i + 1])
        gy = 2 * (w.abs() ** 2) * yb
        for i in range(B):
            p_b.execute(gy[i:i + 1], gb[i:i + 1])

    psteps = max(1, a.steps // 3)
    pms = timed(plain_step, psteps)

    # e2e: inputs from pinned host memory, gradient back to host memory, every step
    xpin = torch.from_numpy(xh).pin_memory()
    gpin = torch.empty_like(xpin).pin_memory()

    def e2e_step():
        x.data.copy_(xpin, non_blocking=True)
        step()
        gpin.copy_(x.grad, non_blocking=True)

    esteps = max(1, a.steps // 3)
    ems = timed(e2e_step, esteps)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # gradient check on signal 0 against torch's binary64 FFT on the CPU
    xc = torch.from_numpy(xh[:1]).requires_grad_()
    (torch.fft.fft(xc) * w[:1].cpu()).abs().square().sum().backward()
    step()
    g0 = x.grad[:1].cpu()
    rel = (torch.linalg.vector_norm(g0 - xc.grad) / torch.linalg.vector_norm(xc.grad)).item()
    cfg = {"workload": f"forward+backward of sum |FFT(x) w|^2, complex128 n=2^{n.bit_length() - 1} x {B} "
                       f"signals, Gaussian parts, complex Gaussian w, K={a.K}, L={a.L}, {a.nprimes} primes",
           "n": n, "batch_per_gpu": B, "K": a.K, "L": a.L, "nprimes": a.nprimes, "seed": a.seed,
           "parallelism": f"replicas x{world}", "l2": "inputs (batch x n x 16 B) exceed L2 each step; no flush"}
    line = {"metric": "FP64-accurate FFT forward+backward signals/s (autograd)", "value": value,
            "unit": "signal/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": cfg,
            "plain": {"value": job_value(psteps, B, world, pms), "unit": "signal/s", "steps": psteps,
                      "executions_per_step": 2 * B},
            "e2e": {"value": job_value(esteps, B, world, ems), "unit": "signal/s", "steps": esteps,
                    "h2d_bytes_per_step": B * n * 16, "d2h_bytes_per_step": B * n * 16},
            "clocks": clk, "gpu_launches": int(launches * a.steps),
            "accuracy": {"grad_rel_l2_vs_torch_cpu_signal0": rel}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------- stress workload
def run_stress(a, rank, world, local):
    """NTT-domain accumulation stress: batches of 8 signals of n = 2^20 and 2^22,
    uniform [-1, 1) parts with 1% spikes of +-1e12 (every split vector needs all
    K = 3 levels), the plain form (L = 1, 96 NTTs per transform) against the
    accumulated form (L = 3, 64 NTTs); error of signal 0 against the binary128 FFT."""
    import numpy as np
    import torch
    dist = init_dist(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2603_29129_gb300 import build as bld
    if rank == 0:
        bld.build()
    if dist:
        dist.barrier()
    from paper_2603_29129_gb300 import ozfft, synth
    import oracle
    if rank == 0 and not a.skip_cpu:
        oracle.build()
    B = 8
    stream = torch.cuda.current_stream(dev)
    results = []
    clocks = ClockSampler(local)
    for lg in (20, 22):
        n = 1 << lg
        xh = synth.complex_signal("spikes", n, a.seed + 1000 * rank, batch=B)
        x = torch.from_numpy(xh).to(dev)
        y = torch.empty_like(x)
        if rank == 0 and not a.skip_cpu:
            hi, lo = oracle.fft_q(xh[0])
        for L, merge, K in ((1, False, a.K), (3, False, a.K), (3, True, a.K), (1, False, ozfft.K_INF),
                            (3, False, ozfft.K_INF)):
            plan = ozfft.Plan(n, B, ozfft.FORWARD, K=K, L=L, nprimes=a.nprimes, merge=merge)
            for _ in range(a.warmup):
                plan.execute(x, y)
            if dist:
                dist.barrier()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(a.steps):
                plan.execute(x, y)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = max_over_ranks(dist, e0.elapsed_time(e1), dev)
            st = plan.stats()
            ok = plan.status() == ozfft.OK
            r = {"n": n, "K": "inf" if K == ozfft.K_INF else K, "L": L, "merge": merge,
                 "value": job_value(a.steps, B, world, ms), "unit": UNIT,
                 "ms_per_step": ms / a.steps, "status_ok": ok, "alpha": st["alpha"],
                 "x_split_levels_mean": st["ntt_forward_runtime"] / (2 * B * a.nprimes),
                 "ntt_per_transform_runtime": (st["ntt_forward_runtime"] + st["ntt_inverse"]) / B,
                 "ntt_per_transform_total": (st["ntt_forward_runtime"] + st["ntt_inverse"]) / B
                 + st["ntt_forward_plan"]}
            if rank == 0 and not a.skip_cpu:
                r["rel_l2_err_signal0_vs_binary128"] = oracle.rel_l2_error(y[0].cpu().numpy(), hi, lo)
            results.append(r)
            del plan
    clk = clocks.stop()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    tot_ms = sum(r["ms_per_step"] for r in results)
    line = {"metric": "FP64-accurate Ozaki-NTT FFTs/s, accumulation stress (n=2^20, 2^22; L=1 vs L=3)",
            "value": len(results) * B * world / (tot_ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": tot_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "complex128 n=2^20 and n=2^22 x 8 signals, uniform[-1,1) parts with 1% spikes "
                                   "of +-1e12, forward, K=3 (L=1, L=3, L=3 merged) and K=inf (L=1, L=3), two primes",
                       "batch_per_gpu": B, "seed": a.seed, "parallelism": f"replicas x{world}",
                       "l2": "inputs (8 x n x 16 B) exceed L2 each step; no flush"},
            "results": results, "clocks": clk}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------- uneven workload
def run_uneven(a, rank, world, local):
    """Signals of uneven lengths n = round(exp U[ln 1000, ln 300000]) (powers of
    two redrawn), parts +-10^U[-8, 8], forward, in one ozfft_plan_many plan (length
    classes batched, replayed as one CUDA graph, autotuned NTT splits), with L = 3
    and L = 1; against the plain pipeline (one batch-1 plan per signal) on a
    sample of the same signals."""
    import numpy as np
    cpu_pool = OraclePool(host_cores()) if (rank == 0 and not a.skip_cpu) else None
    import torch
    dist = init_dist(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2603_29129_gb300 import build as bld
    if rank == 0:
        bld.build()
    if dist:
        dist.barrier()
    from paper_2603_29129_gb300 import ozfft, synth
    import oracle
    if rank == 0 and not a.skip_cpu:
        oracle.build()
    cnt = a.uneven_count
    lens = synth.uneven_lengths(cnt, 3 + 1000 * rank)
    total = int(lens.sum())
    xh = synth.complex_signal("loguniform", total, 3 + 1000 * rank)[0]
    x = torch.from_numpy(xh).to(dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, steps):
        for _ in range(a.warmup):
            fn()
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        return max_over_ranks(dist, e0.elapsed_time(e1), dev)

    out = {}
    clocks = ClockSampler(local)
    for L in (3, 1):
        # the autotuner's candidate timings per length class (OZFFT_TUNE_LOG)
        tlog = tempfile.NamedTemporaryFile("w+", suffix=".tune", delete=False)
        tlog.close()
        os.environ["OZFFT_TUNE_LOG"] = tlog.name
        t0 = time.perf_counter()
        plan = ozfft.PlanMany(lens, ozfft.FORWARD, K=a.K, L=L, nprimes=a.nprimes, autotune=True)
        tplan = time.perf_counter() - t0
        os.environ.pop("OZFFT_TUNE_LOG", None)
        tune_rows = [ln.split() for ln in open(tlog.name).read().splitlines()]
        os.unlink(tlog.name)
        ms = timed(lambda: plan.execute(x, y), a.steps)
        st = plan.stats()
        # whole-step roofline (the graph's kernels of every length class together): modular
        # multiplications of the NTT butterflies and of the Alg. 8 products, live vectors per
        # signal taken as the plan's mean, each signal at its own N
        Ns = np.array([n if n & (n - 1) == 0 else 1 << int(2 * n - 2).bit_length() for n in lens], dtype=np.float64)
        fwd_v, inv_v = st["ntt_forward_runtime"] / cnt, st["ntt_inverse"] / cnt
        prods = inv_v * (L if L > 1 else 1)   # products per signal: at most L per group (upper bound)
        mm = float(np.sum((fwd_v + inv_v) * Ns / 2 * np.log2(Ns) + prods * Ns))
        peak_alu = 152 * 4 * 32 * 2.07e9 / BUTTERFLY_INSTR / 1e12
        # stage-minimal bytes per signal (the fused pipeline's count, 856 N at n = N, K = 3, L = 1):
        # split 32 n + 8 K N, forward NTTs 8 N per vector, MAC reads X and Y (4 N per vector, 2 K P
        # w~* vectors per signal here), inverse outputs written and read once (4 N each), output 32 n
        wv = 2 * a.K * a.nprimes
        alg_bytes = float(np.sum(64 * lens + Ns * (8 * a.K + 8 * fwd_v + 4 * fwd_v + 4 * wv + 8 * inv_v)))
        pk = peaks()
        r = {"value": job_value(a.steps, cnt, world, ms), "unit": "signal/s", "ms_per_step": ms / a.steps,
             "roofline": {"bound": "alu", "kernel": "whole step (CUDA graph of every length class)",
                          "achieved": mm / (ms / a.steps / 1e3) / 1e12, "peak": peak_alu, "unit": "Tmodmul/s",
                          "frac": mm / (ms / a.steps / 1e3) / 1e12 / peak_alu, "traffic": None,
                          "modmuls_per_step": mm,
                          "hbm_view": {"algorithmic_bytes_per_step": alg_bytes,
                                       "achieved": alg_bytes / (ms / a.steps / 1e3) / 1e9,
                                       "peak": pk["hbm_gbs"] if pk else 6800.0, "unit": "GB/s"},
                          "note": "live vectors per signal are the plan's means; products per group counted "
                                  "as L (an upper bound for L > 1)"},
             "bytes_per_s": 2 * 16 * total * world * a.steps / (ms / 1e3), "status_ok": plan.status() == ozfft.OK,
             "plan_seconds": tplan, "workspace_GB": st["workspace_bytes"] / 1e9,
             "ntt_runtime_per_signal": (st["ntt_forward_runtime"] + st["ntt_inverse"]) / cnt,
             "gpu_launches_per_step": st["kernel_launches"],
             "tuning": {"classes": st["classes"], "crt_fused_classes": st["crt_fused_classes"],
                        "split_fused_classes": st["split_fused_classes"],
                        "inv_vecs_largest_class": st["inv_vecs"], "row_log_inv_largest_class": st["row_log_inv"],
                        "candidates": [" ".join(r) for r in tune_rows]}}
        if rank == 0 and not a.skip_cpu:
            yh = y.cpu().numpy()
            xs, ys = plan.split(xh), plan.split(yh)
            order = np.argsort(lens)
            same, errs = True, []
            for i in (int(order[0]), int(order[-1])):
                yo, _ = oracle.ozfft(xs[i], K=a.K, L=L, nprimes=a.nprimes)
                same = same and np.array_equal(yo.view(np.uint64), ys[i].view(np.uint64))
            for i in range(0, cnt, max(1, cnt // 8)):
                bins = np.array([0, len(xs[i]) // 3, len(xs[i]) - 1])
                hi, lo = oracle.dft_q(xs[i], bins=bins)
                errs.append(float(np.max(np.abs(ys[i][bins] - (hi + lo))) / np.linalg.norm(xs[i])))
            r["bit_exact_vs_oracle"] = f"shortest and longest signal: {'yes' if same else 'NO'}"
            r["max_sampled_bin_err_over_norm"] = max(errs)
        out[f"L={L}"] = r
        del plan
    clk = clocks.stop()

    # the plain pipeline: one batch-1 plan per signal, on a sample of the signals
    m = min(a.plain_sample, cnt)
    offs = np.concatenate([[0], np.cumsum(lens)])
    plans = [ozfft.Plan(int(lens[i]), 1, ozfft.FORWARD, K=a.K, L=3, nprimes=a.nprimes) for i in range(m)]
    xv = [x[offs[i]:offs[i + 1]] for i in range(m)]
    yv = [y[offs[i]:offs[i + 1]] for i in range(m)]

    def plain_step():
        for i in range(m):
            plans[i].execute(xv[i], yv[i])

    pms = timed(plain_step, max(1, a.steps // 3))
    psteps = max(1, a.steps // 3)
    del plans
    # the same sample through one uneven-length plan
    sub = ozfft.PlanMany(lens[:m], ozfft.FORWARD, K=a.K, L=3, nprimes=a.nprimes, autotune=True)
    xs_ = x[:offs[m]]
    ys_ = y[:offs[m]]
    sms = timed(lambda: sub.execute(xs_, ys_), psteps)
    del sub
    cpu = None
    if cpu_pool is not None:
        # the oracle on a seeded sample of the same signals, one process per host core
        rng = np.random.default_rng(11)
        pick = rng.choice(cnt, size=min(cnt, 4 * cpu_pool.workers), replace=False)
        xs_all = [xh[offs[i]:offs[i + 1]] for i in pick]
        t0 = time.perf_counter()
        cpu_pool.run(xs_all, a.K, 3, a.nprimes)
        dt = time.perf_counter() - t0
        cpu_pool.close()
        cpu = {"value": len(pick) / dt, "unit": "signal/s", "cores": cpu_pool.workers, "kind": "oracle",
               "cpu_model": cpu_model(),
               "sample": f"{len(pick)} signals drawn (seed 11) from the {cnt} of the workload, L=3, one "
                         f"single-threaded C oracle process per host core, one timed run"}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {"metric": "FP64-accurate Ozaki-NTT FFTs of uneven lengths, signals/s (one plan, CUDA graph)",
            "value": out["L=3"]["value"], "unit": "signal/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": out["L=3"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{cnt} complex128 signals, n log-uniform in [1000, 300000] (powers of two "
                                   f"redrawn, seed 3), parts +-10^U[-8,8], forward, K={a.K}, L=3 (and L=1), "
                                   f"{a.nprimes} primes", "total_elements": total,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs (total x 16 B) exceed L2 each step; no flush"},
            "by_L": out,
            "plain": {"signals": m, "value": job_value(psteps, m, world, pms), "unit": "signal/s",
                      "executions_per_step": m},
            "uneven_plan_same_sample": {"signals": m, "value": job_value(psteps, m, world, sms), "unit": "signal/s"},
            "roofline": out["L=3"]["roofline"], "cpu_baseline": cpu,
            "tuning": out["L=3"]["tuning"], "clocks": clk}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------- our arm
def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if a.workload == "autograd":
        run_autograd(a, rank, world, local)
        return
    if a.workload == "stress":
        run_stress(a, rank, world, local)
        return
    if a.workload == "uneven":
        run_uneven(a, rank, world, local)
        return

    import numpy as np
    # the oracle's host-core pool starts (spawned) before any GPU work
    cpu_pool = OraclePool(min(host_cores(), a.batch)) if (rank == 0 and not a.skip_cpu) else None
    import torch

    dist = init_dist(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2603_29129_gb300 import build as bld
    if rank == 0:
        bld.build()
    if dist:
        dist.barrier()
    from paper_2603_29129_gb300 import ozfft, synth

    def barrier():
        if dist:
            dist.barrier()

    def rank_max(v):
        return max_over_ranks(dist, v, dev)

    B, n = a.batch, a.n
    # host buffers on the GPU's own NUMA node: this thread runs on the GPU's local
    # CPUs before the pinned buffers are allocated (the oracle's pool was spawned
    # earlier and keeps every core)
    loc = gpu_host_locality(local)
    if loc["gpu_local_cpus"]:
        try:
            os.sched_setaffinity(0, loc["gpu_local_cpus"])
        except OSError:
            pass
    x_host = synth.complex_signal("uniform", n, a.seed + 1000 * rank, batch=B)
    x_pin = torch.from_numpy(x_host).pin_memory()
    x = x_pin.to(dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)
    plan = ozfft.Plan(n, B, ozfft.FORWARD, K=a.K, L=a.L, nprimes=a.nprimes, autotune=a.autotune, merge=a.merge,
                      ts=a.ts, row_log=a.row_log, inv_vecs=a.inv_vecs, crt_fuse=a.crt_fuse,
                      split_fuse=a.split_fuse)

    # ---- batched, device-resident (the headline value), with per-kernel events
    for _ in range(a.warmup):
        plan.execute(x, y)
    torch.cuda.synchronize(dev)
    plan.profile()                      # drop anything recorded so far
    plan.set_profiling(True)
    clocks = ClockSampler(local)
    time.sleep(0.25)
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        plan.execute(x, y)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    plan.set_profiling(False)
    prof = plan.profile()
    ms = rank_max(e0.elapsed_time(e1))
    value = job_value(a.steps, B, world, ms)
    stats = plan.stats()
    if plan.status() != ozfft.OK:
        raise RuntimeError("device status flagged the benchmark input")

    # ---- plain pipeline: one execution of a batch-1 plan per transform
    plain = None
    if not a.skip_plain:
        p1 = ozfft.Plan(n, 1, ozfft.FORWARD, K=a.K, L=a.L, nprimes=a.nprimes, autotune=a.autotune, merge=a.merge,
                        ts=a.ts, row_log=a.row_log, inv_vecs=a.inv_vecs, crt_fuse=a.crt_fuse,
                        split_fuse=a.split_fuse)
        xs = [x[i:i + 1] for i in range(B)]
        ys = [y[i:i + 1] for i in range(B)]
        for _ in range(a.warmup):
            for i in range(B):
                p1.execute(xs[i], ys[i])
        psteps = max(1, a.steps // 3)
        barrier()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(psteps):
            for i in range(B):
                p1.execute(xs[i], ys[i])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        pms = rank_max(e0.elapsed_time(e1))
        plain = {"value": job_value(psteps, B, world, pms), "unit": UNIT, "steps": psteps,
                 "ms_per_step": pms / psteps, "executions_per_step": B}
        del p1

    # ---- end to end through the C ABI with host buffers
    e2e = None
    out_pin = torch.empty_like(x_pin).pin_memory()
    if not a.skip_e2e:
        nbytes = B * n * 16
        # standalone pinned copies of one step's input and output, the bounds of the pipeline
        dbuf = torch.empty_like(x)
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

        def copy_ms(fn, reps=5):
            best = None
            for _ in range(reps + 1):
                torch.cuda.synchronize(dev)
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                fn()
                c1.record(stream)
                torch.cuda.synchronize(dev)
                t = c0.elapsed_time(c1)
                best = t if best is None else min(best, t)
            return best

        def both():
            ev = torch.cuda.Event()
            ev.record(stream)
            s_in.wait_event(ev)
            s_out.wait_event(ev)
            with torch.cuda.stream(s_in):
                dbuf.copy_(x_pin, non_blocking=True)
            with torch.cuda.stream(s_out):
                out_pin.copy_(y, non_blocking=True)
            stream.wait_stream(s_in)
            stream.wait_stream(s_out)

        h2d_ms = copy_ms(lambda: dbuf.copy_(x_pin, non_blocking=True))
        d2h_ms = copy_ms(lambda: out_pin.copy_(y, non_blocking=True))
        both_ms = copy_ms(both)
        copy_gbs = {"h2d": nbytes / (h2d_ms / 1e3) / 1e9, "d2h": nbytes / (d2h_ms / 1e3) / 1e9,
                    "h2d_d2h_concurrent_each": nbytes / (both_ms / 1e3) / 1e9, "bytes": nbytes,
                    "how": "best of 5 pinned copies of one step's input (and output), CUDA events"}
        del dbuf
        esteps = max(20, a.steps)
        # synchronous calls (ozfft_execute_host: a four-part pipeline inside each call)
        for _ in range(a.warmup):
            plan.execute_host(x_pin, out_pin)
        barrier()
        call_ms = []
        t0 = time.perf_counter()
        for _ in range(esteps):
            tc = time.perf_counter()
            plan.execute_host(x_pin, out_pin)
            call_ms.append(1e3 * (time.perf_counter() - tc))
        dt_sync = rank_max(time.perf_counter() - t0)
        # asynchronous calls (ozfft_execute_host_async: each call's copies overlap the
        # neighbouring calls' computation), all waited for inside the timed region
        for _ in range(a.warmup):
            plan.execute_host_async(x_pin, out_pin)
        plan.host_wait()
        barrier()
        eclocks = ClockSampler(local)
        time.sleep(0.25)
        t0 = time.perf_counter()
        for _ in range(esteps):
            plan.execute_host_async(x_pin, out_pin)
        plan.host_wait()
        dt = rank_max(time.perf_counter() - t0)
        eclk = eclocks.stop()
        # device time of the kernels inside those calls (per-kernel events, all four parts)
        plan.profile()
        plan.set_profiling(True)
        for _ in range(5):
            plan.execute_host(x_pin, out_pin)
        plan.set_profiling(False)
        hprof = plan.profile()
        host_kernel_ms = sum(v["ms"] for v in hprof["slots"].values()) / 5
        # the host pipeline of ozfft_execute_host: parts of 1/14, 6/14, 6/14 and 1/14 of the batch;
        # copies in on one stream, computation on the caller's, copies out on a third
        wts = [1, 6, 6, 1] if B >= 28 else [1, 1, 1, 1]
        dev_ms = ms / a.steps
        r_in = h2d_ms / B
        r_out = d2h_ms / B
        cuts = [0]
        acc_w = 0
        for w_ in wts:
            acc_w += w_
            cuts.append(B * acc_w // sum(wts) if B >= 28 else min(B, len(cuts) * ((B + 3) // 4)))
        t_in = t_comp = t_out = 0.0
        for i in range(4):
            nb = cuts[i + 1] - cuts[i]
            if nb <= 0:
                continue
            t_in += nb * r_in
            t_comp = max(t_comp, t_in) + nb * dev_ms / B
            t_out = max(t_out, t_comp) + nb * r_out
        # async steady state: a step costs the longest of device time, copy in and copy out,
        # and the first copy in and the last copy out are exposed once per run
        model_async = max(dev_ms, h2d_ms, d2h_ms) + (h2d_ms + d2h_ms) / esteps
        e2e = {"value": job_value(esteps, B, world, 1e3 * dt), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": esteps, "ms_per_step": 1e3 * dt / esteps,
               "api": "ozfft_execute_host_async per step, ozfft_execute_host_wait at the end (copies in and "
                      "out of every step inside the timed region)",
               "model_ms_per_step": model_async,
               "model": "max(device step, copy in, copy out) + (copy in + copy out) / steps",
               "copy_gbs": copy_gbs, "clocks": eclk,
               "sync": {"value": job_value(esteps, B, world, 1e3 * dt_sync), "ms_per_step": 1e3 * dt_sync / esteps,
                        "api": "ozfft_execute_host per step (returns after its copy out)",
                        "model_ms_per_step": t_out,
                        "model": "four-part pipeline inside a call from the measured copy times and the device "
                                 "step time",
                        "kernel_ms_per_step_in_pipeline": host_kernel_ms,
                        "call_ms": {"min": min(call_ms), "median": statistics.median(call_ms), "max": max(call_ms)}},
               "host": {"cpu_model": cpu_model(), "cores": host_cores(),
                        "gpu_numa_node": loc["gpu_numa_node"],
                        "thread_cpus": len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else None,
                        "pinned_in_numa_pages": numa_nodes_of(x_pin.data_ptr()),
                        "pinned_out_numa_pages": numa_nodes_of(out_pin.data_ptr())}}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (live CUDA events over the timed region)
    N = plan.N
    lgN = N.bit_length() - 1
    runtime_fwd = stats["ntt_forward_runtime"]        # live forward vectors per execution
    inv_vecs = stats["ntt_inverse"]                   # live inverse vectors per execution
    m2f, m2i = stats["row_log_fwd"], stats["row_log_inv"]
    # algorithmic bytes per execution (stage-minimal: every input read once, every output written
    # once).  A pass of the NTT reads and writes each live vector (4N + 4N).  The inverse row pass
    # with the fused multiply-accumulate reads each signal's forward spectra X once (4N per live
    # forward vector) and the w~* spectra Ym once per transform (4N per w~* vector), and writes the
    # inverse vectors (4N each): 384N per transform at K = 3, L = 1.  The fused column pass + CRT
    # reads the inverse vectors and writes the output (with the chirp).
    prods = sum(len(pairs) for b in range(B) for conv in plan.dump(ozfft.DUMP_SCHED, b)
                for _, pairs in conv) * a.nprimes
    wvecs = (stats["wstar_levels"][0] + stats["wstar_levels"][1]) * a.nprimes
    alg = {"ntt_fwd_col": 8 * N * runtime_fwd, "ntt_fwd_row": 8 * N * runtime_fwd,
           "ntt_inv_col": 8 * N * inv_vecs, "ntt_inv_row": 4 * N * runtime_fwd + 4 * N * wvecs * B + 4 * N * inv_vecs,
           "premul": B * (16 * n + 16 * n + 16 * N), "crt": 4 * N * inv_vecs + B * 32 * n}
    # algorithmic modular multiplications per execution: one per radix-2 butterfly
    # ((N/2) per stage and vector) and one per NTT-domain product and element
    mm = {"ntt_fwd_col": runtime_fwd * (lgN - m2f) * N // 2, "ntt_fwd_row": runtime_fwd * m2f * N // 2,
          "ntt_inv_col": inv_vecs * (lgN - m2i) * N // 2, "ntt_inv_row": inv_vecs * m2i * N // 2 + prods * N}
    slots = prof["slots"]
    dom = max(slots, key=lambda k: slots[k]["ms"])
    execs = max(1, prof["executions"])
    launches_per_exec = max(1, slots[dom]["launches"] // execs)
    dom_ms = slots[dom]["ms"] / max(1, slots[dom]["launches"])
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else 6800.0
    roof = None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(tfile):
        t = json.load(open(tfile))
        ent = t.get(dom)
        if ent and ent.get("source_hash") == kernel_source_hash() and ent.get("config") == f"n={n},B={B},L={a.L}":
            traffic = ent.get("bytes_per_launch")
    hbm_view = None
    if alg.get(dom):
        alg_launch = alg[dom] / launches_per_exec          # the slot's bytes are per execution
        hbm_view = {"achieved": alg_launch / (dom_ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": alg_launch / (dom_ms / 1e3) / 1e9 / hbm_peak,
                    "algorithmic_bytes_per_launch": alg_launch,
                    "traffic_frac": (traffic / (dom_ms / 1e3) / 1e9 / hbm_peak) if traffic else None,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if pk else "fallback 6.8 TB/s"}
    if mm.get(dom):
        # integer roofline: the NTT kernels are bound by integer issue (ncu: DRAM well below
        # peak, issue slots busy); peak = 152 SMs x 4 schedulers x 32 lanes x 2.07 GHz lane
        # instructions / the lane instructions of one butterfly as compiled (ncu
        # smsp__inst_executed over the register-only kernel of the inverse butterfly: 7.17)
        mm_launch = mm[dom] / launches_per_exec
        peak_derived = 152 * 4 * 32 * 2.07e9 / BUTTERFLY_INSTR / 1e12
        inv = dom.startswith("ntt_inv")
        measured = ozfft.butterfly_rate(inverse=inv) / 1e12
        achieved = mm_launch / (dom_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_derived, "unit": "Tmodmul/s",
                "frac": achieved / peak_derived, "traffic": traffic,
                "traffic_frac": hbm_view["traffic_frac"] if hbm_view else None,
                "peak_source": f"derived: 152 SMs x 4 x 32 lanes x 2.07 GHz / {BUTTERFLY_INSTR} lane instructions "
                               "per butterfly (ncu count of the register-only butterfly kernel)",
                "register_only_rate_floor": measured,
                "register_only_rate_note": "rate of the register-only butterfly kernel: a floor of the "
                                           "attainable rate, not the roof",
                "modmuls_per_launch": mm_launch, "launch_ms": dom_ms, "hbm_view": hbm_view}
    elif hbm_view:
        roof = dict(hbm_view, bound="hbm", kernel=dom, traffic=traffic, launch_ms=dom_ms)
    total_ntt = runtime_fwd + inv_vecs
    ntt_ms = sum(slots[k]["ms"] for k in slots if k.startswith("ntt")) / execs
    breakdown = {k: round(v["ms"] / execs, 4) for k, v in slots.items()}

    # ---- accuracy of one signal and bit parity with the oracle, CPU baseline
    acc = {}
    cpu = None
    if not a.skip_cpu:
        import oracle
        oracle.build()
        y0 = y[0].cpu().numpy()
        hi, lo = oracle.fft_q(x_host[0])
        acc["rel_l2_err_signal0"] = oracle.rel_l2_error(y0, hi, lo)
        cnt = min(a.cpu_signals or cpu_pool.workers, B)
        sig = [x_host[i] for i in range(cnt)]
        ys = cpu_pool.run(sig, a.K, a.L, a.nprimes, a.ts)          # warm-up (and the parity sample)
        runs = []
        for _ in range(a.cpu_runs):
            t0 = time.perf_counter()
            cpu_pool.run(sig, a.K, a.L, a.nprimes, a.ts)
            runs.append(time.perf_counter() - t0)
        cpu_pool.close()
        dt = statistics.median(runs)
        yg = y[:cnt].cpu().numpy()
        same = all(np.array_equal(ys[i].view(np.uint64), yg[i].view(np.uint64)) for i in range(cnt))
        acc["bit_exact_vs_oracle"] = f"{cnt} signals: {'yes' if same else 'NO'}"
        cpu = {"value": cnt / dt, "unit": UNIT, "cores": min(cnt, cpu_pool.workers), "kind": "oracle",
               "cpu_model": cpu_model(), "runs": len(runs), "warmup_runs": 1, "statistic": "median",
               "run_seconds": runs, "build": "gcc -O3 -ffp-contract=off (no -march=native: portable host code)",
               "sample": f"{cnt} of the {B} signals (n={n}) per run, one single-threaded C oracle process "
                         f"per host core"}

    cfg = workload(a)
    cfg.update({"mode": "batched (one ozfft_execute per step)", "parallelism": f"replicas x{world}",
                "N": N, "alpha": stats["alpha"]})
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": cfg,
        "plain": plain, "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
        "gpu_launches": int(stats["kernel_launches"] * a.steps),
        "ntt": {"per_transform_runtime": total_ntt / B, "per_transform_total": (total_ntt + stats["ntt_forward_plan"] * B) / B,
                "row_pass_stages": {"forward": m2f, "inverse": m2i},
                "GBps_algorithmic": total_ntt * 8 * N / (ntt_ms / 1e3) / 1e9},
        "kernel_ms_per_step": breakdown, "accuracy": acc,
        "tuning": {"row_log_fwd": stats["row_log_fwd"], "row_log_inv": stats["row_log_inv"],
                   "inv_vecs": stats["inv_vecs"], "crt_fused": bool(stats["crt_fused_classes"]),
                   "split_fused": bool(stats["split_fused_classes"])},
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
