"""Benchmark: order-4 Hubbard self-energy, batched AMI evaluation on GB300.

Metric: evals/s, one eval = one (sample, flat term, external frequency) triple of the flat
term table (FACTORIZE=false form); the step is one pass of the hot path over 2^24 Philox
momentum samples and 16 Matsubara frequencies.  Inputs are generated in-kernel from the
counter-based stream (no input buffers); L2 is flushed before every timed step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tami|reference]

--impl reference times the CPU oracle (the reference for this method) on the host cores, on
a bounded sample of the same workload, and prints the same JSON line with "impl": "reference".
Under torchrun each rank owns a disjoint block of the sample stream (weak scaling, no
data-path collective); rank 0 prints one JSON line with the max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2311_17189_gb300 import workloads as W  # noqa: E402

CFG = W.ORDER4
FP64_PEAK_TFLOPS = 1.2586   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)


def _hbm_peak_gbs():
    """Measured copy bandwidth (read + write) from MEASURED_PEAKS.json, else 6800 GB/s (the
    fallback measurement on a GB300)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_PEAK_GBS = _hbm_peak_gbs()
METRIC = "order-4 Sigma evals/s (samples x terms x frequencies, FP64), forward + adjoint"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel from one ncu
# capture of this workload at 2^22 samples, per sample; every sample does the same work, so a
# launch's traffic is this times its samples.  It holds only for the kernel it was taken on: the
# step must have run that kernel, and the kernel's identity -- the generated source of the
# diagram's fused kind with the device arithmetic it includes, the identity under which the library
# caches the compilation (whose options are fixed in the library) -- must hash to the captured
# one, else the bench reports traffic as null.
TRAFFIC = {"kernel": "tami_jit_fused (the diagram's specialised fused forward + adjoint)",
           "bytes_per_sample": (4.650301e9 + 5.725492e9) / 4194304,
           "kernel_sha256": "cc21cf574bb547fa71c92372ed461d9c6e83bd460e6a6fa46c67ef91d21e9a88",
           "profile": "profiles/jit_kernels_order4_sigma.md"}


FP64_RATE_VARIANTS = 4   # operand patterns of tami_selftest_fp64_rate (TAMI_FP64_RATE_VARIANTS)


def fp64_rate_measured(stream, target_s=0.25):
    """FP64 fma rate of this GPU from libtami's probe (tami_selftest_fp64_rate: independent fma
    recurrences, 8 blocks of 256 threads per SM), timed with CUDA events on `stream`: for each of
    its operand patterns one warm-up and three launches of about `target_s`; the fastest launch
    of all, in TFLOP/s (the FP64 unit's rate depends on the operands' register placement)."""
    import ctypes
    import torch
    from paper_2311_17189_gb300 import _lib as L
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = 8 * sms
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    fl = ctypes.c_double()
    sp = ctypes.c_void_p(stream.cuda_stream)
    trips = 256

    def launch(v, tr):
        L.check(L.lib().tami_selftest_fp64_rate(v, blocks, tr, ctypes.c_void_p(out.data_ptr()), ctypes.byref(fl), sp))

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best, best_v, best_s, rates = None, None, None, []
    for v in range(FP64_RATE_VARIANTS):
        tr = 256
        launch(v, tr)
        torch.cuda.synchronize()
        e0.record(stream)
        launch(v, tr)
        e1.record(stream)
        e1.synchronize()
        tr = max(1, int(tr * target_s / max(e0.elapsed_time(e1) * 1e-3, 1e-6)))
        vbest = None
        for _ in range(3):
            e0.record(stream)
            launch(v, tr)
            e1.record(stream)
            e1.synchronize()
            rate = fl.value / (e0.elapsed_time(e1) * 1e-3) / 1e12
            if vbest is None or rate > vbest:
                vbest = rate
            if best is None or rate > best:
                best, best_v, best_s = rate, v, e0.elapsed_time(e1) * 1e-3
        rates.append(round(vbest, 4))
    return {"tflops": best, "launch_s": best_s, "blocks": blocks, "variant": best_v, "variants_tflops": rates,
            "probe": "tami_selftest_fp64_rate: independent fma recurrences, the fastest of its operand patterns, "
                     "best of 3 launches each"}


def roofline_peak(measured):
    """The FP64 denominator: the measured fma rate where it is below the derived unit-count peak
    (the pipe cannot be faster than it shows here), else the derived peak."""
    if measured and measured["tflops"] < FP64_PEAK_TFLOPS:
        return measured["tflops"], "measured on this GPU in this run (tami_selftest_fp64_rate, FP64 fma)"
    return FP64_PEAK_TFLOPS, "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz (nominal 1.25 TFLOP/s)"


def kernel_sha256(D):
    """sha256 over the fused kernel source generated for diagram D and the device-arithmetic
    header that source includes."""
    import hashlib
    h = hashlib.sha256(D.jit_source("fused").encode())
    with open(os.path.join(ROOT, "paper_2311_17189_gb300", "csrc", "tami_devmath.cuh"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def oracle_step(S, offset, n, X, cores):
    """One forward + adjoint step of the oracle: the mean, then dual-number derivatives along
    omega, mu, kx_ext and ky_ext."""
    S.eval_momenta(W.lattice(CFG), CFG["seed"], offset, n, X, CFG["beta"], per_sample=False, threads=cores)
    for which in ("omega", "mu", "kx", "ky"):
        S.eval_momenta_deriv(W.lattice(CFG), CFG["seed"], offset, n, X, CFG["beta"], which, threads=cores)


def cpu_baseline(diagram, X, target_s=10.0):
    """The oracle as it stands on all host cores, on the first samples of the same stream."""
    import oracle as O
    S = O.Solution(diagram["alpha"], eps=diagram["eps"])
    cores = os.cpu_count() or 1
    n = 256
    while True:
        t0 = time.perf_counter()
        oracle_step(S, 0, n, X, cores)
        dt = time.perf_counter() - t0
        if dt * 4 > target_s or n >= (1 << 22):
            break
        n *= 4
    info = S.info()
    n1 = max(n // cores, 64)                        # one thread: a proportionally smaller sample
    t0 = time.perf_counter()
    oracle_step(S, 0, n1, X, 1)
    dt1 = time.perf_counter() - t0
    return {"value": n * info["terms"] * len(X) / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"first {n} of the {CFG['n_samples']} samples (same seed), {len(X)} frequencies, "
                      f"forward + 4 dual-number derivative passes, {dt:.2f} s wall",
            "single_thread": {"value": n1 * info["terms"] * len(X) / dt1, "unit": "evals/s", "cores": 1,
                              "sample": f"first {n1} samples, {dt1:.2f} s wall"}}


def order4_diagram(lib):
    return next(d for d in lib.enumerate_sigma(CFG["order"]) if d["code"] == tuple(CFG["code"]))


def run_reference(args):
    import oracle as O
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    d = next(x for x in O.enumerate_sigma(CFG["order"]) if x["code"] == tuple(CFG["code"]))
    S = O.Solution(d["alpha"], eps=d["eps"])
    X = W.matsubara(CFG["beta"], CFG["n_freq"])
    cores = os.cpu_count() or 1
    n = args.ref_samples
    T = S.info()["terms"]
    for i in range(args.warmup):
        oracle_step(S, i * n, n, X, cores)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle_step(S, (args.warmup + i) * n, n, X, cores)
    dt = (time.perf_counter() - t0) / args.steps
    value = n * T * len(X) / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (Philox momenta)",
        "config": {"workload": CFG["name"], "samples_per_step": n, "frequencies": len(X), "terms": T,
                   "beta": CFG["beta"], "t": CFG["t"], "tp": CFG["tp"], "mu": CFG["mu"]},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n} samples per step of the {CFG['n_samples']}-sample workload, "
                                   "forward + 4 dual-number derivative passes"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_tami(args):
    import torch
    import paper_2311_17189_gb300 as T

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    stream = torch.cuda.current_stream()
    d = order4_diagram(T)
    D = T.Diagram(d["alpha"], eps=d["eps"]).upload(local)
    info = D.info()
    X = W.matsubara(CFG["beta"], CFG["n_freq"])
    n = args.samples
    offset, n = T.mc.shard(rank, world, n)
    lat = W.lattice(CFG)
    n_f = len(X)
    Xd = torch.view_as_real(torch.as_tensor(X, dtype=torch.complex128, device=dev)).contiguous()
    Xc = torch.view_as_complex(Xd)
    mean = torch.empty((n_f, 2), dtype=torch.float64, device=dev)
    var = torch.empty((n_f, 2), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    g_host = W.matsubara(CFG["beta"], CFG["n_freq"]).real * 0 + (1.0 + 0.5j)   # fixed upstream gradient
    G = torch.view_as_real(torch.as_tensor(g_host, dtype=torch.complex128, device=dev)).contiguous()
    Gc = torch.view_as_complex(G)

    # the step keeps each sample's line energies and dE/dK factors from the forward for the
    # adjoint (as torch autograd would); term products are still recomputed in the adjoint
    saved = D.saved_buffer(n)

    def fwd(i, save=True):
        return D.forward(lat, CFG["seed"], offset + i * n * world, n, Xc, CFG["beta"], out=(mean, var),
                         save=saved if save else None)

    def bwd(i):
        return D.backward(lat, CFG["seed"], offset + i * n * world, n, Xc, CFG["beta"], Gc, saved=saved)

    def fused(i):
        return D.forward_backward(lat, CFG["seed"], offset + i * n * world, n, Xc, CFG["beta"], Gc)

    for i in range(args.warmup):
        fused(i)
        fwd(i)
        bwd(i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    mk = lambda: torch.cuda.Event(enable_timing=True)
    # the step: forward and adjoint of the same samples in one pass (tami_forward_backward)
    evf = [(mk(), mk()) for _ in range(args.steps)]
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                       # evict L2 (256 MiB > 129 MB) outside the timed span
        evf[i][0].record(stream)
        fused(args.warmup + i)
        evf[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    fused_ms = [a.elapsed_time(b) for a, b in evf]
    fused_kernel = ("tami_jit_fused (the diagram's specialised fused forward + adjoint)" if D.jit_status()["last_used"]
                    else "bwd_kernel<0,1> (fused forward + adjoint)")
    # the same as two calls, the torch autograd path: forward keeping energies, then the adjoint
    ev = [(mk(), mk(), mk()) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                       # evict L2 (256 MiB > 129 MB) outside the timed span
        ev[i][0].record(stream)
        fwd(args.warmup + i)
        ev[i][1].record(stream)
        bwd(args.warmup + i)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    fwd_ms = [a.elapsed_time(b) for a, b, _ in ev]
    bwd_ms = [b.elapsed_time(c) for _, b, c in ev]
    # the plain forward (mean and variance only, nothing kept for an adjoint), timed on its own
    evp = [(mk(), mk()) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        evp[i][0].record(stream)
        fwd(args.warmup + i, save=False)
        evp[i][1].record(stream)
    torch.cuda.synchronize()
    plain_ms = [a.elapsed_time(b) for a, b in evp]
    # end-to-end through the public API: pinned host inputs in, host results out, every step
    Xh = torch.view_as_real(torch.as_tensor(X, dtype=torch.complex128)).contiguous().pin_memory()
    Gh = torch.view_as_real(torch.as_tensor(g_host, dtype=torch.complex128)).contiguous().pin_memory()
    mh = torch.empty((n_f, 2), dtype=torch.float64).pin_memory()
    vh = torch.empty((n_f, 2), dtype=torch.float64).pin_memory()
    gh = torch.empty((n_f + 3,), dtype=torch.float64).pin_memory()
    e0, e1 = mk(), mk()
    e2e_ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        e0.record(stream)
        Xd.copy_(Xh, non_blocking=True)
        G.copy_(Gh, non_blocking=True)
        out = fused(args.warmup + i)
        mh.copy_(torch.view_as_real(out["mean"]), non_blocking=True)
        vh.copy_(out["var"], non_blocking=True)
        gh[:n_f].copy_(out["grad_X_re"], non_blocking=True)
        gh[n_f:].copy_(out["grad_params"], non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    fp64 = fp64_rate_measured(stream)
    clk = clocks.stop()
    tf, tb, tp = float(np.mean(fwd_ms)), float(np.mean(bwd_ms)), float(np.mean(plain_ms))
    ms = float(np.mean(fused_ms))
    e2e = float(np.mean(e2e_ms))
    if world > 1:
        t = torch.tensor([ms, e2e, tf, tb, tp], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, e2e, tf, tb, tp = (float(v) for v in t)
    evals = float(n) * info["n_terms"] * n_f * world
    value = evals / (ms * 1e-3)
    fl_f = n * (info["fwd_save_flops_per_sample"] + n_f * info["flops_per_sample_freq"])
    fl_b = n * (info["bwd_saved_flops_per_sample"] + n_f * info["bwd_flops_per_sample_freq"])
    fl_p = n * (info["flops_per_sample"] + n_f * info["flops_per_sample_freq"])
    fl_x = n * (info["bwd_flops_per_sample"] + n_f * info["fused_flops_per_sample_freq"])
    dom = (fused_kernel, fl_x, ms)
    achieved = dom[1] / (dom[2] * 1e-3) / 1e12
    peak, peak_src = roofline_peak(fp64)
    traffic = None
    if dom[0] == TRAFFIC["kernel"] and kernel_sha256(D) == TRAFFIC["kernel_sha256"]:
        traffic = TRAFFIC["bytes_per_sample"] * n
    h2d = 2 * n_f * 16
    d2h = n_f * 32 + (n_f + 3) * 8
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "step": "forward + adjoint of the same samples in one pass (tami_forward_backward: mean, "
                    "variance, dSigma/dX per frequency and the gradients for a fixed upstream gradient)",
            "two_call": {"value": evals / ((tf + tb) * 1e-3), "unit": "evals/s", "ms": tf + tb,
                         "fwd_ms": tf, "adjoint_ms": tb,
                         "step": "tami_forward keeping per-sample energies, then tami_backward (the autograd path)",
                         "fwd_tflops": fl_f / (tf * 1e-3) / 1e12, "adjoint_tflops": fl_b / (tb * 1e-3) / 1e12},
            "plain_fwd": {"value": evals / (tp * 1e-3), "unit": "evals/s", "ms": tp,
                          "tflops": fl_p / (tp * 1e-3) / 1e12},
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (Philox momenta, in-kernel)",
            "config": {"workload": CFG["name"], "samples_per_gpu": n, "frequencies": n_f,
                       "terms": info["n_terms"], "beta": CFG["beta"], "t": CFG["t"], "tp": CFG["tp"],
                       "mu": CFG["mu"], "l2": "flushed before every step (256 MiB write)",
                       "parallelism": f"samples sharded over {world} GPU(s)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_unit": "bytes per launch (ncu capture, scaled per sample)",
                         "kernel": dom[0], "flops_per_launch": dom[1], "peak_source": peak_src,
                         "peak_derived": FP64_PEAK_TFLOPS, "frac_of_derived": achieved / FP64_PEAK_TFLOPS,
                         "peak_measured": fp64},
            "e2e": {"value": evals / (e2e * 1e-3), "unit": "evals/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": 2 * args.steps,
            "clocks": clk,
            "wall_s_timed": wall,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(d, X)
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_workload(args):
    """The other configurations of the method, timed on one GPU (parity for each is in tests/):
    order5 and order6 (forward + adjoint at four temperatures), order3_real (forward + adjoint on the real
    axis), all_orders (every order-2..5 diagram in one graph launch, forward),
    energy_x1 (the paper's energy-input example) and two_freq_x1 (two external frequencies per
    frequency row, energy input).  Prints one JSON line; not the headline metric."""
    import torch
    import paper_2311_17189_gb300 as T

    torch.cuda.set_device(0)
    dev = "cuda:0"
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    wl = args.workload
    launches_per_step = 0
    if wl in ("order5", "order6", "order3_real"):
        c = {"order5": W.ORDER5, "order6": W.ORDER6, "order3_real": W.ORDER3_REAL}[wl]
        if wl in ("order5", "order6"):
            d = next(x for x in T.enumerate_sigma(c["order"]) if x["code"] == tuple(c["code"]))
            betas = c["betas"]
            Xs = [W.matsubara(b, c["n_freq"]) for b in betas]
        else:
            d = T.enumerate_sigma(c["order"])[c["diagram_index"]]
            betas = (c["beta"],)
            Xs = [W.real_axis(*c["omega"], c["gamma"])]
        D = T.Diagram(d["alpha"], eps=d["eps"]).upload(0)
        info = D.info()
        n = c["n_samples"]
        lat = W.lattice(c)
        Xd = [torch.as_tensor(X, dtype=torch.complex128, device=dev) for X in Xs]
        Gd = [torch.full_like(x, 1.0 + 0.5j) for x in Xd]
        n_f = len(Xs[0])

        def step(i):
            for b, X, G in zip(betas, Xd, Gd):
                D.forward_backward(lat, c["seed"], i * n, n, X, b, G)
        launches_per_step = 2 * len(betas)
        evals = float(n) * info["n_terms"] * n_f * len(betas)
        flops = len(betas) * n * (info["bwd_flops_per_sample"] + n_f * info["fused_flops_per_sample_freq"])
        config = {"workload": c["name"], "samples": n, "frequencies": n_f, "terms": info["n_terms"],
                  "betas": list(betas), "step": "forward + adjoint in one pass (tami_forward_backward) at every beta"}
        bytes_step = None
    elif wl == "all_orders":
        c = W.ALL_ORDERS
        lib = []
        for m in c["orders"]:
            for d in T.enumerate_sigma(m):
                lib.append(T.Diagram(d["alpha"], eps=d["eps"], prefactor=(-1.0) ** m * (-1.0) ** d["loops"]))
        counts = [W.all_orders_samples(k) for k in range(len(lib))]
        seeds = [c["seed"] + k for k in range(len(lib))]
        X = W.matsubara(c["beta"], c["n_freq"])
        n_f = len(X)
        for D in lib:
            D.upload(0)
        B = T.Batch(lib, counts, seeds, n_f)            # chunk size from the autotuner
        lat = W.lattice(c)
        Xd = torch.as_tensor(X, dtype=torch.complex128, device=dev)

        def step(i):
            B.launch(lat, Xd, c["beta"])
        plan = B.info()
        launches_per_step = (1 if plan["items"] else 0) + plan["specialised"] + 1
        infos = [D.info() for D in lib]
        evals = float(sum(k * inf["n_terms"] * n_f for k, inf in zip(counts, infos)))
        flops = sum(k * (inf["flops_per_sample"] + n_f * inf["flops_per_sample_freq"]) for k, inf in zip(counts, infos))
        config = {"workload": c["name"], "diagrams": len(lib), "samples": int(sum(counts)), "frequencies": n_f,
                  "terms": int(sum(inf["n_terms"] for inf in infos)), "beta": c["beta"],
                  "step": ("one graph launch (forward): %d diagrams on their specialised kernels, %d on the "
                           "persistent kernel's work queue, one reduction" % (plan["specialised"], len(lib) - plan["specialised"])),
                  "plan": {k: v for k, v in plan.items() if k != "specialised_diagrams"}}
        bytes_step = None
    elif wl == "energy_x1":
        c = dict(W.ENERGY_X1)
        if args.rows:
            c["n_e"] = args.rows
        D = T.Diagram(c["alpha"]).upload(0)
        info = D.info()
        E = torch.as_tensor(W.random_energies(c["n_e"], c["alpha"].shape[0], a=c["a"], seed=c["seed"]), device=dev)
        X = torch.as_tensor(W.matsubara(c["beta"], c["n_freq"]), dtype=torch.complex128, device=dev)
        n_f = c["n_freq"]

        def step(i):
            D.eval_energies(E, X, c["beta"])
        launches_per_step = 1
        evals = float(c["n_e"]) * info["n_terms"] * n_f
        flops = c["n_e"] * (info["energy_in_flops_per_sample"] + n_f * info["energy_in_flops_per_sample_freq"])
        bytes_step = c["n_e"] * (8 * c["alpha"].shape[0] + 16 * n_f)
        config = {"workload": c["name"], "rows": c["n_e"], "frequencies": n_f, "terms": info["n_terms"],
                  "beta": c["beta"], "step": "tami_eval_energies, full [n_f][n_e] output"}
    elif wl == "two_freq_x1":
        c = dict(W.TWO_FREQ_X1)
        if args.rows:
            c["n_e"] = args.rows
        d = next(x for x in T.enumerate_sigma(c["order"]) if x["code"] == tuple(c["code"]))
        alpha = W.hold_external(d["alpha"], c["held"])
        D = T.Diagram(alpha, eps=d["eps"], n_ext=2).upload(0)
        info = D.info()
        N = alpha.shape[0]
        E = torch.as_tensor(W.random_energies(c["n_e"], N, a=c["a"], seed=c["seed"]), device=dev)
        X = torch.as_tensor(W.matsubara_grid(c["beta"], c["n_grid"], c["n_grid"]), dtype=torch.complex128, device=dev)
        n_f = X.shape[0]

        def step(i):
            D.eval_energies(E, X, c["beta"])
        launches_per_step = 1
        evals = float(c["n_e"]) * info["n_terms"] * n_f
        flops = c["n_e"] * (info["energy_in_flops_per_sample"] + n_f * info["energy_in_flops_per_sample_freq"])
        bytes_step = c["n_e"] * (8 * N + 16 * n_f) + n_f * 32
        config = {"workload": c["name"], "rows": c["n_e"], "frequency_rows": n_f, "externals": 2,
                  "terms": info["n_terms"], "beta": c["beta"],
                  "step": "tami_eval_energies, full [n_f][n_e] output"}
    else:
        raise SystemExit(f"unknown workload {wl}")
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    time.sleep(0.3)
    ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(args.warmup + i)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    fp64 = fp64_rate_measured(stream)
    clk = clocks.stop()
    t = float(np.mean(ms))
    tflops = flops / (t * 1e-3) / 1e12
    peak, peak_src = roofline_peak(fp64)
    line = {"metric": f"{config['workload']} evals/s (samples x terms x frequencies, FP64)",
            "value": evals / (t * 1e-3), "unit": "evals/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "config": config,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "flops_per_step": flops, "peak_source": peak_src,
                         "frac_of_derived": tflops / FP64_PEAK_TFLOPS, "peak_measured": fp64},
            "gpu_launches": launches_per_step * args.steps, "clocks": clk}
    if bytes_step is not None:
        gbs = bytes_step / (t * 1e-3) / 1e9
        line["hbm"] = {"achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s", "frac": gbs / HBM_PEAK_GBS,
                       "algorithmic_bytes_per_step": bytes_step}
    print(json.dumps(line))
    return 0


def run_construct(args):
    """Host-side construction (step a11: residues, flattening into the device table, validation;
    no GPU): wall time per diagram for the paper's order-2 example and the largest enumerated
    tables at orders 4-6, and for enumerating and constructing every order-6 diagram, one by one
    and on a pool of host threads (construct_many).  Not the metric; one JSON line."""
    import resource
    import paper_2311_17189_gb300 as T

    def per_call_ms(make, reps):
        make()
        t0 = time.perf_counter()
        for _ in range(reps):
            make()
        return (time.perf_counter() - t0) / reps * 1e3

    rss0 = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss
    example = np.array([[1, 0, 0], [0, 1, 0], [-1, 1, 1]], dtype=np.int8)   # the paper's order-2 example
    rows = [{"diagram": "order2_paper_example", "terms": T.Diagram(example).info()["n_terms"],
             "ms": per_call_ms(lambda: T.Diagram(example), 200)}]
    for c in (W.ORDER4, W.ORDER5, W.ORDER6):
        d = next(x for x in T.enumerate_sigma(c["order"]) if x["code"] == tuple(c["code"]))
        make = lambda: T.Diagram(d["alpha"], eps=d["eps"])
        rows.append({"diagram": c["name"], "terms": make().info()["n_terms"],
                     "ms": per_call_ms(make, max(2, args.steps))})
    rss1 = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss
    t0 = time.perf_counter()
    ds = T.enumerate_sigma(6)
    t1 = time.perf_counter()
    lib = [T.Diagram(x["alpha"], eps=x["eps"]) for x in ds]       # all held at once
    t2 = time.perf_counter()
    terms = sum(D.info()["n_terms"] for D in lib)
    rss2 = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss
    threads = os.cpu_count() or 1
    t3 = time.perf_counter()
    lib2 = T.construct_many([dict(alpha=x["alpha"], eps=x["eps"]) for x in ds], threads=threads)
    t4 = time.perf_counter()
    assert len(lib2) == len(lib)
    print(json.dumps({"metric": "host construction wall time (AMI residues + flattening + validation)",
                      "unit": "ms", "diagrams": rows,
                      "order6_all": {"diagrams": len(lib), "terms": terms, "enumerate_ms": (t1 - t0) * 1e3,
                                     "construct_ms": (t2 - t1) * 1e3, "held_rss_mb": (rss2 - rss1) / 1024.0,
                                     "construct_many_ms": (t4 - t3) * 1e3, "construct_many_threads": threads},
                      "single_diagrams_peak_rss_growth_mb": (rss1 - rss0) / 1024.0, "cores": 1,
                      "host": os.uname().machine}))
    return 0


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="tami", choices=["tami", "reference"])
    p.add_argument("--ref-samples", type=int, default=1 << 12)
    p.add_argument("--samples", type=int, default=CFG["n_samples"], help="samples per GPU (profiling runs)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--rows", type=int, default=0, help="energy rows of energy_x1 / two_freq_x1 (profiling runs)")
    p.add_argument("--workload", default="order4",
                   choices=["order4", "order5", "order6", "order3_real", "all_orders", "energy_x1", "two_freq_x1",
                            "construct"],
                   help="order4 is the headline metric; the others time the remaining configurations on one GPU "
                        "(construct: the host-side construction, no GPU)")
    p.add_argument("--jit", default="auto", choices=["auto", "never", "always"],
                   help="specialised kernels: auto (large calls), never (generic kernels) or always (profiling runs)")
    args = p.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "construct":
        return run_construct(args)
    import paper_2311_17189_gb300 as T
    T.set_jit(args.jit)
    if args.workload != "order4":
        return run_workload(args)
    return run_tami(args)


if __name__ == "__main__":
    sys.exit(main())
