#!/usr/bin/env python3
"""Benchmark of the LRE hot path (steps i+ii: counts -> theta -> rho).

Default workload (the configuration the headline metric is quoted on):
n = 14 qubits, GHZ state mixed with 5% white noise, 3^14 = 4,782,969 Pauli
bases x 2^14 outcomes, 1000 shots per basis, int16 counts (156.7 GB) drawn
on the device by the counter-based generator in synth/ before timing.
A step is one lre_estimate call (count ingest, parity transform + fold +
1/(N 3^k) weight, Pauli-to-matrix assembly of the complex64 rho).  The
projection (step iii) is timed once, separately, on the rho of the last step
and reported with its FP64 roofline and as a total with the step
(--no-project skips it).

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle (the
paper's zero-dropped direct sum) on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "n14": dict(n=14, state="ghz", p=0.05, shots=1000, kind="i16", seed=14,
                desc="n=14 GHZ+5% white noise, 4782969 bases x 16384 outcomes, 1000 shots/basis, "
                     "int16 counts generated on device"),
    "n12": dict(n=12, state="product", shrink=0.95, shots=4096, kind="i32", seed=12,
                desc="n=12 product of Haar single-qubit states, 5% depolarising, 531441 bases x "
                     "4096 outcomes, 4096 shots/basis, int32 counts"),
    "n12s": dict(n=12, state="ghz", p=0.05, shots=1000, kind="i16", seed=12,
                 desc="n=12 GHZ+5% white noise, 531441 bases x 4096 outcomes, 1000 shots/basis, "
                      "int16 counts (profiling-size case of the n=14 kernels)"),
    "n11p": dict(n=11, state="product", shrink=0.95, shots=4096, kind="i32", seed=11,
                 desc="n=11 product of Haar single-qubit states, 5% depolarising, 177147 bases x 2048 "
                      "outcomes, 4096 shots/basis, int32 counts (profiling-size case of the n=12 kernels)"),
    "n10": dict(n=10, state="ghz", p=0.10, shots=1000, kind="i32", seed=10,
                desc="n=10 GHZ+10% white noise, 59049 bases x 1024 outcomes, 1000 shots/basis, int32"),
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, device=None):
    """Slowest rank's value (every rank gets it); CPU tensors under gloo."""
    import torch
    import torch.distributed as dist
    use_cpu = device is None or dist.get_backend() == "gloo"
    t = torch.tensor([float(x)], dtype=torch.float64, device="cpu" if use_cpu else device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_per_step):
    """Units all ranks processed per second (each rank runs its own instance:
    weak scaling, no data-path collective)."""
    return units_per_rank * world / (ms_per_step / 1000.0)


def fp64_gemm_tflops(torch, device):
    """FP64 peak for the projection's roofline: a cuBLAS DGEMM of 8192^3."""
    nn = 8192
    a = torch.randn(nn, nn, dtype=torch.float64, device=device)
    b = torch.randn(nn, nn, dtype=torch.float64, device=device)
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        a @ b
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 3 / 1e3
    del a, b
    torch.cuda.empty_cache()
    return round(2 * nn ** 3 / t / 1e12, 3)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def source_digest(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# sources whose digest pins a recorded DRAM traffic figure to the kernel it was taken on
KERNEL_SOURCES = {
    "fold_first6": ["paper_1602_08604_gb300/csrc/fold.cu", "paper_1602_08604_gb300/csrc/passes.cuh",
                    "paper_1602_08604_gb300/csrc/sm103.cuh"],
    "fold_first6_mma": ["paper_1602_08604_gb300/csrc/fold_mma.cu", "paper_1602_08604_gb300/csrc/passes.cuh",
                        "paper_1602_08604_gb300/csrc/sm103.cuh"],
    "fold_first7_mma": ["paper_1602_08604_gb300/csrc/fold_mma.cu", "paper_1602_08604_gb300/csrc/passes.cuh",
                        "paper_1602_08604_gb300/csrc/sm103.cuh"],
}


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from profiles/traffic.txt when the kernel's
    sources are unchanged since the capture; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p) or kernel not in KERNEL_SOURCES:
        return None
    digest = source_digest(KERNEL_SOURCES[kernel])
    with open(p) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[1] == workload:
                return float(parts[2]) if parts[3] == digest else None
    return None


def make_counts(torch, wl, device):
    from synth import gen
    n = wl["n"]
    dt = torch.int16 if wl["kind"] == "i16" else torch.int32
    counts = torch.empty((3 ** n, 2 ** n), dtype=dt, device=device)
    if wl["state"] == "ghz":
        gen.gen_ghz(n, wl["p"], wl["shots"], wl["seed"], counts)
    elif wl["state"] == "product":
        from synth import states as st
        bloch = st.haar_bloch_vectors(n, seed=wl["seed"], shrink=wl["shrink"])
        gen.gen_product(bloch, wl["shots"], wl["seed"], counts)
    torch.cuda.synchronize()
    return counts


def cpu_rows(wl, bases):
    import numpy as np
    from synth import counts as sc
    n = wl["n"]
    dt = np.int16 if wl["kind"] == "i16" else np.int32
    if wl["state"] == "ghz":
        return sc.sample_ghz(n, wl["p"], wl["shots"], wl["seed"], bases=bases, dtype=dt)
    from synth import states as st
    bloch = st.haar_bloch_vectors(n, seed=wl["seed"], shrink=wl["shrink"])
    return sc.sample_product(bloch, wl["shots"], wl["seed"], bases=bases, dtype=dt)


def oracle_sample(wl, seconds_target=15.0, max_bases=None):
    """Time the CPU oracle's direct sum (steps i, per basis) on the first
    bases of the workload; returns (bases/s, bases, seconds, threads)."""
    import numpy as np
    from oracle import direct
    n = wl["n"]
    threads = direct.set_threads(0)
    P = 4 ** n
    S = np.zeros(P, np.int64)
    diag = np.zeros(P, np.int64)
    probe = 16
    rows = cpu_rows(wl, np.arange(probe))
    # first call builds the oracle's 2^n x 2^n nonzero matrix (kept for later calls)
    direct.parity_sums(rows[:1], n, b0=0, b1=1, S=np.zeros(P, np.int64), diag=np.zeros(P, np.int64))
    t0 = time.perf_counter()
    direct.parity_sums(rows, n, b0=0, b1=probe, S=S, diag=diag)
    dt = time.perf_counter() - t0
    k = max(probe, int(seconds_target / max(dt / probe, 1e-9)))
    k = min(k, 3 ** n) if max_bases is None else min(k, max_bases, 3 ** n)
    rows = cpu_rows(wl, np.arange(probe, probe + k))
    t0 = time.perf_counter()
    direct.parity_sums(rows, n, b0=probe, b1=probe + k, S=S, diag=diag)
    dt = time.perf_counter() - t0
    return k / dt, k, dt, threads


def spot_check(torch, wl, theta, rho, n_entries=96, n_rho=32):
    """Bit-exact theta on sampled Pauli strings and rho on sampled elements
    against the oracle (counts regenerated on the CPU)."""
    import numpy as np
    from oracle import direct
    n = wl["n"]
    rng = np.random.default_rng(2024)
    idx = []
    for _ in range(n_entries):
        k = int(rng.integers(0, min(n, 4) + 1))         # biased to few identity letters
        dig = rng.integers(1, 4, size=n)
        dig[rng.choice(n, size=k, replace=False)] = 0
        idx.append(int(sum(int(dig[q]) << (2 * (n - 1 - q)) for q in range(n))))
    want = direct.estimate_entries(n, idx, lambda b: cpu_rows(wl, b), wl["shots"])
    got = theta[torch.tensor(idx, device=theta.device)].cpu().numpy()
    ok_theta = bool(np.array_equal(got, want))
    t_host = theta.cpu().numpy()
    d = 2 ** n
    r = rng.integers(0, d, n_rho)
    c = rng.integers(0, d, n_rho)
    ref = direct.mu_elements(t_host, n, r, c)
    gr = rho[torch.from_numpy(r).to(rho.device), torch.from_numpy(c).to(rho.device)].cpu().numpy()
    err = float(np.max(np.abs(gr - ref)) / max(np.max(np.abs(ref)), 1e-30))
    return {"theta_entries": len(idx), "theta_bit_exact": ok_theta,
            "rho_entries": n_rho, "rho_max_rel_err": err}


def run_e2e(args, wl, lre, torch, device, theta_dev):
    """Same metric through lre_estimate_host: every step copies the step's
    input from pinned host memory and reads theta and rho back."""
    n, N = wl["n"], wl["shots"]
    B, d = 3 ** n, 2 ** n
    if wl["state"] == "ghz":
        from synth import gen
        rec = torch.empty((B, N), dtype=torch.int16, device=device)
        gen.gen_ghz_records(n, wl["p"], wl["seed"], rec)
        host_in = torch.empty((B, N), dtype=torch.int16, pin_memory=True)
        host_in.copy_(rec)
        del rec
        kind, what = lre.LRE_HOST_RECORDS_U16, "uint16 shot records"
    else:
        c = make_counts(torch, wl, device)
        host_in = torch.empty(c.shape, dtype=c.dtype, pin_memory=True)
        host_in.copy_(c)
        del c
        kind = lre.LRE_HOST_COUNTS_I16 if wl["kind"] == "i16" else lre.LRE_HOST_COUNTS_I32
        what = f"{wl['kind']} dense counts"
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    theta_h = torch.empty(4 ** n, dtype=torch.float64, pin_memory=True)
    rho_h = torch.empty((d, d), dtype=torch.complex64, pin_memory=True)
    ctx = lre.lre_create(device.index)
    stream = torch.cuda.current_stream(device)
    for _ in range(args.warmup):
        lre.lre_estimate_host(ctx, host_in, kind, N, n, theta_h, rho_h, stream=stream)
    torch.cuda.synchronize()
    per_step = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t1 = time.perf_counter()
        lre.lre_estimate_host(ctx, host_in, kind, N, n, theta_h, rho_h, stream=stream)  # returns synchronised
        per_step.append(time.perf_counter() - t1)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    same = bool(torch.equal(theta_h, theta_dev.cpu())) if theta_dev is not None else None
    lre.lre_destroy(ctx)
    per_step.sort()
    return {"value": round(B / dt, 1), "unit": "Pauli bases/s", "seconds_per_step": round(dt, 4),
            "step_seconds_median_min_max": [round(per_step[len(per_step) // 2], 4), round(per_step[0], 4),
                                            round(per_step[-1], 4)],
            "h2d_bytes_per_step": host_in.numel() * host_in.element_size(),
            "d2h_bytes_per_step": theta_h.numel() * 8 + rho_h.numel() * 8,
            "input": f"pinned host {what}; lre_estimate_host (chunked H2D on a copy stream overlapped "
                     f"with the device ingest and first fold pass per chunk, remaining passes, theta D2H "
                     f"during the assembly, rho D2H)",
            "theta_equals_device_path": same}


FIRST_PASS_KERNELS = ("fold_first6", "fold_first6_mma", "fold_first6_mma_split", "fold_first9_fused",
                      "fold_first6_mma_records", "fold_first9_mma", "fold_first7_mma")


def timed_steps(lre, ctx, torch, stream, step, steps, warmup):
    """warmup untimed steps, then `steps` steps between CUDA events on the
    launching stream, with the library's per-launch event records on.
    Returns (ms per step, [(kernel, ms)], own kernel launches)."""
    for _ in range(warmup):
        step()
    lre.lre_sync(ctx, stream)
    torch.cuda.synchronize()
    launches0 = lre.lre_launch_count(ctx)
    lre.lre_profile(ctx, True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    total_ms = ev0.elapsed_time(ev1)
    lre.lre_sync(ctx, stream)
    recs = lre.lre_profile_records(ctx)
    lre.lre_profile(ctx, False)
    return total_ms, recs, lre.lre_launch_count(ctx) - launches0


def kernel_roofline(recs, steps, wl, workload):
    """Per-kernel device time and the roofline of the step's dominant kernel
    (algorithmic bytes per launch: the counts it reads once)."""
    per = {}
    for name, t in recs:
        a = per.setdefault(name, [0.0, 0])
        a[0] += t
        a[1] += 1
    top_name, (top_ms, top_n) = max(per.items(), key=lambda kv: kv[1][0])
    avg_ms = top_ms / top_n
    n = wl["n"]
    count_bytes = 2 if wl["kind"] == "i16" else 4
    alg_bytes = 3 ** n * (2 ** n) * count_bytes if top_name in FIRST_PASS_KERNELS else None
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9 if alg_bytes else None
    roofline = {"bound": "hbm", "kernel": top_name,
                "achieved": round(achieved, 1) if achieved else None,
                "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
                "frac": round(achieved / peak, 4) if achieved else None,
                "traffic": recorded_traffic(top_name, workload),
                "kernel_ms": round(avg_ms, 3),
                "alg_bytes_per_launch": alg_bytes}
    kernels = {k: {"ms_per_step": round(v[0] / steps, 3), "launches": v[1]} for k, v in per.items()}
    return roofline, kernels


def step_alg_bytes(wl):
    """Counts read once, theta written (and read by the assembly), rho written."""
    n = wl["n"]
    return 3 ** n * (2 ** n) * (2 if wl["kind"] == "i16" else 4) + 8 * 4 ** n * 2 + 8 * 4 ** n


def set_first_variant(lre, ctx, variant, consumers=0, discard=0):
    """Test hooks: the first-pass variant (2: fused with the second pass), the
    CTAs the fused tensor-core pass gives the second pass (0: default) and
    whether that pass drops the ring lines it has read from L2."""
    import ctypes
    f = lre.load().lre_debug_set_first_pass
    f.argtypes = [ctypes.c_void_p, ctypes.c_int]
    f.restype = ctypes.c_int
    if f(ctx, int(variant)) != 0:
        raise RuntimeError("first-pass variant rejected")
    g = lre.load().lre_debug_set_fused_consumers
    g.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    g.restype = ctypes.c_int
    if g(ctx, int(consumers), int(discard)) != 0:
        raise RuntimeError("fused-pass consumer count rejected")


def set_first7(lre, ctx, on):
    """Test hook: the raw tensor-core first pass folds seven qubits where it
    applies (1) or six (0, the library default)."""
    import ctypes
    f = lre.load().lre_debug_set_first7
    f.argtypes = [ctypes.c_void_p, ctypes.c_int]
    f.restype = ctypes.c_int
    if f(ctx, int(on)) != 0:
        raise RuntimeError("first7 setting rejected")


def arm_record(lre, torch, device, stream, counts, wl, workload, path, steps, warmup, theta_ref=None,
               first_variant=None, consumers=0, discard=0, first7=None):
    """One timed arm of lre_estimate on resident counts with the first fold
    pass on the tensor cores or on the ALUs (FWHT), in a context of its own;
    first_variant 2: the first pass fused with the second through L2;
    first7 1: the raw tensor-core first pass folds seven qubits, not six."""
    n = wl["n"]
    ctx = lre.lre_create(device.index)
    try:
        if first_variant is not None:
            set_first_variant(lre, ctx, first_variant, consumers, discard)
        if first7 is not None:
            set_first7(lre, ctx, first7)
        lre.lre_set_fold_path(ctx, {"tensor": lre.LRE_FOLD_TENSOR, "tensor_split": lre.LRE_FOLD_TENSOR_SPLIT,
                                    "fwht": lre.LRE_FOLD_FWHT}[path])
        theta = torch.empty(4 ** n, dtype=torch.float64, device=device)
        rho = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device=device)
        total_ms, recs, launches = timed_steps(
            lre, ctx, torch, stream, lambda: lre.lre_estimate(ctx, counts, wl["shots"], n, theta, rho, stream=stream),
            steps, warmup)
    finally:
        lre.lre_destroy(ctx)
    ms = total_ms / steps
    roofline, kernels = kernel_roofline(recs, steps, wl, workload)
    peak, _ = load_peaks()
    sa = step_alg_bytes(wl)
    out = {"fold_path": path, "ms_per_step": round(ms, 3), "value": round(3 ** n / (ms / 1e3), 1),
           "unit": "Pauli bases/s", "steps": steps, "warmup": warmup, "gpu_launches": launches,
           "roofline": roofline, "kernels": kernels, "step_alg_bytes": sa,
           "step_frac": round(sa / (ms / 1e3) / 1e9 / peak, 4)}
    if theta_ref is not None:
        out["theta_equal_to_headline_arm"] = bool(torch.equal(theta, theta_ref))
    return out, theta


def fused_generation_arm(lre, torch, device, stream, wl, theta_ref, steps, warmup, chunk_rows=4 * 729):
    """Generation fused with the fold: the device generator fills one slot of
    a two-slot ring of count chunks (whole tile rows), lre_stream_chunk folds
    it at once, so the count matrix never exists; a step is generation plus
    estimate.  Beside it, the materialised path's generation of the whole
    matrix, timed the same way (the headline step then adds its ms)."""
    from synth import gen
    n, N = wl["n"], wl["shots"]
    B, d = 3 ** n, 2 ** n
    ring = [torch.empty((chunk_rows, d), dtype=torch.int16, device=device) for _ in range(2)]
    theta = torch.empty(4 ** n, dtype=torch.float64, device=device)
    rho = torch.empty((d, d), dtype=torch.complex64, device=device)
    ctx = lre.lre_create(device.index)
    try:
        def step():
            lre.lre_stream_begin(ctx, n, lre.LRE_COUNTS_I16, N)
            for k, b0 in enumerate(range(0, B, chunk_rows)):
                buf = ring[k % 2][: min(chunk_rows, B - b0)]
                gen.gen_ghz(n, wl["p"], N, wl["seed"], buf, b0=b0)
                lre.lre_stream_chunk(ctx, buf, b0, stream=stream)
            lre.lre_stream_end(ctx, theta, rho, stream=stream)

        total_ms, recs, launches = timed_steps(lre, ctx, torch, stream, step, steps, warmup)
    finally:
        lre.lre_destroy(ctx)
    ms = total_ms / steps
    same = bool(torch.equal(theta, theta_ref))
    del theta, rho, ring
    torch.cuda.empty_cache()
    # the materialised path's generation of the whole matrix, same events
    full = torch.empty((B, d), dtype=torch.int16, device=device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    gen.gen_ghz(n, wl["p"], N, wl["seed"], full)
    e0.record(stream)
    gen.gen_ghz(n, wl["p"], N, wl["seed"], full)
    e1.record(stream)
    torch.cuda.synchronize()
    gen_ms = e0.elapsed_time(e1)
    del full
    torch.cuda.empty_cache()
    per = {}
    for name, t in recs:
        per[name] = per.get(name, 0.0) + t
    lre_ms = sum(per.values()) / steps
    return {"ms_per_step": round(ms, 3), "value": round(B / (ms / 1e3), 1), "unit": "Pauli bases/s",
            "steps": steps, "warmup": warmup, "chunk_bases": chunk_rows,
            "count_buffer_bytes": 2 * chunk_rows * d * 2, "library_kernels_ms_per_step": round(lre_ms, 3),
            "generator_and_gaps_ms_per_step": round(ms - lre_ms, 3), "gpu_launches": launches,
            "materialised_generation_ms": round(gen_ms, 3),
            "theta_equal_to_headline_arm": same,
            "note": "a step generates the counts (GHZ sampler, device) and estimates theta and rho; the "
                    "materialised path needs the 156.7 GB count matrix, generated in "
                    "materialised_generation_ms, before its step"}


def run_ours(args, wl):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_1602_08604_gb300 import lre
    n = wl["n"]
    counts = make_counts(torch, wl, device)
    theta = torch.empty(4 ** n, dtype=torch.float64, device=device)
    rho = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device=device)
    ctx = lre.lre_create(local)
    lre.lre_set_fold_path(ctx, {"tensor": lre.LRE_FOLD_TENSOR, "tensor_split": lre.LRE_FOLD_TENSOR_SPLIT,
                                "fwht": lre.LRE_FOLD_FWHT}[args.fold_path])
    if args.fused_first:
        set_first_variant(lre, ctx, 2, args.fused_consumers, args.fused_discard)
    if args.first7:
        set_first7(lre, ctx, 1)
    stream = torch.cuda.current_stream(device)

    def step():
        lre.lre_estimate(ctx, counts, wl["shots"], n, theta, rho, stream=stream)

    for _ in range(args.warmup):
        step()
    lre.lre_sync(ctx, stream)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    total_ms, recs, launches = timed_steps(lre, ctx, torch, stream, step, args.steps, 0)
    clk = clocks.stop()
    if world > 1:
        total_ms = max_over_ranks(total_ms, device)
        dist.barrier()
    ms = total_ms / args.steps
    B = 3 ** n
    value = whole_job_rate(B, world, ms)
    roofline, kernels = kernel_roofline(recs, args.steps, wl, args.workload)
    peak, _ = load_peaks()
    step_alg = step_alg_bytes(wl)
    check = spot_check(torch, wl, theta, rho) if args.check and rank == 0 else None
    compare = {}
    if args.compare and rank == 0 and world == 1:
        # the other first-pass arm on the same resident counts (spec:
        # tensor-core form against the plain FWHT path, same accuracy)
        other = "fwht" if args.fold_path != "fwht" else "tensor"
        compare[f"{args.workload}_{other}"], _ = arm_record(
            lre, torch, device, stream, counts, wl, args.workload, other, args.compare_steps, 2, theta_ref=theta)
        torch.cuda.empty_cache()
        if args.fold_path == "tensor" and not args.fused_first and not args.first7 and n >= 8:
            # the tensor-core first pass folding seven qubits (then one later pass fewer)
            compare[f"{args.workload}_first_pass_seven_qubits"], _ = arm_record(
                lre, torch, device, stream, counts, wl, args.workload, "tensor", args.compare_steps, 2,
                theta_ref=theta, first7=1)
            torch.cuda.empty_cache()
        if args.fold_path == "tensor" and not args.fused_first:
            # the first pass fused with the second through an L2 ring
            compare[f"{args.workload}_fused_first_second"], _ = arm_record(
                lre, torch, device, stream, counts, wl, args.workload, "tensor", args.compare_steps, 2,
                theta_ref=theta, first_variant=2, consumers=args.fused_consumers,
                discard=args.fused_discard)
            torch.cuda.empty_cache()
    projection = None
    if args.project and rank == 0:
        # step (iii), timed once on its own on the rho of the last step: the
        # Lanczos path (double-float products with the complex64 mu, FP64
        # vectors, full reorthogonalisation, the threshold from the converged
        # end of the spectrum, a certification run, the rank-k rebuild), or
        # the tridiagonal reduction where it falls back (achieved FP64 rate
        # against a DGEMM measured in the same run)
        fp64_peak = fp64_gemm_tflops(torch, device)
        small = torch.eye(256, dtype=torch.complex64, device=device) / 256
        lre.lre_project(ctx, small, 8, torch.empty_like(small), stream=stream)  # handles and libraries warm
        torch.cuda.synchronize()
        rho_p = torch.empty_like(rho)
        eig = torch.empty(2 ** n, dtype=torch.float64, device=device)
        lre.lre_profile(ctx, True)
        t0 = time.perf_counter()
        lre.lre_project(ctx, rho, n, rho_p, eig_rho=eig, stream=stream)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        precs = lre.lre_profile_records(ctx)
        lre.lre_profile(ctx, False)
        ev = eig.cpu().numpy()
        kept = int((ev > 0).sum())
        d = 2 ** n
        m = min(kept, d - kept)
        ptab = {}
        for k, v in precs:
            a_ = ptab.setdefault(k, [0.0, 0])
            a_[0] += v
            a_[1] += 1
        if "kry_matvec" in ptab:
            # Lanczos path: the dominant kernel is the product with mu, read
            # once per step as complex64 (8 d^2 bytes) and formed in
            # double-float arithmetic on the FP32 pipes
            mv_ms, steps = ptab["kry_matvec"]
            peak, peak_kind = load_peaks()
            gbs = 8.0 * d * d * steps / (mv_ms / 1e3) / 1e9
            fp64 = {"bound": "hbm", "kernel": "kry_matvec", "achieved": round(gbs, 1), "peak": peak,
                    "peak_source": peak_kind, "unit": "GB/s", "frac": round(gbs / peak, 4),
                    "lanczos_steps": steps,
                    "byte_model": "8 d^2 per Lanczos step (mu as complex64, once)",
                    "fp64_dgemm_tflops_same_run": fp64_peak}
        else:
            if "hetrd(cusolver)" in ptab:
                flops = 16.0 / 3.0 * d ** 3 + 8.0 * d * d * m + 4.0 * d * d * m
                model = "16/3 d^3 (tridiagonal reduction) + 12 d^2 m (back-transformation, rank-m rebuild)"
            else:
                flops = 16.0 / 3.0 * d ** 3 + 8.0 * d ** 3 + 4.0 * d * d * m
                model = "16/3 d^3 + 8 d^3 (full eigendecomposition) + 4 d^2 m (rank-m rebuild)"
            achieved = flops / secs / 1e12
            fp64 = {"bound": "fp64", "achieved_tflops": round(achieved, 3), "peak_tflops": fp64_peak,
                    "peak_source": "cuBLAS DGEMM 8192^3, same run", "frac": round(achieved / fp64_peak, 4),
                    "flop_model": model}
        projection = {"seconds": round(secs, 4),
                      "kernels": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in ptab.items()},
                      "kept_eigenvalues": kept, "trace": float(ev.sum()), "min_eigenvalue": float(ev.min()),
                      "roofline": fp64}
        del rho_p
    lre.lre_destroy(ctx)
    ctx = None
    e2e = None
    if not args.no_e2e:
        theta_keep = theta
        del counts, rho
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        e2e = run_e2e(args, wl, lre, torch, device, theta_keep)
    else:
        theta_keep = theta
        del counts, rho
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if args.compare and rank == 0 and world == 1 and args.workload == "n14":
        compare["n14_fused_generation"] = fused_generation_arm(lre, torch, device, stream, wl, theta_ref=theta_keep,
                                                               steps=2, warmup=1)
        del theta_keep
        torch.cuda.empty_cache()
        # the int32 precision workload (n = 12, 4096 shots per basis): the
        # tensor-core form (two fp16 planes per count) against the FWHT path
        wl12 = WORKLOADS["n12"]
        c12 = make_counts(torch, wl12, device)
        rec_t, th_t = arm_record(lre, torch, device, stream, c12, wl12, "n12", "tensor_split", args.compare_steps, 3)
        rec_f, _ = arm_record(lre, torch, device, stream, c12, wl12, "n12", "fwht", args.compare_steps, 3,
                              theta_ref=th_t)
        compare["n12_tensor"], compare["n12_fwht"] = rec_t, rec_f
        del c12, th_t
        torch.cuda.empty_cache()
        compare["batched"] = run_batched(args, summary=True)
        torch.cuda.empty_cache()

    out = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            bps, k, dt, thr = oracle_sample(wl, seconds_target=args.cpu_seconds)
            cpu = {"value": round(bps, 3), "unit": "Pauli bases/s", "cores": thr, "kind": "oracle",
                   "sample": f"oracle direct zero-dropped sum over the first {k} bases of the same "
                             f"n={n} workload (counts regenerated on the CPU), {dt:.1f} s"}
        out = {
            "metric": "Pauli bases/sec and end-to-end LRE seconds at n=14; fraction of HBM roofline",
            "value": round(value, 1), "unit": "Pauli bases/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "lre_seconds": round(ms / 1000, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/f64",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "n": n, "shots_per_basis": wl["shots"],
                       "counts_dtype": wl["kind"], "step": "lre_estimate: counts -> theta (FP64) -> rho (c64)",
                       "fold_path": args.fold_path, "fused_first_second": bool(args.fused_first),
                       "l2": "inputs larger than L2 (no flush needed)",
                       "parallelism": "independent instance per GPU" if world > 1 else "1 GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clk, "gpu_launches": launches,
            "e2e": None,
            "kernels": kernels,
            "step_alg_bytes": step_alg,
            "step_alg_gbs": round(step_alg / (ms / 1e3) / 1e9, 1),
            "step_frac": round(step_alg / (ms / 1e3) / 1e9 / peak, 4),
        }
        if check:
            out["parity"] = check
        out["e2e"] = e2e
        if projection:
            out["projection"] = projection
            out["total_seconds_with_projection"] = round(ms / 1000 + projection["seconds"], 4)
        if compare:
            out["comparisons"] = compare
    return out


def batched_specs(count=256, seed=256):
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.integers(3, 10))
        rank = int(rng.integers(1, 5))
        shots = int(np.exp(rng.uniform(np.log(500), np.log(10000))))
        out.append((n, rank, shots, seed * 1000 + k))
    return out


def batched_alg_bytes(ns, jmax):
    """Algorithmic DRAM bytes of one batched launch over instances of these n
    (int32 counts, theta and rho requested): every pass reads its whole input
    and writes its whole output once -- the fold passes of up to jmax qubits
    (the final pass at most two), theta and the exact integers T, then the
    assembly (16-byte intermediates, complex64 rho)."""
    total = 0
    for n in ns:
        r, C, in_sz = n, 1, 4
        while r > 0:
            J = min(r, jmax)
            if r == 3 and J == 3:
                J = 2
            total += 6 ** r * C * in_sz
            total += 4 ** n * 16 if J == r else 6 ** (r - J) * 4 ** J * C * 4
            r, C, in_sz = r - J, C * 4 ** J, 4
        t = 0
        if n >= 6:
            total += 4 ** n * 8 + 4 ** n * (16 if n > 6 else 8)
            t = 6
        while t < n:
            J = 2 if n - t >= 2 else 1
            total += 4 ** n * (8 if t == 0 else 16) + 4 ** n * (8 if t + J == n else 16)
            t += J
    return total


def run_batched(args, summary=False):
    """256 instances (n ~ U{3..9}, random-rank Ginibre mixtures, shots
    log-uniform in 500..10000, int32 counts) in one persistent launch, against
    one lre_estimate call per instance.  summary: the record for the headline
    line's comparisons (args.compare_steps timed steps)."""
    import numpy as np
    import torch
    from paper_1602_08604_gb300 import lre
    from synth import counts as sc
    from synth import gen
    from synth import states as st
    device = torch.device("cuda", 0)
    specs = batched_specs()
    items = []
    for n, rank, shots, seed in specs:
        rho = st.ginibre_mixture(n, rank, seed)
        thr = sc.cdf_thresholds(st.born_probabilities(st.pauli_expectations(rho), n))
        c = torch.empty((3 ** n, 2 ** n), dtype=torch.int32, device=device)
        gen.gen_cdf(torch.from_numpy(thr.view(np.int32)).to(device), n, shots, seed, c)
        theta = torch.empty(4 ** n, dtype=torch.float64, device=device)
        rh = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device=device)
        items.append((c, shots, n, theta, rh))
    torch.cuda.synchronize()
    ctx = lre.lre_create(0)
    stream = torch.cuda.current_stream(device)
    tuned_ms = lre.lre_batch_tune(ctx, items, stream=stream)
    bases = sum(3 ** n for n, _, _, _ in specs)
    count_bytes = sum(3 ** n * 2 ** n * 4 for n, _, _, _ in specs)

    steps = args.compare_steps if summary else args.steps
    warmup = args.warmup if not summary else 3

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    launches0 = lre.lre_launch_count(ctx)
    ms_batch = timed(lambda: lre.lre_batch_run(ctx, items, stream=stream))
    batch_launches = (lre.lre_launch_count(ctx) - launches0) // (steps + warmup)
    theta_b = [it[3].clone() for it in items]
    # the same launch captured once in a CUDA graph and replayed
    side = torch.cuda.Stream(device)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        lre.lre_batch_run(ctx, items, stream=torch.cuda.current_stream(device))
    ms_graph = timed(graph.replay)
    same_graph = all(torch.equal(a, it[3]) for a, it in zip(theta_b, items))
    launches0 = lre.lre_launch_count(ctx)
    ms_single = timed(lambda: [lre.lre_estimate(ctx, c, s, n, t, r, stream=stream) for c, s, n, t, r in items])
    single_launches = (lre.lre_launch_count(ctx) - launches0) // (steps + warmup)
    same = all(torch.equal(a, it[3]) for a, it in zip(theta_b, items))
    lre.lre_sync(ctx, stream)
    peak, peak_kind = load_peaks()
    sched = lre.lre_batch_schedule(ctx)
    alg = batched_alg_bytes([n for n, _, _, _ in specs], sched["jmax"])
    achieved = alg / (ms_batch / 1e3) / 1e9
    out = {
        "metric": "Pauli bases/sec (batched instances)", "value": round(bases / (ms_batch / 1e3), 1),
        "unit": "Pauli bases/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
        "ms_per_step": round(ms_batch, 4), "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None, "dtype": "int32/f64", "data": "synthetic",
        "config": {"workload": "256 instances, n ~ U{3..9}, random-rank (1..4) Ginibre mixtures, "
                               "shots/basis log-uniform 500..10000, int32 counts",
                   "bases": bases, "count_bytes": count_bytes,
                   "schedule": dict(sched, tuned_ms=round(tuned_ms, 4))},
        "roofline": {"bound": "hbm", "kernel": "batch_kernel", "achieved": round(achieved, 1), "peak": peak,
                     "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": None, "alg_bytes_per_launch": alg,
                     "alg_bytes": "every pass reads its input and writes its output once: counts, fold "
                                  "partials, theta and T, assembly intermediates, rho"},
        "batched": {"ms": round(ms_batch, 4), "launches_per_step": batch_launches,
                    "count_gbs": round(count_bytes / (ms_batch / 1e3) / 1e9, 1),
                    "frac_hbm_counts": round(count_bytes / (ms_batch / 1e3) / 1e9 / peak, 4)},
        "graph_replay": {"ms": round(ms_graph, 4), "theta_equal": same_graph},
        "one_launch_per_instance": {"ms": round(ms_single, 4), "launches_per_step": single_launches},
        "speedup_vs_per_instance": round(ms_single / ms_batch, 2),
        "theta_equal_batched_vs_single": same, "gpu_launches": batch_launches * steps,
    }
    lre.lre_destroy(ctx)
    del items
    if summary:
        for k in ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "dtype", "data"):
            out.pop(k, None)
    return out


def accuracy_point(lre, ctx, torch, n, shots, seed):
    """One point of the Sec. V / Fig. 3 study: the maximally mixed n-qubit
    state measured with `shots` shots per basis (counts drawn on the device by
    binary splitting of each basis' shots; int16 while the counts stay far
    below 32767, int32 above), through lre_estimate and lre_project.  For the
    true state I/d every error needs only theta and spectra: ||mu - I/d||_F^2 =
    sum_{P != I} t_P^2 / d, ||rho_hat - I/d||_F^2 = sum (l_i - 1/d)^2 and the
    fidelity with I/d = (sum sqrt(l_i))^2 / d."""
    from synth import gen
    d = 2 ** n
    dev = torch.device("cuda", 0)
    counts = torch.empty((3 ** n, d), dtype=torch.int16 if shots // d <= 16384 else torch.int32, device=dev)
    gen.gen_mixed(n, shots, seed, counts)
    theta = torch.empty(4 ** n, dtype=torch.float64, device=dev)
    rho = torch.empty((d, d), dtype=torch.complex64, device=dev)
    lre.lre_estimate(ctx, counts, shots, n, theta, rho)
    del counts
    rho_p = torch.empty_like(rho)
    eig = torch.empty(d, dtype=torch.float64, device=dev)
    lre.lre_project(ctx, rho, n, rho_p, eig_rho=eig)
    lre.lre_sync(ctx)
    hs_mu = float((theta[1:] ** 2).sum().item() / d)
    lam = eig.clamp(min=0.0)
    hs_rho = float(((eig - 1.0 / d) ** 2).sum().item())
    fid = float(lam.sqrt().sum().item() ** 2 / d)
    n0 = shots / d  # shots per basis = 2^n N_0 (N = 6^n N_0 copies in all)
    want = ((10.0 / 3.0) ** n - 3.0 ** (-n)) / (d * shots)
    return {"shots_per_basis": shots, "N0": n0, "hs_mu": hs_mu, "hs_mu_expected": want,
            "hs_mu_ratio": hs_mu / want, "paper_hs_law": (5.0 / 6.0) ** n / n0,
            "hs_rho_hat": hs_rho, "infidelity_rho_hat": 1.0 - fid,
            "paper_infidelity_law": (5.0 / 3.0) ** n / (4.0 * n0),
            "kept_eigenvalues": int((eig > 0).sum().item()), "theta_I": float(theta[0].item())}


def run_accuracy(args):
    """Sec. V / Fig. 3 analogue on the GPU: estimation error against shots
    for the maximally mixed state (the paper's own workload), one JSON line."""
    import torch
    from paper_1602_08604_gb300 import lre
    ctx = lre.lre_create(0)
    try:
        pts = [accuracy_point(lre, ctx, torch, args.study_n, int(round(n0 * 2 ** args.study_n)), 1000 + i)
               for i, n0 in enumerate(args.study_n0)]
    finally:
        lre.lre_destroy(ctx)
    return {"study": "estimation error vs shots, maximally mixed state (Sec. V, Fig. 3)", "n": args.study_n,
            "data": "synthetic", "expected": "E||mu - rho||_F^2 = ((10/3)^n - 3^-n)/(d S)", "points": pts}


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    vals = []
    for i in range(args.warmup + args.steps):
        bps, k, dt, thr = oracle_sample(wl, seconds_target=args.ref_step_seconds)
        if i >= args.warmup:
            vals.append((bps, k, dt))
    bps = sum(v[0] for v in vals) / len(vals)
    ms = sum(v[2] for v in vals) / len(vals) * 1000
    sample = (f"oracle direct zero-dropped sum over {vals[0][1]} bases of the n={wl['n']} workload "
              f"per step")
    return {"impl": "reference", "metric": "Pauli bases/sec and end-to-end LRE seconds at n=14; fraction of HBM roofline",
            "value": round(bps, 3), "unit": "Pauli bases/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": wl["desc"]},
            "cpu_baseline": {"value": round(bps, 3), "unit": "Pauli bases/s", "cores": thr,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(bps, 3), "unit": "Pauli bases/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="n14", choices=sorted(WORKLOADS) + ["batched", "accuracy"])
    ap.add_argument("--study-n", type=int, default=14, help="qubits of the accuracy study")
    ap.add_argument("--study-n0", type=float, nargs="+", default=[0.125, 1, 4, 16, 64],
                    help="N_0 (shots per basis / 2^n) of the accuracy study's points")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--check", action="store_true", help="spot-check parity against the oracle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-project", dest="project", action="store_false",
                    help="skip the one timed run of step (iii) (the projection)")
    ap.add_argument("--fold-path", default="tensor", choices=["fwht", "tensor", "tensor_split"],
                    help="first fold pass on the tensor cores (the library default: int16 counts), also for "
                         "int32 counts as two fp16 planes (tensor_split), or on the ALUs (FWHT)")
    ap.add_argument("--first7", action="store_true",
                    help="the raw tensor-core first pass folds seven qubits instead of six")
    ap.add_argument("--fused-first", action="store_true",
                    help="the first fold pass fused with the second through an L2 ring (n >= 10)")
    ap.add_argument("--fused-consumers", type=int, default=0,
                    help="fused tensor-core pass: CTAs on the second pass (0: the library's default)")
    ap.add_argument("--fused-discard", type=int, default=0, choices=(0, 1),
                    help="fused tensor-core pass: drop the ring lines the second pass has read from L2")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the comparison arms (the other first-pass path on the same counts; for the "
                         "n=14 workload also the n=12 int32 workload on both paths and the batched launch)")
    ap.add_argument("--compare-steps", type=int, default=5, help="timed steps of each comparison arm")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=8.0)
    args = ap.parse_args()
    if args.workload == "accuracy":
        out = run_accuracy(args) if args.impl == "ours" else None
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.workload == "batched":
        out = run_batched(args) if args.impl == "ours" else None
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    wl = WORKLOADS[args.workload]
    out = run_reference(args, wl) if args.impl == "reference" else run_ours(args, wl)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
