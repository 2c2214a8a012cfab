"""Benchmark: emulated FP64 GEMM (Ozaki-II, INT8 residue path) on GB300.

One step = one full emulated product C = A B at m = n = k = 8192 (Scale,
Reduce, the Q residue GEMMs with their epilogue, Reconstruct), inputs resident
in HBM. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--n 8192] [--q 16] [--bits 0] [--phi 0.5] [--engine auto|imma|tc]

--impl reference times the CPU oracle (the plain restatement of the method)
on the host cores, on a bounded sample of the same workload.

Under torchrun (N > 1) every rank runs its own independent product (weak
scaling, no collective on the data path); the step time is the max over ranks.
"""
from __future__ import annotations

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

METRIC = "emulated-FP64 GEMM TFLOP/s at m=n=k=8192 vs cuBLAS DGEMM, at err ≤2u|A||B|"
UNIT = "TFLOP/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100,
                    help="timed steps (the default keeps the timed region above a second, so that the "
                         "clock samples, taken every 200 ms, fall under load)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--q", type=int, default=16)
    ap.add_argument("--bits", type=int, default=0)
    ap.add_argument("--phi", type=float, default=0.5)
    ap.add_argument("--operands", default="phi", choices=["phi", "paper"],
                    help="phi: entries U(-0.5,0.5)*exp(phi*N(0,1)); paper: the paper's timing operands, row i "
                         "of each operand N(0,1)*2^e_i with e_i an integer drawn from [-20, 20)")
    ap.add_argument("--engine", default="auto", choices=["auto", "imma", "tc", "tc1"])
    ap.add_argument("--format", default="int8", choices=["int8", "E4M3", "E5M2", "E2M3", "E3M2", "E2M1"],
                    help="residue alphabet: the INT8 path, or a float-format configuration")
    ap.add_argument("--no-dgemm", action="store_true", help="skip the cuBLAS DGEMM comparison")
    ap.add_argument("--cpu-sample-s", type=float, default=15.0, help="target seconds of oracle work")
    ap.add_argument("--workload", default="dgemm",
                    choices=["dgemm", "batch", "blocked", "autograd", "fp-sweep", "precision", "peaks"],
                    help="dgemm: one m=n=k product (the headline); batch: 256 uneven products; blocked: the "
                         "inner dimension in slabs; autograd: forward + backward of the differentiable matmul; "
                         "fp-sweep: every float format next to the INT8 path; precision: throughput over n, phi, "
                         "Q and beta; peaks: library GEMM rates of this GPU (the roofline denominators)")
    ap.add_argument("--sweep-n", type=int, nargs="+", default=None, help="fp-sweep / precision: sizes")
    ap.add_argument("--sweep-phi", type=float, nargs="+", default=None, help="fp-sweep / precision: phi values")
    ap.add_argument("--sweep-q", type=int, nargs="+", default=None, help="precision: modulus counts")
    ap.add_argument("--formats", nargs="+", default=["E4M3", "E5M2", "E2M3", "E3M2", "E2M1"],
                    help="fp-sweep: float formats")
    ap.add_argument("--reps", type=int, default=5, help="sweeps: timed repetitions (median)")
    ap.add_argument("--cooldown", type=float, default=2.0,
                    help="sweeps: idle seconds before each row, so that every row starts below the power cap")
    ap.add_argument("--autograd-shapes", nargs="+", default=None,
                    help="autograd: m,k,n triples (default 4096,4096,4096 65536,256,256)")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-mode", default="auto", choices=["auto", "grouped", "streams"],
                    help="batch: autotuned over launch structure and modulus counts (auto), one launch per "
                         "phase over grouped products, or products on autotuned streams")
    ap.add_argument("--e2e-rows", type=int, default=0, help="e2e: rows of a block of C (0: about n/4)")
    ap.add_argument("--e2e-cols", type=int, default=0, help="e2e: columns of a block of C (0: about n/4)")
    ap.add_argument("--k", type=int, default=65536, help="blocked: the inner dimension")
    ap.add_argument("--k-slab", type=int, default=8192, help="blocked: terms per slab")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples, each stamped with the
    host time it arrived. One sampler runs for a whole measurement: started
    before the warm-up (so that nvidia-smi's start-up falls outside every
    timed region), it is summarised per timed region by the samples that
    fall inside it (summary(t0, t1)), which reflect the region itself rather
    than the idle moments around it."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []            # (host time, csv line)
        self.thread = None

    def start(self, settle_s: float = 3.0):
        """Start sampling and return once the first sample has arrived (at
        most settle_s)."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t_end = time.time() + settle_s
        while not self.lines and time.time() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def summary(self, t0=None, t1=None):
        """Median SM clock, maximum clock, throttle reasons and peak power of
        the samples that arrived in [t0, t1] (all samples when t0 is None);
        a region shorter than the sampling period takes the first sample
        after t0 (or the last one before it)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        lines = list(self.lines)
        if t0 is not None:
            inside = [ln for t, ln in lines if t0 <= t <= t1]
            if not inside:
                after = [ln for t, ln in lines if t >= t0]
                before = [ln for t, ln in lines if t < t0]
                inside = after[:1] or before[-1:]
            lines = inside
        else:
            lines = [ln for _, ln in lines]
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}

    def stop(self):
        """End sampling; the summary of every sample taken."""
        if self.proc is None:
            return self.summary()
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summary()


def operands(args, m, n, k, seed):
    """A (m x k) and B (k x n), float64, of the family --operands names."""
    import synth
    if args.operands == "paper":
        return synth.row_scaled_pair(n, seed=seed, m=m, k=k)
    return synth.phi_pair(m, n, k, args.phi, seed=seed)


def operands_name(args):
    if args.operands == "paper":
        return "rows N(0,1)*2^e_i, e_i integer in [-20,20)"
    return f"entries U(-0.5,0.5)*exp({args.phi}*N(0,1))"


def workload_name(n, args, q, bits, fmt="int8", channels=None):
    head = f"emulated dgemm m=n=k={n}, {operands_name(args)} seed 0 (rank r: seed r), "
    if fmt == "int8":
        return head + f"INT8 residue path Q={q} moduli<=239, beta={bits}"
    return head + f"{fmt} configuration, {q} low-precision GEMMs over {channels} channels, beta={bits}"


def make_plan(oz, args, n, engine=None):
    if args.format == "int8":
        return oz.Plan(args.q, args.bits, n, engine if engine is not None else oz.OZ_ENGINE_AUTO)
    return oz.PlanFP(args.format, n, args.bits)


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest of one float per rank (the step time every rank reports);
    x itself without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput_tflops(flops_per_step: float, steps: int, elapsed_ms: float, world: int) -> float:
    """Whole-job rate: every rank runs its own product of flops_per_step per
    step (weak scaling), timed by the slowest rank."""
    return world * flops_per_step * steps / (elapsed_ms * 1e-3) / 1e12


def gemm_traffic(plan, n, oz):
    """DRAM bytes per launch of the TC GEMM from its last ncu capture, scaled to
    this size by n^2; None for another engine, modulus count, or once the
    kernel source differs from the one the counters were taken on."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "gemm_tc_traffic.json")))
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
    except (OSError, ValueError, KeyError):
        return None
    if plan.engine != oz.OZ_ENGINE_TC or plan.q != rec["q"]:
        return None
    if hashlib.sha256(src).hexdigest()[:16] != rec["source_sha256_16"]:
        return None
    per = (rec["dram_bytes_read"] + rec["dram_bytes_write"]) * (n / rec["captured_n"]) ** 2
    return {"bytes": per, "captured_n": rec["captured_n"], "scaled_by": "n^2",
            "algorithmic_bytes": 2.0 * plan.q * 2 * n * n + plan.q * n * n}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def load_library_peaks():
    """FP8 and INT8 library GEMM rates measured on this GPU model by
    `bench.py --workload peaks` (profiles/library_gemm_peaks.json)."""
    try:
        return json.load(open(os.path.join(ROOT, "profiles", "library_gemm_peaks.json")))["tflops"]
    except (OSError, ValueError, KeyError):
        return {}


# ---------------------------------------------------------------------------
# CPU oracle leg (the only place bench.py runs the oracle)
# ---------------------------------------------------------------------------

def oracle_rate(A, B, n, mods, bits, seconds):
    """Time the oracle on a bounded sample of entries of the same product;
    returns (TFLOP/s of the emulated product, entries, seconds, threads)."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(123)
    count = 64
    done, elapsed = 0, 0.0
    while elapsed < seconds:
        r = rng.integers(0, n, size=count)
        c = rng.integers(0, n, size=count)
        t0 = time.perf_counter()
        oracle.dgemm_entries(A, B, mods, bits, r, c)
        dt = time.perf_counter() - t0
        done += count
        elapsed += dt
        if dt < seconds / 8:
            count *= 2
    flops = 2.0 * n * done          # each entry stands for 2k flops of the emulated product
    return flops / elapsed / 1e12, done, elapsed, oracle.threads()


def run_reference(args, rank, world):
    if rank != 0:
        return
    n = args.n
    A, B = operands(args, n, n, n, seed=0)
    import oracle
    if args.format == "int8":
        mods = oracle.max_product_moduli(args.q, 239)
        bits = args.bits or oracle.beta_max(mods, n)
        q, channels = args.q, args.q
    else:
        import paper_2609_37693_gb300 as oz      # the configuration tables only (host side)
        plan = oz.PlanFP(args.format, n, args.bits)
        mods, bits, q, channels = plan.moduli, plan.bits, plan.q, plan.channels
    per_step = max(0.2, min(args.cpu_sample_s, 20.0) / max(args.steps, 1))
    for _ in range(args.warmup):
        oracle_rate(A, B, n, mods, bits, per_step / 4)
    vals, ents, secs = [], 0, 0.0
    threads = oracle.threads()
    for _ in range(args.steps):
        v, e, s, threads = oracle_rate(A, B, n, mods, bits, per_step)
        vals.append(v)
        ents += e
        secs += s
    value = 2.0 * n * ents / secs / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": workload_name(n, args, q, bits, args.format, channels),
                   "m": n, "n": n, "k": n, "q": q, "bits": bits, "phi": args.phi, "operands": args.operands,
                   "format": args.format},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{ents} entries of C ({n}x{n}), each a full k={n} oracle evaluation "
                                   f"(scale, residues, {len(mods)} int64 dot products, CRT, rounding)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Our path
# ---------------------------------------------------------------------------

def bind_host_to_gpu(local):
    """Run this process on the CPUs attached to the GPU (its PCI device's
    local_cpulist), so that pinned host buffers allocated meanwhile live in
    the memory next to it: e2e runs whose buffers landed elsewhere copied
    about a third slower. Returns a note for the JSON line."""
    import torch
    try:
        p = torch.cuda.get_device_properties(local)
        dev = f"/sys/bus/pci/devices/{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        cpus = set()
        for part in open(os.path.join(dev, "local_cpulist")).read().strip().split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        cpus &= os.sched_getaffinity(0)
        node = open(os.path.join(dev, "numa_node")).read().strip()
        if not cpus:
            return "not bound (no local CPU in this process's set)"
        os.sched_setaffinity(0, cpus)
        return f"bound to the {len(cpus)} CPUs local to the GPU (NUMA node {node})"
    except (OSError, ValueError, AttributeError) as e:
        return f"not bound ({type(e).__name__})"


def host_copy_rates(A_pin, C_pin, stream):
    """One timed host-to-device copy of A_pin and one device-to-host copy into
    C_pin (CUDA events on the stream), in GB/s, and the NUMA nodes that hold
    A_pin's pages as /proc/self/numa_maps reports them: the host-operand
    product's speed follows these copies."""
    import torch
    dev_buf = torch.empty(A_pin.shape, dtype=A_pin.dtype, device=stream.device)
    rates = {}
    for name, dst, src in (("h2d", dev_buf, A_pin), ("d2h", C_pin, dev_buf[: C_pin.shape[0]])):
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):
                dst.copy_(src, non_blocking=True)
            e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        rates[name] = src.numel() * src.element_size() / best / 1e6
    del dev_buf
    rates["numa"] = "unknown"
    try:
        addr, start = A_pin.data_ptr(), None
        for line in open("/proc/self/maps"):
            lo, hi = (int(x, 16) for x in line.split()[0].split("-"))
            if lo <= addr < hi:
                start = lo
                break
        for line in open("/proc/self/numa_maps"):
            f = line.split()
            if start is not None and int(f[0], 16) == start:
                rates["numa"] = " ".join(x for x in f[1:] if x[:1] == "N" or x.split(":")[0] in
                                         ("bind", "default", "prefer", "interleave", "local")) or f[1]
                break
    except (OSError, ValueError, IndexError):
        pass
    return rates


def run_ours(args, rank, world, local):
    import torch
    import paper_2609_37693_gb300 as oz

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n = args.n
    engine = {"auto": oz.OZ_ENGINE_AUTO, "imma": oz.OZ_ENGINE_IMMA, "tc": oz.OZ_ENGINE_TC,
              "tc1": oz.OZ_ENGINE_TC1}[args.engine]
    plan = make_plan(oz, args, n, engine)
    is_fp = args.format != "int8"
    A_h, B_h = operands(args, n, n, n, seed=rank)
    A = torch.from_numpy(A_h).to(dev)
    B = torch.from_numpy(B_h).to(dev)
    C = torch.empty((n, n), dtype=torch.float64, device=dev)
    ws = oz.workspace(plan, n, n, n, dev)
    stream = torch.cuda.current_stream(dev)
    sh = oz._stream_handle(stream)

    def step():
        st = oz.oz_dgemm(plan.handle, 0, 0, n, n, n, A.data_ptr(), n, B.data_ptr(), n, C.data_ptr(), n,
                         ws.data_ptr(), ws.numel(), sh)
        if st != oz.OZ_OK:
            raise RuntimeError(f"oz_dgemm: {oz.oz_status_str(st)}")

    # one clock sampler for the whole run, started before the warm-up (see
    # ClockSampler); each timed region reads the samples inside it
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    st = oz.query_status(ws, stream)
    if st != oz.OZ_OK:
        raise RuntimeError(f"status after warm-up: {oz.oz_status_str(st)}")

    # The paper's gate for a timed call (Table tab:setup): relative Frobenius
    # difference from native DGEMM below 1e-12. Native DGEMM is also the
    # throughput comparison.
    dgemm_tflops = None
    rel_frob = None
    if not args.no_dgemm:
        Cn = A @ B
        torch.cuda.synchronize()
        rel_frob = (torch.linalg.norm(C - Cn) / torch.linalg.norm(Cn)).item()
        ts = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.matmul(A, B, out=Cn)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        dgemm_tflops = 2.0 * n**3 / (min(ts) * 1e-3) / 1e12
        del Cn
        if rel_frob > 1e-12:
            raise RuntimeError(f"result differs from native DGEMM by {rel_frob:.3e} (relative Frobenius)")

    # ---- timed region: K steps of oz_dgemm, inputs (1 GiB) larger than L2 ----
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_region = time.time()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.summary(t_region, time.time())
    if dist:
        dist.barrier()
    elapsed_ms = e0.elapsed_time(e1)
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)
    ms_per_step = elapsed_ms / args.steps
    flops = 2.0 * n**3
    value = throughput_tflops(flops, args.steps, elapsed_ms, world)

    # ---- e2e: host buffers through the public host-I/O call (oz_dgemm_host),
    # every step copying A and B in and C out inside the timed region; timed
    # after the device region (C_pin is compared with C, which holds the same
    # product) ----
    all_cpus = os.sched_getaffinity(0)
    host_binding = bind_host_to_gpu(local)            # the pinned buffers land next to the GPU
    A_pin = torch.from_numpy(A_h).pin_memory()
    B_pin = torch.from_numpy(B_h).pin_memory()
    C_pin = torch.empty((n, n), dtype=torch.float64).pin_memory()
    os.sched_setaffinity(0, all_cpus)
    copy_gbs = host_copy_rates(A_pin, C_pin, stream)
    hg = oz.HostGemm(plan, n, n, n, args.e2e_rows, dev, cols_per_chunk=args.e2e_cols)
    for _ in range(max(3, args.warmup)):
        hg(A_pin, B_pin, C_pin, stream)
    torch.cuda.synchronize()
    e2e_steps = max(2, min(args.steps, 10))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps + 1)]
    t_region = time.time()
    host_ms = []
    ev[0].record(stream)
    for i in range(e2e_steps):
        h0 = time.perf_counter()
        hg(A_pin, B_pin, C_pin, stream)
        ev[i + 1].record(stream)
        host_ms.append(round((time.perf_counter() - h0) * 1e3, 3))
    torch.cuda.synchronize()
    e2e_clk = clocks.summary(t_region, time.time())
    e2e_step_ms = [round(ev[i].elapsed_time(ev[i + 1]), 3) for i in range(e2e_steps)]
    e2e_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]) / e2e_steps, dist, dev)
    e2e_value = throughput_tflops(flops, 1, e2e_ms, world)
    e2e_exact = bool(np.array_equal(C_pin.numpy().view(np.uint64), C.cpu().numpy().view(np.uint64)))
    hg_rows, hg_cols = hg.block
    del hg

    # ---- per-phase times through the phase entry points (same kernels) ----
    _, lay = oz.oz_workspace_layout(plan.handle, n, n, n)
    m_pad, n_pad, k_pad = lay["m_pad"], lay["n_pad"], lay["k_pad"]
    base = ws.data_ptr()
    phase_ms = {"split_a": 0.0, "split_b": 0.0, "gemm": 0.0, "reconstruct": 0.0}
    reps = max(3, min(args.steps, 10))
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        oz.oz_split(plan.handle, 1, n, n, A.data_ptr(), n, m_pad, k_pad, base + lay["s"], base + lay["u"],
                    base + lay["flag"], None, sh)
        ev[1].record(stream)
        if is_fp or plan.engine != oz.OZ_ENGINE_IMMA:   # as oz_dgemm does: B's columns split in place
            oz.oz_split(plan.handle, 0, n, n, B.data_ptr(), n, n_pad, k_pad, base + lay["t"], base + lay["v"],
                        base + lay["flag"], base + lay["colmax"], sh)
        else:                                   # int8 planes: B^T, then its rows split
            oz.oz_transpose(n, n, B.data_ptr(), n, base + lay["bt"], sh)
            oz.oz_split(plan.handle, 1, n, n, base + lay["bt"], n, n_pad, k_pad, base + lay["t"], base + lay["v"],
                        base + lay["flag"], None, sh)
        ev[2].record(stream)
        oz.oz_residue_gemm(plan.handle, n, n, m_pad, n_pad, k_pad, base + lay["u"], base + lay["v"],
                           base + lay["y"], 0, base + lay["flag"], sh)
        ev[3].record(stream)
        oz.oz_reconstruct(plan.handle, n, n, base + lay["y"], base + lay["s"], base + lay["t"], C.data_ptr(), n,
                          sh)
        ev[4].record(stream)
        torch.cuda.synchronize()
        for i, key in enumerate(phase_ms):
            phase_ms[key] += ev[i].elapsed_time(ev[i + 1]) / reps
    phase_sum = sum(phase_ms.values())
    clocks.stop()

    # ---- roofline of the dominant kernel (the residue GEMMs) ----
    peaks = load_peaks()
    gemm_ops = 2.0 * plan.q * n**3                       # algorithmic low-precision ops per launch
    gemm_s = phase_ms["gemm"] * 1e-3
    achieved = gemm_ops / gemm_s / 1e12
    lib = load_library_peaks()
    if is_fp and args.format != "E2M1" and "fp8_e4m3" in lib:
        peak = lib["fp8_e4m3"]
        peak_src = "FP8 E4M3 dense, measured (torch._scaled_mm, profiles/library_gemm_peaks.json)"
    elif is_fp and "fp8_e4m3" in lib:
        peak = lib["fp8_e4m3"] * 3.0
        peak_src = ("FP4 dense = measured FP8 E4M3 (profiles/library_gemm_peaks.json) x 3, the nominal dense "
                    "ratio 13.5 / 4.5 PFLOP/s (no block-scaled FP4 library GEMM could be timed)")
    elif is_fp:
        ratio = 6.0 if args.format == "E2M1" else 2.0
        peak = peaks.get("bf16_tflops", 1900.0) * ratio
        peak_src = (f"{'FP4' if ratio == 6.0 else 'FP8'} dense = measured bf16 burst (MEASURED_PEAKS.json "
                    f"bf16_tflops) x {ratio:g}, the nominal dense ratio")
    elif plan.engine in (oz.OZ_ENGINE_TC, oz.OZ_ENGINE_TC1):
        peak = peaks.get("bf16_tflops", 1900.0)
        peak_src = "bf16 dense, measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    elif "int8" in lib:
        peak = lib["int8"]
        peak_src = "INT8 dense, measured (torch._int_mm, cuBLASLt; profiles/library_gemm_peaks.json)"
    else:
        peak = 167.0
        peak_src = "INT8 dense on B300 as stated in the paper (Sec. 'Speedup'); no measured INT8 peak exists"
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": "residue GEMM (+fused epilogue)",
                "peak_source": peak_src}
    if not is_fp and plan.engine in (oz.OZ_ENGINE_TC, oz.OZ_ENGINE_TC1) and "bf16_tflops_sustained" in peaks:
        # the timed region is long enough to meet the power cap: the sustained
        # (seconds-long, power-capped) cuBLAS figure is the other denominator
        roofline["frac_of_sustained_peak"] = achieved / peaks["bf16_tflops_sustained"]
    tr = gemm_traffic(plan, n, oz)
    if tr is not None:
        roofline["traffic"] = tr.pop("bytes")
        roofline["traffic_source"] = dict(tr, unit="bytes per launch")
    hbm = peaks.get("hbm_gbs", 6768.8)
    _, row_bytes = plan.plane_geometry(n)
    nplanes = plan.planes if is_fp else plan.q
    ybytes = (2 * plan.channels) if is_fp else plan.q       # residue bytes per output entry
    bytes_split = 8.0 * 2 * n * n + nplanes * 2.0 * n * row_bytes
    bytes_rec = ybytes * n * n + 8.0 * n * n
    gemm_peak_s = gemm_ops / (peak * 1e12)
    t_roof = gemm_peak_s + (bytes_split + bytes_rec + ybytes * n * n) / (hbm * 1e9)

    line = None
    if rank == 0:
        cpu = None
        if world == 1:
            v, ents, secs, thr = oracle_rate(A_h, B_h, n, plan.moduli, plan.bits, args.cpu_sample_s)
            cpu = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                   "sample": f"{ents} sampled entries of the same {n}^3 product, each a full oracle evaluation "
                             f"({secs:.1f} s on the host cores)"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": args.format.lower() if is_fp else ("int8" if plan.engine == oz.OZ_ENGINE_IMMA else "bf16"),
            "data": "synthetic",
            "config": {"workload": workload_name(n, args, plan.q, plan.bits, args.format,
                                                 getattr(plan, "channels", plan.q)),
                       "m": n, "n": n, "k": n, "q": plan.q, "bits": plan.bits, "phi": args.phi, "operands": args.operands,
                       "format": args.format,
                       "engine": {1: "imma", 2: "tc", 3: "fp", 4: "tc1"}[plan.engine], "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (A and B 512 MiB each); no flush",
                       "cublas_dgemm_tflops": dgemm_tflops, "speedup_vs_cublas_dgemm":
                           (value / world / dgemm_tflops) if dgemm_tflops else None,
                       "rel_frobenius_vs_dgemm": rel_frob,
                       "phase_ms": phase_ms, "phase_share": {k: v / phase_sum for k, v in phase_ms.items()},
                       "roofline_time_ms": t_roof * 1e3, "roofline_step_frac": t_roof * 1e3 / ms_per_step},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * n * n,
                    "d2h_bytes_per_step": 8 * n * n, "ms_per_step": e2e_ms, "step_ms": e2e_step_ms,
                    "host_enqueue_ms": host_ms,
                    "copy_gbs": copy_gbs, "clocks": e2e_clk,
                    "api": "oz_dgemm_host (pinned host A, B, C; blocks of C overlap copies and phases)",
                    "block": [hg_rows, hg_cols], "host": host_binding,
                    "equals_device_result": e2e_exact},
            "gpu_launches": (oz.launches_per_dgemm(False, False) if args.format == "int8" else 6) * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_batch(args, rank, world, local):
    """256 products with m, n, k log-uniform on [64, 4096] (phi = 1), captured
    into one CUDA graph, next to a loop of cuBLAS DGEMM calls on the same
    operands. --batch-mode grouped: oz_group_run, one launch per phase over
    the products of alike plans; streams: oz_dgemm_batched over an autotuned
    number of streams."""
    import torch
    import paper_2609_37693_gb300 as oz
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    shapes = [tuple(int(x) for x in s) for s in synth.batch_shapes(args.batch_count, 64, 4096, seed=0)]
    As, Bs, Cs = [], [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B = synth.phi_pair(m, n, k, 1.0, seed=i)
        As.append(torch.from_numpy(A).to(dev))
        Bs.append(torch.from_numpy(B).to(dev))
        Cs.append(torch.empty((m, n), dtype=torch.float64, device=dev))
    flops = sum(2.0 * m * n * k for (m, n, k) in shapes)
    if args.batch_mode == "auto":
        bg, label, tune = oz.autotune_batch(shapes, As, Bs, Cs)
        mode_desc = "autotuned: " + label
        launches = bg.launches() if isinstance(bg, oz.GroupedGemm) else \
            sum(oz.launches_per_dgemm(False, False) for _ in shapes)
    elif args.batch_mode == "grouped":
        bg = oz.GroupedGemm(As, Bs, Cs)
        bg.capture()
        tune, mode_desc, launches = None, "grouped products, one launch per phase", bg.launches()
    else:
        bg, tune = oz.autotune_batched(shapes, As, Bs, Cs, candidates=(1, 2, 4, 8, 16))
        mode_desc = f"oz_dgemm_batched on {bg.nstreams} streams"
        launches = sum(oz.launches_per_dgemm() for _ in shapes)
    for _ in range(max(args.warmup, 1)):
        bg.replay()
    torch.cuda.synchronize()
    s0 = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    e0.record(s0)
    for _ in range(args.steps):
        bg.replay()
    e1.record(s0)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # the same products through cuBLAS DGEMM, one call each
    ref = [torch.empty_like(c) for c in Cs]
    for A, B, R in zip(As, Bs, ref):
        torch.matmul(A, B, out=R)
    torch.cuda.synchronize()
    e0.record(s0)
    reps = 2
    for _ in range(reps):
        for A, B, R in zip(As, Bs, ref):
            torch.matmul(A, B, out=R)
    e1.record(s0)
    torch.cuda.synchronize()
    ms_dgemm = e0.elapsed_time(e1) / reps
    num = sum(float(torch.linalg.norm(C - R) ** 2) for C, R in zip(Cs, ref))
    den = sum(float(torch.linalg.norm(R) ** 2) for R in ref)
    if rank == 0:
        line = {
            "metric": "batched emulated-FP64 GEMM TFLOP/s, 256 products m,n,k log-uniform on [64,4096]",
            "value": flops / (ms * 1e-3) / 1e12, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"{len(shapes)} uneven products, m,n,k log-uniform [64,4096] seed 0, "
                                   f"phi=1, least Q at 53 bits per product, one CUDA graph",
                       "mode": mode_desc, "total_flops": flops, "autotune_ms": tune,
                       "q_histogram": {str(q): sum(1 for p in bg.plans if p.q == q) for q in sorted({p.q for p in bg.plans})},
                       "cublas_dgemm_loop_tflops": flops / (ms_dgemm * 1e-3) / 1e12,
                       "speedup_vs_cublas_dgemm_loop": ms_dgemm / ms,
                       "rel_frobenius_vs_dgemm": (num / den) ** 0.5},
            "gpu_launches": launches * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def run_blocked(args, rank, world, local):
    """One product m = n = --n with inner dimension --k through the blocked
    call in slabs of --k-slab terms (Sec. "Slabs"), next to the unblocked
    oz_dgemm of the same product (whose planes for the whole K must fit): the
    cost of running the epilogue once per slab and of the per-slab launches,
    and a check that both give the same bits."""
    import torch
    import paper_2609_37693_gb300 as oz
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, k, kt = args.n, args.k, args.k_slab
    A, B = operands(args, n, n, k, seed=rank)
    Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    del A, B
    engine = {"auto": oz.OZ_ENGINE_TC, "imma": oz.OZ_ENGINE_IMMA, "tc": oz.OZ_ENGINE_TC,
              "tc1": oz.OZ_ENGINE_TC1}[args.engine]
    # the window must admit the whole K; an IMMA plan is made for one slab (its
    # INT32 cap), at 53 bits unless given, and the call checks K against k_rec
    plan = oz.Plan(args.q, args.bits or (53 if engine == oz.OZ_ENGINE_IMMA else 0),
                   min(k, kt) if engine == oz.OZ_ENGINE_IMMA else k, engine)
    Cb = torch.empty((n, n), dtype=torch.float64, device=dev)
    wsb = torch.empty(oz.oz_blocked_workspace_bytes(plan.handle, n, n, kt), dtype=torch.uint8, device=dev)
    s0 = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s0)
        for _ in range(steps):
            fn()
        e1.record(s0)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms = timed(lambda: oz.dgemm_blocked(Ad, Bd, plan, kt, out=Cb, ws=wsb), args.steps)
    clk = clocks.stop()
    del wsb
    ms_u, same = None, None
    if k <= plan.k_max:
        Cu = torch.empty_like(Cb)
        wsu = oz.workspace(plan, n, n, k, dev)
        ms_u = timed(lambda: oz.dgemm(Ad, Bd, plan, out=Cu, ws=wsu), max(args.steps // 2, 1))
        same = bool(torch.equal(Cb.view(torch.int64), Cu.view(torch.int64)))
    flops = 2.0 * n * n * k
    nslabs = -(-k // kt)
    if rank == 0:
        line = {
            "metric": "emulated-FP64 GEMM TFLOP/s, blocked call", "value": flops / (ms * 1e-3) / 1e12,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": f"m=n={n}, k={k} in {nslabs} slabs of {kt}, {operands_name(args)}, Q={plan.q}, "
                                   f"beta={plan.bits}, engine {args.engine}",
                       "unblocked_ms": ms_u,
                       "unblocked_tflops": flops / (ms_u * 1e-3) / 1e12 if ms_u else None,
                       "blocked_over_unblocked": ms / ms_u if ms_u else None,
                       "equals_unblocked_bits": same,
                       "workspace_gb_blocked": oz.oz_blocked_workspace_bytes(plan.handle, n, n, kt) / 1e9,
                       "workspace_gb_unblocked": plan.workspace_bytes(n, n, k) / 1e9},
            # shifts of A's rows (1) and B's columns (2); per slab two splits and the
            # GEMM; one Reconstruct
            "gpu_launches": (4 + 3 * nslabs) * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def _median_ms(fn, reps):
    """Median of reps timed calls (CUDA events on the current stream) after one
    untimed call."""
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(statistics.median(ts))


def _best_ms(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def run_peaks(args, rank, world, local):
    """Library GEMM rates of this GPU at m = n = k = --n, best of 10 (CUDA
    events, one untimed call first): cuBLAS DGEMM, bf16 (torch.matmul), FP8
    E4M3 (torch._scaled_mm, unit scales, bf16 output), INT8 (torch._int_mm,
    cuBLASLt, int32 output) and block-scaled FP4 E2M1 (torch._scaled_mm with
    UE8M0 block scales of 1) where this PyTorch has it. These are the
    denominators of the INT8 and float-format rooflines."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    g = torch.Generator(device=dev).manual_seed(0)
    out = {}
    a64 = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
    b64 = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
    out["fp64_dgemm"] = 2.0 * n**3 / (_best_ms(lambda: a64 @ b64, 3) * 1e-3) / 1e12
    a = a64.to(torch.bfloat16)
    b = b64.to(torch.bfloat16)
    del a64, b64
    out["bf16"] = 2.0 * n**3 / (_best_ms(lambda: a @ b, 10) * 1e-3) / 1e12
    one = torch.ones((), dtype=torch.float32, device=dev)
    a8 = (a * 4).to(torch.float8_e4m3fn)
    b8 = (b * 4).to(torch.float8_e4m3fn).t().contiguous().t()        # column-major second operand
    out["fp8_e4m3"] = 2.0 * n**3 / (_best_ms(lambda: torch._scaled_mm(a8, b8, one, one, out_dtype=torch.bfloat16),
                                              10) * 1e-3) / 1e12
    ai = torch.randint(-100, 100, (n, n), dtype=torch.int8, device=dev, generator=g)
    bi = torch.randint(-100, 100, (n, n), dtype=torch.int8, device=dev, generator=g).t().contiguous().t()
    out["int8"] = 2.0 * n**3 / (_best_ms(lambda: torch._int_mm(ai, bi), 10) * 1e-3) / 1e12
    notes = {}
    try:
        a4 = torch.randint(0, 256, (n, n // 2), dtype=torch.uint8, device=dev, generator=g).view(torch.float4_e2m1fn_x2)
        b4 = torch.randint(0, 256, (n, n // 2), dtype=torch.uint8, device=dev, generator=g).view(torch.float4_e2m1fn_x2)
        sa = torch.full((n * (n // 32),), 127, dtype=torch.uint8, device=dev).view(torch.float8_e8m0fnu)
        sb = torch.full((n * (n // 32),), 127, dtype=torch.uint8, device=dev).view(torch.float8_e8m0fnu)
        fn = lambda: torch._scaled_mm(a4, b4.t(), sa, sb, out_dtype=torch.bfloat16)  # noqa: E731
        out["fp4_e2m1_mx"] = 2.0 * n**3 / (_best_ms(fn, 10) * 1e-3) / 1e12
    except Exception as e:                        # not every PyTorch build has a block-scaled FP4 GEMM
        notes["fp4_e2m1_mx"] = f"unavailable: {type(e).__name__}: {str(e)[:160]}"
    if rank == 0:
        print(json.dumps({"metric": f"library GEMM TFLOP/s at m=n=k={n}", "value": out.get("fp8_e4m3"),
                          "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
                          "config": {"workload": "library GEMM peaks", "n": n, "rates": out, "notes": notes,
                                     "torch": torch.__version__,
                                     "how": "best of 10 after one untimed call, CUDA events"}}), flush=True)


def run_autograd(args, rank, world, local):
    """Forward + backward of EmuMatmul (C = A B, dA = dC B^T, dB = A^T dC
    through the emulated product) against float64 autograd, at m = n = k =
    4096 and at m = 65536, k = n = 256. Operands and dC ~ N(0, 1) (torch
    generator seeded 0); best of 3 timed passes after one untimed pass;
    TFLOP/s counts the three products, 3 * 2mnk."""
    import torch
    import paper_2609_37693_gb300 as oz
    torch.cuda.set_device(local)
    rows = []
    shapes = [tuple(int(x) for x in t.split(",")) for t in args.autograd_shapes] if args.autograd_shapes else \
        [(4096, 4096, 4096), (65536, 256, 256)]
    for (m, k, n) in shapes:
        g = torch.Generator(device="cuda").manual_seed(0)
        A = torch.randn(m, k, dtype=torch.float64, device="cuda", generator=g).requires_grad_()
        B = torch.randn(k, n, dtype=torch.float64, device="cuda", generator=g).requires_grad_()
        dC = torch.randn(m, n, dtype=torch.float64, device="cuda", generator=g)

        def emu():
            A.grad = None
            B.grad = None
            oz.EmuMatmul.apply(A, B).backward(dC)

        def nat():
            A.grad = None
            B.grad = None
            (A @ B).backward(dC)

        te, tn = _best_ms(emu, 3), _best_ms(nat, 3)
        fl = 3 * 2.0 * m * n * k
        rows.append({"m": m, "k": k, "n": n, "emulated_ms": te, "emulated_tflops": fl / te / 1e9,
                     "fp64_autograd_ms": tn, "fp64_autograd_tflops": fl / tn / 1e9, "speedup": tn / te})
    if rank == 0:
        print(json.dumps({"metric": "emulated-FP64 matmul forward+backward TFLOP/s (3 products)",
                          "value": rows[0]["emulated_tflops"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
                          "data": "synthetic", "config": {"workload": "EmuMatmul fwd+bwd", "rows": rows}}),
              flush=True)


def run_fp_sweep(args, rank, world, local):
    """Every float-format configuration (E4M3, E5M2, E2M3, E3M2, E2M1) next to
    the INT8 path at m = n = k = n: GEMM count Q, channels, bit budget beta
    (the widest the window allows at K = n, and the paper's 53), median
    product time, emulated TFLOP/s, GEMM-phase time and its low-precision
    TFLOP/s, and cuBLAS DGEMM on the same operands. One JSON line per row.
    The error of each row is a property of beta alone (every configuration
    returns the oracle's bits at its beta; tests/test_gpu_fp.py checks this):
    oracle/precision.py tabulates it."""
    import torch
    import paper_2609_37693_gb300 as oz
    import synth
    torch.cuda.set_device(local)
    st = oz._stream_handle()
    for n in args.sweep_n or [8192]:
        for phi in args.sweep_phi or [0.5, 2.0]:
            A, B = synth.phi_pair(n, n, n, phi, seed=0)
            Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
            del A, B
            dg = 2.0 * n**3 / (_median_ms(lambda: Ad @ Bd, 2) * 1e-3) / 1e12
            for fmt in ["INT8"] + list(args.formats):
                for bits in (0, 53):
                    time.sleep(args.cooldown)
                    plan = oz.Plan(16, bits, n) if fmt == "INT8" else oz.PlanFP(fmt, n, bits)
                    ws = oz.workspace(plan, n, n, n)
                    C = torch.empty((n, n), dtype=torch.float64, device="cuda")
                    ms = _median_ms(lambda: oz.dgemm(Ad, Bd, plan, out=C, ws=ws), args.reps)
                    lay = oz.oz_workspace_layout(plan.handle, n, n, n)[1]
                    base = ws.data_ptr()
                    gms = _median_ms(lambda: oz.oz_residue_gemm(
                        plan.handle, n, n, lay["m_pad"], lay["n_pad"], lay["k_pad"], base + lay["u"],
                        base + lay["v"], base + lay["y"], 0, base + lay["flag"], st), args.reps)
                    row = {"workload": "fp-sweep", "n": n, "phi": phi, "format": fmt, "q": plan.q,
                           "channels": getattr(plan, "channels", plan.q), "bits": plan.bits, "ms": ms,
                           "tflops": 2.0 * n**3 / (ms * 1e-3) / 1e12, "gemm_ms": gms,
                           "gemm_lp_tflops": 2.0 * n**3 * plan.q / (gms * 1e-3) / 1e12, "dgemm_tflops": dg}
                    if rank == 0:
                        print(json.dumps(row), flush=True)
                    del C, ws
                    torch.cuda.empty_cache()
            del Ad, Bd
            torch.cuda.empty_cache()


def run_precision(args, rank, world, local):
    """The emulated product's throughput over sizes n, exponent spreads phi and
    modulus counts Q, each Q at the widest beta its window allows at K = n and,
    where the window holds, at the paper's 53: median product time and
    emulated TFLOP/s next to cuBLAS DGEMM, one JSON line per row. The error of
    each (n, phi, Q, beta) is the oracle's (the GPU returns its bits, checked
    by the parity tests): oracle/precision.py tabulates it."""
    import torch
    import paper_2609_37693_gb300 as oz
    import synth
    torch.cuda.set_device(local)
    for n in args.sweep_n or [1024, 4096, 8192]:
        for phi in args.sweep_phi or [0.5, 1.0, 2.0, 4.0]:
            A, B = synth.phi_pair(n, n, n, phi, seed=0)
            Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
            del A, B
            dg = 2.0 * n**3 / (_median_ms(lambda: Ad @ Bd, 2) * 1e-3) / 1e12
            for q in args.sweep_q or list(range(10, 21)):
                bmax = oz.Plan(q, 0, n).bits
                for bits in [bmax] + ([53] if 53 < bmax else []):
                    plan = oz.Plan(q, bits, n)
                    ws = oz.workspace(plan, n, n, n)
                    C = torch.empty((n, n), dtype=torch.float64, device="cuda")
                    ms = _median_ms(lambda: oz.dgemm(Ad, Bd, plan, out=C, ws=ws), args.reps)
                    row = {"workload": "precision", "n": n, "phi": phi, "q": q, "bits": plan.bits, "ms": ms,
                           "tflops": 2.0 * n**3 / (ms * 1e-3) / 1e12, "dgemm_tflops": dg}
                    if rank == 0:
                        print(json.dumps(row), flush=True)
                    del C, ws
            del Ad, Bd
            torch.cuda.empty_cache()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch":
        run_batch(args, rank, world, local)
        return
    if args.workload == "blocked":
        run_blocked(args, rank, world, local)
        return
    others = {"autograd": run_autograd, "fp-sweep": run_fp_sweep, "precision": run_precision, "peaks": run_peaks}
    if args.workload in others:
        others[args.workload](args, rank, world, local)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
