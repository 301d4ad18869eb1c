"""Benchmark: coupled Gibbs nonzero-updates/s on the pedigree workload.

Workload "pedigree50k": pedigree-shaped real non-symmetric C, n = 50,000, about
7 nnz per row, K = 1024 chains, FP32 sweeps; estimates = the full diagonal of
C^-1 and the 512-column block C^-1[:, 0:512] (BF16 tensor-core accumulation).
A step = one sampling batch: B cycles of the coupled sweep (Eqs. 4/5) with
the fused diagonal partials, one block contraction over the batch, and the FP64
folds.  value = nnz(C) * K * cycles / seconds.  The rows are swept in the colour
order by default (Sec. 4 reordering: the sampler of P C P^T, 7 dependency levels
instead of 80); the same step in the given row order is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

With N > 1 (torchrun) every rank runs its own K chains (disjoint chain ids):
chains are independent, so there is no exchange on the data path ("weak").
The reference arm is the FP64 CPU oracle on the host cores, timed on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled Gibbs nonzero-updates/s"
UNIT = "nonzero-updates/s"
WORKLOAD = "pedigree50k"


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.lines = []
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "mine" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# the sweep kernels (mcinv_info sweep_kernel): name, the sources that define it, and
# the committed ncu summary of its launch on pedigree50k
SWEEP_KERNELS = {
    0: ("cc_sweep_kernel", ("sweep.cu", "sweep_core.cuh", "internal.h"), "cc_sweep_pedigree50k.txt"),
    1: ("cc_sweep_staged_kernel", ("sweep_staged.cu", "sweep_core.cuh", "internal.h"), None),
    2: ("cc_sweep_grid_kernel", ("sweep_grid.cu", "sweep_ring.cuh", "sweep_core.cuh", "internal.h"), None),
    3: ("cc_sweep_grid_kernel (bulk-staged gathers)", ("sweep_grid.cu", "sweep_ring.cuh", "sweep_core.cuh", "internal.h"),
        "cc_sweep_grid_bulk_pedigree50k.txt"),
    4: ("cc_sweep_grid_kernel (bulk-staged gathers, pair layout)",
        ("sweep_grid.cu", "sweep_ring.cuh", "sweep_core.cuh", "internal.h"), "cc_sweep_grid_pair_pedigree50k.txt"),
    5: ("cc_sweep_tiled_kernel (tile-staged neighbours, pair layout)",
        ("sweep_tiled.cu", "sweep_tiled.h", "sweep_ring.cuh", "sweep_core.cuh", "internal.h"), None),
    6: ("cc_sweep_wave_kernel (chain-sliced wavefront, sliced layout)",
        ("sweep_wave.cu", "sweep_wave.h", "sweep_ring.cuh", "sweep_core.cuh", "internal.h"), None),
}

# bytes a cycle must move per (row, chain) of a complex64 sweep: z and w read and
# written once (32), or, for the wavefront sweep, the black half read once and every
# row written once (24: it keeps the red half in shared memory for the black rows)
def kernel_bytes_per_unit(sweep_kernel):
    return 24.0 if sweep_kernel == 6 else 32.0


def traffic_from_profiles(kernel_file, units_per_launch, sources=("sweep.cu", "sweep_core.cuh", "internal.h"),
                          threads=None):
    """DRAM bytes per launch of the sweep from the committed ncu summary, if the
    summary was taken on the current source of the kernel and its layout (matching
    hash of its source files) and, where it names one, the same CTA shape."""
    import hashlib
    if kernel_file is None:
        return None
    p = os.path.join(ROOT, "profiles", kernel_file)
    if not os.path.exists(p):
        return None
    src = b"".join(open(os.path.join(ROOT, "paper_cs_0412107_gb300", "csrc", f), "rb").read()
                   for f in sources
                   if os.path.exists(os.path.join(ROOT, "paper_cs_0412107_gb300", "csrc", f)))
    digest = hashlib.sha256(src).hexdigest()[:16]
    per_unit, ok, shape_ok = None, False, True
    for line in open(p):
        if line.startswith("source_sha256_16:"):
            ok = line.split(":", 1)[1].strip() == digest
        if line.startswith("threads_per_cta:") and threads is not None:
            shape_ok = int(line.split(":", 1)[1]) == threads
        if line.startswith("dram_bytes_per_unit:"):
            per_unit = float(line.split(":", 1)[1])
    if ok and shape_ok and per_unit is not None:
        return per_unit * units_per_launch
    return None


def kernel_flags(args):
    """The sweep kernel: timed on the matrix by the autotuner (auto), or fixed: the
    chain-sliced kernel in its default shape, the grid-wide kernel (register
    gathers, 512 threads), the grid-wide kernel with bulk-staged gathers on
    separate z, w buffers (bulk) or on the pair layout (pair), the tile-staged
    sweep (tile) or the wavefront sweep (wave)."""
    from paper_cs_0412107_gb300 import mcinv
    if args.kernel == "auto":
        return (0 if args.no_autotune else mcinv.MCINV_F_AUTOTUNE), {}
    if args.kernel == "sliced":
        return 0, {}
    if args.kernel == "grid":
        return mcinv.MCINV_F_GRID, {"threads_per_cta": 512}
    if args.kernel == "bulk":
        return mcinv.MCINV_F_GRID | mcinv.MCINV_F_GRID_BULK | mcinv.MCINV_F_GRID_NOPAIR, {}
    if args.kernel == "tile":
        return mcinv.MCINV_F_GRID | mcinv.MCINV_F_GRID_BULK | mcinv.MCINV_F_GRID_TILE, {}
    if args.kernel == "wave":
        return mcinv.MCINV_F_GRID | mcinv.MCINV_F_GRID_BULK | mcinv.MCINV_F_GRID_WAVE, {}
    # the pair layout in the shape --threads names (384 by default)
    return mcinv.MCINV_F_GRID | mcinv.MCINV_F_GRID_BULK | mcinv.MCINV_F_GRID_PAIR, {}


def shape_kw(args):
    """Explicit slice shape (--W, --threads) or the kernel's own."""
    kw = dict(kernel_flags(args)[1])
    if args.W:
        kw["chains_per_cta"] = args.W
    if args.threads:
        kw["threads_per_cta"] = args.threads
    return kw


def order_flag(args):
    """The sweep order: the rows as given (Eqs. 4/5 for i = 1..n), or the colour order
    (Sec. 4 reordering: the sampler of P C P^T, one dependency level per colour)."""
    from paper_cs_0412107_gb300 import mcinv
    return mcinv.MCINV_F_COLOR_ORDER if args.order == "colour" else 0


def run_mine(args, world, rank, local):
    import torch

    from paper_cs_0412107_gb300 import mcinv
    from paper_cs_0412107_gb300 import workloads as wl

    torch.cuda.set_device(local)
    w = wl.WORKLOADS[WORKLOAD]
    csr = w.build()
    K = args.chains
    acc = mcinv.MCINV_ACC_BF16_TC if args.acc == "tc" else mcinv.MCINV_ACC_FP32_SIMT
    S = np.arange(512)
    R = np.arange(csr.n)
    stream = torch.cuda.current_stream()
    h = mcinv.create_from_csr(csr, K=K, seed=args.seed, chain_base=rank * K, acc=acc,
                              batch_cycles=args.batch, block_rows=R, block_cols=S,
                              flags=kernel_flags(args)[0] | order_flag(args), **shape_kw(args))
    info0 = mcinv.mcinv_info(h)
    B = info0["batch_cycles"]
    mcinv.mcinv_burnin(h, args.burnin)
    for _ in range(args.warmup):
        mcinv.mcinv_sample(h, B)
    mcinv.mcinv_sync(h)
    launches0 = mcinv.mcinv_info(h)["kernel_launches"]
    mcinv.mcinv_profile(h, True)
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            mcinv.mcinv_sample(h, B)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    mcinv.mcinv_sync(h)
    ms = ev0.elapsed_time(ev1)
    prof = {mcinv.KERNEL_NAMES[k]: mcinv.mcinv_profile_read(h, k) for k in range(5)}
    mcinv.mcinv_profile(h, False)
    launches = mcinv.mcinv_info(h)["kernel_launches"] - launches0
    ms_max = max_over_ranks(ms, world)
    cycles = args.steps * B
    updates = float(csr.nnz) * K * cycles * world
    value = updates / (ms_max / 1e3)

    hbm, bf16, bf16_sus, peak_kind = read_peaks()
    sw_launches, sw_ms = prof["sweep"]
    cyc_per_launch = cycles / max(sw_launches, 1)
    units_per_launch = csr.n * K * cyc_per_launch  # (row, chain) coupled updates per sweep launch
    # algorithmic bytes of one sweep launch: each stored off-diagonal c_ij of C and of
    # C^dagger gathers one z_j / w_j and each row writes z_i and w_i (FP32), per chain
    # and cycle; the pedigree's random parents give no reuse, so every gather counts
    nnz_off = csr.nnz - csr.n
    alg_bytes = (4.0 * (2 * nnz_off + 2 * csr.n)) * K * cyc_per_launch
    achieved = alg_bytes / (sw_ms / sw_launches / 1e3) / 1e9 if sw_launches else None
    compulsory_bytes = 16.0 * units_per_launch  # read + write z and w once
    bl_launches, bl_ms = prof["block"]
    kname, ksrc, kprof = SWEEP_KERNELS[info0["sweep_kernel"]]
    gemm_flops = 2.0 * csr.n * 512 * K * B  # one contraction per batch
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded pedigree-shaped matrix, Philox noise)",
        "config": {"workload": WORKLOAD, "n": csr.n, "nnz": csr.nnz, "K": K, "batch_cycles": B,
                   "cycles_per_step": B, "estimates": "diagonal + C^-1[:, 0:512]",
                   "block_accumulation": "bf16 tensor cores" if acc else "fp32 simt",
                   "sweep_kernel": kname, "grid_ctas": info0["grid_ctas"],
                   "chains_per_cta": info0["chains_per_cta"], "threads_per_cta": info0["threads_per_cta"], "ctas_per_slice": info0["ctas_per_slice"],
                   "levels": info0["levels"], "sweep_order": args.order,
                   "l2": "inputs larger than L2 (z, w double-buffered: %.0f MB)" % (4 * 4 * csr.n * K / 1e6),
                   "parallelism": f"replicas x{world} (disjoint chains)"},
        "roofline": {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": (achieved / hbm) if achieved else None,
                     "traffic": traffic_from_profiles(kprof, units_per_launch, ksrc, info0["threads_per_cta"]),
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "bytes_per_unit": alg_bytes / units_per_launch,
                     "units_per_launch": units_per_launch,
                     "compulsory_bytes_per_launch": compulsory_bytes,
                     "compulsory_gbs": compulsory_bytes / (sw_ms / sw_launches / 1e3) / 1e9 if sw_launches else None},
        "kernels_ms": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()},
        "block_tflops": (gemm_flops * bl_launches / (bl_ms / 1e3) / 1e12) if bl_launches and acc else None,
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    mcinv.mcinv_destroy(h)
    if args.order == "colour" and not args.no_natural:
        # the same step with the rows swept in their given order (Eqs. 4/5 for i = 1..n),
        # for comparison: same kernels, 80 dependency levels instead of 7
        hn = mcinv.create_from_csr(csr, K=K, seed=args.seed, chain_base=rank * K, acc=acc,
                                   batch_cycles=args.batch, block_rows=R, block_cols=S,
                                   flags=kernel_flags(args)[0], **shape_kw(args))
        mcinv.mcinv_burnin(hn, args.burnin)
        for _ in range(args.warmup):
            mcinv.mcinv_sample(hn, B)
        mcinv.mcinv_profile(hn, True)
        nsteps = max(3, args.steps // 3)
        barrier(world)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(nsteps):
            mcinv.mcinv_sample(hn, B)
        ev1.record(stream)
        torch.cuda.synchronize()
        msn = max_over_ranks(ev0.elapsed_time(ev1), world)
        nl, nms = mcinv.mcinv_profile_read(hn, mcinv.MCINV_KERNEL_SWEEP)
        ni = mcinv.mcinv_info(hn)
        mcinv.mcinv_destroy(hn)
        ach_n = alg_bytes / (nms / nl / 1e3) / 1e9 if nl else None
        result["natural_order"] = {"value": float(csr.nnz) * K * nsteps * B * world / (msn / 1e3),
                                   "ms_per_step": msn / nsteps, "steps": nsteps, "levels": ni["levels"],
                                   "sweep_gbs": ach_n, "sweep_frac": ach_n / hbm if ach_n else None}
    if rank == 0 and world == 1 and args.order == "colour" and not args.no_natural and not args.no_extras:
        result["order_efficiency"] = guarded(order_efficiency, args, csr)
    if rank == 0 and not args.no_e2e:
        result["e2e"] = run_e2e(args, csr, K, acc, rank)
    if rank == 0 and world == 1 and not args.no_cpu:
        base, accuracy = cpu_baseline_and_accuracy(args, csr, kernel_flags(args)[0] | order_flag(args),
                                                   shape_kw(args))
        result["cpu_baseline"] = base
        result["accuracy"] = accuracy
    if rank == 0 and world == 1 and not args.no_extras:
        result["configs"] = run_configs(args, local)
    return result


def order_efficiency(args, csr):
    """Statistical efficiency of the two sweep orders on the pedigree workload.

    The colour order (Sec. 4's reordering: the sampler of P C P^T) sweeps faster than
    the given order, but the order changes the Gauss-Seidel contraction and so the
    autocorrelation of the chains; updates per second only mean faster answers if
    the error per sampling cycle stays about the same.  Both orders run the
    benchmark's handle (K chains, 500 burn-in cycles, BF16 block) and, after a
    doubling series of sampling cycles, the RMS errors of the diagonal on 24 sampled
    rows and of C^-1[:, 0:512] on 16 sampled columns are taken against FP64 BiCGSTAB
    solves (the clock stops while they are read).  Reported: the curves, seconds to
    each error, and the error variance per sampling cycle (RMS^2 x cycles, the Monte
    Carlo part), whose ratio is the statistical efficiency of one order against
    the other."""
    import scipy.sparse.linalg as spl
    import torch

    from paper_cs_0412107_gb300 import mcinv
    n = csr.n
    rows = np.linspace(0, n - 1, 24).astype(np.int64)
    cols = np.linspace(0, 511, 16).astype(np.int64)
    A = csr.to_scipy().tocsr()

    def column(j):
        e = np.zeros(n)
        e[j] = 1.0
        x, info = spl.bicgstab(A, e, rtol=1e-12, atol=0.0, maxiter=2000)
        assert info == 0, info
        return x

    dtruth = np.array([column(j)[j] for j in rows])
    btruth = np.stack([column(j) for j in cols], axis=1)
    K, B, burn = args.chains, 8, 500
    checks = [8, 16, 32, 64, 128, 256, 512, 1024, 2048]
    rms = lambda d: float(np.sqrt(np.mean(d ** 2)))
    out = {"K": K, "burnin": burn, "diag_rows": len(rows), "block_columns": len(cols),
           "truth": "FP64 BiCGSTAB columns of C^-1 (rtol 1e-12)"}
    for name, oflag in (("colour", mcinv.MCINV_F_COLOR_ORDER), ("given", 0)):
        h = mcinv.create_from_csr(csr, K=K, seed=args.seed + 202, acc=mcinv.MCINV_ACC_BF16_TC, batch_cycles=B,
                                  block_rows=np.arange(n), block_cols=np.arange(512),
                                  flags=kernel_flags(args)[0] | oflag, **shape_kw(args))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mcinv.mcinv_burnin(h, burn)
        mcinv.mcinv_sync(h)
        t_burn = time.perf_counter() - t0
        t, done, curve = t_burn, 0, []
        for c in checks:
            t0 = time.perf_counter()
            mcinv.mcinv_sample(h, c - done)
            mcinv.mcinv_sync(h)
            t += time.perf_counter() - t0
            done = c
            dm, _ = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_DIAG)
            bm, _ = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)
            curve.append({"sampling_cycles": c, "seconds": t, "rms_diag": rms(dm[rows] - dtruth),
                          "rms_block": rms(bm[:, cols] - btruth)})
        levels = mcinv.mcinv_info(h)["levels"]
        mcinv.mcinv_destroy(h)
        tail = curve[-4:]
        out[name] = {"levels": levels, "burnin_seconds": t_burn, "curve": curve,
                     "seconds_per_sampling_cycle": (curve[-1]["seconds"] - curve[0]["seconds"]) /
                                                   (checks[-1] - checks[0]),
                     "diag_error_var_per_cycle": float(np.mean([p["rms_diag"] ** 2 * p["sampling_cycles"]
                                                                for p in tail])),
                     "block_error_var_per_cycle": float(np.mean([p["rms_block"] ** 2 * p["sampling_cycles"]
                                                                 for p in tail]))}
        for eps in (3e-3, 1e-3):
            for est in ("diag", "block"):
                hit = next((p["seconds"] for p in curve if p[f"rms_{est}"] <= eps), None)
                out[name][f"seconds_to_{est}_rms_{eps:g}"] = hit
    c, g = out["colour"], out["given"]
    for est in ("diag", "block"):
        eff = g[f"{est}_error_var_per_cycle"] / c[f"{est}_error_var_per_cycle"]
        out[f"{est}_statistical_efficiency_colour_over_given"] = eff
        out[f"{est}_effective_speedup_colour_over_given"] = eff * g["seconds_per_sampling_cycle"] / \
            c["seconds_per_sampling_cycle"]
    return out


def run_e2e(args, csr, K, acc, rank):
    """The same metric through the public C ABI from host buffers: one job =
    mcinv_create from a pinned host CSR (H2D), burn-in, sampling, the diagonal
    and block estimates read back to pinned host memory (D2H), destroy."""
    import torch

    from paper_cs_0412107_gb300 import mcinv
    rp = torch.from_numpy(csr.row_ptr).pin_memory()
    col = torch.from_numpy(csr.col).pin_memory()
    val = torch.from_numpy(np.ascontiguousarray(csr.val)).pin_memory()
    S = np.arange(512)
    R = np.arange(csr.n)
    burn, samp = args.e2e_burnin, args.e2e_samples
    h2d = rp.numel() * 8 + col.numel() * 4 + val.numel() * 8
    d2h = csr.n * 8 * 2 + csr.n * 512 * 8 * 2
    out_d = torch.empty(csr.n, dtype=torch.float64).pin_memory()
    se_d = torch.empty(csr.n, dtype=torch.float64).pin_memory()
    out_b = torch.empty(csr.n * 512, dtype=torch.float64).pin_memory()
    se_b = torch.empty(csr.n * 512, dtype=torch.float64).pin_memory()
    L = mcinv.lib()
    import ctypes

    def job():
        opt = mcinv.mcinv_default_options(K=K, seed=args.seed + 1, chain_base=rank * K, acc=acc,
                                          batch_cycles=args.batch,
                                          flags=kernel_flags(args)[0] | order_flag(args), **shape_kw(args))
        opt.stream = mcinv.current_stream()
        Ra = np.ascontiguousarray(R, dtype=np.int64)
        Sa = np.ascontiguousarray(S, dtype=np.int64)
        opt.block_rows = Ra.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        opt.block_cols = Sa.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        opt.n_block_rows, opt.n_block_cols = len(Ra), len(Sa)
        hp = ctypes.c_void_p()
        mcinv._check(L.mcinv_create(ctypes.byref(hp), csr.n, ctypes.c_void_p(rp.data_ptr()),
                                    ctypes.c_void_p(col.data_ptr()), ctypes.c_void_p(val.data_ptr()),
                                    mcinv.MCINV_REAL64, ctypes.byref(opt)))
        mcinv._check(L.mcinv_burnin(hp, burn), hp)
        mcinv._check(L.mcinv_sample(hp, samp), hp)
        mcinv._check(L.mcinv_estimate(hp, mcinv.MCINV_EST_DIAG, None, ctypes.c_void_p(out_d.data_ptr()),
                                      ctypes.c_void_p(se_d.data_ptr())), hp)
        mcinv._check(L.mcinv_estimate(hp, mcinv.MCINV_EST_BLOCK, None, ctypes.c_void_p(out_b.data_ptr()),
                                      ctypes.c_void_p(se_b.data_ptr())), hp)
        L.mcinv_destroy(hp)

    job()  # warm-up (allocator, module load)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_jobs):
        job()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.e2e_jobs
    return {"value": float(csr.nnz) * K * (burn + samp) / dt, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "step": f"one job: create + {burn} burn-in + {samp} sampling cycles + diag and block readback",
            "seconds_per_job": dt}


def batch_workload(count, seed=0):
    """The batched workload: `count` random-dominant matrices (4 off-diagonals per
    row, diagonal 1.5 x row sum) with n log-uniform in [64, 4096], seeds 0.."""
    from paper_cs_0412107_gb300 import workloads as wl
    sizes = wl.batch_sizes(count, 64, 4096, seed=seed)
    return [wl.random_dominant(int(n), 4, 1.5, k) for k, n in enumerate(sizes)]


def run_batch(args, world, rank, local):
    """512 matrices in one pool (one persistent launch per kernel per step,
    graph-replayed), full inverse each: throughput of the whole batch, then the
    same matrices as a Poisson request stream through the server at 50% and 90%
    of that throughput, with p50/p99 latency."""
    import torch

    from paper_cs_0412107_gb300 import mcinv
    torch.cuda.set_device(local)
    mats = batch_workload(args.batch_count)
    burn, samp, K, B = args.batch_burnin, args.batch_samples, 256, 8
    budget = int(args.batch_mem_gb * (1 << 30))
    nnz_total = sum(c.nnz for c in mats)
    pool = mcinv.mcinv_pool_create(K=K, seed=args.seed, chain_base=rank * K, mem_budget=budget,
                                   max_slots=len(mats), batch_cycles=B, flags=order_flag(args))
    # warm-up pool: tuning steps and graph capture on a few members
    for k in range(min(8, len(mats))):
        mcinv.mcinv_pool_submit(pool, mats[k], matrix_id=10_000 + k, burnin=2 * B, samples=6 * B)
    for _ in range(8):
        mcinv.mcinv_pool_step(pool)
    mcinv.mcinv_pool_destroy(pool)
    pool = mcinv.mcinv_pool_create(K=K, seed=args.seed, chain_base=rank * K, mem_budget=budget,
                                   max_slots=len(mats), batch_cycles=B, flags=order_flag(args))
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t0 = time.perf_counter()
        tickets = [mcinv.mcinv_pool_submit(pool, c, matrix_id=k, burnin=burn, samples=samp)
                   for k, c in enumerate(mats)]
        t_admit = time.perf_counter() - t0
        steps = 0
        while not all(mcinv.mcinv_pool_poll(pool, t) for t in tickets):
            mcinv.mcinv_pool_step(pool)
            steps += 1
        mcinv.mcinv_pool_sync(pool)
        dt = time.perf_counter() - t0
    info = mcinv.mcinv_pool_info(pool)
    # accuracy on a few members against the dense inverse
    errs = []
    for k in range(0, len(mats), max(1, len(mats) // 8)):
        m, se = mcinv.mcinv_pool_estimate(pool, tickets[k], mcinv.MCINV_EST_BLOCK, mats[k].n)
        truth = np.linalg.inv(mats[k].to_dense())
        errs.append(float(np.sqrt(np.mean((m - truth) ** 2))))
    mcinv.mcinv_pool_destroy(pool)
    updates = float(nnz_total) * K * (burn + samp)
    value = updates / dt
    flops = sum(2.0 * c.n * c.n for c in mats) * K * samp
    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "impl": "mine",
           "dtype": "f32 sweep, bf16 tensor-core accumulation",
           "config": {"workload": "batch512", "matrices": len(mats), "K": K, "burnin": burn, "samples": samp,
                      "sum_n": int(sum(c.n for c in mats)), "sum_nnz": int(nnz_total),
                      "estimate": "full inverse of every matrix", "batch_cycles": B,
                      "chains_per_cta": info["chains_per_cta"], "threads_per_cta": info["threads_per_cta"],
                      "sweep_order": args.order},
           "seconds": dt, "admission_seconds": t_admit, "steps": steps,
           "block_tflops_effective": flops / dt / 1e12,
           "rms_error_vs_dense_inverse": {"median": float(np.median(errs)), "max": float(np.max(errs))},
           "kernel_launches": info["kernel_launches"], "clocks": clocks.summary()}
    # time to 1e-2 RMS error of every inverse: the same schedule through the batched
    # BF16 pool and through the plain path (one FP32 handle per matrix, SIMT
    # accumulation, launches issued one by one), RMS checked on every 64th matrix
    if args.rms_samples > 0:
        res["time_to_rms"] = time_to_rms(args, mats, burn, K, B, budget, rank)
    if args.serve_requests <= 0:
        return res
    # serving: Poisson arrivals at 50% and 90% of the batch throughput (matrices/s)
    rate_max = len(mats) / dt
    serving = {}
    for frac in (0.5, 0.9):
        srv = mcinv.mcinv_server_create(K=K, seed=args.seed, mem_budget=budget, max_slots=len(mats), batch_cycles=B, flags=order_flag(args))
        rng = np.random.default_rng(1)
        n_req = min(len(mats), args.serve_requests)
        gaps = rng.exponential(1.0 / (frac * rate_max), size=n_req)
        ids = []
        t0 = time.perf_counter()
        for k in range(n_req):
            ids.append(mcinv.mcinv_server_submit(srv, mats[k], k, burn, samp, mcinv.MCINV_EST_DIAG))
            time.sleep(gaps[k])
        lat = [mcinv.mcinv_server_wait(srv, ids[k], mats[k].n, mcinv.MCINV_EST_DIAG, 3600)[2] for k in range(n_req)]
        el = time.perf_counter() - t0
        st = mcinv.mcinv_server_stats(srv)
        mcinv.mcinv_server_destroy(srv)
        serving[f"{int(frac * 100)}pct"] = {"offered_matrices_per_s": frac * rate_max, "requests": n_req,
                                           "p50_ms": float(np.percentile(lat, 50)),
                                           "p99_ms": float(np.percentile(lat, 99)),
                                           "completed_per_s": n_req / el, "engine_steps": st["steps"]}
    res["serving"] = serving
    return res


def time_to_rms(args, mats, burn, K, B, budget, rank, target=1e-2, max_samples=2000):
    """Time to an RMS inverse error <= target on every monitored matrix (every 64th,
    against its dense inverse), checked after every B sampling cycles, for the batched
    BF16 form and for the plain path (one handle per matrix, FP32 CUDA-core
    accumulation, launches issued one matrix at a time).  Both forms draw the same
    noise (seed, matrix id), so they need about the same number of cycles; the clock
    stops while the error is checked.  Setup (pool creation and admission, or handle
    creation and destruction) and the read-back of every matrix's inverse and SE to
    the host are reported apart from accumulation (burn-in and sampling until the
    estimates on the device reach the target)."""
    import torch

    from paper_cs_0412107_gb300 import mcinv
    check = list(range(0, len(mats), 64))
    truth = {k: np.linalg.inv(mats[k].to_dense()) for k in check}
    rms = lambda k, m: float(np.sqrt(np.mean((m - truth[k]) ** 2)))
    out = {"target_rms": target, "burnin": burn, "checked_every_cycles": B, "monitored_matrices": len(check)}
    # batched form: every matrix admitted at once, steps until the monitored ones reach the target
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    # one step's product a batch: the estimates can be checked after every step
    pool = mcinv.mcinv_pool_create(K=K, seed=args.seed, chain_base=rank * K, mem_budget=budget,
                                   max_slots=len(mats), batch_cycles=B, fold_steps=1, flags=order_flag(args))
    tickets = [mcinv.mcinv_pool_submit(pool, c, matrix_id=k, burnin=burn, samples=max_samples)
               for k, c in enumerate(mats)]
    mcinv.mcinv_pool_sync(pool)
    t_setup = time.perf_counter() - t0
    t_acc, cycles, worst = 0.0, 0, None
    while cycles < burn + max_samples:
        t0 = time.perf_counter()
        mcinv.mcinv_pool_step(pool)
        mcinv.mcinv_pool_sync(pool)
        t_acc += time.perf_counter() - t0
        cycles += B
        if cycles <= burn:
            continue
        worst = max(rms(k, mcinv.mcinv_pool_estimate(pool, tickets[k], mcinv.MCINV_EST_BLOCK, mats[k].n)[0])
                    for k in check)  # the check: not timed
        if worst <= target:
            break
    t0 = time.perf_counter()
    for k, c in enumerate(mats):  # the answer: every matrix's inverse and its SE, read back
        mcinv.mcinv_pool_estimate(pool, tickets[k], mcinv.MCINV_EST_BLOCK, c.n)
    t_read = time.perf_counter() - t0
    mcinv.mcinv_pool_destroy(pool)
    out["batched_bf16"] = {"seconds": t_setup + t_acc, "setup_seconds": t_setup, "accumulation_seconds": t_acc,
                           "readback_seconds": t_read, "sampling_cycles": cycles - burn, "rms_max": worst}
    # plain path: the monitored matrices first, each until it reaches the target, which
    # fixes the sampling cycles every other matrix then runs
    torch.cuda.synchronize()
    t_setup = t_acc = t_read = 0.0
    need, rms_plain = 0, []

    def plain(k, c, samples=None):
        nonlocal t_setup, t_acc, t_read, need
        t0 = time.perf_counter()
        h = mcinv.create_from_csr(c, K=K, seed=args.seed, chain_base=rank * K, matrix_id=k,
                                  acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=B, flags=order_flag(args),
                                  block_rows=np.arange(c.n), block_cols=np.arange(c.n))
        mcinv.mcinv_sync(h)
        t1 = time.perf_counter()
        t_setup += t1 - t0
        mcinv.mcinv_burnin(h, burn)
        if samples is not None:
            mcinv.mcinv_sample(h, samples)
        mcinv.mcinv_sync(h)
        t_acc += time.perf_counter() - t1
        if samples is None:
            done = 0
            while True:
                t2 = time.perf_counter()
                mcinv.mcinv_sample(h, B)
                mcinv.mcinv_sync(h)
                t_acc += time.perf_counter() - t2
                done += B
                m, _ = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)  # the check: not timed
                if rms(k, m) <= target or done >= max_samples:
                    rms_plain.append(rms(k, m))
                    need = max(need, done)
                    break
        t2 = time.perf_counter()
        mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)  # the answer, read back
        t3 = time.perf_counter()
        mcinv.mcinv_destroy(h)
        t_read += t3 - t2
        t_setup += time.perf_counter() - t3

    for k in check:
        plain(k, mats[k])
    for k, c in enumerate(mats):
        if k not in truth:
            plain(k, c, samples=need)
    out["plain_fp32"] = {"seconds": t_setup + t_acc, "setup_seconds": t_setup, "accumulation_seconds": t_acc,
                         "readback_seconds": t_read, "sampling_cycles": need, "rms_max": max(rms_plain)}
    out["note"] = ("seconds = setup + accumulation: the estimates are on the device at the target error; "
                   "readback_seconds is the copy of every matrix's inverse and SE to the host (about 16 GB)")
    out["speedup"] = out["plain_fp32"]["seconds"] / out["batched_bf16"]["seconds"]
    out["speedup_accumulation"] = out["plain_fp32"]["accumulation_seconds"] / out["batched_bf16"]["accumulation_seconds"]
    return out


def lattice_truth(csr, cols):
    """Columns of C^-1 by FP64 BiCGSTAB on the host (C is strictly diagonally dominant, so
    the solves converge quickly): the truth for the RMS error of the block estimate."""
    import scipy.sparse.linalg as spl
    A = csr.to_scipy()
    out = np.empty((csr.n, len(cols)), dtype=np.complex128)
    for k, j in enumerate(cols):
        e = np.zeros(csr.n, dtype=np.complex128)
        e[j] = 1.0
        x, info = spl.bicgstab(A, e, rtol=1e-12, atol=0.0, maxiter=2000)
        assert info == 0, info
        out[:, k] = x
    return out


def run_lattice(args, world, rank, local):
    """The 4D lattice (16^4, K = 8192, complex64): the 4096 x 4096 block C^-1[0:4096, 0:4096]
    accumulated with BF16 operands on the tensor cores against FP32 CUDA-core accumulation,
    after 50 burn-in cycles; RMS error against FP64 solves on 64 of its columns after every
    batch of 8 sampling cycles, and the time each form takes to reach 1e-2 and 3e-3."""
    import torch

    from paper_cs_0412107_gb300 import mcinv
    from paper_cs_0412107_gb300 import workloads as wl
    torch.cuda.set_device(local)
    csr = wl.WORKLOADS["lattice4d16"].build()
    K, B, burn, nb = 8192, 8, 50, args.lattice_batches
    R = np.arange(4096)
    check = np.arange(0, 4096, 64)
    truth = lattice_truth(csr, check)[:4096]
    res = {"metric": "time to RMS inverse error", "unit": "s", "higher_is_better": False, "n_gpus": world,
           "impl": "mine", "config": {"workload": "lattice4d16", "n": csr.n, "nnz": csr.nnz, "K": K,
                                      "block": "C^-1[0:4096, 0:4096]", "burnin": burn, "batch_cycles": B,
                                      "sweep_order": args.order,
                                      "rms_over": "4096 x 64 columns of the block (FP64 BiCGSTAB truth)"},
           "forms": {}}
    for name, acc in (("bf16_tensor_cores", mcinv.MCINV_ACC_BF16_TC), ("fp32_cuda_cores", mcinv.MCINV_ACC_FP32_SIMT)):
        h = mcinv.create_from_csr(csr, K=K, seed=args.seed, acc=acc, batch_cycles=B, block_rows=R, block_cols=R,
                                  flags=mcinv.MCINV_F_AUTOTUNE | order_flag(args))
        torch.cuda.synchronize()
        with ClockSampler(local) as clocks:
            t0 = time.perf_counter()
            mcinv.mcinv_burnin(h, burn)
            curve = []
            for k in range(nb):
                mcinv.mcinv_sample(h, B)
                m, _ = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)  # synchronises
                rms = float(np.sqrt(np.mean(np.abs(m[:, check] - truth) ** 2)))
                curve.append({"cycles": burn + (k + 1) * B, "seconds": time.perf_counter() - t0, "rms": rms})
        mcinv.mcinv_destroy(h)
        first = lambda tgt: next((c["seconds"] for c in curve if c["rms"] <= tgt), None)
        res["forms"][name] = {"curve": curve, "seconds_to_1e-2": first(1e-2), "seconds_to_3e-3": first(3e-3),
                              "clocks": clocks.summary()}
    a, b = res["forms"]["bf16_tensor_cores"], res["forms"]["fp32_cuda_cores"]
    res["value"] = a["seconds_to_3e-3"]
    for t in ("1e-2", "3e-3"):
        ta, tb = a[f"seconds_to_{t}"], b[f"seconds_to_{t}"]
        res[f"speedup_to_{t}"] = tb / ta if ta and tb else None
    return res

def run_lattice2d(args, world, rank, local):
    """The complex 2D lattice (L = 128, K = 4096 chains, diagonal and tr(QC^-1) with q ~ U(0,1)),
    or with --workload lattice4d16-rate the 4D one (16^4, K = 8192, the same estimates):
    coupled updates per second of the sampling step, with the sweep's bytes against the
    copy bandwidth both as gathered (every stored c_ij of C and of C^dagger reads one
    complex64 z_j / w_j) and as compulsory (z and w read and written once a cycle)."""
    import torch

    from paper_cs_0412107_gb300 import mcinv
    from paper_cs_0412107_gb300 import workloads as wl

    torch.cuda.set_device(local)
    name = "lattice4d16" if args.workload == "lattice4d16-rate" else "lattice2d128"
    w = wl.WORKLOADS[name]
    csr = w.build()
    K = args.lattice_chains or w.K  # fewer chains: a smaller case of the same kernel (for ncu)
    h = mcinv.create_from_csr(csr, K=K, seed=args.seed, chain_base=rank * K, acc=mcinv.MCINV_ACC_FP32_SIMT,
                              batch_cycles=args.batch, flags=kernel_flags(args)[0] | order_flag(args),
                              **shape_kw(args))
    mcinv.mcinv_set_trace_weights(h, wl.q_diag(csr.n, args.seed))
    info0 = mcinv.mcinv_info(h)
    B = info0["batch_cycles"]
    mcinv.mcinv_burnin(h, args.burnin)
    for _ in range(args.warmup):
        mcinv.mcinv_sample(h, B)
    mcinv.mcinv_sync(h)
    launches0 = mcinv.mcinv_info(h)["kernel_launches"]
    mcinv.mcinv_profile(h, True)
    stream = torch.cuda.current_stream()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            mcinv.mcinv_sample(h, B)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    mcinv.mcinv_sync(h)
    ms_max = max_over_ranks(ev0.elapsed_time(ev1), world)
    prof = {mcinv.KERNEL_NAMES[k]: mcinv.mcinv_profile_read(h, k) for k in range(5)}
    launches = mcinv.mcinv_info(h)["kernel_launches"] - launches0
    tr, tse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_TRACE, q_diag=wl.q_diag(csr.n, args.seed))
    mcinv.mcinv_destroy(h)
    cycles = args.steps * B
    hbm, _, _, peak_kind = read_peaks()
    sw_launches, sw_ms = prof["sweep"]
    cyc_per_launch = cycles / max(sw_launches, 1)
    units_per_launch = csr.n * K * cyc_per_launch
    nnz_off = csr.nnz - csr.n
    alg_bytes = 8.0 * (2 * nnz_off + 2 * csr.n) * K * cyc_per_launch
    compulsory_bytes = 32.0 * units_per_launch
    t_launch = sw_ms / sw_launches / 1e3 if sw_launches else None
    achieved = alg_bytes / t_launch / 1e9 if t_launch else None
    kname, ksrc, kprof = SWEEP_KERNELS[info0["sweep_kernel"]]
    kprof = {4: f"cc_sweep_grid_pair_{name}.txt", 5: f"cc_sweep_tiled_{name}.txt",
             6: f"cc_sweep_wave_{name}.txt"}.get(info0["sweep_kernel"])
    own_bytes = kernel_bytes_per_unit(info0["sweep_kernel"]) * units_per_launch
    return {
        "metric": METRIC, "value": float(csr.nnz) * K * cycles * world / (ms_max / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
        "data": "synthetic (seeded U(1) lattice, Philox noise)",
        "config": {"workload": name, "n": csr.n, "nnz": csr.nnz, "K": K, "batch_cycles": B,
                   "estimates": "diagonal + tr(QC^-1), q ~ U(0,1)", "sweep_kernel": kname,
                   "threads_per_cta": info0["threads_per_cta"], "levels": info0["levels"],
                   "sweep_order": args.order,
                   "l2": "inputs larger than L2 (z, w double-buffered: %.0f MB)" % (4 * 8 * csr.n * K / 1e6)},
        "roofline": {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm if achieved else None, "peak_source": f"{peak_kind} hbm_gbs",
                     "traffic": traffic_from_profiles(kprof, units_per_launch, ksrc, info0["threads_per_cta"]),
                     "algorithmic_bytes_per_launch": alg_bytes, "bytes_per_unit": alg_bytes / units_per_launch,
                     "units_per_launch": units_per_launch, "compulsory_bytes_per_launch": compulsory_bytes,
                     "compulsory_frac": compulsory_bytes / t_launch / 1e9 / hbm if t_launch else None,
                     "kernel_bytes_per_launch": own_bytes,
                     "kernel_frac": own_bytes / t_launch / 1e9 / hbm if t_launch else None},
        "trace": {"re": float(np.real(tr)), "im": float(np.imag(tr)), "se_re": float(np.real(tse)),
                  "se_im": float(np.imag(tse)), "cycles": args.burnin + (args.warmup + args.steps) * B},
        "kernels_ms": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }


def cpu_baseline(csr, K, seconds, workload=WORKLOAD):
    """The FP64 oracle on the host cores, on a bounded sample of the workload:
    `chains` chains (one OpenMP thread per chain group) for `cycles` cycles."""
    import oracle
    threads = os.cpu_count() or 1
    chains = threads
    t0 = time.perf_counter()
    oracle.run(csr, chains, seed=0, ncycles=1, cpg=1, diag=False, threads=threads)
    one = time.perf_counter() - t0
    cycles = max(1, int(seconds / max(one, 1e-6)))
    t0 = time.perf_counter()
    oracle.run(csr, chains, seed=0, ncycles=cycles, cpg=1, diag=False, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": float(csr.nnz) * chains * cycles / dt, "unit": UNIT, "cores": threads,
            "kind": "oracle", "sample": f"{chains} chains x {cycles} cycles of {workload} (of K={K})",
            "seconds": dt}


def cpu_baseline_and_accuracy(args, csr, flags, shape):
    """The CPU-baseline leg of the pedigree line.

    The FP64 oracle is timed on a bounded sample of the workload: Ks chains of the
    colour-ordered matrix P C P^T for 16 burn-in and 112 sampling cycles, with the
    diagonal and 256 sampled rows x 512 columns of the block C^-1[:, 0:512]
    accumulated, on every host core (one OpenMP thread per chain group).  A second,
    smaller sample (no accumulation) is timed on one core.

    The same all-core run is the FP64 reference of the accuracy report (the error of
    each result against the oracle, next to its Monte Carlo standard error): a GPU
    handle in the benchmark's configuration (FP32 sweep, BF16 tensor-core block,
    FP64 folds, colour order, autotuned kernel) runs the same Ks chains, and its
    diagonal and block estimates are compared entry by entry with the oracle's."""
    import oracle
    from oracle.colour import greedy_order, permuted
    from paper_cs_0412107_gb300 import mcinv
    nproc = os.cpu_count() or 1
    Ks, B, burn, samp = 128, 8, 16, 112
    seed = args.seed + 101
    order, _ = greedy_order(csr)
    cp = permuted(csr, order)
    pos = np.empty(csr.n, dtype=np.int64)
    pos[order] = np.arange(csr.n)  # row r of C is row pos[r] of P C P^T
    R = np.linspace(0, csr.n - 1, 256).astype(np.int64)
    S = np.arange(512)
    cpg = max(1, Ks // nproc)
    t0 = time.perf_counter()
    _, dacc, bacc = oracle.run(cp, Ks, seed=seed, ncycles=burn + samp, acc_from=burn, cpg=cpg, R=pos[R], S=pos[S],
                               threads=nproc)
    t_all = time.perf_counter() - t0
    od = dacc.sum(0).real[pos] / (Ks * samp)
    ob = bacc.sum(0).real / (Ks * samp)
    # one core: 8 chains, no accumulation, sized to about 5 s
    t0 = time.perf_counter()
    oracle.run(cp, 8, seed=seed, ncycles=1, diag=False, threads=1)
    c1 = max(1, int(5.0 / max(time.perf_counter() - t0, 1e-6)))
    t0 = time.perf_counter()
    oracle.run(cp, 8, seed=seed, ncycles=c1, diag=False, threads=1)
    t_one = time.perf_counter() - t0
    base = {"value": float(csr.nnz) * Ks * (burn + samp) / t_all, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "nproc": nproc,
            "sample": f"{Ks} chains x {burn + samp} cycles of {WORKLOAD} in colour order, diagonal and 256 x 512 "
                      f"entries of C^-1[:, 0:512] accumulated over the last {samp} (of K={args.chains})",
            "seconds": t_all,
            "one_core": {"value": float(csr.nnz) * 8 * c1 / t_one, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"8 chains x {c1} cycles of {WORKLOAD} in colour order, no accumulation",
                         "seconds": t_one}}
    h = mcinv.create_from_csr(csr, K=Ks, seed=seed, acc=mcinv.MCINV_ACC_BF16_TC, batch_cycles=B,
                              block_rows=np.arange(csr.n), block_cols=S, flags=flags, **shape)
    mcinv.mcinv_burnin(h, burn)
    mcinv.mcinv_sample(h, samp)
    dm, dse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_DIAG)
    bm, bse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)
    info = mcinv.mcinv_info(h)
    mcinv.mcinv_destroy(h)
    bm, bse = bm[R], bse[R]

    def report(m, se, ref):
        err = np.abs(m - ref)
        return {"max_abs_error": float(err.max()), "rms_error": float(np.sqrt(np.mean(err ** 2))),
                "max_rel_error": float(err.max() / np.abs(ref).max()),
                "mc_se_median": float(np.median(se)), "mc_se_min": float(np.min(se)),
                "max_error_over_se": float(np.max(err / se))}

    acc = {"reference": "FP64 oracle, same draws (the CPU-baseline sample)", "K": Ks, "burnin": burn,
           "samples": samp, "batch_cycles": B, "sweep_kernel": SWEEP_KERNELS[info["sweep_kernel"]][0],
           "diagonal": dict(report(dm, dse, od), precision="FP32 sweep partials, FP64 fold", entries=int(csr.n)),
           "block": dict(report(bm, bse, ob), precision="BF16 operands on the tensor cores, FP32 accumulation, "
                                                        "FP64 fold", entries=f"{len(R)} sampled rows x {len(S)}")}
    return base, acc


def guarded(fn, *a, **kw):
    """Run one sub-record; a failure is reported in the record, not raised."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 -- the main line must still print
        return {"error": f"{type(e).__name__}: {e}"}


def run_configs(args, local):
    """The other workloads of the benchmark, each one bounded: the complex 2D lattice's
    update rate and roofline, the 4D lattice's time to 1e-2 and 3e-3 RMS error with the
    tensor cores against CUDA-core accumulation, and the batched form (throughput,
    time to 1e-2 RMS against the plain path, serving latency)."""
    import copy
    out = {}
    a = copy.copy(args)
    # a step is one sampling batch of 128 cycles, as on the headline line
    a.steps, a.warmup, a.batch, a.burnin = 8, 3, 128, 20
    a.kernel, a.order, a.W, a.threads, a.no_autotune = "auto", "colour", 0, 0, False
    r = guarded(run_lattice2d, a, 1, 0, local)
    if "error" not in r:
        r = {k: r[k] for k in ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "dtype", "config",
                               "roofline", "trace", "kernels_ms", "gpu_launches", "clocks")}
    out["lattice2d128"] = r
    a = copy.copy(args)
    a.lattice_batches, a.order = 6, "colour"
    out["lattice4d16"] = guarded(run_lattice, a, 1, 0, local)
    a = copy.copy(args)
    a.order = "colour"
    out["batch512"] = guarded(run_batch, a, 1, 0, local)
    return out


DIRAC_PAPER = {"exact": 413007.84, "cc_cycles": 10832 + 18, "cc_se": 4.128, "cpu_seconds": 10859.0}


def run_dirac(args, world, rank, local):
    """Algorithm 1 in full on the paper's Example 2, case 1 (Table 3): the free Wilson-Dirac
    matrix on an 18^4 lattice (n = 419,904, 14 nonzeros per row, K = 0.1).

    Coupling burn-in at tol 1e-5 (Eq. 12), then sampling until the trace's MC error
    (Geyer's effective length) is below 1e-5 of the estimate, checked every 100 cycles,
    the rule behind Tables 4 and 5.  The whole run is timed on the device; the estimate
    is compared with the exact trace from the momentum-space closed form."""
    import torch

    from paper_cs_0412107_gb300 import mcinv
    from paper_cs_0412107_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dims = (18, 18, 18, 18)
    csr = wl.wilson_dirac(dims, 0.1)
    exact = wl.wilson_dirac_inverse_trace(dims, 0.1).real
    K = args.chains
    stream = torch.cuda.current_stream()
    h = mcinv.create_from_csr(csr, K=K, seed=args.seed, chain_base=rank * K, acc=mcinv.MCINV_ACC_FP32_SIMT,
                              batch_cycles=10, flags=kernel_flags(args)[0] | order_flag(args), **shape_kw(args))
    info0 = mcinv.mcinv_info(h)
    mcinv.mcinv_set_trace_weights(h, np.ones(csr.n))
    mcinv.mcinv_sync(h)
    launches0 = info0["kernel_launches"]
    mcinv.mcinv_profile(h, True)
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    evm = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        p = mcinv.mcinv_burnin_coupled(h, 1e-5, 1000)
        evm.record(stream)
        used = mcinv.mcinv_sample_until(h, 1e-5, 100, 100_000)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    ms_sampling = evm.elapsed_time(ev1)
    prof = {mcinv.KERNEL_NAMES[k]: mcinv.mcinv_profile_read(h, k) for k in range(5)}
    mcinv.mcinv_profile(h, False)
    g = mcinv.mcinv_trace_mc_error(h)
    launches = mcinv.mcinv_info(h)["kernel_launches"] - launches0
    mcinv.mcinv_destroy(h)
    ms_max = max_over_ranks(ms, world)
    cycles = p + used
    value = float(csr.nnz) * K * cycles * world / (ms_max / 1e3)
    hbm, _, _, peak_kind = read_peaks()
    sw_launches, sw_ms = prof["sweep"]
    # the coupled-difference sweeps (one chain, no noise) are launched as well; count the
    # units of every launch: K chains per chain cycle, one per difference cycle
    units = float(csr.n) * (K * cycles + p)
    compulsory = 32.0 * units  # read + write z and w once, complex64
    gather = 8.0 * (2 * (csr.nnz - csr.n) + 2 * csr.n) / csr.n * units
    achieved = compulsory / (sw_ms / 1e3) / 1e9 if sw_ms else None
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 0,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "complex64 (f32)", "data": "synthetic: the paper's own matrix (free Wilson-Dirac, 18^4, K=0.1)",
        "config": {"workload": "dirac18", "n": csr.n, "nnz": csr.nnz, "K": K, "step": "one Algorithm 1 run",
                   "burnin": "coupled, tol 1e-5", "stop": "MC error < 1e-5 of tr, checked every 100 cycles",
                   "chains_per_cta": info0["chains_per_cta"], "threads_per_cta": info0["threads_per_cta"],
                   "ctas_per_slice": info0["ctas_per_slice"], "levels": info0["levels"], "sweep_order": args.order,
                   "l2": "inputs larger than L2 (z, w double-buffered: %.1f GB)" % (4 * 8 * csr.n * K / 1e9)},
        "result": {"burnin_cycles": p, "sampling_cycles": used, "trace": g["mean"], "mc_error": g["se"],
                   "effective_length": g["ess"], "exact": exact, "z": (g["mean"] - exact) / g["se"],
                   "seconds": ms_max / 1e3, "sampling_seconds": ms_sampling / 1e3,
                   "effective_samples_per_second": g["ess"] / (ms_sampling / 1e3),
                   "effective_length_per_cycle": g["ess"] / used},
        "paper_table4": DIRAC_PAPER,
        "roofline": {"kernel": SWEEP_KERNELS[info0["sweep_kernel"]][0], "bound": "hbm", "achieved": achieved,
                     "peak": hbm, "unit": "GB/s", "frac": achieved / hbm if achieved else None, "traffic": None,
                     "peak_source": f"{peak_kind} hbm_gbs", "bytes_per_unit": 32.0,
                     "bytes": "compulsory (stencil neighbours are reuse)",
                     "gather_inclusive_gbs": gather / (sw_ms / 1e3) / 1e9 if sw_ms else None,
                     "sweep_ms_per_chain_cycle": sw_ms / cycles},
        "kernels_ms": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(csr, K, args.cpu_seconds, "dirac18")
    return result


def run_reference(args, world, rank):
    """The reference arm: the FP64 CPU oracle (there is no upstream code), one
    bounded sample of the workload per step, on rank 0 only."""
    if rank != 0:
        return None
    import oracle
    from paper_cs_0412107_gb300 import workloads as wl
    csr = wl.WORKLOADS[WORKLOAD].build()
    threads = os.cpu_count() or 1
    chains = threads
    st = None
    for k in range(args.warmup):
        st, _, _ = oracle.run(csr, chains, seed=0, cycle0=k, ncycles=1, cpg=1, diag=False, threads=threads, state=st)
    t0 = time.perf_counter()
    for k in range(args.steps):
        st, _, _ = oracle.run(csr, chains, seed=0, cycle0=args.warmup + k, ncycles=1, cpg=1, diag=False,
                              threads=threads, state=st)
    dt = time.perf_counter() - t0
    value = float(csr.nnz) * chains * args.steps / dt
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded pedigree-shaped matrix, Philox noise)",
            "config": {"workload": WORKLOAD, "n": csr.n, "nnz": csr.nnz, "K": args.chains},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{chains} chains x 1 cycle per step of {WORKLOAD}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--acc", default="tc", choices=["tc", "simt"])
    ap.add_argument("--chains", type=int, default=1024)
    ap.add_argument("--batch", type=int, default=128, help="cycles per sampling batch = per step")
    ap.add_argument("--burnin", type=int, default=20)
    ap.add_argument("--W", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-jobs", type=int, default=2)
    ap.add_argument("--e2e-burnin", type=int, default=500)
    ap.add_argument("--e2e-samples", type=int, default=5000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "batch512", "dirac18", "lattice4d16",
                                                             "lattice2d128", "lattice4d16-rate"],
                    help="lattice4d16: time to RMS error; lattice4d16-rate: the update rate, as lattice2d128")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-burnin", type=int, default=200)
    ap.add_argument("--batch-samples", type=int, default=2000)
    ap.add_argument("--batch-mem-gb", type=float, default=64.0)
    ap.add_argument("--serve-requests", type=int, default=128)
    ap.add_argument("--rms-samples", type=int, default=16)
    ap.add_argument("--order", default="colour", choices=["natural", "colour"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "sliced", "grid", "bulk", "pair", "tile", "wave"])
    ap.add_argument("--no-natural", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads' sub-records")
    ap.add_argument("--lattice-batches", type=int, default=6)
    ap.add_argument("--lattice-chains", type=int, default=0, help="chains of the lattice rate runs (0: the workload's)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    args = ap.parse_args()
    assert args.warmup >= 3 or args.impl == "reference" or os.environ.get("BENCH_ALLOW_SHORT"), "warmup >= 3"
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        res = run_reference(args, world, rank)
    elif args.workload == "batch512":
        res = run_batch(args, world, rank, local)
    elif args.workload == "dirac18":
        res = run_dirac(args, world, rank, local)
    elif args.workload == "lattice4d16":
        res = run_lattice(args, world, rank, local)
    elif args.workload in ("lattice2d128", "lattice4d16-rate"):
        res = run_lattice2d(args, world, rank, local)
    else:
        res = run_mine(args, world, rank, local)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
