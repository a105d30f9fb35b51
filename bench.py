#!/usr/bin/env python
"""Benchmark of the stabilised fermion log-weight ln det(I + B_L ... B_1) on one or more
GB300 GPUs (one process per GPU; chains are independent, so N GPUs run N independent
batches: weak scaling, no collective on the data path).

Workload (default): 16x16 periodic lattice (N = 256), beta = 16 (L = 160 slices,
dtau = 0.1), stabilisation every n_s = 8 slices, t = 1, mu = 0, omega0 = 1, lambda = 1;
512 seeded synthetic fields per GPU, half iid N(0, 1) and half the CDW pattern
0.8 (-1)^(ix+iy) + N(0, 0.3^2). The fields (168 MB) and the workspace (1.5 GB) are larger
than L2, so no explicit flush is needed between steps.

One step = one pass of the whole hot path over the batch: a cumulative update of every
chain (effective-model checkerboard sweeps, E_eff, exact ln w with the stabilised
determinant and G, the Eq. (6) acceptance, S(pi,pi)) followed by the regression of E_eff
on the batch. value = ln det evaluations per second = chains / step time, in the mixed
precision mode (slice products in --precision, default the exact sliced BF16x9 mode on the
tensor cores; FP64 QR / D scales / LU / log-ratio; the T update of the stabilisation FP64-accurate
on the tensor cores). Every mode's ln det is scored against the oracle over the whole batch
(max and RMS of |d ln det|), and the FP64 mode's full step is timed beside the headline.

--probe prints the cuBLAS FP64 / FP32 / TF32 / BF16 GEMM rates and the copy bandwidth of the
GPU (the rates the bench reports beside its nominal alu peaks) and exits.

--impl reference times the CPU oracle (plain FP64 numpy) on the host cores instead.

--mode dqmc measures the conventional DQMC updates instead (chain-sweeps/s, one chain per SM,
12x12 / L = 120 by default) with the roofline of its local-update kernel; with --impl reference
it times the DQMC oracle.
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "stabilised ln det(I+B_L...B_1) evals/s, mixed vs FP64 on one GB300, % of peak"
UNIT = "evals/s"

# Roofline denominators. HBM and BF16 come from MEASURED_PEAKS.json when present (the tensor
# kernels are taken against its BF16 burst rate; TF32 against that rate times the nominal
# TF32 / BF16 ratio 1.1 / 2.25). The FP64 and FP32 pipes are not in that file: "alu" peaks are the
# nominal figures (FP64 1.25 TFLOP/s), with the rates that this run measures with cuBLAS
# (probe_rates, also `python bench.py --probe`) reported beside them.
NOMINAL = {"fp64_tflops": 1.25, "fp32_tflops": 152 * 128 * 2 * 2.07e9 / 1e12, "hbm_gbs": 6800.0,
           "tf32_per_bf16": 1.1 / 2.25}
MIXED_BAR_DLNW = 1e-4  # |d ln w| of a mixed-precision mode against the FP64 oracle


def probe_rates(dev):
    """Pipe rates measured now with library GEMMs (cuBLAS through torch.matmul; CUDA events, best
    of a few repetitions after a warm-up): FP64, FP32 (TF32 off), TF32 and BF16 in TFLOP/s, and a
    device-to-device copy of 1 Gi BF16 elements in GB/s (bytes read + written)."""
    import torch

    def best_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    def gemm(n, dtype, reps, tf32=False):
        a = torch.randn(n, n, device=dev).to(dtype)
        b = torch.randn(n, n, device=dev).to(dtype)
        old = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        try:
            ms = best_ms(lambda: torch.matmul(a, b), reps)
        finally:
            torch.backends.cuda.matmul.allow_tf32 = old
        return 2.0 * n ** 3 / (ms / 1e3) / 1e12

    out = {"fp64_tflops": gemm(4096, torch.float64, 3), "fp32_tflops": gemm(8192, torch.float32, 3),
           "tf32_tflops": gemm(8192, torch.float32, 5, tf32=True), "bf16_tflops": gemm(8192, torch.bfloat16, 5)}
    src = torch.empty(1 << 30, dtype=torch.bfloat16, device=dev)
    dst = torch.empty_like(src)
    out["copy_gbs"] = 2.0 * src.numel() * 2 / (best_ms(lambda: dst.copy_(src), 5) / 1e3) / 1e9
    out["how"] = "torch.matmul 4096^3 FP64, 8192^3 FP32 / TF32 / BF16 (2 n^3 flop), copy of 1 Gi BF16; best of 3-5"
    del src, dst
    torch.cuda.empty_cache()
    return out


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = {"hbm_gbs": 6800.0, "source": "fallback"}
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained"):
                if k in d:
                    peaks[k] = float(d[k])
            peaks["source"] = "measured"
        except Exception:
            pass
    return peaks


# ---------------------------------------------------------------------------------------
# CPU oracle timing (spawned workers, one BLAS thread each)
# ---------------------------------------------------------------------------------------
def _oracle_logdet_worker(args):
    wl_name, nf, fids = args
    from oracle import HolsteinParams
    from oracle.fermion import fermion_logdet
    from oracle.lattice import exp_hopping
    from paper_1802_06177_gb300 import inputs
    from paper_1802_06177_gb300.workloads import WORKLOADS
    wl = WORKLOADS[wl_name]
    p = HolsteinParams(wl.Lx, wl.Lx, wl.L, n_s=wl.n_s)
    E = exp_hopping(wl.Lx, wl.Lx, 1.0, 0.0, 0.1)
    gen = inputs.mixed_fields if wl.fields == "mixed" else inputs.gaussian_fields
    x = gen(nf, wl.Lx, wl.Lx, wl.L, seed=wl.seed)
    out = []
    for fid in fids:
        lndet, sign, _ = fermion_logdet(p, x[fid], E=E, want_G=False)
        out.append((fid, lndet, sign))
    return out


def oracle_pool(nproc):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("MKL_NUM_THREADS", "1")
    return mp.get_context("spawn").Pool(nproc)


def oracle_logdets(pool, wl_name, nf, field_ids):
    """Oracle ln|det| of fields of the benchmark batch (seeded exactly as on rank 0)."""
    ids = list(field_ids)
    nchunk = max(1, min(len(ids), 64))
    chunks = [ids[k::nchunk] for k in range(nchunk)]
    return {f: (l, sg) for part in pool.map(_oracle_logdet_worker, [(wl_name, nf, c) for c in chunks if c])
            for f, l, sg in part}


# ---------------------------------------------------------------------------------------
# GPU clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        reasons = sorted({n for r in rows for n, v in zip(self.NAMES, r[5:9]) if "Active" in v and "Not" not in v})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------
# algorithmic work per launch call of each kernel class (flops or bytes), per field
# ---------------------------------------------------------------------------------------
QR_PANEL_OVERRIDE = [0]  # --qr-panel


def qr_panel_width(N):
    return QR_PANEL_OVERRIDE[0] or (32 if N <= 256 else 16)


def qrt_panel_sizes(N):
    """(p, m, n_t) of every panel of the pre-pivoted blocked QR: first row, rows m = N - p, trailing
    columns n_t after the panel."""
    bp = qr_panel_width(N)
    return [(p, N - p, max(0, N - p - bp)) for p in range(0, N, bp)]


def qr_panel_flops(N):
    """FP64 flops of the panel kernels of one QR: Householder QR of each m x BP panel (2 m BP^2 - 2/3 BP^3);
    the last panel also forms its Gram matrix V^T V (m BP^2) and compact-WY triangle S (BP^3 / 3), which
    the tensor-core products form for the other panels."""
    bp = qr_panel_width(N)
    sizes = qrt_panel_sizes(N)
    w = sum(2.0 * m * bp * bp - 2.0 / 3.0 * bp ** 3 for _, m, _ in sizes)
    m_last = sizes[-1][1]
    return w + m_last * bp * bp + bp ** 3 / 3.0


def qr_trailing_flops(N):
    """FP64-equivalent flops of the trailing updates of one QR: W = V^T C and C - V W' (2 x 2 m n_t BP)."""
    bp = qr_panel_width(N)
    return sum(4.0 * m * nt * bp for _, m, nt in qrt_panel_sizes(N))


def qr_trailing_issued(N):
    """BF16 MMA flops the tensor-core trailing updates of one QR issue: 28 slice products each of
    W^T = C^T V (128-row tiles of trailing columns x BP x K chunks of 64 from the chunk of row p)
    and of V W' (128-row tiles from the tile of row p x 64-column tiles x BP)."""
    bp = qr_panel_width(N)
    kpad, mpad = -(-N // 64) * 64, -(-N // 128) * 128
    t = 0.0
    for p, _, nt in qrt_panel_sizes(N):
        if nt == 0:
            continue
        t += 28 * 2.0 * (128 * -(-nt // 128)) * bp * (kpad - 64 * (p // 64))
        t += 28 * 2.0 * (mpad - 128 * (p // 128)) * (64 * -(-nt // 64)) * bp
    return t


def class_work(cls, wl, nsl_mean, precision="fp32", qrt=False):
    N, L = wl.N, wl.L
    if cls == "slice" and precision == "fp64":  # separable exp(-dtau K): N^2 (Lx + Ly) FMAs per slice
        return 2.0 * N ** 2 * (2 * wl.Lx) * nsl_mean, "flop"
    if cls == "slice":
        return 2.0 * N ** 3 * nsl_mean, "flop"
    if cls == "qr":  # per field and QR: with the tensor-core trailing updates, the FP64 panels alone
        return (qr_panel_flops(N) if qrt else 4.0 / 3.0 * N ** 3), "flop"
    if cls == "qrtc":
        return qr_trailing_flops(N), "flop"
    if cls == "formq":
        return 4.0 / 3.0 * N ** 3, "flop"
    if cls == "tupdate":
        return 1.0 * N ** 3, "flop"
    if cls == "greens":
        return 2.0 * N ** 3, "flop"
    if cls == "sweep":
        return 8.0 * N * L * 1.5, "byte"  # read the field once, write the updated half
    return None, None


# DRAM traffic per field of the dominant kernel, from the committed ncu summary of that
# kernel; valid only while the kernel source is the one the counters were taken on.
TRAFFIC_SOURCES = {"qr": ("profiles/k_qrt_16x16_L160.md", "paper_1802_06177_gb300/csrc/k_qrt.cu"),
                   "qrtc": ("profiles/k_qrt_16x16_L160.md", "paper_1802_06177_gb300/csrc/k_qrt.cu")}


def kernel_traffic(cls, fields_per_call):
    import hashlib
    import re
    if cls not in TRAFFIC_SOURCES:
        return None
    prof_md, src = (os.path.join(ROOT, q) for q in TRAFFIC_SOURCES[cls])
    if not (os.path.exists(prof_md) and os.path.exists(src)):
        return None
    m = re.search(r"traffic-per-field %s: ([0-9.eE+]+) bytes \(source sha256 ([0-9a-f]+)\)" % cls, open(prof_md).read())
    if not m:
        return None
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if not digest.startswith(m.group(2)):
        return None  # the kernel changed since the counters were taken
    return float(m.group(1)) * fields_per_call


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return rank, local, world


def max_over_ranks(value, world, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.mode == "dqmc":
        return run_reference_dqmc(args)
    from paper_1802_06177_gb300.workloads import WORKLOADS
    wl = WORKLOADS[args.workload]
    nproc = min(16, os.cpu_count() or 1)
    pool = oracle_pool(nproc)
    times = []
    for s in range(args.warmup + args.steps):
        done, _, wall = time_oracle_step(pool, nproc, wl.name, args.nsweeps)
        if s >= args.warmup:
            times.append((done, wall))
    pool.close()
    done = sum(d for d, _ in times)
    wall = sum(w for _, w in times)
    value = done / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, args, args.precision),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle",
                             "sample": "per step: %d chains (one per core), one oracle cumulative update each "
                                       "(%d E_eff sweeps, exact ln w with UDT log-det and G, Eq. 6 accept) on %s"
                                       % (nproc, args.nsweeps, wl.name)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _oracle_step_worker(args):
    wl_name, chain, nsweeps = args
    import numpy as np

    from oracle import HolsteinParams
    from oracle.chain import cumulative_update
    from oracle.lattice import exp_hopping
    from oracle.weight import log_weight
    from paper_1802_06177_gb300 import inputs
    from paper_1802_06177_gb300.workloads import WORKLOADS
    wl = WORKLOADS[wl_name]
    p = HolsteinParams(wl.Lx, wl.Lx, wl.L, n_s=wl.n_s)
    E = exp_hopping(wl.Lx, wl.Lx, 1.0, 0.0, 0.1)
    x = inputs.gaussian_fields(1, wl.Lx, wl.Lx, wl.L, seed=wl.seed + 7 * chain)[0]
    J = np.array([50.25, 0.05, 0.0, 0.0, 0.5])
    lw = log_weight(p, x, E)[0]
    t0 = time.perf_counter()
    cumulative_update(p, x, lw, 0.0, J, nsweeps, 0, chain, wl.seed, 0.3, E=E)
    return time.perf_counter() - t0


def time_oracle_step(pool, nproc, wl_name, nsweeps):
    t0 = time.perf_counter()
    per = pool.map(_oracle_step_worker, [(wl_name, c, nsweeps) for c in range(nproc)])
    return nproc, max(per), time.perf_counter() - t0


def config_of(wl, args, precision):
    return {"workload": wl.name, "model": "holstein_2d", "N": wl.N, "Lx": wl.Lx, "L": wl.L, "beta": wl.beta,
            "n_s": wl.n_s, "chains_per_gpu": args.fields or wl.nfields, "nsweeps": args.nsweeps,
            "sub_batches": getattr(args, "sub_batches", 0) or 3,
            "slice_groups": getattr(args, "slice_groups", 0) or (4 if wl.N <= 256 else 1),
            "precision": precision,
            "fp64_slices": "dense" if getattr(args, "dense_slices", False) else "separable",
            "global_batch": (args.fields or wl.nfields) * args.gpus,
            "parallelism": "replicas x%d" % args.gpus,
            "l2": "inputs larger than L2 (fields %.0f MB + workspace), no flush" % (
                (args.fields or wl.nfields) * wl.N * wl.L * 8 / 1e6)}


def tensor_use(wl, nf, ngroups, precision, prof, peaks):
    """Tensor-pipe use of the tensor-core kernel classes over a profiled region: issued MMA flops
    (every slice product the kernels issue, padding included) of all the class's calls (the
    profiler counts the fields of each call; one call per stabilisation group) over the class's
    busy time, against the measured BF16 burst rate (TF32: times the nominal TF32 / BF16 ratio)."""
    bf16 = peaks.get("bf16_tflops")
    if not bf16:
        return {}
    N = wl.N
    npad, mtiles = -(-N // 64) * 64, -(-N // 128)
    nsl_mean = wl.L / ngroups
    out = {}
    src = "MEASURED_PEAKS.json bf16_tflops (burst)"
    sl = prof.get("slice")
    if precision in ("bf16x9", "tf32x3") and sl and sl[2] > 0:
        if precision == "bf16x9":  # 9 products of 128-row tiles x K chunks of 64 per slice
            nt = 128 if mtiles == 1 and N > 64 else (64 if mtiles <= 2 else (32 if mtiles <= 4 else 16))
            per_field_slice = 9 * 2.0 * (128 * mtiles) * npad * (nt * -(-N // nt))
            peak, how = bf16, src
        else:  # 3 products, K padded to 32
            per_field_slice = 3 * 2.0 * (128 * mtiles) * (-(-N // 32) * 32) * N
            peak, how = bf16 * NOMINAL["tf32_per_bf16"], src + " x 1.1/2.25 (nominal TF32/BF16)"
        issued = per_field_slice * nsl_mean * sl[3]
        t = issued / (sl[2] / 1e3) / 1e12
        out["slice:" + precision] = {"issued_tflops": t, "peak_tflops": peak, "frac_of_peak": t / peak,
                                     "busy_ms": sl[2], "dense_fp32_equivalent_tflops":
                                     2.0 * N ** 3 * nsl_mean * sl[3] / (sl[2] / 1e3) / 1e12, "peak_source": how}
    qt = prof.get("qrtc")
    if qt and qt[2] > 0:
        field_qrs = qt[3] / max(1, len(qrt_panel_sizes(N)) - 1)  # one call per panel but the last
        issued = qr_trailing_issued(N) * field_qrs
        t = issued / (qt[2] / 1e3) / 1e12
        out["qrtc:" + precision] = {"issued_tflops": t, "peak_tflops": bf16, "frac_of_peak": t / bf16,
                                    "busy_ms": qt[2], "includes": "the slicing of the trailing columns",
                                    "fp64_equivalent_tflops": qr_trailing_flops(N) * field_qrs / (qt[2] / 1e3) / 1e12,
                                    "peak_source": src}
    tu = prof.get("tupdate")
    if tu and tu[2] > 0:
        nk = npad // 64
        chunks = sum(nk - 2 * mt for mt in range(mtiles))  # K chunks per column tile (triangular start)
        issued = chunks * (npad // 64) * 28 * 2.0 * 128 * 64 * 64 * tu[3]
        t = issued / (tu[2] / 1e3) / 1e12
        out["tupdate:" + precision] = {"issued_tflops": t, "peak_tflops": bf16, "frac_of_peak": t / bf16,
                                       "busy_ms": tu[2], "includes": "the two slicing kernels",
                                       "fp64_equivalent_tflops": float(N) ** 3 * tu[3] / (tu[2] / 1e3) / 1e12,
                                       "peak_source": src}
    return out


def run_gpu(args):
    import numpy as np
    import torch

    from paper_1802_06177_gb300 import inputs
    from paper_1802_06177_gb300.dist import fit_eff_distributed
    from paper_1802_06177_gb300.slmc import Context
    from paper_1802_06177_gb300.workloads import WORKLOADS

    rank, local, world = dist_setup(args)
    wl = WORKLOADS[args.workload]
    nf = args.fields or wl.nfields
    QR_PANEL_OVERRIDE[0] = args.qr_panel
    pool = None
    nproc = min(16, os.cpu_count() or 1)
    if rank == 0 and not args.no_cpu_baseline:
        pool = oracle_pool(nproc)  # spawn before the first GPU call
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seed = wl.seed + 1000003 * rank
    xh = inputs.mixed_fields(nf, wl.Lx, wl.Lx, wl.L, seed=seed) if wl.fields == "mixed" else \
        inputs.gaussian_fields(nf, wl.Lx, wl.Lx, wl.L, seed=seed)
    x0 = torch.from_numpy(xh).to(dev)

    def make(prec):
        c = Context(wl.Lx, wl.Lx, wl.L, n_s=wl.n_s, precision=prec, max_fields=nf, seed=seed, sweep_delta=0.3,
                    device=dev)
        if args.sub_batches:
            c.set_sub_batches(args.sub_batches)
        if args.slice_groups:
            c.set_slice_groups(args.slice_groups)
        if args.sub_priorities >= 0:
            c.set_sub_batch_priorities(args.sub_priorities)
        if args.qr_cluster:
            c.set_qr_cluster(args.qr_cluster)
        if args.dense_slices:
            c.set_dense_slices(1)
        if args.qr_panel:
            c.set_tuning(args.qr_panel, 0)
        if args.qr_path >= 0:
            c.set_qr_path(args.qr_path)
        return c

    def setup(ctx):
        x = x0.clone()
        lnw0, _, _ = ctx.log_weight(x)
        J, _ = ctx.fit_eff(x, lnw0)  # self-learned couplings of the initial batch
        lnw, s = ctx.chain_init(x)
        n_acc = torch.zeros(nf, dtype=torch.int64, device=dev)
        n_sw = torch.zeros(nf, dtype=torch.int64, device=dev)
        return {"x": x, "J": J, "lnw": lnw, "s": s, "n_acc": n_acc, "n_sw": n_sw}

    def step(ctx, st, k):
        if args.mode == "logdet":
            ctx.logdet(st["x"])
            return
        ctx.cumulative_update(st["x"], st["J"], args.nsweeps, 1, k, st["lnw"], st["s"], st["n_acc"], st["n_sw"])
        # Eq. (5) over the chains of every process: partial state, all-gather (N > 1), merge
        st["J_fit"], _ = fit_eff_distributed(ctx, st["x"], st["lnw"])

    def timed(ctx, st, steps, warmup, k0, profile=False, clocks=False):
        for k in range(warmup):
            step(ctx, st, k0 + k)
        torch.cuda.synchronize()
        barrier(world)
        sampler = ClockSampler(local) if clocks else None
        if profile:
            ctx.profile(True)
        n0 = ctx.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for k in range(steps):
            step(ctx, st, k0 + warmup + k)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = ctx.launch_count() - n0
        prof = ctx.profile_read_detail() if profile else None
        if profile:
            ctx.profile(False)
        clk = sampler.stop() if sampler else None
        ctx.get_error()
        barrier(world)
        return max_over_ranks(ms, world, dev), launches, prof, clk

    # ---- pipe rates of this GPU (cuBLAS), reported beside the nominal alu peaks -----------
    probed = probe_rates(dev)

    # ---- headline: mixed precision --------------------------------------------------
    ctx = make(args.precision)
    st = setup(ctx)
    ms, launches, _, clk = timed(ctx, st, args.steps, args.warmup, 0, clocks=True)
    ms_step = ms / args.steps
    value = nf * world / (ms_step / 1e3)
    # per-class device time of the same step, from a separate profiled pass (CUDA events around every
    # launch call on its stream; the events cost a few per cent, so the headline above runs without)
    psteps = max(1, min(args.steps, 5))
    ms_prof, _, prof, _ = timed(ctx, st, psteps, 0, args.steps + args.warmup, profile=True)

    # ---- e2e through host buffers, over as many steps as the device-timed value ------------
    xh_pin = torch.from_numpy(st["x"].cpu().numpy()).pin_memory()
    lnw_h = torch.empty(nf, dtype=torch.float64).pin_memory()
    s_h = torch.empty(nf, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        st["x"].copy_(xh_pin, non_blocking=True)
        step(ctx, st, 10 ** 6 + k)
        xh_pin.copy_(st["x"], non_blocking=True)
        lnw_h.copy_(st["lnw"], non_blocking=True)
        s_h.copy_(st["s"], non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    h2d = nf * wl.N * wl.L * 8
    d2h = h2d + 2 * nf * 8

    # ---- logdet-only rates, tensor-pipe use and ln det of every mode over the whole batch -----
    peaks = load_peaks()
    ngroups = math.ceil(wl.L / wl.n_s)
    rates, lndets, tensor = {}, {}, {}
    old_mode = args.mode
    args.mode = "logdet"

    def logdet_mode(c, m):
        ms_l, _, pr, _ = timed(c, {"x": x0.clone()}, 1, 2, 0, profile=True)
        rates[m] = nf * world / (ms_l / 1e3)
        lndets[m] = c.logdet(x0)[0].cpu().numpy()
        tensor.update(tensor_use(wl, nf, ngroups, m, pr, peaks))

    logdet_mode(ctx, args.precision)
    ctx.close()
    fp64_value = None
    for extra in ([] if args.no_fp64 else ["fp64", "fp32", "tf32x3", "bf16x9"]):
        if extra == args.precision:
            continue
        ce = make(extra)
        logdet_mode(ce, extra)
        if extra == "fp64" and old_mode == "step":
            args.mode = old_mode
            ms64s, _, _, _ = timed(ce, setup(ce), 1, 2, 0)
            fp64_value = nf * world / (ms64s / 1e3)
            args.mode = "logdet"
        ce.close()
    args.mode = old_mode

    batched = None if args.no_batch else run_uneven_batch(args, dev, seed)

    if rank != 0:
        return 0

    # ---- roofline of the dominant kernel class -------------------------------------------
    nsl_mean = wl.L / ngroups
    # calls of one class on concurrent sub-batch streams overlap: rank classes by busy time
    # (union of their call intervals) and divide the class's work by it
    dom = max(prof, key=lambda k: prof[k][2])
    dom_ms, dom_calls, dom_busy, dom_units = prof[dom]
    # with the tensor-core trailing updates a QR is one "qr" call per panel and one "qrtc" call per
    # panel but the last: count QRs of all fields (field-QRs) and calls per QR
    qrt = bool(prof.get("qrtc") and prof["qrtc"][1] > 0)
    npan = len(qrt_panel_sizes(wl.N))
    per_qr = {"qr": npan, "qrtc": max(1, npan - 1)}.get(dom, 1) if qrt else 1
    dom_calls, dom_units = dom_calls / per_qr, dom_units / per_qr
    work, kind = class_work(dom, wl, nsl_mean, args.precision, qrt)
    roof = None
    if work:
        fields_per_call = dom_units / max(dom_calls, 1)
        per_call = work * fields_per_call
        busy_s = dom_busy / 1e3
        fp64_cls = dom in ("qr", "formq", "greens") or (dom == "slice" and args.precision == "fp64")
        traffic = kernel_traffic(dom, fields_per_call)
        common = {"kernel_class": dom, "algorithmic_per_launch": per_call, "fields_per_launch": fields_per_call,
                  "launches_timed": dom_calls, "busy_ms": dom_busy, "sum_launch_ms": dom_ms,
                  "avg_launch_ms": dom_ms / max(dom_calls, 1),
                  "timing": "achieved = work of all timed launches / their busy time (union of launch "
                            "intervals on the sub-batch streams, CUDA events on the launching streams) over "
                            "a profiled pass of %d steps after the headline's timed steps" % psteps}
        if kind == "flop" and (fp64_cls or dom == "slice"):
            achieved = work * dom_units / busy_s / 1e12
            if fp64_cls:
                peak, pk, src = NOMINAL["fp64_tflops"], probed["fp64_tflops"], \
                    "nominal FP64 1.25 TFLOP/s (alu, not in MEASURED_PEAKS.json); cuBLAS DGEMM rate of this run beside it"
            else:
                peak, pk, src = NOMINAL["fp32_tflops"], probed["fp32_tflops"], \
                    "nominal FP32 SIMT rate 152 SM x 128 lanes x 2 x 2.07 GHz (alu); cuBLAS SGEMM rate beside it"
            roof = dict(common, bound="alu", pipe="fp64" if fp64_cls else "fp32", achieved=achieved, peak=peak,
                        unit="TFLOP/s", frac=achieved / peak, peak_probed=pk, frac_of_probed=achieved / pk,
                        traffic=traffic, peak_source=src)
        elif kind == "flop" and dom == "qrtc":
            t = tensor_use(wl, nf, ngroups, args.precision, prof, peaks).get("qrtc:" + args.precision)
            if t:
                roof = dict(common, bound="tensor", achieved=t["issued_tflops"], peak=t["peak_tflops"],
                            unit="TFLOP/s", frac=t["frac_of_peak"], traffic=traffic, peak_source=t["peak_source"],
                            fp64_equivalent_tflops=t["fp64_equivalent_tflops"])
        elif kind == "flop":  # tensor-core classes: issued BF16 flops against the measured BF16 rate
            t = tensor_use(wl, nf, ngroups, args.precision, prof, peaks).get(dom + ":" + args.precision)
            if t:
                roof = dict(common, bound="tensor", achieved=t["issued_tflops"], peak=t["peak_tflops"],
                            unit="TFLOP/s", frac=t["frac_of_peak"], traffic=None, peak_source=t["peak_source"])
        else:
            achieved = work * dom_units / busy_s / 1e9
            roof = dict(common, bound="hbm", achieved=achieved, peak=peaks["hbm_gbs"], unit="GB/s",
                        frac=achieved / peaks["hbm_gbs"], traffic=traffic, peak_source=peaks["source"])
    # E_eff sweeps: algorithmic bytes per half-sweep and chain = read the field, write the updated half
    sweep_roof = None
    if prof.get("sweep") and prof["sweep"][2] > 0:
        sb = 12.0 * wl.N * wl.L * prof["sweep"][3] / (prof["sweep"][2] / 1e3) / 1e9
        sweep_roof = {"bound": "hbm", "achieved": sb, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "frac": sb / peaks["hbm_gbs"], "algorithmic_bytes_per_half_sweep_and_chain": 12 * wl.N * wl.L,
                      "peak_source": peaks["source"]}
    total_prof = sum(v[2] for v in prof.values())
    shares = {k: round(v[2] / total_prof, 4) for k, v in prof.items() if v[2] > 0}
    step_tensor = tensor_use(wl, nf, ngroups, args.precision, prof, peaks)

    # ---- accuracy of every mode against the FP64 oracle over the batch, and CPU baseline ----
    acc = None
    cpu = None
    if pool is not None:
        ids = list(range(nf)) if not args.acc_fields else \
            sorted(set(range(min(args.acc_fields // 2, nf))) |
                   set(range(nf // 2, min(nf, nf // 2 + args.acc_fields - args.acc_fields // 2))))
        ref = oracle_logdets(pool, wl.name, nf, ids)
        r = np.array([ref[i][0] for i in ids])
        acc = {}
        for m, v in lndets.items():
            d = np.abs(v[ids] - r)
            acc[m] = {"max": float(d.max()), "rms": float(np.sqrt(np.mean(d ** 2))), "n": len(ids),
                      "max_dlnw": float(2 * d.max()), "rms_dlnw": float(2 * np.sqrt(np.mean(d ** 2))),
                      "meets_mixed_bar": bool(2 * d.max() <= MIXED_BAR_DLNW)}
        acc["fields"] = "all %d fields of the batch" % nf if len(ids) == nf else ids
        acc["note"] = "|d ln w| = 2 |d ln det| (two spin species; the bosonic part is exact FP64 in both)"
        done, busy, wall = time_oracle_step(pool, nproc, wl.name, args.nsweeps)
        done2, busy2, wall2 = time_oracle_step(pool, nproc, wl.name, args.nsweeps)
        cpu = {"value": (done + done2) / (wall + wall2), "unit": UNIT, "cores": nproc, "kind": "oracle",
               "sample": "%d chains x 2 rounds (one per core, 1 BLAS thread each): one oracle cumulative update "
                         "per chain (%d E_eff sweeps, exact ln w with UDT log-det and G, Eq. 6 accept) on %s"
                         % (nproc, args.nsweeps, wl.name)}
        pool.close()

    # FP64-pipe work of one evaluation of the step (QR per group, Q of the final group (FP64 in
    # every mode; the other groups' Q is FP64 only in FP64 mode), final LU, G, and FP64 slices in
    # FP64 mode; the T update runs on the tensor cores) against the step time
    N3 = float(wl.N) ** 3
    w_qr = qr_panel_flops(wl.N) if qrt else (4.0 / 3.0) * N3  # the panels alone when the trailing updates are TC
    w64 = ngroups * w_qr + (4.0 / 3.0) * N3 * (ngroups if args.precision == "fp64" else 1) \
        + (2.0 / 3.0 + (2.0 if args.mode == "step" else 0.0)) * N3
    if args.precision == "fp64":  # slices through the separable exp(-dtau K): N^2 (Lx + Ly) FMAs each
        w64 += 2.0 * float(wl.N) ** 2 * (2 * wl.Lx) * wl.L
    ach64 = w64 * nf * world / (ms_step / 1e3) / 1e12 / world
    fp64_step = {"flop_per_eval": w64, "achieved_per_gpu": ach64, "unit": "TFLOP/s",
                 "frac_of_nominal": ach64 / NOMINAL["fp64_tflops"], "frac_of_probed": ach64 / probed["fp64_tflops"],
                 "excludes": "T update (tensor cores)" + (", QR trailing updates (tensor cores)" if qrt else "")}
    dtype = {"fp64": "f64", "fp32": "f32 slices + f64 stabilisation",
             "tf32x3": "tf32x3 slices (tensor cores) + f64 stabilisation",
             "bf16x9": "bf16x9 exact-sliced slices (tensor cores) + f64 stabilisation"}[args.precision] + \
        "; T update f64-accurate on the tensor cores (bf16 slices)" + \
        ("; QR trailing updates f64-accurate on the tensor cores (bf16 slices)" if qrt else "")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config_of(wl, args, args.precision),
            "e2e": {"value": nf * world / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.steps},
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
            "fp64_value": fp64_value, "logdet_only_evals_per_s": rates, "accuracy_max_abs_dlndet": acc,
            "fp64_step": fp64_step, "sweep_roofline": sweep_roof, "tensor_step": step_tensor,
            "tensor_logdet_only": tensor, "probed_rates": probed, "time_shares": shares, "mode": args.mode,
            "batched_uneven": batched}
    print(json.dumps(line), flush=True)
    return 0


def run_uneven_batch(args, dev, seed):
    """Uneven batch: 64 chains each of 8x8/L=80, 10x10/L=100, 12x12/L=120, 16x16/L=160 (beta = L dtau),
    slices in the --batch-precision mode, n_s and tiles autotuned per class, advanced round by round (one
    cumulative update of every chain per round, 20 E_eff sweeps each) by replaying one captured CUDA graph. Per update the
    E_eff sweeps of all 256 chains run in one persistent queue launch; the same batch with each
    class's kernel-per-half-sweep sequence instead is timed beside it."""
    from paper_1802_06177_gb300.slmc import autotune
    from paper_1802_06177_gb300.workloads import UNEVEN_BATCH
    tuned, classes = {}, []
    for Lx, L, n in UNEVEN_BATCH:
        r = autotune(Lx, Lx, L, precision=args.batch_precision, ntune=16, tol=5e-5, seed=seed)
        tuned["%dx%d_L%d" % (Lx, Lx, L)] = {"n_s": r["n_s"], "qr_panel": r["qr_panel"],
                                            "slice_cols": r["slice_cols"], "max_abs_dlndet": r["max_abs_dlndet"]}
        classes.append(dict(Lx=Lx, L=L, nchains=n, n_s=r["n_s"], precision=args.batch_precision, seed=seed,
                            sweep_delta=0.3,
                            tuning=(r["qr_panel"], r["slice_cols"])))
    out = _time_uneven(args, dev, seed, classes, queue=True)
    out["per_class_kernels"] = _time_uneven(args, dev, seed, classes, queue=False)
    out["tuned"] = tuned
    out["precision"] = args.batch_precision
    return out


def _time_uneven(args, dev, seed, classes, queue):
    import torch

    from paper_1802_06177_gb300 import inputs
    from paper_1802_06177_gb300.slmc import Batch
    b = Batch([{k: v for k, v in cl.items() if k != "tuning"} for cl in classes], device=dev)
    b.set_sweep_queue(queue)
    keep = []
    with torch.cuda.stream(b.stream):
        for q, cl in enumerate(classes):
            ctx = b.context(q)
            ctx.set_tuning(*cl["tuning"])
            x = torch.from_numpy(inputs.gaussian_fields(cl["nchains"], cl["Lx"], cl["Lx"], cl["L"],
                                                        seed=seed + 17 * q)).to(dev)
            lnw0, _, _ = ctx.log_weight(x)
            J, _ = ctx.fit_eff(x, lnw0)
            lnw, s = ctx.chain_init(x)
            n_acc = torch.zeros(cl["nchains"], dtype=torch.int64, device=dev)
            ctx.set_update_counter(0)
            b.bind(q, x, J, lnw, s, n_acc)
            keep.append((x, J, lnw, s, n_acc, ctx))
    b.stream.synchronize()
    b.capture(args.nsweeps, 1)
    b.launch(2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.launch(args.batch_rounds)
    e1.record(b.stream)
    b.stream.synchronize()
    ms = e0.elapsed_time(e1)
    with torch.cuda.stream(b.stream):
        for k in keep:
            k[5].get_error()
    nch = sum(cl["nchains"] for cl in classes)
    acc = sum(int(k[4].sum().item()) for k in keep) / float(nch * (args.batch_rounds + 2))
    b.close()
    return {"evals_per_s": nch * args.batch_rounds / (ms / 1e3), "chains": nch, "rounds_timed": args.batch_rounds,
            "ms_per_round": ms / args.batch_rounds, "graph_launch_per_round": 1, "nsweeps": args.nsweeps,
            "sweep_queue": queue, "acceptance": acc}


# ---------------------------------------------------------------------------------------
# DQMC sweeps (the conventional updates the self-learning method is compared with)
# ---------------------------------------------------------------------------------------
def _oracle_dqmc_worker(args):
    wl_name, chain, seed = args
    from oracle import HolsteinParams
    from oracle.dqmc import dqmc_sweeps
    from oracle.lattice import exp_hopping
    from paper_1802_06177_gb300 import inputs
    from paper_1802_06177_gb300.workloads import WORKLOADS
    wl = WORKLOADS[wl_name]
    p = HolsteinParams(wl.Lx, wl.Lx, wl.L, n_s=wl.n_s)
    E = exp_hopping(wl.Lx, wl.Lx, 1.0, 0.0, 0.1)
    x = inputs.mixed_fields(2, wl.Lx, wl.Lx, wl.L, seed=wl.seed + 7 * chain)[chain % 2]
    t0 = time.perf_counter()
    dqmc_sweeps(p, x, 1, 0, chain, seed, 0.5, E=E)
    return time.perf_counter() - t0


DQMC_METRIC = "DQMC sweeps (local updates, fast ratio + Sherman-Morrison + wrapping) per second on one GB300"
DQMC_UNIT = "chain-sweeps/s"


def run_reference_dqmc(args):
    """The DQMC oracle on the host cores (one chain per core, one sweep each per step), with the
    metric, unit and config of the DQMC mode's GPU line."""
    from paper_1802_06177_gb300.workloads import WORKLOADS
    wl = WORKLOADS[args.workload]
    nproc = min(16, os.cpu_count() or 1)
    pool = oracle_pool(nproc)
    seed = wl.seed
    done, wall = 0, 0.0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pool.map(_oracle_dqmc_worker, [(wl.name, c, seed) for c in range(nproc)])
        if s >= args.warmup:
            done += nproc
            wall += time.perf_counter() - t0
    pool.close()
    value = done / wall
    sample = "per step: %d chains (one per core, 1 BLAS thread each), one oracle DQMC sweep each on %s" % (
        nproc, wl.name)
    line = {"impl": "reference", "metric": DQMC_METRIC, "value": value, "unit": DQMC_UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "model": "holstein_2d", "N": wl.N, "Lx": wl.Lx, "L": wl.L,
                       "n_s": wl.n_s, "chains_per_step": nproc, "block_updates_per_sweep": 0, "sweep_delta": 0.5,
                       "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": DQMC_UNIT, "cores": nproc, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": DQMC_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "mode": "dqmc"}
    print(json.dumps(line), flush=True)
    return 0


def run_dqmc(args):
    import torch

    from paper_1802_06177_gb300 import inputs
    from paper_1802_06177_gb300.slmc import Context
    from paper_1802_06177_gb300.workloads import WORKLOADS

    rank, local, world = dist_setup(args)
    wl = WORKLOADS[args.workload]
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    probed = probe_rates(dev)
    nproc = min(16, os.cpu_count() or 1)
    pool = oracle_pool(nproc) if rank == 0 and not args.no_cpu_baseline else None
    nf = args.fields or torch.cuda.get_device_properties(dev).multi_processor_count  # one chain per SM
    seed = wl.seed + 1000003 * rank
    ctx = Context(wl.Lx, wl.Lx, wl.L, n_s=wl.n_s, precision="fp64", max_fields=nf, seed=seed, sweep_delta=0.5,
                  device=dev)
    x = torch.from_numpy(inputs.mixed_fields(nf, wl.Lx, wl.Lx, wl.L, seed=seed)).to(dev)
    n_loc = torch.zeros(nf, dtype=torch.int64, device=dev)
    n_blk = torch.zeros(nf, dtype=torch.int64, device=dev)
    ctx.dqmc_sweep(x, args.warmup, sweep0=0, nblock=args.dqmc_block, n_acc_local=n_loc, n_acc_block=n_blk)
    torch.cuda.synchronize()
    barrier(world)
    acc0 = int(n_loc.sum().item())
    sampler = ClockSampler(local)
    ctx.profile(True)
    n0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    ctx.dqmc_sweep(x, args.steps, sweep0=args.warmup, nblock=args.dqmc_block, n_acc_local=n_loc, n_acc_block=n_blk)
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    launches = ctx.launch_count() - n0
    prof = ctx.profile_read_detail()
    ctx.profile(False)
    clk = sampler.stop()
    accepted = int(n_loc.sum().item()) - acc0
    ctx.get_error()
    # e2e: fields from pinned host memory, one sweep, fields and counts back
    xh = torch.from_numpy(x.cpu().numpy()).pin_memory()
    nh = torch.empty(nf, dtype=torch.int64).pin_memory()
    torch.cuda.synchronize()
    e0.record()
    for k in range(max(1, min(args.steps, 2))):
        x.copy_(xh, non_blocking=True)
        ctx.dqmc_sweep(x, 1, sweep0=10 ** 6 + k, nblock=args.dqmc_block, n_acc_local=n_loc, n_acc_block=n_blk)
        xh.copy_(x, non_blocking=True)
        nh.copy_(n_loc, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / max(1, min(args.steps, 2)), world, dev)
    ctx.close()
    barrier(world)
    if rank != 0:
        return 0
    N, Lx, L = wl.N, wl.Lx, wl.L
    ms_step = ms / args.steps
    value = nf * world / (ms_step / 1e3)
    # k_dqmc_slices: per slice 2 N^2 (Lx + Ly) FMAs of the wrap (four circulant passes), N^2 per
    # accepted move (Sherman-Morrison); FP64 pipe (alu)
    flops = 2.0 * (2.0 * N * N * (2 * Lx) * L * nf * args.steps + float(N) * N * accepted)
    dq_ms, dq_calls, dq_busy, dq_units = prof["dqmc"]
    achieved = flops / (dq_busy / 1e3) / 1e12
    roof = {"kernel_class": "dqmc", "kernel": "k_dqmc_slices", "bound": "alu", "pipe": "fp64",
            "algorithmic_per_launch": flops / max(dq_calls, 1), "launches_timed": dq_calls, "busy_ms": dq_busy,
            "achieved": achieved, "peak": NOMINAL["fp64_tflops"], "unit": "TFLOP/s",
            "frac": achieved / NOMINAL["fp64_tflops"], "peak_probed": probed["fp64_tflops"],
            "frac_of_probed": achieved / probed["fp64_tflops"], "traffic": None,
            "peak_source": "nominal FP64 1.25 TFLOP/s (alu, not in MEASURED_PEAKS.json); cuBLAS DGEMM rate of this run beside it"}
    total_prof = sum(v[2] for v in prof.values())
    shares = {k: round(v[2] / total_prof, 4) for k, v in prof.items() if v[2] > 0}
    cpu = None
    if pool is not None:
        t0 = time.perf_counter()
        pool.map(_oracle_dqmc_worker, [(wl.name, c, seed) for c in range(nproc)])
        wall = time.perf_counter() - t0
        pool.close()
        cpu = {"value": nproc / wall, "unit": DQMC_UNIT, "cores": nproc, "kind": "oracle",
               "sample": "%d chains (one per core, 1 BLAS thread each), one oracle DQMC sweep each on %s"
                         % (nproc, wl.name)}
    h2d = nf * N * L * 8
    line = {"metric": DQMC_METRIC, "value": value, "unit": DQMC_UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "model": "holstein_2d", "N": N, "Lx": Lx, "L": L, "n_s": wl.n_s,
                       "chains_per_gpu": nf, "block_updates_per_sweep": args.dqmc_block, "sweep_delta": 0.5,
                       "parallelism": "replicas x%d" % world,
                       "l2": "per-chain G in shared memory (N <= 160) or L2; fields %.0f MB" % (h2d / 1e6)},
            "e2e": {"value": nf * world / (e2e_ms / 1e3), "unit": DQMC_UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": h2d + 8 * nf},
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
            "acceptance_local": accepted / float(nf * args.steps * N * L), "time_shares": shares, "mode": "dqmc"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="slmc", choices=["slmc", "reference"])
    ap.add_argument("--workload", default=None, help="default holstein_16x16_L160 (dqmc mode: holstein_12x12_L120)")
    ap.add_argument("--precision", default="bf16x9", choices=["fp64", "fp32", "tf32x3", "bf16x9"])
    ap.add_argument("--nsweeps", type=int, default=20)
    ap.add_argument("--fields", type=int, default=0, help="override chains per GPU (small profiling cases)")
    ap.add_argument("--mode", default="step", choices=["step", "logdet", "dqmc"])
    ap.add_argument("--dqmc-block", type=int, default=0, help="DQMC mode: block updates per sweep")
    ap.add_argument("--acc-fields", type=int, default=0, help="oracle-scored fields (0 = the whole batch)")
    ap.add_argument("--probe", action="store_true", help="print the cuBLAS / copy rates of this GPU and exit")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-rounds", type=int, default=100)
    ap.add_argument("--batch-precision", default="bf16x9", choices=["fp64", "fp32", "tf32x3", "bf16x9"],
                    help="slice precision of the uneven batch")
    ap.add_argument("--sub-batches", type=int, default=0, help="forked streams per batch (0 = library default)")
    ap.add_argument("--slice-groups", type=int, default=0, help="FP32 slice kernel column groups (0 = default)")
    ap.add_argument("--sub-priorities", type=int, default=-1, help="descending sub-batch stream priorities (1/0)")
    ap.add_argument("--qr-cluster", type=int, default=0, help="CTAs per field of the QR (0 = automatic, 1, 2, 4)")
    ap.add_argument("--dense-slices", action="store_true", help="FP64 mode: dense exp(-dtau K) slice products")
    ap.add_argument("--qr-panel", type=int, default=0, help="QR panel width 16 or 32 (0 = default)")
    ap.add_argument("--qr-path", type=int, default=-1, help="0 = QR trailing updates on the tensor cores, 1 = FP64")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "slmc":
        args.warmup = 3
    if args.workload is None:
        args.workload = "holstein_12x12_L120" if args.mode == "dqmc" else "holstein_16x16_L160"
    if args.probe:
        import torch
        print(json.dumps(probe_rates(torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0"))))), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "dqmc":
        return run_dqmc(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
