"""Benchmark of the pass-efficient randomized low-rank SVD on one GB300 (or N replicas).

Workload (the configuration the headline metric -- "sketch-pass GB/s vs HBM
peak; rank-k SVD time BF16 vs FP32 at equal error" -- is quoted on): block
Krylov (Alg. 9 of Bjarkason 2018) with v = 4 views of a 65536 x 16384 matrix
stored in BF16, A = U diag(j^-1.5) V^T with Haar U, V (synthetic, seeded),
target rank k = 100, oversampling p = 20.  One step is one complete
factorisation: four views of A on the tensor cores, block CholeskyQR2 after
each inner view, the Krylov-basis QR, the core SVD and the lift.  The same
matrix widened to FP32 runs the FP32 form of the identical schedule for the
BF16-versus-FP32 comparison at equal error.

value = bytes of A streamed by the step's views (4 x 2 GiB) / step time.
A (2 GiB) is larger than L2 (129 MB), so every view reads it from HBM.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun with N > 1 every rank runs the same workload on its own GPU
(replicas: the method has no cross-GPU exchange on one matrix per GPU) and
rank 0 reports the aggregate over ranks with max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, K_RANK, P_OVER, VIEWS = 65536, 16384, 100, 20, 4
METRIC = "sketch-pass GB/s (A bytes streamed by the views per factorisation / time)"
WORKLOAD = "block_krylov_v4_bf16_65536x16384_k100_p20"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            backend = os.environ.get("BENCH_BACKEND", "nccl")
            dist.init_process_group(backend=backend)
        return dist, dist.get_rank(), ws
    return None, 0, 1


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _max_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------- inputs
def make_inputs(device):
    """Seeded synthetic A (BF16, 65536 x 16384) and Omega (16384 x 120)."""
    import torch

    from paper_1804_07531_gb300 import synth
    cfg = synth.CONFIGS["krylov_65536x16384_v4"]
    r = N
    u = synth.haar_torch(M, r, cfg["seed_u"], device=device)
    v = synth.haar_torch(N, r, cfg["seed_v"], device=device)
    sig = torch.tensor(synth.sigma_config("pow15", r), dtype=torch.float32, device=device)
    a = torch.empty(M, N, dtype=torch.bfloat16, device=device)
    prev_tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    for i0 in range(0, M, 8192):
        a[i0:i0 + 8192] = ((u[i0:i0 + 8192] * sig[None, :]) @ v.t()).bfloat16()
    torch.backends.cuda.matmul.allow_tf32 = prev_tf32
    del u, v
    gen = torch.Generator(device=device)
    gen.manual_seed(cfg["seed_omega"])
    omega = torch.randn(N, K_RANK + P_OVER, generator=gen, device=device)
    torch.cuda.synchronize()
    return a, omega


def recon_error(a, u, s, v):
    """|A - U diag(s) V^T|_F in FP64 on the device (chunked, test metric only)."""
    import torch
    tot = 0.0
    vt = (v.double() * s.double()[None, :]).t()
    for i0 in range(0, a.shape[0], 4096):
        blk = a[i0:i0 + 4096].double() - u[i0:i0 + 4096].double() @ vt
        tot += float((blk * blk).sum())
    return math.sqrt(tot)


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# DRAM traffic of one view_bf16_kernel launch per algorithmic byte, from the
# ncu capture of the 16384 x 16384, ell = 120 range view (read 558.62 MB +
# write 9.47 MB against 548.67 MB algorithmic: A, the BF16 operand, Y).
# Traffic is proportional to A's size for this kernel (A is streamed once per
# launch, the thin operands stay in L2), so a full launch scales by bytes.
VIEW_TRAFFIC_PER_ALG_BYTE = (558.832128e6 + 9.545728e6) / (16384 * 16384 * 2 + 16384 * 120 * 2 + 16384 * 120 * 4)
VIEW_TRAFFIC_SOURCE = "ncu --set full capture of the 16384 x 16384 ell=120 range view, scaled by bytes"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "fallback"


# ------------------------------------------------------- dual sketch
DUAL_WIDTHS = ((32, 64), (64, 128), (120, 240))


def dual_sketch_cases(a, hbm, bf16_pk, reps=10):
    """The one-read dual sketch Y = A X, Z = A^T W (Alg. 7 steps a, b) on the
    workload's matrix: the fused kernel (each staged tile of A feeds both
    products, A read once) against two full passes, at two narrow width pairs
    and at the single-pass workload's (ell1, ell2) = (120, 240).  Kernel times
    come from the library's CUDA-event trace; call times include the operand
    conversion and output zeroing."""
    import torch

    from paper_1804_07531_gb300 import api
    from paper_1804_07531_gb300._binding import Handle
    h = Handle.get(a.device)
    m, n = a.shape
    a_bytes = a.numel() * a.element_size()
    gen = torch.Generator(device=a.device)
    gen.manual_seed(31)
    out = {}
    for ell1, ell2 in DUAL_WIDTHS:
        x = torch.randn(n, ell1, generator=gen, device=a.device)
        w = torch.randn(m, ell2, generator=gen, device=a.device)
        res = {"default": "fused" if ell2 <= 64 or (ell2 <= 128 and ell1 <= 64) else "two_pass"}
        flops = 2.0 * m * n * (ell1 + ell2)
        for name, band in (("fused", -2), ("two_pass", -1)):
            for _ in range(2):
                api.sketch(a, x, w, band_mb=band)
            torch.cuda.synchronize()
            h.set_trace(True)
            h.trace_read("view_range", reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                api.sketch(a, x, w, band_mb=band)
            e1.record()
            torch.cuda.synchronize()
            d_ms, d_n = h.trace_read("view_dual")
            r_ms, r_n = h.trace_read("view_range")
            c_ms, c_n = h.trace_read("view_corange", reset=True)
            h.set_trace(False)
            k_ms = (d_ms + r_ms + c_ms) / reps
            res[name] = {
                "ms_call": round(e0.elapsed_time(e1) / reps, 4), "ms_kernels": round(k_ms, 4),
                "kernel_launches": int((d_n + r_n + c_n) // reps), "a_reads": 1 if name == "fused" else 2,
                "a_gbs": round(a_bytes / (k_ms * 1e-3) / 1e9, 1),
                "frac_hbm": round(a_bytes / (k_ms * 1e-3) / 1e9 / hbm, 4),
                "frac_tensor": round(flops / (k_ms * 1e-3) / 1e12 / bf16_pk, 4),
            }
        out[f"ell1_{ell1}_ell2_{ell2}"] = res
    return out


# ------------------------------------------------ the other workloads
def _timed(fn, reps):
    """Median of `reps` CUDA-event timings of fn() (ms), after one warm-up call."""
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
    return statistics.median(ts)


def _tf32_peak(bf16_pk):
    """TF32 dense peak: the measured BF16 peak times the nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s)."""
    return bf16_pk * 1.1 / 2.25


def workload_c2(dev, hbm, bf16_pk, reps=5):
    """Single pass (Alg. 7) on A = U_256 diag(10^(-j/25)) V_256^T + 1e-4 N(0,1),
    20000 x 10000 FP32, k = 50, Omega 10000 x 120, Psi 20000 x 240: the dual
    sketch (FP32 form: three TF32 products per product, tensor-bound) and the
    whole factorisation."""
    import torch

    from paper_1804_07531_gb300 import api, synth
    from paper_1804_07531_gb300._binding import Handle
    cfg = synth.CONFIGS["single_pass_20000x10000"]
    m, n, r, k = cfg["m"], cfg["n"], cfg["rank"], cfg["k"]
    u = synth.haar_torch(m, r, cfg["seed_u"], device=dev)
    v = synth.haar_torch(n, r, cfg["seed_v"], device=dev)
    sig = torch.tensor(synth.sigma_config("exp25", r), dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(cfg["seed_noise"])
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    a = (u * sig) @ v.t() + cfg["noise"] * torch.randn(m, n, generator=gen, device=dev)
    torch.backends.cuda.matmul.allow_tf32 = prev
    del u, v
    om = torch.randn(n, cfg["ell1"], generator=gen, device=dev)
    ps = torch.randn(m, cfg["ell2"], generator=gen, device=dev)
    h = Handle.get(dev)
    ms_sketch = _timed(lambda: api.sketch(a, om, ps), reps)
    h.set_trace(True)
    h.trace_read("view_range", reset=True)
    api.sketch(a, om, ps)
    torch.cuda.synchronize()
    r_ms, _ = h.trace_read("view_range")
    c_ms, _ = h.trace_read("view_corange", reset=True)
    h.set_trace(False)
    ms_fact = _timed(lambda: api.single_pass(a, k, om, ps), reps)
    st = api.device_status(dev.index or 0)
    flops = 3 * 2.0 * m * n * (cfg["ell1"] + cfg["ell2"])
    k_ms = r_ms + c_ms
    a_bytes = m * n * 4
    return {
        "workload": "single_pass_f32_20000x10000_k50_l120_240", "status": st,
        "sketch_ms_call": round(ms_sketch, 4), "sketch_ms_kernels": round(k_ms, 4),
        "sketch_a_gbs": round(a_bytes / (k_ms * 1e-3) / 1e9, 1),
        "roofline": {"bound": "tensor", "dtype": "tf32x3", "achieved": round(flops / (k_ms * 1e-3) / 1e12, 1),
                     "peak": round(_tf32_peak(bf16_pk), 1), "unit": "TFLOP/s",
                     "frac": round(flops / (k_ms * 1e-3) / 1e12 / _tf32_peak(bf16_pk), 4),
                     "flops": flops, "note": "3 TF32 MMAs per product (hi*hi + hi*lo + lo*hi); peak = measured "
                                             "BF16 burst x 1.1/2.25 (nominal TF32/BF16)"},
        "factorisation_ms": round(ms_fact, 4),
    }


def workload_c3b(a, omega, reps=5):
    """Block Krylov with the row-streamed variant of Sec. 7.3 (enhanced, v = 4)
    on the workload's BF16 matrix: views 1-3 give A X and A^T (A X) each."""
    from paper_1804_07531_gb300 import api
    ms = _timed(lambda: api.block_krylov(a, K_RANK, P_OVER, VIEWS, omega, enhanced=True), reps)
    a_bytes = a.numel() * a.element_size()
    st = api.device_status(a.device.index or 0)
    return {"workload": "block_krylov_enhanced_v4_bf16_65536x16384_k100_p20", "status": st,
            "ms_per_factorisation": round(ms, 4),
            "a_reads": 7, "paper_views": VIEWS,
            "a_gbs_read": round(7 * a_bytes / (ms * 1e-3) / 1e9, 1),
            "note": "views 1-3 each read A twice (A X, then A^T (A X) by a second pass), the last once"}


def workload_c4(dev, reps=10):
    """Differentiation: Alg. 2 (v = 4, k = 32, p = 8) forward and reverse on
    A = U diag(sigma) V^T, 8192 x 4096 FP32, sigma_j = exp(-j/40) with a x0.1
    gap after j = 32; loss = sum of the top-k singular values."""
    import torch

    from oracle import algorithms as Al
    from paper_1804_07531_gb300 import api, synth
    cfg = synth.CONFIGS["grad_8192x4096_v4"]
    m, n, k, p, v = cfg["m"], cfg["n"], cfg["k"], cfg["p"], cfg["v"]
    u = synth.haar_torch(m, n, cfg["seed_u"], device=dev)
    vv = synth.haar_torch(n, n, cfg["seed_v"], device=dev)
    sig = torch.tensor(synth.sigma_config("gap32", n), dtype=torch.float32, device=dev)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    a = ((u * sig) @ vv.t()).contiguous()
    torch.backends.cuda.matmul.allow_tf32 = prev
    del u, vv
    gen = torch.Generator(device=dev)
    gen.manual_seed(cfg["seed_omega"])
    om = torch.randn(n, k + p, generator=gen, device=dev)
    ds = torch.ones(k, device=dev)
    ms_f = _timed(lambda: api.subspace_iter(a, k, p, v, om), reps)
    ms_b = _timed(lambda: api.subspace_iter_backward(a, k, p, v, om, ds), reps)
    du = torch.randn(m, k, generator=gen, device=dev)
    dv = torch.randn(n, k, generator=gen, device=dev)
    ms_buv = _timed(lambda: api.subspace_iter_backward(a, k, p, v, om, ds=ds, du=du, dv=dv), reps)
    st = api.device_status(dev.index or 0)
    a64 = a.double().cpu().numpy()
    om64 = om.double().cpu().numpy()
    t0 = time.perf_counter()
    Al.gen_subspace_iteration(a64, om64, k, v)
    t_orc = time.perf_counter() - t0
    return {"workload": "grad_subspace_v4_f32_8192x4096_k32_p8", "status": st,
            "forward_ms": round(ms_f, 4), "backward_ms": round(ms_b, 4),
            "forward_plus_backward_ms": round(ms_f + ms_b, 4),
            "backward_u_s_v_ms": round(ms_buv, 4),
            "cpu_oracle_forward_s": round(t_orc, 3), "cpu_oracle_cores": _threads()}


def _host_matrix(m, n, r, seed, dev, pc):
    """Pinned host A = U_r diag(1/j) V_r^T + 1e-5 N(0,1), m x n FP32 (U, V Haar,
    r = 1024 terms of the sigma_j = 1/j spectrum), stored as n / pc contiguous
    column panels of pc columns (a (n / pc, m, pc) tensor), built on the
    device in 4096-row blocks and copied out; None when the pinned allocation
    fails."""
    import torch

    from paper_1804_07531_gb300 import synth
    try:
        a_host = torch.empty(n // pc, m, pc, dtype=torch.float32).pin_memory()
    except RuntimeError:
        return None
    u = synth.haar_torch(m, r, seed, device=dev)
    v = synth.haar_torch(n, r, seed + 1, device=dev)
    sig = 1.0 / torch.arange(1, r + 1, device=dev, dtype=torch.float32)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed + 2)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    for i0 in range(0, m, 4096):
        blk = (u[i0:i0 + 4096] * sig) @ v.t()
        blk += 1e-5 * torch.randn(blk.shape, generator=gen, device=dev)
        for p in range(n // pc):
            a_host[p, i0:i0 + 4096].copy_(blk[:, p * pc:(p + 1) * pc])
    torch.backends.cuda.matmul.allow_tf32 = prev
    del u, v
    torch.cuda.synchronize()
    return a_host


def workload_c5(dev, sweep=True):
    """Host-streamed single pass and Alg. 2 (A in pinned host memory as 4096-column
    panels, each stored contiguously) at the largest of 262144 / 131072 / 65536
    rows x 65536 columns that can be pinned, against a plain pinned H2D copy of
    one panel measured in the same run (the host link's roof); plus the v = 1..6 accuracy sweep against the FP64
    oracle on a scaled matrix of the same family (8192 x 2048, k = 50,
    ell1 = 100, ell2 = 200, ell = 100 for v >= 2)."""
    import torch

    from paper_1804_07531_gb300 import api
    n, k, ell1, ell2, pc = 65536, 200, 400, 800, 4096
    out = {"workload": "host_stream_f32_k200_l400_800_panels4096"}
    a_host = None
    for m in (262144, 131072, 65536):
        a_host = _host_matrix(m, n, 1024, 51, dev, pc)
        if a_host is not None:
            break
    if a_host is None:
        out["unavailable"] = "no pinned host allocation of 16 GiB or more"
        return out
    a_bytes = a_host.numel() * 4
    out.update({"m": m, "n": n, "a_gib": round(a_bytes / 2 ** 30, 1), "layout": "contiguous 4096-column panels"})
    # the link: plain pinned copies of every panel (m x pc each, contiguous) into
    # one device buffer, the host-to-device traffic of one view without the
    # sketches; a single panel alone copies faster than the whole buffer does
    d = torch.empty(m, pc, device=dev)
    d.copy_(a_host[0], non_blocking=True)
    torch.cuda.synchronize()

    def copy_all():
        for i in range(a_host.shape[0]):
            d.copy_(a_host[i], non_blocking=True)

    t = _timed(copy_all, 1)
    link = a_bytes / (t * 1e-3) / 1e9
    t1 = _timed(lambda: d.copy_(a_host[0], non_blocking=True), 3)
    out["one_panel_h2d_gbs"] = round(m * pc * 4 / (t1 * 1e-3) / 1e9, 1)
    del d
    torch.cuda.empty_cache()
    out["link_h2d_gbs"] = round(link, 1)
    gen = torch.Generator(device=dev)
    gen.manual_seed(53)
    om = torch.randn(n, ell1, generator=gen, device=dev)
    ps = torch.randn(m, ell2, generator=gen, device=dev)
    for name, views, fn in (("single_pass_v1", 1, lambda: api.single_pass_host(a_host, k, om, ps)),
                            ("subspace_v2", 2, lambda: api.subspace_iter_host(a_host, k, ell1 - k, 2, om))):
        ms = _timed(fn, 1)
        gbs = views * a_bytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": round(ms, 1), "a_gbs": round(gbs, 1), "frac_of_link": round(gbs / link, 3),
                     "status": api.device_status(dev.index or 0)}
    del a_host
    if sweep:
        out["accuracy_sweep"] = _c5_sweep(dev)
    return out


def _c5_sweep(dev):
    import torch

    from oracle import algorithms as Al
    from paper_1804_07531_gb300 import api, synth
    m, n, k, l1, l2 = 8192, 2048, 50, 100, 200
    a64 = synth.usv(m, n, synth.sigma_config("inv", n), 61, 62) + 1e-5 * synth.gaussian(m, n, seed=63)
    a32 = a64.astype(np.float32)
    a = a32.astype(np.float64)
    om = synth.gaussian(n, l1, seed=64).astype(np.float32)
    ps = synth.gaussian(m, l2, seed=65).astype(np.float32)
    ah = torch.tensor(a32).pin_memory()
    tom, tps = torch.tensor(om, device=dev), torch.tensor(ps, device=dev)
    best = float(np.sqrt(np.sum(np.linalg.svd(a, compute_uv=False)[k:] ** 2)))
    rows = []
    for v in range(1, 7):
        if v == 1:
            ug, sg, vg = api.single_pass_host(ah, k, tom, tps, panel_cols=512)
            uo, so, vo = Al.single_pass(a, om.astype(np.float64), ps.astype(np.float64), k)
        else:
            ug, sg, vg = api.subspace_iter_host(ah, k, l1 - k, v, tom, panel_cols=512)
            uo, so, vo = Al.gen_subspace_iteration(a, om.astype(np.float64), k, v)
        e_g = Al.frob_error(a, ug.double().cpu().numpy(), sg.double().cpu().numpy(), vg.double().cpu().numpy())
        e_o = Al.frob_error(a, uo, so, vo)
        rows.append({"v": v, "rel_err_gpu": e_g / np.linalg.norm(a), "rel_err_oracle": e_o / np.linalg.norm(a),
                     "gpu_vs_oracle": abs(e_g - e_o) / e_o, "err_over_optimal": e_g / best})
    return {"shape": [m, n], "k": k, "ell1": l1, "ell2": l2, "panels": 512, "rows": rows}


# --------------------------------------------------------- CPU baseline
CPU_ROWS = 1024


def cpu_sample():
    """A row sample of the workload's matrix family for the FP64 oracle: the
    same n = 16384 and spectrum law (sigma_j = j^-1.5, Haar factors), 1024
    rows instead of 65536, and the same Omega shape."""
    from paper_1804_07531_gb300 import synth
    a = synth.usv(CPU_ROWS, N, synth.sigma_config("pow15", CPU_ROWS), 101, 102)
    om = synth.gaussian(N, K_RANK + P_OVER, seed=103)
    return a, om


def _threads():
    try:
        from threadpoolctl import threadpool_info
        return max(i.get("num_threads", 1) for i in threadpool_info())
    except Exception:
        return os.cpu_count()


def cpu_time_one(a, om):
    """Seconds for one FP64 oracle factorisation (Alg. 9, v = 4) of the sample."""
    from oracle import algorithms as Al
    t0 = time.perf_counter()
    Al.block_krylov(a, om, K_RANK, VIEWS)
    return time.perf_counter() - t0


def cpu_baseline(budget_s: float = 10.0):
    """The FP64 oracle's block Krylov on the row sample, scaled to the metric:
    A bytes (BF16 element size, as in the workload) streamed by the 4 views
    per second."""
    a, om = cpu_sample()
    runs, el = 0, 0.0
    while runs < 1 or (el < budget_s and runs < 3):
        el += cpu_time_one(a, om)
        runs += 1
    per = el / runs
    return {
        "value": VIEWS * CPU_ROWS * N * 2 / per / 1e9, "unit": "GB/s", "cores": _threads(), "kind": "oracle",
        "sample": f"FP64 oracle Alg. 9 (v=4, k=100, p=20) on a {CPU_ROWS} x {N} row sample of the same "
                  f"matrix family, {runs} run(s), {per:.2f} s each; bytes counted at BF16 size",
    }


# ------------------------------------------------------------ main arm
def run_ours(args):
    import torch

    from paper_1804_07531_gb300 import api
    from paper_1804_07531_gb300._binding import Handle

    dist, rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    a, omega = make_inputs(dev)
    h = Handle.get(local)
    a_bytes = a.numel() * a.element_size()
    stream = torch.cuda.current_stream()

    def step():
        return api.block_krylov(a, K_RANK, P_OVER, VIEWS, omega)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = api.device_status(local)
    if st != 0:
        raise RuntimeError(f"device status {st} after warm-up")

    # ---- timed region (device events on the launching stream)
    h.set_trace(True)
    h.trace_read("view_range", reset=True)
    launches0 = h.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        _barrier(dist)
        torch.cuda.synchronize()
        e0.record(stream)
        torch.cuda.nvtx.range_push("bench_timed")  # profiler filter for the timed launches
        for _ in range(args.steps):
            u, s, v = step()
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        torch.cuda.synchronize()
        _barrier(dist)
    launches = h.kernel_launches() - launches0
    ms_step = e0.elapsed_time(e1) / args.steps
    rng_ms, rng_n = h.trace_read("view_range")
    cor_ms, cor_n = h.trace_read("view_corange")
    orth_ms, orth_n = h.trace_read("orth")
    svd_ms, svd_n = h.trace_read("core_svd", reset=True)
    h.set_trace(False)
    ms_max = _max_over_ranks(dist, ms_step, dev)
    total_bytes = _sum_over_ranks(dist, VIEWS * a_bytes * args.steps, dev)
    value = total_bytes / (ms_max * args.steps * 1e-3) / 1e9

    # ---- the one-read dual sketch, and the enhanced block Krylov, on the same matrix
    hbm0, bf16_pk0, _ = _peaks()
    extra = rank == 0 and not args.no_extra
    dual = dual_sketch_cases(a, hbm0, bf16_pk0) if extra else None
    workloads = {"c3b": workload_c3b(a, omega)} if extra else {}

    # ---- accuracy of the BF16 form, and the FP32 form at equal error
    e_bf16 = recon_error(a, u, s, v)
    a32 = a.float()
    del a
    torch.cuda.empty_cache()
    for _ in range(1):
        api.block_krylov(a32, K_RANK, P_OVER, VIEWS, omega)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fsteps = max(1, min(3, args.steps))
    f0.record(stream)
    for _ in range(fsteps):
        u32, s32, v32 = api.block_krylov(a32, K_RANK, P_OVER, VIEWS, omega)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_fp32 = f0.elapsed_time(f1) / fsteps
    e_fp32 = recon_error(a32, u32, s32, v32)
    a = a32.bfloat16()
    del a32
    torch.cuda.empty_cache()

    # ---- end to end through the C ABI with host buffers: lr_block_krylov_host
    # copies A and Omega from pinned host memory into the device workspace,
    # factorises, and copies U, S, V back into pinned host buffers, every step
    a_host = a.cpu().pin_memory()
    om_host = torch.empty(K_RANK + P_OVER, N, dtype=torch.float32).pin_memory().t()
    om_host.copy_(omega)
    del a
    torch.cuda.empty_cache()
    e2e_steps = max(1, min(args.steps, 5))
    outs_host = (torch.empty(K_RANK, M, dtype=torch.float32).pin_memory().t(),
                 torch.empty(K_RANK, dtype=torch.float32).pin_memory(),
                 torch.empty(K_RANK, N, dtype=torch.float32).pin_memory().t())

    def e2e_step():
        res = api.block_krylov_host(a_host, K_RANK, P_OVER, VIEWS, om_host, out=outs_host)
        torch.cuda.current_stream().synchronize()
        return res

    e2e_step()
    torch.cuda.synchronize()
    _barrier(dist)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        out = e2e_step()
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    t_e2e = _max_over_ranks(dist, t_e2e, dev)
    e2e_val = _sum_over_ranks(dist, VIEWS * a_bytes, dev) / t_e2e / 1e9
    h2d = a_host.numel() * a_host.element_size() + om_host.numel() * 4
    d2h = sum(t.numel() * t.element_size() for t in out)
    e_e2e = float(np.abs(out[1].numpy() - s.cpu().numpy()).max() / float(s[0]))
    # the host link as this run sees it: one plain pinned copy of A, timed
    # with events (the e2e step cannot be faster than this plus the views
    # that follow the first)
    a_dev = torch.empty(a_host.shape, dtype=a_host.dtype, device=dev)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_dev.copy_(a_host, non_blocking=True)
    h0.record()
    a_dev.copy_(a_host, non_blocking=True)
    h1.record()
    torch.cuda.synchronize()
    a_h2d_ms = h0.elapsed_time(h1)
    del a_dev
    torch.cuda.empty_cache()
    del a_host
    if extra:
        workloads["c2"] = workload_c2(dev, hbm0, bf16_pk0)
        workloads["c4"] = workload_c4(dev)
        workloads["c5"] = workload_c5(dev)

    if rank != 0:
        return
    hbm, bf16_pk, src = _peaks()
    view_launch_ms = (rng_ms + cor_ms) / max(1, rng_n + cor_n)
    # algorithmic bytes of one view launch: A once + the thin operand (BF16) + the FP32 output
    ell_avg = (3 * (K_RANK + P_OVER) + 2 * (K_RANK + P_OVER)) / 4.0
    alg_bytes = a_bytes + (M + N) * ell_avg * (2 + 4) / 2
    achieved = alg_bytes / (view_launch_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16",
        "data": "synthetic (seeded Haar U, V; sigma_j = j^-1.5), A 2 GiB > L2 so every view reads HBM",
        "config": {
            "workload": WORKLOAD, "m": M, "n": N, "k": K_RANK, "p": P_OVER, "views": VIEWS,
            "a_dtype": "bf16", "l2": "inputs larger than L2 (no flush needed)",
            "parallelism": "replicas" if world > 1 else "single GPU",
        },
        "roofline": {
            "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": round(VIEW_TRAFFIC_PER_ALG_BYTE * alg_bytes),
            "traffic_source": VIEW_TRAFFIC_SOURCE, "alg_bytes_per_launch": round(alg_bytes),
            "kernel": "view_bf16_kernel (range + co-range views)",
            "launches_timed": rng_n + cor_n, "avg_launch_ms": round(view_launch_ms, 4),
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback 6.8 TB/s",
        },
        "breakdown_ms_per_step": {
            "views": round((rng_ms + cor_ms) / args.steps, 4),
            "orth": round(orth_ms / args.steps, 4),
            "core_svd": round(svd_ms / args.steps, 4),
        },
        "fp32_form": {
            "ms_per_step": round(ms_fp32, 3), "recon_error": e_fp32, "bf16_recon_error": e_bf16,
            "bf16_over_fp32_error": e_bf16 / e_fp32, "bf16_speedup": ms_fp32 / ms_max,
        },
        "dual_sketch": dual,
        "workloads": workloads,
        "e2e": {"value": round(e2e_val, 2), "unit": "GB/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": round(t_e2e * 1e3, 3),
                "call": "lr_block_krylov_host (pinned host A, Omega in; U, S, V out)",
                "sigma_vs_device_run": e_e2e,
                "a_h2d_ms": round(a_h2d_ms, 3), "a_h2d_gbs": round(a_bytes / (a_h2d_ms * 1e-3) / 1e9, 1)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


def run_reference(args):
    """The FP64 oracle as it stands, on the host cores, same metric and config:
    each step is one oracle factorisation of the bounded row sample."""
    dist, rank, world = _dist()
    if rank != 0:
        return
    a, om = cpu_sample()
    for _ in range(args.warmup):
        cpu_time_one(a, om)
    times = [cpu_time_one(a, om) for _ in range(args.steps)]
    per = statistics.mean(times)
    val = VIEWS * CPU_ROWS * N * 2 / per / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "m": M, "n": N, "k": K_RANK, "p": P_OVER,
                                        "views": VIEWS},
        "cpu_baseline": {"value": round(val, 4), "unit": "GB/s", "cores": _threads(), "kind": "oracle",
                         "sample": f"FP64 oracle Alg. 9 (v=4) on a {CPU_ROWS} x {N} row sample, one "
                                   f"factorisation per step; bytes counted at BF16 size"},
        "e2e": {"value": round(val, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_case(args):
    """One hot kernel on a small case, for profiler captures: `reps` calls of
    one library entry point on seeded inputs (A larger than L2 by default),
    each timed with CUDA events; prints one JSON line per case."""
    import torch

    from paper_1804_07531_gb300 import api
    from paper_1804_07531_gb300._binding import Handle
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    m, n, ell, case = args.case_m, args.case_n, args.case_ell, args.kernel_case
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    bf16 = case in ("view_range", "view_corange", "dual_bf16", "chained_bf16")
    a = torch.randn(m, n, generator=gen, device=dev)
    if bf16:
        a = a.bfloat16()
    x = torch.randn(n, ell, generator=gen, device=dev)
    w = torch.randn(m, ell, generator=gen, device=dev)
    if case in ("view_range", "view_range_f32"):
        def call():
            return api.sketch(a, x)
    elif case in ("view_corange", "view_corange_f32"):
        def call():
            return api.sketch(a, None, w)
    elif case in ("dual_bf16", "dual_f32"):
        w2 = torch.randn(m, 2 * ell, generator=gen, device=dev)

        def call():
            return api.sketch(a, x, w2, band_mb=args.case_band)
    elif case in ("chained_bf16", "chained_f32"):
        def call():
            return api.sketch_chained(a, x, band_mb=args.case_band)
    elif case == "orth":
        y = torch.randn(m, ell, generator=gen, device=dev)

        def call():
            return api.orth(y)
    elif case == "block_krylov":
        # the workload's schedule (Alg. 9, v = 4, k = 100, p = 20: a 240 x 240
        # core) on an m x n BF16 matrix with the same spectrum law
        from paper_1804_07531_gb300 import synth
        u = synth.haar_torch(m, n, 21, device=dev)
        v = synth.haar_torch(n, n, 22, device=dev)
        sig = torch.tensor(synth.sigma_config("pow15", n), dtype=torch.float32, device=dev)
        a = ((u * sig[None, :]) @ v.t()).bfloat16()
        del u, v
        om = torch.randn(n, K_RANK + P_OVER, generator=gen, device=dev)

        def call():
            return api.block_krylov(a, K_RANK, P_OVER, VIEWS, om)
    else:
        raise ValueError(case)
    call()
    torch.cuda.synchronize()
    h = Handle.get(0)
    times = []
    for _ in range(args.case_reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    st = h.status()
    if st != 0:
        raise RuntimeError(f"device status {st}")
    ms = statistics.median(times)
    a_bytes = a.numel() * a.element_size()
    print(json.dumps({"case": case, "band_mb": args.case_band, "m": m, "n": n, "ell": ell,
                      "a_dtype": str(a.dtype).split(".")[-1],
                      "ms_median": round(ms, 4), "a_gbs": round(a_bytes / (ms * 1e-3) / 1e9, 1),
                      "reps": args.case_reps}), flush=True)


def run_host_case(args):
    """Host-streamed views (A in pinned host memory, streamed in 4096-column
    panels) against the host link's own roof, measured in the same run as a
    plain pinned copy of A: Alg. 7 (one view, k = 200, ell1 = 400, ell2 = 800)
    and Alg. 2 with v = 2 and 3 (every view streams A once).  A is a seeded
    synthetic m x n FP32 matrix (sigma_j = 1/j on a 200-dimensional part plus
    1e-5 Gaussian noise), built on the device and copied to the host."""
    import torch

    from paper_1804_07531_gb300 import api, synth
    synth._preload_torch_linalg()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    m, n, k, ell1, ell2, pc = args.case_m, args.case_n, 200, 400, 800, 4096
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    r = 200
    u = torch.linalg.qr(torch.randn(m, r, generator=gen, device=dev))[0]
    v = torch.linalg.qr(torch.randn(n, r, generator=gen, device=dev))[0]
    sig = 1.0 / torch.arange(1, r + 1, device=dev, dtype=torch.float32)
    a_host = torch.empty(m, n, dtype=torch.float32).pin_memory()
    for i0 in range(0, m, 4096):
        blk = (u[i0:i0 + 4096] * sig) @ v.t()
        blk += 1e-5 * torch.randn(blk.shape, generator=gen, device=dev)
        a_host[i0:i0 + 4096].copy_(blk)
    del u, v
    torch.cuda.synchronize()
    a_bytes = a_host.numel() * 4
    # the link's roof: a plain pinned host-to-device copy of A
    d = torch.empty_like(a_host, device=dev)
    d.copy_(a_host, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    d.copy_(a_host, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    link = a_bytes / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del d
    torch.cuda.empty_cache()
    om = torch.randn(n, ell1, generator=gen, device=dev)
    ps = torch.randn(m, ell2, generator=gen, device=dev)
    out = {"case": "host_stream", "m": m, "n": n, "a_gib": round(a_bytes / 2 ** 30, 2), "panel_cols": pc,
           "link_h2d_gbs": round(link, 1)}
    runs = [("single_pass_v1", 1, lambda: api.single_pass_host(a_host, k, om, ps, panel_cols=pc))]
    for vv in (2, 3):
        runs.append((f"subspace_v{vv}", vv,
                     lambda vv=vv: api.subspace_iter_host(a_host, k, ell1 - k, vv, om, panel_cols=pc)))
    for name, views, fn in runs:
        fn()
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        gbs = views * a_bytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": round(ms, 2), "a_gbs": round(gbs, 1), "frac_of_link": round(gbs / link, 3)}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the dual-sketch comparison and the other workloads (C2, C3b, C4, C5)")
    ap.add_argument("--kernel-case", default=None,
                    choices=["view_range", "view_corange", "view_range_f32", "view_corange_f32", "dual_bf16",
                             "dual_f32", "chained_bf16", "chained_f32", "orth", "block_krylov", "host_stream"],
                    help="time one entry point on a small case (profiling) instead of the workload")
    ap.add_argument("--case-m", type=int, default=16384)
    ap.add_argument("--case-n", type=int, default=16384)
    ap.add_argument("--case-ell", type=int, default=120)
    ap.add_argument("--case-reps", type=int, default=3)
    ap.add_argument("--case-band", type=int, default=0,
                    help="opts.band_mb for the dual/chained cases: 0 fused one-read kernel where available, "
                         "-1 two full passes, > 0 L2 bands of that many MiB")
    args = ap.parse_args()
    if args.kernel_case == "host_stream":
        run_host_case(args)
    elif args.kernel_case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
