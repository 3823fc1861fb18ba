"""Benchmark of the RPA epsilon hot path for one q-point on GB300.

One step = one eps~^-1 solve of the mixed-precision large-cell workload
(a = 30.78 bohr, 60^3 FFT grid, 12 Ry wavefunction spheres, 6 Ry epsilon
sphere with N_G = 7180, N_v = 108, N_c = 3000: K = 324,000 pairs): for each
conduction chunk of 500 bands the matrix elements (band and pair transforms,
complex64 M of 3.1 GB) and their chi contribution (split-FP16 products on the
tensor cores, FP32 segments, FP64 sum), then eps~ and its inverse (FP64-level),
all through the C ABI (bgw_mtxel, bgw_chi_sum, bgw_epsinv) on device-resident
inputs.  The e2e figure is the same solve through bgw_epsilon with host
buffers: the coefficient upload and the eps~^-1 download are inside its
timed region.  Sub-objects: the larger FP64 cell (N_G = 2120) solved in the
mixed precision and in plain FP64 on the same GPU (the metric's "vs plain
FP64 GPU" comparison), the c2 error against the FP64 oracle's seeded
256 x 256 subblock (tests/golden), and the batched, served, real-axis,
real-flavor, W/q0 and Sigma paths.

Prints ONE JSON line (rank 0).  Under torchrun each rank runs its own
independent solves (q-points are independent: replicas, weak scaling).

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on bounded samples of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import glob
import json
import math
import os
import re
import shutil
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "χ TFLOP/s & ε̃⁻¹ solves/s at ≤1e-6 rel err vs plain FP64 GPU; p50/p99 latency"
HEADLINE = "c2"
NC_CHUNK = 500   # conduction bands per chunk of the large cell (54,000 pairs, 3.1 GB of complex64 M)
WORKLOAD = ("c2: a=30.78 bohr, fft 60^3, wfn 12 Ry, eps 6 Ry (N_G=7180), N_v=108, N_c=3000 in chunks of "
            f"{NC_CHUNK}, q=(0.1,0,0)")
WORKLOAD_C1 = "c1: a=20.52 bohr, fft 40^3, wfn 12 Ry, eps 6 Ry (N_G=2120), N_v=32, N_c=800, q=(0.1,0,0)"
CONFIG = {"workload": WORKLOAD, "precision": "mix_fp16", "replicas": 1,
          "l2": "working set > L2 (3.1 GB M per chunk, 0.8 GB chi); 256 MiB flush between steps"}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def profile_traffic(tag):
    """DRAM bytes per launch of a kernel, as an ncu summary under profiles/
    records it: a line `traffic[<tag>]: <bytes> bytes per launch`.  None when
    no current capture is recorded."""
    pat = re.compile(r"traffic\[" + re.escape(tag) + r"\]:\s*([0-9.eE+]+)\s*bytes per launch")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                m = pat.search(line)
                if m:
                    return float(m.group(1))
    return None


# Slices per value of the tensor-core update in the mixed solves (the
# library's default: FP64-level updates).
UPDATE_SLICES_MIXED = 7


def oz_tiles(ng, k0):
    """128x32 tiles of the look-ahead and the bulk update launches of the
    sweep step at block k0 (the kernel's work-item decode and skips)."""
    BM, BN, NB = 128, 32, 32
    nI, nJ = (ng + BM - 1) // BM, (ng + BN - 1) // BN
    kb = min(NB, ng - k0)
    k1 = k0 + NB
    has_next = k1 < ng
    In, Jn = k1 // BM, k1 // BN

    def skip(I, J):
        i0, j0 = I * BM, J * BN
        return (j0 >= ng or (k0 <= i0 and min(i0 + BM, ng) <= k0 + kb)
                or (k0 <= j0 and min(j0 + BN, ng) <= k0 + kb))

    ahead = bulk = 0
    for I in range(nI):
        for J in range(min(4 * I + 4, nJ)):
            if skip(I, J):
                continue
            if has_next and (I == In or J == Jn):
                ahead += 1
            else:
                bulk += 1
    return ahead, bulk


# FP64 CUDA-core peak from unit counts and the maximum SM clock: 152 SMs x
# 2 FP64 FMA lanes per SM per clock (the part's 1.25 TFLOP/s FP64 rating at
# 2.07 GHz corresponds to 1.99 FMA/clk/SM) x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bgw_clocks_{os.getpid()}.csv")

    def __enter__(self):
        exe = shutil.which("nvidia-smi")
        if exe:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen([exe, f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_time(t_local: float, ws: int, device) -> float:
    """Time of the whole job of ws replicas (one process per GPU, each solving
    its own q-points): the slowest rank's time, all ranks agreeing."""
    if ws <= 1:
        return t_local
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_rate(units_per_rank: int, t_local: float, ws: int, device) -> float:
    """Whole-job throughput: the units all ranks processed / the job's time."""
    return ws * units_per_rank / replica_time(t_local, ws, device)


def mtxel_flops(s):
    """Algorithmic FP flops of the matrix elements of one solve: per pair the
    pruned product transform, 5 n log2 n per 1D line over n^2 + (2 g_x + 1) n
    + (2 g_x + 1)(2 g_y + 1) lines (g_x, g_y: the epsilon sphere's largest
    |G_x|, |G_y|), plus 6 n^3 for the product; per band the band transform,
    counted as three full passes of n^2 lines (an upper bound)."""
    n = s.fft
    gx, gy = int(np.abs(s.geps[:, 0]).max()), int(np.abs(s.geps[:, 1]).max())
    line = 5.0 * n * math.log2(n)
    per_pair = line * (n * n + (2 * gx + 1) * n + (2 * gx + 1) * (2 * gy + 1)) + 6.0 * n ** 3
    per_band = 3.0 * n * n * line
    return s.npairs * per_pair + (s.nv + s.nc) * per_band, per_pair


def flops_of(s):
    """Algorithmic flop counts of one solve (per stage)."""
    K, ng = s.npairs, s.ng
    # chi: ZGEMM-equivalent 8 N_G^2 K, Hermitian minimum 4 N_G^2 K
    return {"mtxel": mtxel_flops(s)[0],
            "chi_zgemm": 8.0 * ng * ng * K, "chi_herm": 4.0 * ng * ng * K,
            "inv": 8.0 * ng ** 3,          # general complex inverse (Gauss-Jordan / LU + solves)
            "inv_herm": 4.0 * ng ** 3}     # Hermitian positive-definite inverse (what the sweep does)


def _set_inverse_options(ctx, prec):
    from paper_1111_4429_gb300 import bgw
    # the mixed precisions invert with the tensor-core trailing update (seven
    # slices, the sweep's critical chain in double FP32), the plain path with
    # FP64 FMA, as bgw_epsilon does
    ctx.set_option(bgw.BGW_OPT_INVERSE, 0 if prec == bgw.BGW_PREC_FP64 else 1)
    ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, 0 if prec == bgw.BGW_PREC_FP64 else UPDATE_SLICES_MIXED)
    ctx.set_option(bgw.BGW_OPT_DOUBLE_FP32, 0 if prec == bgw.BGW_PREC_FP64 else 1)


def _reset_inverse_options(ctx):
    from paper_1111_4429_gb300 import bgw
    ctx.set_option(bgw.BGW_OPT_INVERSE, -1)
    ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, 0)
    ctx.set_option(bgw.BGW_OPT_DOUBLE_FP32, -1)


def _solve_steps(ctx, s, prec, steps, warmup, flush, timing, nc_chunk=None, timing_steps=None):
    """Timed one-q solves through bgw_mtxel / bgw_chi_sum per conduction chunk
    and bgw_epsinv, on a dedicated stream (capturable: repeated bgw_epsinv
    calls replay a CUDA graph).  Returns per-step stage times [steps][3] (ms:
    matrix elements, chi, inverse; summed over the chunks), the library's
    kernel-group totals per step (timing: from further steps run with
    BGW_OPT_TIMING on, which run directly), the last chi and eps~^-1 and the
    library kernel launches of the timed steps."""
    import torch
    from paper_1111_4429_gb300 import bgw
    cell = bgw.system_cell(s)
    nc_chunk = nc_chunk or s.nc
    chunks = [(c0, min(s.nc, c0 + nc_chunk)) for c0 in range(0, s.nc, nc_chunk)]
    sstream = torch.cuda.Stream()
    cv = torch.from_numpy(s.cv).cuda()
    cc = torch.from_numpy(s.cc).cuda()
    cdt = torch.complex128 if prec == bgw.BGW_PREC_FP64 else torch.complex64
    M = torch.empty((s.nv * nc_chunk, s.ng), dtype=cdt, device="cuda")
    chi = torch.empty((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    inv = torch.empty_like(chi)
    torch.cuda.synchronize()

    def step(evs=None):
        for k, (c0, c1) in enumerate(chunks):
            if evs:
                evs[k][0].record(sstream)
            ctx.mtxel(cell, s.gv, cv, s.gc, cc[c0:c1], s.geps, prec, M[:s.nv * (c1 - c0)])
            if evs:
                evs[k][1].record(sstream)
            ctx.chi_sum(cell, s.nv, c1 - c0, s.ng, M[:s.nv * (c1 - c0)], s.ev, s.ec[c0:c1], None, prec, k > 0, chi)
            if evs:
                evs[k][2].record(sstream)
        ctx.epsinv([cell], [s.geps], [chi], None, [inv])
        if evs:
            evs[-1][0].record(sstream)

    _set_inverse_options(ctx, prec)
    with torch.cuda.stream(sstream):
        for _ in range(warmup):
            step()
        ctx.sync()
        ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(len(chunks) + 1)]
              for _ in range(steps)]
        l0 = ctx.launch_count()
        for k in range(steps):
            flush.fill_(k & 0xff)       # evict L2 between steps (outside the events)
            step(ev[k])
        sstream.synchronize()
        launches = ctx.launch_count() - l0
        kt = {}
        if timing:
            nt = timing_steps or steps
            ctx.set_option(bgw.BGW_OPT_TIMING, 1)
            ctx.timing_report(reset=True)
            for k in range(nt):
                flush.fill_(k & 0xff)
                step()
            sstream.synchronize()
            kt = {k: (v[0] / nt, v[1] / nt) for k, v in ctx.timing_report(reset=True).items()}
            ctx.set_option(bgw.BGW_OPT_TIMING, 0)
    torch.cuda.synchronize()
    _reset_inverse_options(ctx)
    stage = []
    for e in ev:
        m = sum(c[0].elapsed_time(c[1]) for c in e[:-1])
        x = sum(c[1].elapsed_time(c[2]) for c in e[:-1])
        stage.append([m, x, e[-2][2].elapsed_time(e[-1][0])])
    return np.array(stage), kt, chi, inv, launches


def _roofline(s, kt, step_ms, peaks, peak_src, size_tag="c2"):
    """Roofline of the kernel group with the largest time per step (kt:
    kernel group -> (launches per step, ms per step)); size_tag names the
    workload in the profiles' traffic records."""
    per_step_ms = {k: v[1] for k, v in kt.items() if k != "inverse"}
    if "inverse" in kt and "oz_update" not in kt:
        per_step_ms["inverse"] = kt["inverse"][1]
    dom = max(per_step_ms, key=per_step_ms.get)
    fl = flops_of(s)
    bf16 = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    n_launch, ms = kt[dom]
    t_launch = ms / 1e3 / n_launch
    if dom == "chi_tc":
        # per launch: one chunk of pairs; algorithmic = the Hermitian product
        # 4 N_G^2 K (complex multiply-adds of the lower triangle, 8 flop per
        # complex multiply-add counted once per G >= G' pair ... as 4 N_G^2 K);
        # issued = the tiles' 12 real 128x128x16 MMAs per 16 pairs
        ntr = (s.ng + 127) // 128
        tiles = ntr * (ntr + 1) // 2
        kpad = (s.npairs + 31) // 32 * 32
        issued = tiles * 12 * 2.0 * 128 * 128 * kpad
        alg = fl["chi_herm"]
        roof = {"bound": "tensor", "kernel": "chi_tc_kernel (tcgen05 kind::f16 M128 N128, TMA-fed split-FP16 chi)",
                "achieved": alg / n_launch / t_launch / 1e12, "peak": bf16, "unit": "TFLOP/s",
                "algorithmic": "4 N_G^2 K flop per step (Hermitian product, lower triangle) over "
                               f"{n_launch:.0f} launches per step (chunks of pairs)",
                "peak_source": f"{peak_src} bf16 sustained (FP16 has the same nominal rate; the kernel runs inside "
                               "back-to-back solves)",
                "issued_tensor_tflops": issued / n_launch / t_launch / 1e12,
                "issued_frac_of_peak": issued / n_launch / t_launch / 1e12 / bf16,
                "zgemm_equivalent_tflops": fl["chi_zgemm"] / n_launch / t_launch / 1e12,
                "launch_ms": t_launch * 1e3,
                "traffic_tag": "chi_tc"}
    elif dom == "oz_update":
        sl = UPDATE_SLICES_MIXED
        pairs = sl * (sl + 1) // 2
        nsteps = (s.ng + 31) // 32
        bulk_tiles = sum(oz_tiles(s.ng, k0)[1] for k0 in range(0, s.ng, 32)) / nsteps
        issued = bulk_tiles * pairs * 8 * 2.0 * 128 * 32 * 16
        # FP64-equivalent: 128x32 complex elements x 32 complex multiply-adds
        # of 8 flop each per tile (the sweep's 4 N_G^3 in total)
        fp64eq = bulk_tiles * 8.0 * 128 * 32 * 32
        roof = {"bound": "tensor", "kernel": f"oz::update_pipe_kernel<{sl} slices> (tcgen05 kind::f16 M128, one MMA "
                                             "per U slice and K quarter over its V slices: the sweep's trailing "
                                             "update from exact FP16 slices)",
                "achieved": issued / t_launch / 1e12, "peak": bf16, "unit": "TFLOP/s",
                "algorithmic": f"issued tensor flops of the bulk launch: {bulk_tiles:.0f} tiles of 128x32 x "
                               f"{pairs * 8} slice-pair products of 2x128x32x16 ({sl * 8} MMAs of N = 32 (SL - a))",
                "peak_source": f"{peak_src} bf16 sustained",
                "fp64_equivalent_tflops": fp64eq / t_launch / 1e12,
                "fp64_equivalent_frac_of_fp64_pipe": fp64eq / t_launch / 1e12 / FP64_PEAK_TFLOPS,
                "fp64_pipe_peak_tflops": FP64_PEAK_TFLOPS,
                "launch_ms": t_launch * 1e3, "traffic_tag": "oz_update"}
    elif dom in ("pair_yxpass", "pair_zgather", "band_transform"):
        roof = {"bound": "alu", "kernel": f"{dom} (FP32 FFT passes of the matrix elements)",
                "achieved": fl["mtxel"] / (sum(kt[k][1] for k in ("pair_yxpass", "pair_zgather", "band_transform")
                                               if k in kt) / 1e3) / 1e12,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "algorithmic": "pruned FFT flops of all matrix-element passes per step (5 n log2 n per line)",
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz",
                "launch_ms": t_launch * 1e3, "traffic_tag": dom}
    elif dom == "chi_f64":
        roof = {"bound": "alu", "kernel": "chi_f64_kernel (FP64 FMA)",
                "achieved": fl["chi_herm"] / n_launch / t_launch / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "algorithmic": "4 N_G^2 K flop (Hermitian lower triangle)",
                "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 x 2.07 GHz", "traffic_tag": "chi_f64"}
    else:
        roof = {"bound": "alu", "kernel": dom, "achieved": None, "peak": None, "unit": "TFLOP/s"}
    if roof.get("achieved") is not None:
        roof["frac"] = roof["achieved"] / roof["peak"]
    tag = roof.pop("traffic_tag", None)
    roof["traffic"] = profile_traffic(f"{tag}_{size_tag}") if tag else None
    roof["share_of_step"] = per_step_ms[dom] / step_ms
    roof["launches_per_step"] = n_launch
    return roof


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1111_4429_gb300 import bgw, synth

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    s = synth.config_system(HEADLINE)
    ctx = bgw.Context(local)
    cell = bgw.system_cell(s)
    prec = bgw.PREC[args.prec]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    fl = flops_of(s)
    peaks, peak_src = _peaks()

    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        stage, kt, chi, inv, launches = _solve_steps(ctx, s, prec, args.steps, args.warmup, flush, timing=False,
                                                     nc_chunk=NC_CHUNK)
        wall = time.perf_counter() - t0
    if ws > 1:
        dist.barrier()
    t_total = replica_time(float(stage.sum()) / 1e3, ws, "cuda")
    mean = stage.mean(0)
    step_ms = float(stage.sum(1).mean())
    # kernel groups from a few further steps with the library's event timing
    _, kt, _, _, _ = _solve_steps(ctx, s, prec, 1, 1, flush, timing=True, nc_chunk=NC_CHUNK,
                                  timing_steps=min(3, args.steps))
    kms = {k: v[1] for k, v in kt.items()}
    roof = _roofline(s, kt, step_ms, peaks, peak_src)

    # error against the FP64 oracle: the seeded 256 x 256 principal subblock
    # of chi and eps~^-1 (tests/golden, written by a script that runs only the
    # oracle) -- the plain FP64 GPU solve of this size takes about a minute
    golden = None
    gpath = os.path.join(ROOT, "tests", "golden", "c2_oracle.npz")
    if os.path.exists(gpath) and prec != bgw.BGW_PREC_FP64:
        g = np.load(gpath)
        idx = torch.from_numpy(g["idx"]).cuda()

        def rel(a, b):
            return float(np.linalg.norm(a - b) / np.linalg.norm(b))
        golden = {"epsinv_subblock_rel_err_vs_fp64_oracle": rel(inv[0][idx][:, idx].cpu().numpy(), g["epsinv_sub"]),
                  "chi_subblock_rel_err_vs_fp64_oracle": rel(chi[0][idx][:, idx].cpu().numpy(), g["chi_sub"]),
                  "epsinv_diag_rel_err_vs_fp64_oracle": rel(torch.diagonal(inv[0]).cpu().numpy(), g["epsinv_diag"]),
                  "subblock": "256 x 256 principal, indices from the workload's subblock sub-seed"}
    del chi, inv
    torch.cuda.empty_cache()

    # end to end through bgw_epsilon with pinned host buffers, on a stream of
    # its own (repeated calls replay the library's graph of the whole path)
    cvh = torch.from_numpy(s.cv).pin_memory()
    cch = torch.from_numpy(s.cc).pin_memory()
    invh = torch.empty((1, s.ng, s.ng), dtype=torch.complex128).pin_memory()
    es = torch.cuda.Stream()
    _set_inverse_options(ctx, prec)
    torch.cuda.synchronize()
    with torch.cuda.stream(es):
        for _ in range(2):
            ctx.epsilon(cell, s.gv, cvh, s.ev, s.gc, cch, s.ec, s.geps, None, prec, NC_CHUNK, None, invh)
        e2e_steps = max(2, min(args.steps, 5))
        es.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ctx.epsilon(cell, s.gv, cvh, s.ev, s.gc, cch, s.ec, s.geps, None, prec, NC_CHUNK, None, invh)
        es.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    _reset_inverse_options(ctx)
    ctx.close()
    del cvh, cch
    torch.cuda.empty_cache()

    extra = ws == 1 and not args.skip_extra
    ctx = bgw.Context(local)
    c1 = run_c1(ctx, prec, flush, args) if ws == 1 else None
    batch = run_batch_c3(ctx, prec) if extra else None
    f2 = run_f2(ctx, prec, flush) if extra else None
    ra = run_real_axis(ctx, prec, flush) if extra else None
    rf = run_real_flavor(ctx, prec, flush) if extra else None
    sg = run_sigma(ctx, prec, flush) if extra else None
    serve = run_serve_c4(prec, nreq=args.serve_requests) if extra else None

    out = {
        "metric": METRIC,
        "value": ws * args.steps / t_total,   # = replica_rate over the ranks
        "unit": "solves/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_total * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if prec == bgw.BGW_PREC_FP64 else "c64 M + fp16x3 chi (fp32 acc, fp64 sum) + f64 inverse",
        "data": "synthetic (seeded QR-orthonormal complex Gaussian coefficients, uniform sorted energies)",
        "config": dict(CONFIG, precision=args.prec, replicas=ws),
        "chi_tflops_zgemm_eq": fl["chi_zgemm"] / (mean[1] / 1e3) / 1e12,
        "chi_tflops_hermitian": fl["chi_herm"] / (mean[1] / 1e3) / 1e12,
        "mtxel_tflops": fl["mtxel"] / (mean[0] / 1e3) / 1e12,
        "stage_ms": {"mtxel": mean[0], "chi_sum": mean[1], "epsinv": mean[2]},
        "kernel_ms_per_step": kms,
        "roofline": roof,
        "c2_vs_fp64_oracle": golden,
        "c1": c1,
        "batch_c3": batch,
        "serve_c4": serve,
        "w_and_q0": f2,
        "real_axis_c1": ra,
        "real_flavor_c1": rf,
        "sigma_cohsex_c1": sg,
        "e2e": {"value": 1.0 / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(s.cv.nbytes + s.cc.nbytes),
                "d2h_bytes_per_step": int(invh.numel() * 16)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "wall_s_timed": wall,
        "peaks_file": peak_src,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(s)
        if c1 is not None:
            out["c1"]["cpu_oracle_full_solve"] = oracle_full_c1()
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_c1(ctx, prec, flush, args, steps=5, warmup=2):
    """The larger FP64 cell (N_G = 2120, K = 25,600) in one chunk: the mixed
    solve and the plain FP64 solve of the same inputs on the same GPU (the
    metric's comparison), the eps~^-1 difference between them, and the e2e
    solve through bgw_epsilon with pinned host buffers."""
    import torch
    from paper_1111_4429_gb300 import bgw, synth
    s = synth.config_system("c1")
    fl = flops_of(s)
    st, kt, _, inv, _ = _solve_steps(ctx, s, prec, steps, warmup, flush, timing=True)
    st64, kt64, _, inv64, _ = _solve_steps(ctx, s, bgw.BGW_PREC_FP64, 2, 1, flush, timing=True)
    m, m64 = st.mean(0), st64.mean(0)
    err = float(torch.linalg.matrix_norm(inv - inv64) / torch.linalg.matrix_norm(inv64))
    peaks, peak_src = _peaks()
    roof = _roofline(s, kt, float(st.sum(1).mean()), peaks, peak_src, size_tag="c1")
    cell = bgw.system_cell(s)
    cvh = torch.from_numpy(s.cv).pin_memory()
    cch = torch.from_numpy(s.cc).pin_memory()
    invh = torch.empty((1, s.ng, s.ng), dtype=torch.complex128).pin_memory()
    es = torch.cuda.Stream()
    _set_inverse_options(ctx, prec)
    with torch.cuda.stream(es):
        for _ in range(2):
            ctx.epsilon(cell, s.gv, cvh, s.ev, s.gc, cch, s.ec, s.geps, None, prec, 0, None, invh)
        es.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            ctx.epsilon(cell, s.gv, cvh, s.ev, s.gc, cch, s.ec, s.geps, None, prec, 0, None, invh)
        es.synchronize()
        e2e_s = (time.perf_counter() - t0) / 5
    _reset_inverse_options(ctx)
    return {"workload": WORKLOAD_C1,
            "mixed": {"solves_per_s": 1e3 / float(st.sum(1).mean()),
                      "stage_ms": {"mtxel": m[0], "chi_sum": m[1], "epsinv": m[2]},
                      "chi_tflops_hermitian": fl["chi_herm"] / (m[1] / 1e3) / 1e12,
                      "kernel_ms_per_step": {k: v[1] for k, v in kt.items()}, "roofline": roof,
                      "e2e_solves_per_s": 1.0 / e2e_s},
            "plain_fp64": {"solves_per_s": 1e3 / float(st64.sum(1).mean()),
                           "stage_ms": {"mtxel": m64[0], "chi_sum": m64[1], "epsinv": m64[2]},
                           "chi_tflops_zgemm_eq": fl["chi_zgemm"] / (m64[1] / 1e3) / 1e12,
                           "chi_tflops_hermitian": fl["chi_herm"] / (m64[1] / 1e3) / 1e12,
                           "kernel_ms_per_step": {k: v[1] for k, v in kt64.items()}},
            "mixed_over_plain_fp64": float(st64.sum(1).mean() / st.sum(1).mean()),
            "epsinv_rel_err_vs_plain_fp64_gpu": err}


def run_f2(ctx, prec, flush, steps=3, warmup=2):
    """W and the q0 head on the c1 sizes.

    screened_w: bgw_screened_w over 8 matrices of the c1 epsilon sphere
    (N_G = 2120, one per frequency of an imaginary-axis grid), out of place:
    32 B of HBM traffic per element (16 read, 16 written), 1.15 GB per call,
    L2 flushed between calls.  q0_c1: bgw_epsilon on device buffers for the
    c1 sizes at q0 = (0.001, 0, 0) with k.p-shaped occupied bands, with the
    FP64 head (default at small q) and without it; the head error is taken
    against the plain FP64 GPU solve of the same input."""
    import torch
    from paper_1111_4429_gb300 import bgw, synth
    st = torch.cuda.current_stream()
    peaks, _ = _peaks()
    s1 = synth.config_system("c1")
    nm, ng = 8, s1.ng
    gen = torch.Generator(device="cuda").manual_seed(7)
    inv = torch.randn((nm, ng, ng), dtype=torch.complex128, device="cuda", generator=gen)
    w = torch.empty_like(inv)
    cells = [bgw.system_cell(s1)] * nm
    gl = [s1.geps] * nm
    ins, outs = list(inv), list(w)
    for _ in range(warmup):
        ctx.screened_w(cells, gl, ins, outs)
    ctx.sync()
    # back-to-back calls: the 1.15 GB working set is far above L2, and the
    # queue stays ahead of the GPU so host marshalling does not show
    reps = 5
    ctx.set_option(bgw.BGW_OPT_TIMING, 1)
    ctx.timing_report(reset=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(1)
    a.record(st)
    for _ in range(reps):
        ctx.screened_w(cells, gl, ins, outs)
    b.record(st)
    b.synchronize()
    kt = ctx.timing_report(reset=True)
    ctx.set_option(bgw.BGW_OPT_TIMING, 0)
    ms = a.elapsed_time(b) / reps
    kms = kt["screened_w"][1] / kt["screened_w"][0] if "screened_w" in kt else None
    bytes_ = nm * ng * ng * 32.0
    wout = {"matrices": nm, "ng": ng, "ms_per_call": ms, "ms_library_events": kms, "bytes": bytes_,
            "gbs": bytes_ / (ms / 1e3) / 1e9, "frac_of_measured_hbm": bytes_ / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
            "bound": "hbm", "launches_per_call": nm + 1}
    del inv, w

    p = dict(synth.CONFIGS["c1"])
    s = synth.q0_system("q0_c1", **p, q_frac=(1e-3, 0.0, 0.0))
    cell = bgw.system_cell(s)
    cv = torch.from_numpy(s.cv).cuda()
    cc = torch.from_numpy(s.cc).cuda()
    out = torch.empty((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")

    def solve(pr, n, nw):
        for _ in range(nw):
            ctx.epsilon(cell, s.gv, cv, s.ev, s.gc, cc, s.ec, s.geps, None, pr, 0, None, out)
        ctx.sync()
        ctx.set_option(bgw.BGW_OPT_TIMING, 1)
        ctx.timing_report(reset=True)
        tt = []
        for k in range(n):
            flush.fill_(k & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            ctx.epsilon(cell, s.gv, cv, s.ev, s.gc, cc, s.ec, s.geps, None, pr, 0, None, out)
            b.record(st)
            b.synchronize()
            tt.append(a.elapsed_time(b))
        kt = ctx.timing_report(reset=True)
        ctx.set_option(bgw.BGW_OPT_TIMING, 0)
        ctx.sync()
        return float(np.mean(tt)), {k: v[1] / v[0] for k, v in kt.items()}, out[0].clone()

    _, _, ref = solve(bgw.BGW_PREC_FP64, 1, 1)
    ms_on, k_on, inv_on = solve(prec, steps, warmup)
    ctx.set_option(bgw.BGW_OPT_HEAD, 0)
    try:
        ms_off, _, inv_off = solve(prec, steps, warmup)
    finally:
        ctx.set_option(bgw.BGW_OPT_HEAD, -1)

    def errs(x):
        return {"epsinv_rel": float(torch.linalg.matrix_norm(x - ref) / torch.linalg.matrix_norm(ref)),
                "head_rel": float(abs(x[0, 0] - ref[0, 0]) / abs(ref[0, 0]))}
    q0 = {"workload": "c1 sizes at q0 = (0.001, 0, 0) b, k.p-shaped occupied bands (N_v 32, N_c 800, N_G 2120)",
          "head_fp64": {"solves_per_s": 1e3 / ms_on, "ms": ms_on, **errs(inv_on),
                        "head_dot_ms": k_on.get("head_dot"), "head_wings_ms": k_on.get("head_wings")},
          "head_fp32": {"solves_per_s": 1e3 / ms_off, "ms": ms_off, **errs(inv_off)},
          "eps_head_00": float(1.0 / ref[0, 0].real)}
    return {"screened_w": wout, "q0_c1": q0}


def run_real_axis(ctx, prec, flush, steps=2, warmup=1):
    """Real-axis (full-frequency) solve of the c1 sizes: bgw_epsilon_real with
    device buffers, retarded, delta = 0.05 Ha, on the paper's grid with
    spacing 0.1 Ha up to 0.5 Ha, then steps growing by 0.1 Ha up to 1.5 Ha
    (9 frequencies).  One frequency of the same input through the plain FP64
    path gives the error figure."""
    import torch
    from paper_1111_4429_gb300 import bgw, synth
    st = torch.cuda.current_stream()
    s = synth.config_system("c1")
    grid = bgw.frequency_grid(0.1, 0.5, 1.5, 0.1)
    cell = bgw.system_cell(s)
    cv = torch.from_numpy(s.cv).cuda()
    cc = torch.from_numpy(s.cc).cuda()
    nf = len(grid)
    out = torch.empty((nf, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    for _ in range(warmup):
        ctx.epsilon_real(cell, s.gv, cv, s.ev, s.gc, cc, s.ec, s.geps, grid, 0.05, False, prec, 0, None, out)
    ctx.sync()
    ctx.set_option(bgw.BGW_OPT_TIMING, 1)
    ctx.timing_report(reset=True)
    tt = []
    for k in range(steps):
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        ctx.epsilon_real(cell, s.gv, cv, s.ev, s.gc, cc, s.ec, s.geps, grid, 0.05, False, prec, 0, None, out)
        b.record(st)
        b.synchronize()
        tt.append(a.elapsed_time(b))
    kt = ctx.timing_report(reset=True)
    ctx.set_option(bgw.BGW_OPT_TIMING, 0)
    ctx.sync()
    ms = float(np.mean(tt))
    one = torch.empty((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    ctx.epsilon_real(cell, s.gv, cv, s.ev, s.gc, cc, s.ec, s.geps, grid[-1:], 0.05, False, bgw.BGW_PREC_FP64, 0,
                     None, one)
    ctx.sync()
    err = float(torch.linalg.matrix_norm(out[-1] - one[0]) / torch.linalg.matrix_norm(one[0]))
    return {"workload": "c1 sizes (N_v 32, N_c 800, N_G 2120), retarded, delta 0.05 Ha, %d real frequencies "
                        "(grid: spacing 0.1, low cutoff 0.5, high cutoff 1.5, increment 0.1 Ha)" % nf,
            "frequencies": [float(x) for x in grid],
            "ms_per_call": ms, "frequency_solves_per_s": nf * 1e3 / ms,
            "kernel_ms_per_call": {k: v[1] / steps for k, v in kt.items()},
            "epsinv_rel_err_vs_plain_fp64_gpu_at_1.4Ha": err}


def run_real_flavor(ctx, prec, flush, steps=3, warmup=2):
    """Real flavor on the c1 sizes: the same spheres, bands and energies with
    real coefficients (inversion and time-reversal symmetry), one static solve
    through bgw_epsilon on device buffers; the plain FP64 real-flavor solve of
    the same input gives the error figure."""
    import torch
    from paper_1111_4429_gb300 import bgw, synth
    st = torch.cuda.current_stream()
    p = dict(synth.CONFIGS["c1"])
    s = synth.make_system("c1_real", **p, real=True)
    cell = bgw.system_cell(s)
    cv = torch.from_numpy(s.cv).cuda()
    cc = torch.from_numpy(s.cc).cuda()
    out = torch.empty((1, s.ng, s.ng), dtype=torch.float64, device="cuda")
    flav = prec | bgw.BGW_FLAVOR_REAL

    def run(pr, n, nw):
        for _ in range(nw):
            ctx.epsilon(cell, s.gv, cv, s.ev, s.gc, cc, s.ec, s.geps, None, pr, 0, None, out)
        ctx.sync()
        ctx.set_option(bgw.BGW_OPT_TIMING, 1)
        ctx.timing_report(reset=True)
        tt = []
        for k in range(n):
            flush.fill_(k & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            ctx.epsilon(cell, s.gv, cv, s.ev, s.gc, cc, s.ec, s.geps, None, pr, 0, None, out)
            b.record(st)
            b.synchronize()
            tt.append(a.elapsed_time(b))
        kt = ctx.timing_report(reset=True)
        ctx.set_option(bgw.BGW_OPT_TIMING, 0)
        ctx.sync()
        return float(np.mean(tt)), {k: v[1] / n for k, v in kt.items()}, out[0].clone()

    ms, kt, inv = run(flav, steps, warmup)
    _, _, ref = run(bgw.BGW_PREC_FP64 | bgw.BGW_FLAVOR_REAL, 1, 1)
    err = float(torch.linalg.matrix_norm(inv - ref) / torch.linalg.matrix_norm(ref))
    return {"workload": "c1 sizes with real coefficients (N_v 32, N_c 800, N_G 2120), static",
            "solves_per_s": 1e3 / ms, "ms": ms, "kernel_ms_per_solve": kt,
            "epsinv_rel_err_vs_plain_fp64_real_flavor_gpu": err}


def run_sigma(ctx, prec, flush, steps=2, warmup=1):
    """Diagonal static COHSEX / bare exchange (bgw_sigma_cohsex) on the c1
    cell: 8 outer bands at k, 832 inner bands at k - q (32 occupied), the
    N_G = 2120 eps~^-1 of the c1 solve.  The quadratic forms are one complex
    GEMM of 8 K N_G^2 flops, K = 8 x 832 pairs: FP64 in the plain path, split
    operands on the tensor cores in the mixed one.  Both are timed."""
    import torch
    from paper_1111_4429_gb300 import bgw, synth
    st = torch.cuda.current_stream()
    s = synth.config_system("c1")
    cell = bgw.system_cell(s)
    inv = torch.empty((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    ctx.epsilon(cell, s.gv, torch.from_numpy(s.cv).cuda(), s.ev, s.gc, torch.from_numpy(s.cc).cuda(), s.ec, s.geps,
                None, prec, 0, None, inv)
    ctx.sync()
    sb = synth.sigma_bands(s, 8, 832, 32, seed=2001)
    co = torch.from_numpy(sb.co).cuda()
    ci = torch.from_numpy(sb.ci).cuda()
    K = 8 * 832
    res = {"workload": "c1 cell, 8 outer x 832 inner bands (32 occupied), N_G 2120"}
    outs = {}
    for name, p in (("fp64", bgw.BGW_PREC_FP64), ("mixed", prec)):
        for _ in range(warmup):
            out = ctx.sigma_cohsex(cell, sb.go, co, sb.gi, ci, sb.nocc, s.geps, inv[0], prec=p)
        tt = []
        for k in range(steps):
            flush.fill_(k & 0xff)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            out = ctx.sigma_cohsex(cell, sb.go, co, sb.gi, ci, sb.nocc, s.geps, inv[0], prec=p)
            b.record(st)
            b.synchronize()
            tt.append(a.elapsed_time(b))
        ms = float(np.mean(tt))
        outs[name] = out
        res[name] = {"ms_per_call": ms, "quad_gemm_tflops_over_call": 8.0 * K * s.ng * s.ng / (ms / 1e3) / 1e12}
    f, m = outs["fp64"], outs["mixed"]
    res["mixed_vs_fp64_max_rel"] = float(max(np.abs(m[k] - f[k]).max() / np.abs(f[k]).max() for k in range(4)))
    res["sigma_ha"] = {"X": f[0].tolist(), "SX": f[1].tolist(), "CH": f[2].tolist(), "CH_exact": f[3].tolist()}
    return res


def run_batch_c3(ctx, prec, steps=2):
    """8 q-points of the c1 cell (q = 0.05 j, j = 1..8: uneven epsilon spheres)
    x 12 imaginary frequencies on a Gauss-Legendre grid over [0, 2] Ha, through
    bgw_epsilon_batch on a side stream: the first call runs directly and
    captures a CUDA graph, the timed calls replay it (96 solves per step)."""
    import torch
    from paper_1111_4429_gb300 import bgw, synth
    systems = synth.batched_q_systems(8)
    om = synth.gauss_legendre_frequencies(12)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        cvs = [torch.from_numpy(s.cv).cuda() for s in systems]
        ccs = [torch.from_numpy(s.cc).cuda() for s in systems]
        outs = [torch.empty((12, s.ng, s.ng), dtype=torch.complex128, device="cuda") for s in systems]
        ctx.epsilon_batch(systems, cvs, ccs, om, prec, outs, stream=st)     # direct run + capture
        st.synchronize()
        l0 = ctx.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            ctx.epsilon_batch(systems, cvs, ccs, om, prec, outs, stream=st)
        e1.record(st)
        st.synchronize()
        graph_launches = ctx.launch_count() - l0
    ms = e0.elapsed_time(e1) / steps
    # error of two (q, omega) results against the plain FP64 path
    s0 = systems[0]
    ref = torch.empty((2, s0.ng, s0.ng), dtype=torch.complex128, device="cuda")
    ctx.epsilon(bgw.system_cell(s0), s0.gv, cvs[0], s0.ev, s0.gc, ccs[0], s0.ec, s0.geps, om[[0, 11]],
                bgw.BGW_PREC_FP64, 0, None, ref)
    ctx.sync()
    err = max(float(torch.linalg.matrix_norm(outs[0][f] - ref[i]) / torch.linalg.matrix_norm(ref[i]))
              for i, f in enumerate((0, 11)))
    chi_flops = sum(12 * 8.0 * s.ng * s.ng * s.npairs for s in systems)
    gap = graph_gap_us()
    return {"workload": "c1 cell, q = (0.05 j, 0, 0) for j = 1..8, 12 Gauss-Legendre iw in [0, 2] Ha, "
                        "N_G " + "/".join(str(s.ng) for s in systems),
            "solves_per_s": 96.0 / (ms / 1e3), "ms_per_batch": ms,
            "chi_zgemm_eq_tflops_over_batch": chi_flops / (ms / 1e3) / 1e12,
            "graph_launches_per_batch": graph_launches / steps,
            "graph_us_per_dependent_launch": gap,
            "launch_overhead_share_bound": gap * 1e-3 * (graph_launches / steps) / ms,
            "epsinv_rel_err_vs_plain_fp64_gpu": err}


def graph_gap_us(n=2000, reps=5):
    """Device time per launch of a replayed CUDA graph of n dependent one-element
    kernels (each waits for the one before): what a graph adds per kernel, and
    so the most that one persistent kernel per stage could save per launch."""
    import torch
    x = torch.zeros(1, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        x.add_(1.0)
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        for _ in range(n):
            x.add_(1.0)
    with torch.cuda.stream(st):
        g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            g.replay()
        e1.record(st)
    st.synchronize()
    return e0.elapsed_time(e1) * 1e3 / (reps * n)


def run_serve_c4(prec, nreq=200, seed=1004, window=16):
    """The served stream: nreq requests (cell scale s in {1,2,3}, eps cutoff
    in {3,4,6} Ry, N_v = 4 s^3, N_c ~ U[50,1500] clamped to the conduction
    plane waves at 10 Ry; bands from one orthonormal set per scale, energies
    per request), 4 slots, 120 GB budget.  A calibration pass submits them as
    fast as a window of `window` outstanding requests allows (capacity); the
    same requests then arrive as a Poisson stream at 0.7 x capacity, each
    submitted at its arrival time.  Latency = arrival -> eps~^-1 on the host
    (the server's submit -> result, plus any lateness of the submission).
    Per request: its size, queue and run time, so the tail is attributed.
    Error: per (s, cutoff) class the request with the fewest pairs against
    the plain FP64 GPU path."""
    import torch
    from paper_1111_4429_gb300 import bgw, synth
    reqs = synth.serve_requests(200, seed)[:nreq]
    systems = synth.serve_systems(reqs, seed)
    keep = {}
    for k, r in enumerate(reqs):     # smallest request of each class: checked against plain FP64
        c = (r["s"], r["ecut_eps"])
        if c not in keep or systems[k].npairs < systems[keep[c]].npairs:
            keep[c] = k
    keep_idx = set(keep.values())
    srv = bgw.Server(bgw.Context(0), hbm_budget_bytes=120 << 30, max_slots=4, prec=prec)

    def stream(arrivals):
        n = len(systems)
        res, outs, late = [None] * n, {}, [0.0] * n
        outstanding = {}
        t0 = time.perf_counter()
        k = 0
        while k < n or outstanding:
            now = time.perf_counter() - t0
            while k < n and (arrivals[k] <= now if arrivals is not None else len(outstanding) < window):
                o = np.empty((systems[k].ng, systems[k].ng), dtype=np.complex128)
                late[k] = max(0.0, now - arrivals[k]) * 1e3 if arrivals is not None else 0.0
                outstanding[srv.submit(systems[k], o)] = (k, o)
                k += 1
                now = time.perf_counter() - t0
            progressed = False
            for t in list(outstanding):
                r = srv.poll(t, timeout_ms=0)
                if r is not None:
                    j, o = outstanding.pop(t)
                    res[j] = r
                    if j in keep_idx:
                        outs[j] = o
                    progressed = True
            if not progressed:
                time.sleep(0.0002)
        return res, outs, late, time.perf_counter() - t0

    stream(None)                                   # warm the slots' plans and tuning
    _, _, _, t_cal = stream(None)
    cap = len(systems) / t_cal
    lam = 0.7 * cap
    gen = np.random.Generator(np.random.PCG64(seed + 1))
    arrivals = np.cumsum(gen.exponential(1.0 / lam, len(systems)))
    res, outs, late, wall = stream(arrivals)
    srv.close()
    ok = all(r["status"] == 0 for r in res)
    lat = np.array([r["latency_ms"] + late[k] for k, r in enumerate(res)])
    que = np.array([r["queue_ms"] + late[k] for k, r in enumerate(res)])
    run = lat - que
    ng = np.array([s.ng for s in systems])
    K = np.array([s.npairs for s in systems])
    by_ng = {}
    for g in sorted(set(ng.tolist())):
        m = ng == g
        by_ng[str(g)] = {"requests": int(m.sum()), "p50_ms": float(np.percentile(lat[m], 50)),
                         "p99_ms": float(np.percentile(lat[m], 99)), "run_p50_ms": float(np.percentile(run[m], 50)),
                         "queue_p50_ms": float(np.percentile(que[m], 50))}
    slow = np.argsort(-lat)[:5]
    p99 = float(np.percentile(lat, 99))
    tail = lat >= p99 - 1e-9
    # the smallest request of each class against the plain FP64 GPU path
    ctx = bgw.Context(0)
    errs = {}
    for (sc, e), j in sorted(keep.items()):
        sk = systems[j]
        ref = np.zeros((1, sk.ng, sk.ng), dtype=np.complex128)
        ctx.epsilon(bgw.system_cell(sk), sk.gv, sk.cv, sk.ev, sk.gc, sk.cc, sk.ec, sk.geps, None, bgw.BGW_PREC_FP64,
                    0, None, ref)
        errs[f"s{sc}_e{e:g}"] = float(np.linalg.norm(outs[j] - ref[0]) / np.linalg.norm(ref[0]))
    ctx.close()
    return {"workload": f"{len(systems)} requests of the served stream (seed {seed}), Poisson arrivals at 0.7 x "
                        f"measured capacity, 4 slots, 120 GB budget",
            "solves_per_s": len(systems) / wall, "capacity_solves_per_s": cap, "arrival_rate_per_s": lam,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": p99,
            "queue_share_of_latency_at_p99": float(que[tail].sum() / lat[tail].sum()),
            "by_ng": by_ng,
            "slowest": [{"index": int(j), "ng": int(ng[j]), "pairs": int(K[j]), "latency_ms": float(lat[j]),
                         "queue_ms": float(que[j]), "run_ms": float(run[j])} for j in slow],
            "all_ok": ok, "epsinv_rel_err_vs_plain_fp64_gpu_per_class": errs,
            "max_epsinv_rel_err_vs_plain_fp64_gpu": max(errs.values()),
            "inputs": "bands from one orthonormal set per cell scale, energies per request"}


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_pairs(s, c0, c1):
    """The oracle's M and chi over all valence x conduction bands c0..c1-1:
    (seconds for M, seconds for chi, chi)."""
    import oracle
    t0 = time.perf_counter()
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc[c0:c1], s.geps, s.fft)
    t1 = time.perf_counter()
    x = oracle.chi(m, oracle.chi_weights(s.ev, s.ec[c0:c1]), s.omega)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, x


def _oracle_inverse(s, x):
    """The oracle's eps~ and full-size inverse (seconds)."""
    import oracle
    t0 = time.perf_counter()
    oracle.epsinv_sym(x, oracle.coulomb(s.bvec, s.q_frac, s.geps))
    return time.perf_counter() - t0


def cpu_baseline(s, nc_sample=30):
    """The FP64 oracle on the host cores, bounded: M and chi over all valence
    x nc_sample conduction bands (the pair sum is linear in the pairs, so the
    full solve's M and chi take nc / nc_sample times as long), plus the
    full-size eps~ and inverse, measured."""
    tm, tx, x = _oracle_pairs(s, 0, nc_sample)
    ti = _oracle_inverse(s, x)
    scale = s.nc / nc_sample
    full = (tm + tx) * scale + ti
    return {"value": 1.0 / full, "unit": "solves/s", "cores": _cores(), "kind": "oracle",
            "sample": f"M and chi over all {s.nv} valence x {nc_sample} of {s.nc} conduction bands "
                      f"({tm:.1f} s + {tx:.1f} s measured, x{scale:.0f} for all pairs) plus the full N_G = {s.ng} "
                      f"eps~ and inverse ({ti:.1f} s measured)",
            "stage_s_full_solve": {"mtxel": tm * scale, "chi_sum": tx * scale, "epsinv": ti}}


def oracle_full_c1():
    """One whole c1 solve by the FP64 oracle on the host cores (measured, no
    sampling)."""
    import oracle
    from paper_1111_4429_gb300 import synth
    s = synth.config_system("c1")
    t0 = time.perf_counter()
    oracle.solve(s)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "solves/s", "seconds": dt, "cores": _cores(), "kind": "oracle",
            "sample": "the whole c1 solve (M, chi, eps~, inverse), not sampled"}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, on the headline
    workload.  A whole large-cell solve takes tens of minutes on a host, so
    each step is a bounded sample: M and chi over all valence x NC_REF
    conduction bands (a different block of bands each step); the full-size
    eps~ and inverse are measured once before the steps.  ms_per_step is the
    measured time of one step; value = one solve's time built from the
    measured parts: (mean step) x N_c / NC_REF + the inverse."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_1111_4429_gb300 import synth
    NC_REF = 20
    s = synth.config_system(HEADLINE)
    blocks = [(c0, c0 + NC_REF) for c0 in range(0, s.nc - NC_REF + 1, NC_REF)]
    x = None
    for k in range(max(1, args.warmup)):
        _, _, x = _oracle_pairs(s, *blocks[k % len(blocks)])
    t_inv = _oracle_inverse(s, x)
    per = []
    t0 = time.perf_counter()
    for k in range(args.steps):
        tm, tx, _ = _oracle_pairs(s, *blocks[(k + args.warmup) % len(blocks)])
        per.append(tm + tx)
    meas = time.perf_counter() - t0
    step = float(np.mean(per))
    full = step * s.nc / NC_REF + t_inv
    val = 1.0 / full
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded QR-orthonormal complex Gaussian coefficients, uniform sorted energies)",
        "config": dict(CONFIG, precision=args.prec, replicas=ws),
        "cpu_baseline": {"value": val, "unit": "solves/s", "cores": _cores(), "kind": "oracle",
                         "sample": f"each step: M and chi over all {s.nv} valence x {NC_REF} of {s.nc} conduction "
                                   f"bands ({s.nv * NC_REF} of {s.npairs} pairs); one solve = mean step x "
                                   f"{s.nc // NC_REF} + the full N_G = {s.ng} inverse measured once "
                                   f"({t_inv:.1f} s); {meas:.1f} s of steps measured",
                         "full_solve_s": full},
        "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_profile_case(args):
    """Small cases for ncu captures (each after one warm-up call):
    solve   -- one solve of the c1 cell and spheres with N_c = 200 (K = 6400
               pairs, M = 217 MB > L2, about 1.5 GB on the device);
    general -- one pivoted general inverse (bgw_epsinv_general, tensor-core
               update) of a seeded random complex N_G = 2120 chi;
    w       -- bgw_screened_w on 8 seeded random N_G = 2120 matrices;
    sigma   -- bgw_sigma_cohsex, mixed, on the c1 cell (8 outer x 832 inner
               bands, N_G = 2120) with a seeded random Hermitian eps~^-1;
    c2      -- one solve of the large cell and spheres (60^3 grid, N_G =
               7180) with N_c = 100 (K = 10,800 pairs, M = 620 MB > L2, chi
               in chunks of 2048 pairs as at full size, the full N_G = 7180
               inverse; about 4 GB on the device);
    mtxel_c2 -- the matrix elements alone of that case (mixed precision),
               with the warp-per-pair y,x kernel that the autotuner picks on
               the 60^3 grid at full size."""
    import torch
    from paper_1111_4429_gb300 import bgw, synth
    ctx = bgw.Context(0)
    case = args.profile_case
    if case == "mtxel_c2":
        s = synth.config_system("c2", nc=100)
        cell = bgw.system_cell(s)
        prec = bgw.PREC[args.prec]
        ctx.set_option(bgw.BGW_OPT_PAIR_KERNEL, 1)
        cv = torch.from_numpy(s.cv).cuda()
        cc = torch.from_numpy(s.cc).cuda()
        M = torch.empty((s.npairs, s.ng), dtype=torch.complex128 if prec == 0 else torch.complex64, device="cuda")
        for _ in range(2):
            ctx.mtxel(cell, s.gv, cv, s.gc, cc, s.geps, prec, M)
        ctx.sync()
        desc = "c2 cell, N_c=100, matrix elements, warp-per-pair kernel"
    elif case in ("solve", "c2"):
        s = synth.config_system("c1", nc=200) if case == "solve" else synth.config_system("c2", nc=100)
        cell = bgw.system_cell(s)
        prec = bgw.PREC[args.prec]
        ctx.set_option(bgw.BGW_OPT_INVERSE, 0 if prec == bgw.BGW_PREC_FP64 else 1)
        ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, 0 if prec == bgw.BGW_PREC_FP64 else UPDATE_SLICES_MIXED)
        ctx.set_option(bgw.BGW_OPT_DOUBLE_FP32, 0 if prec == bgw.BGW_PREC_FP64 else 1)
        cv = torch.from_numpy(s.cv).cuda()
        cc = torch.from_numpy(s.cc).cuda()
        M = torch.empty((s.npairs, s.ng), dtype=torch.complex128 if prec == 0 else torch.complex64, device="cuda")
        chi = torch.empty((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
        inv = torch.empty_like(chi)
        for _ in range(2):
            ctx.mtxel(cell, s.gv, cv, s.gc, cc, s.geps, prec, M)
            ctx.chi_sum(cell, s.nv, s.nc, s.ng, M, s.ev, s.ec, None, prec, False, chi)
            ctx.epsinv([cell], [s.geps], [chi], None, [inv])
        ctx.sync()
        desc = "c1 cell, N_c=200" if case == "solve" else "c2 cell, N_c=100"
    else:
        s = synth.config_system("c1")
        ng = s.ng
        gen = torch.Generator(device="cuda").manual_seed(1)
        cell = bgw.system_cell(s)
        if case == "general":
            x = torch.randn((ng, ng), dtype=torch.complex128, device="cuda", generator=gen) * 1e-3
            inv = torch.empty_like(x)
            ctx.set_option(bgw.BGW_OPT_INVERSE, 1)
            for _ in range(2):
                ctx.epsinv_general([cell], [s.geps], [x], None, [inv])
            desc = "general inverse N_G=2120, tensor-core update"
        elif case == "sigma":
            z = torch.randn((ng, ng), dtype=torch.complex128, device="cuda", generator=gen) * 1e-2
            ei = torch.eye(ng, dtype=torch.complex128, device="cuda") + z + z.conj().T
            sb = synth.sigma_bands(s, 8, 832, 32, seed=2001)
            co = torch.from_numpy(sb.co).cuda()
            ci = torch.from_numpy(sb.ci).cuda()
            for _ in range(2):
                ctx.sigma_cohsex(cell, sb.go, co, sb.gi, ci, sb.nocc, s.geps, ei, prec=bgw.PREC[args.prec])
            desc = "Sigma COHSEX, c1 cell, 8 x 832 bands"
        else:
            x = torch.randn((8, ng, ng), dtype=torch.complex128, device="cuda", generator=gen)
            w = torch.empty_like(x)
            for _ in range(2):
                ctx.screened_w([cell] * 8, [s.geps] * 8, list(x), list(w))
            desc = "screened W, 8 x N_G=2120"
        ctx.sync()
    print(json.dumps({"profile_case": desc, "precision": args.prec, "launches": ctx.launch_count()}))


def run_item_widths(args):
    """Time the mixed-precision inverse (bgw_epsinv, tensor-core update, seven
    slices, double-FP32 chain; graph replays on a side stream, best of 3 x 5
    calls) at several N_G with the bulk update items wide (BGW_OPT_UPDATE_ITEMS
    0), of two column tiles (1) and by the default rule (-1); one JSON line per
    N_G.  The matrices are seeded chi = -1e-3 Z Z^H / N_G on prefixes of the
    60^3 cell's epsilon sphere; the three inverses are checked bit for bit."""
    import numpy as np
    import torch
    from paper_1111_4429_gb300 import bgw, synth
    s2 = synth.config_system("c2")
    cell = bgw.system_cell(s2)
    for ng in (743, 1185, 1600, 2120, 2545, 3000, 3911, 5000, 7180):
        geps = np.ascontiguousarray(s2.geps[:ng])
        gen = torch.Generator(device="cuda").manual_seed(3)
        z = torch.randn((ng, ng), dtype=torch.complex128, device="cuda", generator=gen) / np.sqrt(ng)
        chi = -(z @ z.conj().T) * 1e-3
        inv = torch.empty_like(chi)
        row = {"ng": ng}
        ref = None
        same = True
        for name, items in (("wide_ms", 0), ("narrow_ms", 1), ("rule_ms", -1)):
            ctx = bgw.Context(0)
            ctx.set_option(bgw.BGW_OPT_INVERSE, 1)
            ctx.set_option(bgw.BGW_OPT_DOUBLE_FP32, 1)
            ctx.set_option(bgw.BGW_OPT_UPDATE_ITEMS, items)
            st = torch.cuda.Stream()
            best = float("inf")
            with torch.cuda.stream(st):
                for _ in range(3):
                    ctx.epsinv([cell], [geps], [chi], None, [inv])
                st.synchronize()
                for _ in range(3):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    for _ in range(5):
                        ctx.epsinv([cell], [geps], [chi], None, [inv])
                    e1.record(st)
                    st.synchronize()
                    best = min(best, e0.elapsed_time(e1) / 5)
            h = inv.cpu().numpy()
            ref = h if ref is None else ref
            same = same and bool(np.array_equal(h, ref))
            row[name] = round(best, 3)
            ctx.close()
        row["bit_identical"] = same
        print(json.dumps(row), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", default="mix_fp16", choices=["fp64", "mix_fp16", "mix_bf16"])
    ap.add_argument("--skip-extra", action="store_true", help="skip the batched q x iw and served-stream parts")
    ap.add_argument("--serve-requests", type=int, default=200, help="requests of the served stream")
    ap.add_argument("--profile-case", nargs="?", const="solve", default=None,
                    choices=["solve", "general", "w", "sigma", "c2", "mtxel_c2"],
                    help="small case for ncu captures (solve: reduced c1 solve; general: one pivoted general "
                         "inverse; w: screened W on 8 matrices; sigma: one mixed Sigma call)")
    ap.add_argument("--item-widths", action="store_true",
                    help="time the mixed inverse at several N_G under each bulk update item width")
    args = ap.parse_args()
    if args.item_widths:
        run_item_widths(args)
    elif args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
