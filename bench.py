"""Benchmark of the free-space LGF Poisson solve on one GB300 (replicas when --gpus N > 1).

Workload (the headline configuration): single-level vector Poisson (3 components) for the
streamfunction of a Gaussian-core vortex ring, R = 1, sigma = 0.2 R, h = R/32, 96x96x48 cells in
16^3 blocks (108 blocks; source blocks are those with max|omega| >= 1e-6 max, all 108 here).
A step is one complete ``lgf_poisson_solve`` (forward block transforms, per-frequency block-pair sum,
inverse transforms) with inputs resident in HBM; the one-off LGF table is built before timing.

Reported: Mcells/s of the mixed (double-float, DF32) path, whose error against the FP64 CPU oracle
is checked outside the timed region (<= 1e-10 relative L-infinity), next to the FP64 path; the
roofline of the dominant kernel; the CPU oracle (zero-padded FP64 FFT convolution) on the host
cores; and an end-to-end number through the C ABI with host buffers.

``--impl reference`` times the CPU oracle itself (the reference arm of this comparison).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poisson-solve Mcells/s, mixed vs FP64 at rel err ≤1e-10; % of HBM roofline"
WORKLOAD = "vortex-ring vector Poisson, R=1, sigma=0.2R, h=R/32, 96x96x48 cells, 16^3 blocks, 3 comps"
FP32_INST_PEAK = 152 * 128 * 2.070e9  # FP32 lanes x SMs x max SM clock (instructions/s)
FP64_FLOP_PEAK = 1.25e12              # nominal dense FP64 of GB300
DF_OPS_PER_CMAC = 54                  # FP32 instructions of one renormalised double-float complex multiply-add


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(vals, world, device=None):
    """Element-wise maximum of per-rank values (step times) over the replicas of the job, on whatever
    process group is initialised (NCCL on the GPU machine, gloo in the CPU tests); unchanged on one rank."""
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replica_rate(units_per_rank, ms, world):
    """Whole-job throughput in M units/s of `world` replicas that each process `units_per_rank` units per
    step, a step taking `ms` milliseconds (the maximum over ranks)."""
    return units_per_rank * world / (ms * 1e-3) / 1e6


def _replicas_init(world, local):
    """Process group of the replicas (torchrun, one rank per GPU) for the barrier and the max over ranks."""
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl")
        dist.barrier()


def _replicas_done(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"lgf_clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


MODE_NAMES = {1: "pair", 2: "box"}
PHASE_NAMES = ("restrict", "correction", "forward", "mac", "inverse", "interp", "residual", "heat")


def _phases(ph):
    return {n: float(v) for n, v in zip(PHASE_NAMES, ph) if v}


CADD, CNORM, CMUL, CMUL_W8, DFMUL, RFMA, DOT2, DFADD = 16, 6, 38, 24, 7, 12, 24, 14  # FP32 instructions of the
# double-float operations (common.cuh): lazy complex add, renormalisation of a complex value, complex
# product, product by W_8 or W_8^3 (two lazy sums, two lazy real products), product by a real
# power-of-two-free constant, real multiply-add, real two-term dot product with accumulation,
# renormalised real add (+ renormalisation)


def _fwd_pass_inst(nb, lines, B3, both):
    """Conjugate-pair forward block-index DFT of nb inputs to P = 2 nb outputs (k_bdft_fwd): the j = 0
    term initialises the accumulators, slots q = 0 and q = nb are sums, the nb - 1 general pairs take
    four real multiply-adds per input; `both`: store X_k and X_{P-k} (False: the Hermitian half)."""
    per = (nb - 1) * (2 * CADD + (nb - 1) * 4 * RFMA)
    per += 2 * CNORM + (nb - 1) * (2 if both else 1) * 2 * DFADD
    return lines * B3 * per


def _inv_pass_inst(nb, lines, B3, real):
    """Conjugate-pair inverse of P = 2 nb inputs to nb outputs (k_bdft_inv): X_0 +- X_{P/2} per output,
    then per general input pair U, V (two complex adds) and a two-term real dot product per output part
    (one part for a real field; a sum for output 0)."""
    per = nb * CADD + (nb - 1) * (2 * CADD + CADD + (nb - 1) * (1 if real else 2) * DOT2) + nb * CNORM
    return lines * B3 * per


def df_box_instructions(B, nb, ncomp):
    """FP32 instructions the double-float block-index FFT mode executes per solve, counted from the
    arithmetic of the kernels (not measured): the six block-index DFT passes (k_bdft_fwd / k_bdft_inv)
    and the fused local-FFT kernel (k_box_mid).  Components ride two per complex field; an odd last
    component is a real field kept on the Hermitian half K1x <= Px/2."""
    import math
    nx, ny, nz = nb
    px, py, pz = 2 * nx, 2 * ny, 2 * nz
    B3 = B ** 3
    lg = int(math.log2(B))
    # radix-2 FFT of B points: twiddled butterflies except W = 1 and W = -i (an exact swap); W = W_8 and
    # W_8^3 take two sums and two real products (CMUL_W8), the others a complex product
    def _tw(cls):
        return sum(sum(1 for j in range(1, ln // 2) if cls(j * (64 // ln))) * (B // ln)
                   for ln in [2 ** s for s in range(1, lg + 1)])
    w8 = _tw(lambda k: k in (8, 24))
    general = _tw(lambda k: k not in (8, 16, 24))
    fft1d = general * CMUL + w8 * CMUL_W8 + (B // 2) * lg * 2 * CADD  # lazily added; no renormalisation
    mid_block = 6 * B * B * fft1d + 2 * B3 * CMUL + B3 * 2 * DFMUL  # one twiddle product per cell each way
    dft = mid = 0
    fields = [px] * (ncomp // 2) + [px // 2 + 1] * (ncomp % 2)
    for pxu in fields:
        real = pxu < px
        dft += _fwd_pass_inst(nx, ny * nz, B3, not real)      # forward x
        dft += _fwd_pass_inst(ny, pxu * nz, B3, True)         # forward y
        dft += _fwd_pass_inst(nz, pxu * py, B3, True)         # forward z
        dft += _inv_pass_inst(nz, pxu * py, B3, False)        # inverse z
        dft += _inv_pass_inst(ny, pxu * nz, B3, False)        # inverse y
        dft += _inv_pass_inst(nx, ny * nz, B3, real)          # inverse x
        mid += pxu * py * pz * mid_block
    return dft, mid


# DRAM bytes (read + write) of one k_box_mid<df,16> launch on this workload, from one ncu capture of
# the current kernel (131.22 MB read + 29.95 MB written; set to None when the kernel changes)
MID_DF16_TRAFFIC = 161.17e6


def _alu_entry(kern, inst, ms, launches, traffic=None):
    ach = inst / (ms * 1e-3)
    return {"kernel": kern, "bound": "alu", "achieved": ach / 1e12, "peak": FP32_INST_PEAK / 1e12,
            "unit": "T FP32-inst/s", "frac": ach / FP32_INST_PEAK, "traffic": traffic,
            "launches_per_step": launches, "kernel_ms_per_step": float(ms),
            "note": "algorithmic FP32 instructions of the double-float arithmetic per step / CUDA-event time"
                    " of the kernel on its stream; peak = 152 SMs x 128 FP32 lanes x 2070 MHz (derived, not"
                    " measured); traffic = ncu DRAM read + write bytes of one launch"}


def roofline_entry(case, B, ncomp, rep, ph):
    """Roofline of the dominant kernel of the DF32 solve (FP32-pipe bound), and of the second kernel class."""
    W = (2 * B) ** 2 * (B + 1)
    if rep.mac_mode_used == 1:  # pair
        inst = rep.pairs * W * ncomp * DF_OPS_PER_CMAC
        return _alu_entry("k_mac_pair<df,4,3> (block-pair multiply-accumulate)", inst, ph[3], 1), None
    nz, ny, nx = (n // B for n in case["shape"])
    dft, local = df_box_instructions(B, (nx, ny, nz), ncomp)
    mid = _alu_entry("k_box_mid<df,16> (twiddle + local FFT + kernel + inverse, all fields)", local, ph[3], 1,
                     MID_DF16_TRAFFIC if (B, nx, ny, nz, ncomp) == (16, 6, 6, 3, 3) else None)
    passes = _alu_entry("k_bdft_fwd/inv<df,16> (six block-index DFT passes)", dft, ph[2] + ph[4], 6)
    return mid, passes


def build_case():
    import lgf_synth as S
    case = S.single_level_ring()
    src = {tuple(b) for b in case["src_blocks"]}
    roles = np.array([2 + (1 if tuple(b) in src else 0) for b in case["blocks"]], np.uint8)
    return case, roles


def cpu_oracle_step(case):
    """The oracle's FFT convolution of the full workload (FP64, host cores)."""
    import oracle
    return oracle.solve_box_fft(case["box"], case["h"])


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    import oracle
    case, _ = build_case()
    cells = int(np.prod(case["shape"]))
    for _ in range(args.warmup):
        cpu_oracle_step(case)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_oracle_step(case)
    dt = (time.perf_counter() - t0) / args.steps
    val = cells / dt / 1e6
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mcells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": cells, "ncomp": 3},
            "cpu_baseline": {"value": val, "unit": "Mcells/s", "cores": cores, "kind": "oracle",
                             "sample": "full workload: zero-padded FP64 FFT convolution (scipy/numpy pocketfft)",
                             "threads_used": oracle.num_threads()},
            "e2e": {"value": val, "unit": "Mcells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_line(L, torch, dev, steps, warmup):
    """Batched RK3 stage (config 5): 64 uneven ring instances (1-3 levels, finest boxes 32..192 cells),
    each stage one Poisson solve and one integrating-factor apply per instance in DF32, three chained
    stages captured in one CUDA graph.  value = Poisson target cells of all instances per stage / stage time
    (inputs ~1.7 GB, larger than L2, so no flush)."""
    import lgf_synth as S
    params = S.batch_instances(64, B=16)
    inst = [S.ring_instance(p, B=16, n_ext=16) for p in params]
    table = L.lgf_table_create(16, (14, 14, 14), L.LGF_TBL_BOX_ONLY)
    meshes = [L.Mesh(mh["levels"], 16, mh["h0"], n_ext=16) for mh, _, _ in inst]
    fs = [torch.from_numpy(np.concatenate(f, axis=1)).to(dev) for _, f, _ in inst]
    phis = [torch.zeros_like(f) for f in fs]
    gs = [torch.zeros_like(f) for f in fs]
    tmps = [torch.zeros_like(f) for f in fs]
    cells = 0
    for mh, _, _ in inst:
        n = [len(b) for b in mh["levels"]] + [0]
        cells += sum((n[k] - n[k + 1] // 8) * 16 ** 3 for k in range(len(n) - 1))
    b = L.Batch(table, meshes, 3, L.LGF_F64, alpha=[0.1] * 64, opts=L.make_opts(precision=L.LGF_PREC_DF32),
                nstreams=8)
    bs = torch.cuda.Stream(dev)  # graph capture needs a stream other than the legacy default one
    stream = bs.cuda_stream
    torch.cuda.synchronize()
    ptr = lambda ts: [t.data_ptr() for t in ts]
    b.graph_create(3, ptr(fs), ptr(phis), ptr(gs), ptr(tmps), stream)
    for _ in range(max(1, warmup)):
        b.graph_launch(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bs)
    for _ in range(steps):
        b.graph_launch(stream)
    e1.record(bs)
    torch.cuda.synchronize()
    ms_stage = e0.elapsed_time(e1) / (3 * steps)
    out = {"workload": "64 ring instances, R ~ U[0.5,1.5], sigma/R ~ U[0.1,0.25], 1-3 levels, 16^3 blocks, "
                       "3 components, alpha = 0.1", "instances": 64, "blocks": int(sum(m.total_blocks for m in meshes)),
           "target_cells_per_stage": int(cells), "graph_nodes": int(b.graph_nodes()), "stages_per_graph": 3,
           "ms_per_stage": ms_stage, "value": cells / (ms_stage * 1e-3) / 1e6, "unit": "Mcells/s",
           "dtype": "df32", "note": "each stage: Poisson solve + heat-kernel apply per instance"}
    b.close()
    L.lgf_table_destroy(table)
    return out


def heat_line(L, torch, dev, steps, warmup):
    """Heat-kernel (integrating-factor) apply on the composite mesh (FIF-AMR, Sec. 3.5) in DF32: the
    three-level ring (h = R/16, R/32, R/64; 3 components), alpha_finest = 0.1 and the per-level scaling
    alpha_k = alpha_finest 4^-(K-1-k).  value = target cells of all levels / call time, L2 flushed
    between calls.  Roofline of the separable passes + store (k_heat_line x 3 per level, k_heat_store):
    in double-float the passes are bound by the FP32 pipe (about 20 r + 10 instructions against 16 bytes
    per cell-component and pass), so the algorithmic count is per target cell-component and pass one
    product, r lazy pair sums and r multiply-adds and a renormalisation, with r per level the radius the
    library takes (the last n with e^{-2 alpha} I_n(2 alpha) >= 1e-18); the store counts nothing."""
    import lgf_synth as S
    mesh, f = S.three_level_ring()
    m = L.Mesh(mesh["levels"], mesh["B"], mesh["h0"], n_ext=mesh["n_ext"])
    ncomp = f[0].shape[0]
    ft = torch.from_numpy(np.concatenate(f, axis=1)).to(dev)
    g = torch.zeros_like(ft)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    hs = torch.cuda.Stream(dev)
    st = hs.cuda_stream

    def apply(rep=None, timing=0):
        L.lgf_heat_apply(None, m, ncomp, ft.data_ptr(), g.data_ptr(), L.LGF_F64, 0.1,
                         L.make_opts(precision=L.LGF_PREC_DF32, timing=timing), rep, st)

    ref = L.lgf_report()
    apply(ref)
    for _ in range(warmup):
        apply()
    torch.cuda.synchronize()
    evs = []
    with torch.cuda.stream(hs):
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(hs)
            apply()
            e1.record(hs)
            evs.append((e0, e1))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    ph = []
    rep = L.lgf_report()
    for _ in range(steps):
        with torch.cuda.stream(hs):
            flush.fill_(1.0)
        apply(rep, timing=1)
        ph.append([rep.ms_phase[i] for i in range(8)])
    torch.cuda.synchronize()
    ph = np.mean(np.array(ph), axis=0)
    # end to end through the C ABI: pinned host source in, result out, inside the timed region
    h_in = torch.from_numpy(np.concatenate(f, axis=1)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(hs):
        e0.record(hs)
        for _ in range(steps):
            ft.copy_(h_in, non_blocking=True)
            apply()
            h_out.copy_(g, non_blocking=True)
        e1.record(hs)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / steps
    cells = int(ref.target_cells)
    from scipy.special import ive
    K = len(mesh["levels"])
    n_blk = [len(b) for b in mesh["levels"]] + [0]
    inst = 0
    for k in range(K):
        a2 = 2 * 0.1 * 4.0 ** (-(K - 1 - k))
        r = max([n for n in range(80) if ive(n, a2) >= 1e-18] or [0])
        omega = (n_blk[k] - n_blk[k + 1] // 8) * mesh["B"] ** 3
        inst += 3 * ncomp * omega * (DFMUL + r * (CADD // 2 + RFMA) + CNORM // 2)
    ach = inst / (ph[7] * 1e-3)
    return {"workload": "three-level ring (config 3 mesh: h = R/16, R/32, R/64, 16^3 blocks), 3 components, "
                        "alpha_finest = 0.1, DF32", "blocks": int(m.total_blocks), "target_cells": cells,
            "ms_per_step": ms, "value": cells / (ms * 1e-3) / 1e6, "unit": "Mcells/s", "dtype": "df32",
            "phases_ms": {"restrict": float(ph[0]), "build": float(ph[5]), "passes_and_store": float(ph[7])},
            "gpu_launches": int(ref.kernel_launches),
            "roofline": {"kernel": "k_heat_line x 3 + k_heat_store (per level)", "bound": "alu",
                         "achieved": ach / 1e12, "peak": FP32_INST_PEAK / 1e12, "unit": "T FP32-inst/s",
                         "frac": ach / FP32_INST_PEAK, "traffic": None,
                         "note": "algorithmic FP32 instructions of the double-float passes on the target cells "
                                 "(halo cells not counted) over the library's phase time of the passes and the "
                                 "store; peak = 152 SMs x 128 FP32 lanes x 2070 MHz (derived, not measured)"},
            "e2e": {"value": cells / (e2e_ms * 1e-3) / 1e6, "unit": "Mcells/s",
                    "h2d_bytes_per_step": int(h_in.numel() * 8), "d2h_bytes_per_step": int(h_out.numel() * 8)},
            "l2": "flushed by a 256 MiB write between timed calls (outside the events)"}


def refresh_line(L, torch, dev, case, steps, warmup):
    """Velocity refresh u = -C^T L_E^{-1} omega (Sec. 4.1, Eq. (eq:vel_update)) of the ring vorticity of the
    solve workload (96 x 96 x 48 cells, 16^3 blocks, the three components as edge vorticity): the DF32
    streamfunction solve on the blocks and their -x, -y, -z neighbours (7 x 7 x 4 blocks of box) plus the
    curl kernel.  Error against the oracle's refresh (outside the timed region); value = cells / call
    time, L2 flushed between calls."""
    import oracle.refresh as OR
    B, h = case["B"], case["h"]
    cells = int(np.prod(case["shape"]))
    table = L.lgf_table_create(B, (6, 6, 3), L.LGF_TBL_BOX_ONLY)
    m = L.Mesh([case["blocks"]], B, h)
    om = torch.from_numpy(case["f"]).to(dev)
    u = torch.zeros_like(om)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    rs = torch.cuda.Stream(dev)
    opts = L.make_opts(precision=L.LGF_PREC_DF32)
    rep = L.lgf_report()

    def call(r=None):
        L.lgf_velocity_refresh(table, m, om.data_ptr(), u.data_ptr(), L.LGF_F64, opts, r, rs.cuda_stream)

    call(rep)
    torch.cuda.synchronize()
    import lgf_synth as S
    got = S.blocks_to_box(u.cpu().numpy(), case["blocks"], B, case["shape"])
    ref = OR.velocity_refresh(case["box"], h)
    err = float(max(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max() for c in range(3)))
    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    evs = []
    with torch.cuda.stream(rs):
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(rs)
            call()
            e1.record(rs)
            evs.append((e0, e1))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    L.lgf_table_destroy(table)
    return {"workload": "ring vorticity 96x96x48 cells (edge components), 16^3 blocks, DF32, box mode",
            "ms_per_step": ms, "value": cells / (ms * 1e-3) / 1e6, "unit": "Mcells/s", "rel_err": err,
            "gpu_launches": int(rep.kernel_launches), "dtype": "df32",
            "l2": "flushed by a 256 MiB write between timed calls (outside the events)"}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2010_13213_gb300.lgf as L

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case, roles = build_case()
    B = case["B"]
    cells = int(np.prod(case["shape"]))
    ncomp = 3
    mesh = L.Mesh([case["blocks"]], B, case["h"], roles=roles)
    t_tab = time.perf_counter()
    table = L.lgf_table_create(B, (5, 5, 2), L.LGF_TBL_FP64 | L.LGF_TBL_DF32 | L.LGF_TBL_FP32)
    t_tab = time.perf_counter() - t_tab
    f = torch.from_numpy(case["f"]).to(dev)
    phi = torch.zeros_like(f)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream

    mode = {"auto": L.LGF_MAC_AUTO, "pair": L.LGF_MAC_PAIR, "box": L.LGF_MAC_BOX}[args.mode]

    def solve(prec, rep=None, timing=0, fin=f, fout=phi, m=None, slices=0, st=None):
        L.lgf_poisson_solve(table, mesh, ncomp, fin.data_ptr(), fout.data_ptr(), L.LGF_F64,
                            L.make_opts(precision=prec, mac_mode=mode if m is None else m, timing=timing,
                                        dft_slices=slices), rep, stream if st is None else st)

    # accuracy outside the timed region: against the oracle (rank 0 computes, all ranks check)
    ref = cpu_oracle_step(case)
    import lgf_synth as S
    errs = {}
    for name, prec, sl in (("fp64", L.LGF_PREC_FP64, 0), ("df32", L.LGF_PREC_DF32, 0), ("fp32", L.LGF_PREC_FP32, 0),
                           ("df32_tc5", L.LGF_PREC_DF32, 5), ("df32_tc6", L.LGF_PREC_DF32, 6),
                           ("fp32_tc3", L.LGF_PREC_FP32, 3)):
        solve(prec, slices=sl)
        torch.cuda.synchronize()
        got = S.blocks_to_box(phi.cpu().numpy(), case["blocks"], B, case["shape"])
        errs[name] = float(max(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max() for c in range(2)))

    def timed(prec, m=None, slices=0):
        """Per-step device time from CUDA events recorded on the solve's stream around each solve (no
        events inside, so the kernels of a solve may overlap through programmatic dependent launch),
        then a second pass with the library's phase events for the per-kernel split."""
        for _ in range(args.warmup):
            solve(prec, m=m, slices=slices)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        evs = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)  # L2 flush between timed steps (256 MiB write), outside the events
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            solve(prec, m=m, slices=slices)
            e1.record()
            evs.append((e0, e1))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        wall = time.perf_counter() - t0
        step_ms = [a.elapsed_time(b) for a, b in evs]
        phase_ms = []
        rep = L.lgf_report()
        for _ in range(args.steps):
            flush.fill_(1.0)
            solve(prec, rep, timing=1, m=m, slices=slices)
            phase_ms.append([rep.ms_phase[i] for i in range(8)])
        torch.cuda.synchronize()
        return float(np.mean(step_ms)), np.mean(np.array(phase_ms), axis=0), wall, rep

    with ClockSampler(local) as clk:
        ms_df, ph_df, wall_df, rep_df = timed(L.LGF_PREC_DF32)
        ms_64, ph_64, wall_64, rep_64 = timed(L.LGF_PREC_FP64)
        ms_32, ph_32, wall_32, rep_32 = timed(L.LGF_PREC_FP32)
        ms_dfp, ph_dfp, _, rep_dfp = timed(L.LGF_PREC_DF32, m=L.LGF_MAC_PAIR)
        tc = {name: timed(prec, slices=sl) for name, prec, sl in
              (("df32_tc5", L.LGF_PREC_DF32, 5), ("df32_tc6", L.LGF_PREC_DF32, 6), ("fp32_tc3", L.LGF_PREC_FP32, 3))}
    clocks = clk.summary()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    h_in = torch.from_numpy(case["f"]).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_in = torch.empty_like(f)
    d_out = torch.empty_like(f)
    for _ in range(args.warmup):
        d_in.copy_(h_in, non_blocking=True)
        solve(L.LGF_PREC_DF32, fin=d_in, fout=d_out)
        h_out.copy_(d_out, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        d_in.copy_(h_in, non_blocking=True)
        solve(L.LGF_PREC_DF32, fin=d_in, fout=d_out)
        h_out.copy_(d_out, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_serial_ms = e0.elapsed_time(e1) / args.steps

    # the same with consecutive steps on two streams (each its own device buffers and library workspace):
    # a step's copies overlap the neighbouring step's solve; every step's copies stay in the timed region
    sts = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    dins, douts = [torch.empty_like(f) for _ in sts], [torch.empty_like(f) for _ in sts]
    houts = [torch.empty_like(h_in).pin_memory() for _ in sts]

    def e2e_step(k):
        i = k % 2
        with torch.cuda.stream(sts[i]):
            dins[i].copy_(h_in, non_blocking=True)
            solve(L.LGF_PREC_DF32, fin=dins[i], fout=douts[i], st=sts[i].cuda_stream)
            houts[i].copy_(douts[i], non_blocking=True)

    for k in range(args.warmup):
        e2e_step(k)
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for s_ in sts:
        s_.wait_event(e0)
    for k in range(args.steps):
        e2e_step(k)
    for s_ in sts:
        cur.wait_stream(s_)
    e1.record(cur)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps

    # every reported time is the maximum over the replicas
    tc_names = sorted(tc)
    mx = max_over_ranks([ms_df, ms_64, ms_32, ms_dfp, e2e_ms, e2e_serial_ms] + [tc[n][0] for n in tc_names], world, dev)
    ms_df, ms_64, ms_32, ms_dfp, e2e_ms, e2e_serial_ms = mx[:6]
    tc = {n: (mx[6 + i],) + tuple(tc[n][1:]) for i, n in enumerate(tc_names)}
    L.lgf_table_destroy(table)
    batch = batch_line(L, torch, dev, 5, 2) if args.batch else None
    heat = heat_line(L, torch, dev, 10, 3) if args.batch else None
    vref = refresh_line(L, torch, dev, case, 10, 3) if args.batch else None
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    roof, roof_passes = roofline_entry(case, B, ncomp, rep_df, ph_df)
    cores = os.cpu_count()
    t0 = time.perf_counter()
    cpu_oracle_step(case)
    cpu_dt = time.perf_counter() - t0
    import oracle
    line = {
        "metric": METRIC, "value": replica_rate(cells, ms_df, world), "unit": "Mcells/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_df,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "df32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": cells, "ncomp": ncomp, "blocks": int(len(case["blocks"])),
                   "mac_mode": args.mode, "parallelism": f"replicas{world}",
                   "l2": "flushed by a 256 MiB write between timed steps (outside the step events)"},
        "rel_err": errs,
        "fp64": {"value": replica_rate(cells, ms_64, world), "unit": "Mcells/s", "ms_per_step": ms_64,
                 "mode": MODE_NAMES[rep_64.mac_mode_used], "phases_ms": _phases(ph_64)},
        "fp32": {"value": replica_rate(cells, ms_32, world), "unit": "Mcells/s", "ms_per_step": ms_32,
                 "rel_err": errs["fp32"], "note": "plain FP32: error above the 1e-10 target, reported only"},
        "df32_pair_mode": {"value": replica_rate(cells, ms_dfp, world), "unit": "Mcells/s",
                           "ms_per_step": ms_dfp, "phases_ms": _phases(ph_dfp)},
        "dft_gemm": {name: {"value": replica_rate(cells, v[0], world), "unit": "Mcells/s", "ms_per_step": v[0],
                            "rel_err": errs[name], "phases_ms": _phases(v[1])} for name, v in tc.items()},
        "mode": MODE_NAMES[rep_df.mac_mode_used],
        "phases_ms_df32": _phases(ph_df),
        "table_build_s": t_tab,
        "roofline": roof,
        "roofline_second": roof_passes,
        "cpu_baseline": {"value": cells / cpu_dt / 1e6, "unit": "Mcells/s", "cores": cores, "kind": "oracle",
                         "sample": "full workload once: zero-padded FP64 FFT convolution (pocketfft)",
                         "threads_used": oracle.num_threads()},
        "e2e": {"value": replica_rate(cells, e2e_ms, world), "unit": "Mcells/s",
                "h2d_bytes_per_step": int(h_in.numel() * 8), "d2h_bytes_per_step": int(h_out.numel() * 8),
                "note": "pinned host source copied in and the result copied out every step; consecutive steps"
                        " on two streams, so a step's copies overlap the neighbouring step's solve"},
        "e2e_serial": {"value": replica_rate(cells, e2e_serial_ms, world), "unit": "Mcells/s",
                       "note": "one stream: copy in, solve, copy out, step after step"},
        "batch_rk3_stage": batch,
        "heat_apply": heat,
        "velocity_refresh": vref,
        "gpu_launches": int(rep_df.kernel_launches) * args.steps,
        "clocks": clocks,
        "wall_s_timed": {"df32": wall_df, "fp64": wall_64, "fp32": wall_32},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="auto", choices=["auto", "pair", "box"])
    ap.add_argument("--batch", default=1, type=int,
                    help="also time the 64-instance batched RK3 stage and the composite-mesh heat apply (0: skip)")
    ap.add_argument("--workload", default="ring", choices=["ring", "batch", "heat", "refresh"],
                    help="batch: only the 64-instance batched RK3 stage; heat: only the composite-mesh "
                         "heat apply; refresh: only the velocity refresh (each its own JSON line)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch_only(args)
    elif args.workload == "heat":
        run_heat_only(args)
    elif args.workload == "refresh":
        run_refresh_only(args)
    else:
        run_gpu(args)


def run_batch_only(args):
    """The batched RK3 stage alone (one replica per rank), printed by rank 0."""
    import torch
    import paper_2010_13213_gb300.lgf as L
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _replicas_init(world, local)
    out = batch_line(L, torch, dev, args.steps, args.warmup)
    ms = max_over_ranks([out["ms_per_stage"]], world, dev)[0]
    if rank == 0:
        line = {"metric": "batched RK3 stage, Poisson target Mcells/s",
                "value": replica_rate(out["target_cells_per_stage"], ms, world),
                "unit": "Mcells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "df32", "data": "synthetic", "config": out}
        print(json.dumps(line), flush=True)
    _replicas_done(world)


def run_heat_only(args):
    """The composite-mesh heat apply alone (one replica per rank), printed by rank 0."""
    import torch
    import paper_2010_13213_gb300.lgf as L
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _replicas_init(world, local)
    out = heat_line(L, torch, dev, args.steps, args.warmup)
    ms = max_over_ranks([out["ms_per_step"]], world, dev)[0]
    if rank == 0:
        line = {"metric": "heat-kernel apply (FIF-AMR), target Mcells/s",
                "value": replica_rate(out["target_cells"], ms, world),
                "unit": "Mcells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "df32", "data": "synthetic", "config": out,
                "roofline": out["roofline"], "e2e": out["e2e"], "gpu_launches": out["gpu_launches"] * args.steps}
        print(json.dumps(line), flush=True)
    _replicas_done(world)


def run_refresh_only(args):
    """The velocity refresh alone (one replica per rank), printed by rank 0."""
    import torch
    import paper_2010_13213_gb300.lgf as L
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _replicas_init(world, local)
    case, _ = build_case()
    out = refresh_line(L, torch, dev, case, args.steps, args.warmup)
    ms = max_over_ranks([out["ms_per_step"]], world, dev)[0]
    if rank == 0:
        line = {"metric": "velocity refresh u = -C^T L_E^-1 omega, Mcells/s",
                "value": replica_rate(int(np.prod(case["shape"])), ms, world), "unit": "Mcells/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "df32",
                "data": "synthetic", "config": out, "gpu_launches": out["gpu_launches"] * args.steps}
        print(json.dumps(line), flush=True)
    _replicas_done(world)


if __name__ == "__main__":
    main()
