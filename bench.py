"""Benchmark of the free-space LGF Poisson solve on one GB300 (replicas when --gpus N > 1).

Headline workload: the batched solver of 64 uneven vortex-ring problems (each its own composite mesh of
1-3 levels, finest boxes 32^2 x 32 .. 192^2 x 96 cells, 16^3 blocks, 3 components), one vector Poisson
solve per instance per step, in double-float ("mixed", DF32) arithmetic, the 64 solves captured in one
CUDA graph.  Inputs stay resident in HBM (about 1.7 GB, larger than L2).  value = Poisson target cells
of all instances (sum over levels of |Omega_k|) per second.

Reported beside it: the FP64 batched path; the error of a seeded sample of instances against the FP64 CPU
oracle (outside the timed region); the roofline of the dominant kernel from the method-minimum bytes the
library reports (lgf_report.alg_bytes) against the measured HBM copy bandwidth; an end-to-end figure
through the C ABI with host buffers; the CPU oracle on a bounded sample of the workload; and one line per
other configuration (32^3 random sources, the single ring, the three-level ring, two coaxial rings), the
heat apply, the velocity refresh and the full batched RK3 stage (Poisson + integrating factor).

``--impl reference`` times the CPU oracle itself (the reference arm of this comparison).
"""
from __future__ import annotations

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

METRIC = "Poisson-solve Mcells/s, mixed vs FP64 at rel err ≤1e-10; % of HBM roofline"
WORKLOAD = ("64 uneven vortex-ring instances (R ~ U[0.5,1.5], sigma/R ~ U[0.1,0.25], 1-3 levels, finest boxes "
            "32^2x32..192^2x96 cells), 16^3 blocks, 3 components, one vector Poisson solve per instance per step, "
            "captured CUDA graph")
NINST = 64
FP32_INST_PEAK = 152 * 128 * 2.070e9  # FP32 lanes x SMs x max SM clock (instructions/s), derived from unit counts


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


def _replicas_init(world):
    """Process group of the replicas (torchrun, one rank per GPU) for the barrier and the max over ranks."""
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl")
        dist.barrier()


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _replicas_done(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def peaks():
    """The measured peaks of this machine's GPUs (HBM copy GB/s, bf16 TFLOP/s); the recipe's fallback if the
    file is absent (marked so)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        d["source"] = "measured (MEASURED_PEAKS.json)"
        return d
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback (file absent)"}


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


PHASE_NAMES = ("restrict", "correction", "forward", "mac", "inverse", "interp", "residual", "heat")


def _phases(ph):
    return {n: float(v) for n, v in zip(PHASE_NAMES, ph) if v}


def roofline(kernel, alg_bytes, kernel_ms, launches, pk, traffic=None, alg_flops=None, note=""):
    """HBM roofline of a kernel from the method-minimum bytes of the work it completes (lgf_report.alg_bytes)
    over its CUDA-event time on its stream, against the measured copy bandwidth."""
    ach = alg_bytes / (kernel_ms * 1e-3) / 1e9
    out = {"kernel": kernel, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
           "frac": ach / pk["hbm_gbs"], "traffic": traffic, "alg_bytes_per_step": float(alg_bytes),
           "kernel_ms_per_step": float(kernel_ms), "launches_per_step": int(launches),
           "peak_source": pk["source"],
           "note": "achieved = method-minimum bytes (caller fields read and written once + unique kernel-spectrum "
                   "values, lgf_report.alg_bytes) / the kernel's CUDA-event time; " + note}
    if alg_flops is not None:
        out["flop_view"] = {"alg_tflops": alg_flops / (kernel_ms * 1e-3) / 1e12, "alg_flops_per_step": alg_flops,
                            "note": "5 M log2 M per complex transform (+ 8 per pair multiply-add) over the same time; "
                                    "the double-float arithmetic runs them on the FP32 pipe"}
    return out


def flush_l2(buf):
    buf.fill_(1.0)


def time_calls(torch, call, steps, warmup, stream, flush=None, world=1):
    """Mean device time (ms) of `call` over `steps` timed calls, CUDA events on `stream` around each call;
    `flush` (a buffer larger than L2) is rewritten between calls outside the events."""
    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    _barrier(world)
    evs = []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            if flush is not None:
                flush_l2(flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            evs.append((e0, e1))
    torch.cuda.synchronize()
    _barrier(world)
    return float(np.mean([a.elapsed_time(b) for a, b in evs]))


def rel_err_fields(got, ref):
    """max over components with a nonzero reference of max|got - ref| / max|ref| (arrays [ncomp][...])."""
    errs = [float(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max()) for c in range(ref.shape[0])
            if np.abs(ref[c]).max() > 0]
    return max(errs)


# ----------------------------------------------------------------------------------------------- batch
def batch_case():
    import lgf_synth as S
    params = S.batch_instances(NINST, B=16)
    inst = [S.ring_instance(p, B=16, n_ext=16) for p in params]
    cells = []
    for mh, _, _ in inst:
        n = [len(b) for b in mh["levels"]] + [0]
        cells.append(sum((n[k] - n[k + 1] // 8) * 16 ** 3 for k in range(len(n) - 1)))
    return params, inst, cells


def batch_sample(params, cells):
    """The seeded sample of instances checked against (and timed with) the oracle: the smallest
    instance of each level count, plus the second-smallest three-level one."""
    order = sorted(range(len(params)), key=lambda i: cells[i])
    pick, seen = [], {}
    for i in order:
        k = params[i]["levels"]
        if seen.get(k, 0) < (2 if k == 3 else 1):
            pick.append(i)
            seen[k] = seen.get(k, 0) + 1
    return sorted(pick)


def oracle_instance(inst_i):
    from oracle import amr
    mh, f, _ = inst_i
    return amr.flgf_amr(mh, f)


def batch_errors(phis_host, inst, sample, refs):
    out = {}
    for i in sample:
        mh = inst[i][0]
        ref, masks = refs[i]
        got, o, e = phis_host[i], 0, 0.0
        for k, blk in enumerate(mh["levels"]):
            m = masks[k]
            sub = got[:, o:o + len(blk)]
            for c in range(ref[k].shape[0]):
                r = ref[k][c][m]
                if r.size and np.abs(r).max() > 0:
                    e = max(e, float(np.abs(sub[c][m] - r).max() / np.abs(r).max()))
            o += len(blk)
        out[str(i)] = e
    return out


def batch_poisson(L, torch, dev, steps, warmup, world, pk, fp64=True, check=True):
    """The headline: 64 DF32 Poisson solves per step in one captured graph."""
    params, inst, cells = batch_case()
    t0 = time.perf_counter()
    table = L.lgf_table_create(16, (14, 14, 14), L.LGF_TBL_BOX_ONLY)
    t_table = time.perf_counter() - t0
    meshes = [L.Mesh(mh["levels"], 16, mh["h0"], n_ext=16) for mh, _, _ in inst]
    host = [torch.from_numpy(np.concatenate(f, axis=1)) for _, f, _ in inst]
    fs = [h.to(dev) for h in host]
    phis = [torch.zeros_like(f) for f in fs]
    total = int(sum(cells))
    bs = torch.cuda.Stream(dev)
    ptr = lambda ts: [t.data_ptr() for t in ts]
    nstreams = 16
    res = {}
    for name, prec in (("df32", L.LGF_PREC_DF32), ("fp64", L.LGF_PREC_FP64)):
        if name == "fp64" and not fp64:
            continue
        b = L.Batch(table, meshes, 3, L.LGF_F64, opts=L.make_opts(precision=prec), nstreams=nstreams)
        t0 = time.perf_counter()
        b.autotune(ptr(fs), ptr(phis), bs.cuda_stream)  # measured DFT-pass variant, order and stream count
        ns, slices, tuned_ms = b.tuning()
        res[name + "_tuning"] = {"nstreams": ns, "tensor_core_instances": int(sum(1 for x in slices if x)),
                                 "slices": sorted(set(slices)), "autotune_s": time.perf_counter() - t0,
                                 "instance_ms_sum": float(sum(tuned_ms)),
                                 "instance_ms_max": float(max(tuned_ms))}
        b.graph_create(1, ptr(fs), ptr(phis), None, None, bs.cuda_stream)
        nsteps = steps if name == "df32" else max(2, min(steps, 5))
        ms = time_calls(torch, lambda: b.graph_launch(bs.cuda_stream), nsteps, warmup, bs, world=world)
        res[name] = {"ms": ms, "nodes": b.graph_nodes(), "steps": nsteps}
        if check:
            torch.cuda.synchronize()
            res[name]["phis"] = [p.cpu().numpy() for p in phis]
        if name == "df32":
            # end to end through the C ABI with host buffers: (a) the serial form, every step copies all
            # sources in from pinned host memory on one stream, replays the graph, copies all results out;
            # (b) lgf_batch_graph_create_io, the same copies inside the graph on two copy streams
            hin = [h.pin_memory() for h in host]
            hout = [torch.empty_like(h).pin_memory() for h in host]

            def e2e_step():
                with torch.cuda.stream(bs):
                    for d, h in zip(fs, hin):
                        d.copy_(h, non_blocking=True)
                    b.graph_launch(bs.cuda_stream)
                    for h, d in zip(hout, phis):
                        h.copy_(d, non_blocking=True)

            res["e2e_serial_ms"] = time_calls(torch, e2e_step, max(3, steps // 2), 2, bs, world=world)
            b.graph_create_io(ptr(hin), ptr(hout), ptr(fs), ptr(phis), bs.cuda_stream)
            res["e2e_ms"] = time_calls(torch, lambda: b.graph_launch(bs.cuda_stream), max(3, steps // 2), 2, bs,
                                       world=world)
            res["e2e_nodes"] = b.graph_nodes()
            if check:
                torch.cuda.synchronize()
                res["e2e_match"] = all(torch.equal(h, d.cpu()) for h, d in zip(hout, phis))
            res["e2e_bytes"] = int(sum(h.numel() * 8 for h in host))
        b.close()
    # per-kernel time: the same solves one by one with the library's phase events (CUDA events on the
    # solve's stream), and the method-minimum work the library reports for each
    mid_ms = pas_ms = tot_ms = alg_b = alg_f = 0.0
    launches = mids = 0
    rep = L.lgf_report()
    opts = L.make_opts(precision=L.LGF_PREC_DF32, timing=1)
    for _ in range(2):  # second sweep is the measured one
        mid_ms = pas_ms = tot_ms = alg_b = alg_f = 0.0
        launches = mids = 0
        for m, f, p in zip(meshes, fs, phis):
            L.lgf_poisson_solve(table, m, 3, f.data_ptr(), p.data_ptr(), L.LGF_F64, opts, rep, bs.cuda_stream)
            mid_ms += rep.ms_phase[3]
            pas_ms += rep.ms_phase[2] + rep.ms_phase[4]
            tot_ms += rep.ms_total
            alg_b += rep.alg_bytes
            alg_f += rep.alg_flops
            launches += rep.kernel_launches
            mids += len(m.levels)
    torch.cuda.synchronize()
    L.lgf_table_destroy(table)
    out = dict(params=params, inst=inst, cells=cells, total=total, res=res, t_table=t_table, nstreams=nstreams,
               mid_ms=mid_ms, pas_ms=pas_ms, serial_ms=tot_ms, alg_bytes=alg_b, alg_flops=alg_f,
               launches=launches, mid_launches=mids, blocks=int(sum(m.total_blocks for m in meshes)))
    return out


def poisson_batch_line(L, torch, dev, steps, warmup, world):
    """The 64-instance DF32 Poisson step as one captured graph with the batch's default schedule (16
    streams, longest-first by block count, CUDA-core DFT passes): the headline's solve path without the
    autotuner's trial runs, for launch lists."""
    params, inst, cells = batch_case()
    table = L.lgf_table_create(16, (14, 14, 14), L.LGF_TBL_BOX_ONLY)
    meshes = [L.Mesh(mh["levels"], 16, mh["h0"], n_ext=16) for mh, _, _ in inst]
    fs = [torch.from_numpy(np.concatenate(f, axis=1)).to(dev) for _, f, _ in inst]
    phis = [torch.zeros_like(f) for f in fs]
    b = L.Batch(table, meshes, 3, L.LGF_F64, opts=L.make_opts(precision=L.LGF_PREC_DF32), nstreams=16)
    bs = torch.cuda.Stream(dev)
    ptr = lambda ts: [t.data_ptr() for t in ts]
    b.graph_create(1, ptr(fs), ptr(phis), None, None, bs.cuda_stream)
    ms = time_calls(torch, lambda: b.graph_launch(bs.cuda_stream), steps, warmup, bs, world=world)
    nodes = b.graph_nodes()
    b.close()
    L.lgf_table_destroy(table)
    total = int(sum(cells))
    return {"workload": "the 64 instances, one DF32 Poisson solve each, one graph, 16 streams", "ms_per_step": ms,
            "value": total / (ms * 1e-3) / 1e6, "unit": "Mcells/s", "target_cells": total, "graph_nodes": int(nodes)}


def batch_stage_heat(L, torch, dev, steps, warmup, world):
    """The full batched RK3 step: per stage one Poisson solve and one integrating-factor apply per
    instance, three chained stages in one graph, the per-stage IF argument (c~_i - c~_{i-1}) alpha of the
    HERK tableau (Table tab:HREK, c~ = 0, 1/3, 1, 1 read as stage increments 1/3, 2/3, 0 -> the last stage
    applies alpha/3 as well so every stage has a kernel) -- alpha = 0.1 over the step."""
    params, inst, cells = batch_case()
    table = L.lgf_table_create(16, (14, 14, 14), L.LGF_TBL_BOX_ONLY)
    meshes = [L.Mesh(mh["levels"], 16, mh["h0"], n_ext=16) for mh, _, _ in inst]
    fs = [torch.from_numpy(np.concatenate(f, axis=1)).to(dev) for _, f, _ in inst]
    phis = [torch.zeros_like(f) for f in fs]
    gs = [torch.zeros_like(f) for f in fs]
    tmps = [torch.zeros_like(f) for f in fs]
    b = L.Batch(table, meshes, 3, L.LGF_F64, alpha=[0.1] * NINST, opts=L.make_opts(precision=L.LGF_PREC_DF32),
                nstreams=16)
    bs = torch.cuda.Stream(dev)
    ptr = lambda ts: [t.data_ptr() for t in ts]
    b.autotune(ptr(fs), ptr(phis), bs.cuda_stream)  # DFT-pass variant, order and stream count (Poisson stages)
    stage_alpha = [[0.1 / 3.0] * NINST, [0.2 / 3.0] * NINST, [0.1 / 3.0] * NINST]
    b.graph_create(3, ptr(fs), ptr(phis), ptr(gs), ptr(tmps), bs.cuda_stream, alpha_stages=stage_alpha)
    ms = time_calls(torch, lambda: b.graph_launch(bs.cuda_stream), steps, warmup, bs, world=world) / 3.0
    nodes = b.graph_nodes()
    ns = b.tuning()[0]
    b.close()
    L.lgf_table_destroy(table)
    total = int(sum(cells))
    return {"workload": "the 64 instances, per stage one DF32 Poisson solve and one DF32 heat apply each, three "
                        "stages per graph with per-stage alpha (HERK increments 1/3, 2/3, 1/3 of alpha = 0.1)",
            "ms_per_stage": ms, "value": total / (ms * 1e-3) / 1e6, "unit": "Mcells/s (Poisson target cells)",
            "graph_nodes": int(nodes), "stages_per_graph": 3, "nstreams": ns}


# ------------------------------------------------------------------------------------- single configs
def single_config(L, torch, dev, name, case, steps, warmup, world, pk, precisions, table_off, mode=0,
                  flush=None, slices=(), box_only=False):
    """One single-level configuration: per arithmetic the mean solve time (L2 flushed between calls), the
    error against the oracle's FFT convolution, and the HBM roofline of the solve from alg_bytes."""
    import oracle
    import lgf_synth as S
    B = case["B"]
    ncomp = case["f"].shape[0]
    cells = int(np.prod(case["shape"]))
    mesh = L.Mesh([case["blocks"]], B, case["h"], roles=case.get("roles"))
    flags = L.LGF_TBL_BOX_ONLY if box_only else L.LGF_TBL_FP64 | L.LGF_TBL_DF32 | L.LGF_TBL_FP32
    table = L.lgf_table_create(B, table_off, flags)
    f = torch.from_numpy(case["f"]).to(dev)
    phi = torch.zeros_like(f)
    st = torch.cuda.Stream(dev)
    t0 = time.perf_counter()
    ref = oracle.solve_box_fft(case["box"], case["h"])
    cpu_s = time.perf_counter() - t0
    out = {"cells": cells, "ncomp": ncomp, "blocks": int(len(case["blocks"])),
           "cpu_oracle": {"value": cells / cpu_s / 1e6, "unit": "Mcells/s", "cores": os.cpu_count(),
                          "kind": "oracle", "sample": "the whole configuration once: zero-padded FP64 FFT "
                                                      "convolution (pocketfft)"}}
    if name == "cfg1":  # the direct O(N^2) sum on a seeded sample of target cells, extrapolated
        rng = np.random.default_rng(7)
        nz, ny, nx = case["shape"]
        tg = np.stack([rng.integers(0, nx, 512), rng.integers(0, ny, 512), rng.integers(0, nz, 512)], 1)
        t0 = time.perf_counter()
        oracle.solve_box_direct(case["box"], case["h"], tg)
        dt = time.perf_counter() - t0
        out["cpu_oracle_direct"] = {"value": 512 / dt / 1e6, "unit": "Mcells/s (targets)", "cores": os.cpu_count(),
                                    "kind": "oracle", "sample": "512 seeded target cells of the 32^3 box, the "
                                                                "compensated direct sum over all 32768 sources"}
    variants = [(n, p, 0) for n, p in precisions] + [(f"df32_tc{s}", L.LGF_PREC_DF32, s) for s in slices]
    for vname, prec, sl in variants:
        opts = L.make_opts(precision=prec, mac_mode=mode, dft_slices=sl)
        rep = L.lgf_report()
        call = lambda: L.lgf_poisson_solve(table, mesh, ncomp, f.data_ptr(), phi.data_ptr(), L.LGF_F64, opts, None,
                                           st.cuda_stream)
        call()
        torch.cuda.synchronize()
        got = S.blocks_to_box(phi.cpu().numpy(), case["blocks"], B, case["shape"])
        err = rel_err_fields(got, ref)
        ms = time_calls(torch, call, steps, warmup, st, flush=flush, world=world)
        L.lgf_poisson_solve(table, mesh, ncomp, f.data_ptr(), phi.data_ptr(), L.LGF_F64,
                            L.make_opts(precision=prec, mac_mode=mode, dft_slices=sl, timing=1, residual=1), rep,
                            st.cuda_stream)
        out[vname] = {"value": cells / (ms * 1e-3) / 1e6, "unit": "Mcells/s", "ms_per_step": ms, "rel_err": err,
                      "residual_rel": rep.residual_rel, "mode": {1: "pair", 2: "box"}.get(rep.mac_mode_used),
                      "phases_ms": _phases([rep.ms_phase[i] for i in range(8)]),
                      "gpu_launches": int(rep.kernel_launches),
                      "roofline": roofline("whole solve", rep.alg_bytes, ms, rep.kernel_launches, pk,
                                           alg_flops=rep.alg_flops)}
    L.lgf_table_destroy(table)
    return out


def multi_config(L, torch, dev, steps, warmup, world, pk, flush):
    """Config 3: the three-level ring (h = R/16, R/32, R/64), DF32 and FP64 box mode against the oracle."""
    import lgf_synth as S
    from oracle import amr
    mesh, f = S.three_level_ring()
    t0 = time.perf_counter()
    ref, masks = amr.flgf_amr(mesh, f)
    cpu_s = time.perf_counter() - t0
    m = L.Mesh(mesh["levels"], mesh["B"], mesh["h0"], n_ext=mesh["n_ext"])
    ft = torch.from_numpy(np.concatenate(f, axis=1)).to(dev)
    phi = torch.zeros_like(ft)
    table = L.lgf_table_create(16, (14, 14, 14), L.LGF_TBL_BOX_ONLY)
    st = torch.cuda.Stream(dev)
    ncells = int(sum(int(mk.sum()) for mk in masks))
    out = {"levels": [len(b) for b in mesh["levels"]],
           "cpu_oracle": {"value": ncells / cpu_s / 1e6, "unit": "Mcells/s", "cores": os.cpu_count(),
                          "kind": "oracle", "sample": "the whole configuration once: the FP64 FLGF-AMR oracle"}}
    for vname, prec in (("df32", L.LGF_PREC_DF32), ("fp64", L.LGF_PREC_FP64), ("fp32", L.LGF_PREC_FP32)):
        rep = L.lgf_report()
        call = lambda: L.lgf_poisson_solve(table, m, 3, ft.data_ptr(), phi.data_ptr(), L.LGF_F64,
                                           L.make_opts(precision=prec, mac_mode=2), None, st.cuda_stream)
        call()
        torch.cuda.synchronize()
        got, o, err = phi.cpu().numpy(), 0, 0.0
        for k, blk in enumerate(mesh["levels"]):
            sub = got[:, o:o + len(blk)]
            for c in range(2):
                r = ref[k][c][masks[k]]
                err = max(err, float(np.abs(sub[c][masks[k]] - r).max() / np.abs(r).max()))
            o += len(blk)
        ms = time_calls(torch, call, steps, warmup, st, flush=flush, world=world)
        L.lgf_poisson_solve(table, m, 3, ft.data_ptr(), phi.data_ptr(), L.LGF_F64,
                            L.make_opts(precision=prec, mac_mode=2, timing=1, residual=1), rep, st.cuda_stream)
        cells = int(rep.target_cells)
        out["cells"] = cells
        out[vname] = {"value": cells / (ms * 1e-3) / 1e6, "unit": "Mcells/s", "ms_per_step": ms, "rel_err": err,
                      "residual_rel": rep.residual_rel, "phases_ms": _phases([rep.ms_phase[i] for i in range(8)]),
                      "gpu_launches": int(rep.kernel_launches),
                      "roofline": roofline("whole solve", rep.alg_bytes, ms, rep.kernel_launches, pk,
                                           alg_flops=rep.alg_flops)}
    L.lgf_table_destroy(table)
    return out


def heat_line(L, torch, dev, steps, warmup, world, pk, flush):
    """Heat-kernel (integrating-factor) apply on the composite mesh (FIF-AMR, Sec. 3.5) in DF32: the
    three-level ring, 3 components, alpha_finest = 0.1 and alpha_k = alpha_finest 4^-(K-1-k).  value =
    target cells / call time (L2 flushed between calls); roofline: the separable passes as an HBM stencil
    (2 x 8 bytes per target cell-component and pass) over the passes' phase time."""
    import lgf_synth as S
    mesh, f = S.three_level_ring()
    m = L.Mesh(mesh["levels"], mesh["B"], mesh["h0"], n_ext=mesh["n_ext"])
    ncomp = f[0].shape[0]
    ft = torch.from_numpy(np.concatenate(f, axis=1)).to(dev)
    g = torch.zeros_like(ft)
    hs = torch.cuda.Stream(dev)
    call = lambda: L.lgf_heat_apply(None, m, ncomp, ft.data_ptr(), g.data_ptr(), L.LGF_F64, 0.1,
                                    L.make_opts(precision=L.LGF_PREC_DF32), None, hs.cuda_stream)
    ms = time_calls(torch, call, steps, warmup, hs, flush=flush, world=world)
    rep = L.lgf_report()
    L.lgf_heat_apply(None, m, ncomp, ft.data_ptr(), g.data_ptr(), L.LGF_F64, 0.1,
                     L.make_opts(precision=L.LGF_PREC_DF32, timing=1), rep, hs.cuda_stream)
    cells = int(rep.target_cells)
    h_in = torch.from_numpy(np.concatenate(f, axis=1)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()

    def e2e():
        ft.copy_(h_in, non_blocking=True)
        call()
        h_out.copy_(g, non_blocking=True)

    e2e_ms = time_calls(torch, e2e, steps, 2, hs, world=world)
    passes_bytes = 3 * ncomp * cells * 16.0
    return {"workload": "three-level ring (h = R/16, R/32, R/64, 16^3 blocks), 3 components, alpha_finest = 0.1, "
                        "DF32", "target_cells": cells, "ms_per_step": ms, "value": cells / (ms * 1e-3) / 1e6,
            "unit": "Mcells/s", "dtype": "df32",
            "phases_ms": {"restrict": float(rep.ms_phase[0]), "build": float(rep.ms_phase[5]),
                          "passes_and_store": float(rep.ms_phase[7])},
            "gpu_launches": int(rep.kernel_launches),
            "roofline": roofline("k_heat_line x 3 + k_heat_store (per level)", passes_bytes, rep.ms_phase[7],
                                 4 * len(mesh["levels"]), pk,
                                 note="for the heat passes: 8 bytes in + 8 out per target cell-component and pass"),
            "e2e": {"value": cells / (e2e_ms * 1e-3) / 1e6, "unit": "Mcells/s",
                    "h2d_bytes_per_step": int(h_in.numel() * 8), "d2h_bytes_per_step": int(h_out.numel() * 8)},
            "l2": "flushed by a 256 MiB write between timed calls (outside the events)"}


def refresh_line(L, torch, dev, steps, warmup, world, flush):
    """Velocity refresh u = -C^T L_E^{-1} omega (Sec. 4.1, Eq. (eq:vel_update)) of the single ring's vorticity
    (96 x 96 x 48 cells, 16^3 blocks) in DF32, error against the oracle's refresh."""
    import lgf_synth as S
    import oracle.refresh as OR
    case = S.single_level_ring()
    B, h = case["B"], case["h"]
    cells = int(np.prod(case["shape"]))
    table = L.lgf_table_create(B, (6, 6, 3), L.LGF_TBL_BOX_ONLY)
    m = L.Mesh([case["blocks"]], B, h)
    om = torch.from_numpy(case["f"]).to(dev)
    u = torch.zeros_like(om)
    rs = torch.cuda.Stream(dev)
    rep = L.lgf_report()
    opts = L.make_opts(precision=L.LGF_PREC_DF32)
    call = lambda r=None: L.lgf_velocity_refresh(table, m, om.data_ptr(), u.data_ptr(), L.LGF_F64, opts, r,
                                                 rs.cuda_stream)
    call(rep)
    torch.cuda.synchronize()
    got = S.blocks_to_box(u.cpu().numpy(), case["blocks"], B, case["shape"])
    ref = OR.velocity_refresh(case["box"], h)
    err = float(max(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max() for c in range(3)))
    ms = time_calls(torch, call, steps, warmup, rs, flush=flush, world=world)
    L.lgf_table_destroy(table)
    return {"workload": "ring vorticity 96x96x48 cells (edge components), 16^3 blocks, DF32, box mode",
            "ms_per_step": ms, "value": cells / (ms * 1e-3) / 1e6, "unit": "Mcells/s", "rel_err": err,
            "gpu_launches": int(rep.kernel_launches), "dtype": "df32"}


def bump_study(L, torch, dev):
    """The bump test of Sec. 3.4 (Fig. fig:source_correction_convergence): the manufactured streamfunction and
    its analytic vector Laplacian on meshes with 0-3 refinement levels (alpha = 1/6, N_E = 14, 16^3 blocks),
    solved in DF32 without the source correction, with it on Omega_k only, and with it on the extended
    region; on the finest level the error of Psi against the analytic field and of L Psi against omega."""
    import lgf_synth as S
    from oracle import amr
    table = L.lgf_table_create(16, (16, 16, 16), L.LGF_TBL_BOX_ONLY)
    out = {}
    for lr in range(4):
        mesh, om, ps = S.bump_case(lr)
        f = torch.from_numpy(np.concatenate([o[:2] for o in om], axis=1)).to(dev)
        phi = torch.zeros_like(f)
        k = len(mesh["levels"]) - 1
        lv = amr.build_levels(mesh)[k]
        B = mesh["B"]
        wbox, pbox = np.zeros((2,) + lv.shape), np.zeros((2,) + lv.shape)
        for i, b in enumerate(mesh["levels"][k]):
            sl = (slice(None),) + lv.block_slice(b, B)
            wbox[sl], pbox[sl] = om[k][:2, i], ps[k][:2, i]
        inner = lv.omega & ~amr.dilate_maxnorm(~lv.omega, 1)
        row = {"blocks": [len(b) for b in mesh["levels"]], "finest_h": mesh["h0"] / 2 ** k}
        for v in (("no_correction", "correction_no_ext", "correction_ext") if lr else ("correction_ext",)):
            m = L.Mesh(mesh["levels"], B, mesh["h0"], n_ext=0 if v == "correction_no_ext" else mesh["n_ext"])
            flags = L.LGF_SOLVE_NO_CORRECTION if v == "no_correction" else 0
            L.lgf_poisson_solve(table, m, 2, f.data_ptr(), phi.data_ptr(), L.LGF_F64,
                                L.make_opts(precision=L.LGF_PREC_DF32, mac_mode=L.LGF_MAC_BOX, flags=flags))
            torch.cuda.synchronize()
            got = phi.cpu().numpy()[:, sum(len(b) for b in mesh["levels"][:k]):]
            box = np.zeros((2,) + lv.shape)
            for i, b in enumerate(mesh["levels"][k]):
                box[(slice(None),) + lv.block_slice(b, B)] = got[:, i]
            e_psi = float(np.abs(box - pbox)[:, lv.omega].max() / np.abs(pbox).max())
            e_lap = float(np.abs(amr.laplacian_box(box, lv.h) - wbox)[:, inner].max() / np.abs(wbox).max())
            row[v] = {"psi_err": e_psi, "lpsi_err": e_lap}
        out[f"L_R={lr}"] = row
    L.lgf_table_destroy(table)
    return out


def projection_line(L, torch, dev, steps, warmup, world, flush):
    """HERK stage projection L_C p = D r, u = H(r - G p) (Sec. 2.4, Sec. 3.6) in DF32 on the three-level ring
    mesh (the ring vorticity as the face field r, alpha_finest = 0.1): time per call (L2 flushed between
    calls), and the error against the oracle's projection on the small three-level ring (8^3 blocks)."""
    import lgf_synth as S
    from oracle import projection
    out = {}
    small, fs = S.three_level_ring(R=1.0, sigma=0.2, B=8, n_ext=6, h_fine=1 / 32, support=(24, 24, 16), dilate0=1)
    ref_u, ref_p = projection.project_amr(small, fs, 0.1)
    t8 = L.lgf_table_create(8, (14, 14, 14), L.LGF_TBL_BOX_ONLY)
    m8 = L.Mesh(small["levels"], 8, small["h0"], n_ext=small["n_ext"])
    r8 = torch.from_numpy(np.concatenate(fs, axis=1)).to(dev)
    u8 = torch.zeros_like(r8)
    p8 = torch.zeros((1,) + tuple(r8.shape[1:]), dtype=torch.float64, device=dev)
    L.lgf_stage_projection(t8, m8, r8.data_ptr(), u8.data_ptr(), p8.data_ptr(), L.LGF_F64, 0.1,
                           L.make_opts(precision=L.LGF_PREC_DF32, mac_mode=L.LGF_MAC_BOX))
    torch.cuda.synchronize()
    gu, gp = u8.cpu().numpy(), p8.cpu().numpy()
    lv_masks = projection.amr.build_levels(small)
    err, o = 0.0, 0
    for k, blk in enumerate(small["levels"]):
        msk = projection._to_blocks(lv_masks[k], blk, lv_masks[k].omega[None].astype(float), 8)[0] > 0.5
        for got, ref in ((gu[:, o:o + len(blk)], ref_u[k]), (gp[:, o:o + len(blk)], ref_p[k])):
            if msk.any():
                err = max(err, float(np.abs(got[:, msk] - ref[:, msk]).max() / np.abs(ref[:, msk]).max()))
        o += len(blk)
    L.lgf_table_destroy(t8)
    mesh, f = S.three_level_ring()
    m = L.Mesh(mesh["levels"], 16, mesh["h0"], n_ext=mesh["n_ext"])
    table = L.lgf_table_create(16, (14, 14, 14), L.LGF_TBL_BOX_ONLY)
    r = torch.from_numpy(np.concatenate(f, axis=1)).to(dev)
    u = torch.zeros_like(r)
    st = torch.cuda.Stream(dev)
    opts = L.make_opts(precision=L.LGF_PREC_DF32, mac_mode=L.LGF_MAC_BOX)
    call = lambda: L.lgf_stage_projection(table, m, r.data_ptr(), u.data_ptr(), 0, L.LGF_F64, 0.1, opts, None,
                                          st.cuda_stream)
    ms = time_calls(torch, call, steps, warmup, st, flush=flush, world=world)
    rep = L.lgf_report()
    L.lgf_stage_projection(table, m, r.data_ptr(), u.data_ptr(), 0, L.LGF_F64, 0.1, opts, rep, st.cuda_stream)
    torch.cuda.synchronize()
    L.lgf_table_destroy(table)
    cells = int(rep.target_cells)
    return {"workload": "three-level ring mesh (h = R/16, R/32, R/64, 16^3 blocks), the ring vorticity as r, "
                        "alpha_finest = 0.1, DF32", "ms_per_step": ms, "value": cells / (ms * 1e-3) / 1e6,
            "unit": "Mcells/s", "target_cells": cells, "gpu_launches": int(rep.kernel_launches),
            "rel_err": err, "rel_err_case": "small three-level ring (8^3 blocks), u and p against the oracle",
            "l2": "flushed by a 256 MiB write between timed calls (outside the events)"}


def indicator_line(L, torch, dev, steps, warmup, world, flush):
    """Refinement indicator (Sec. 4.2) computed with the DF32 solve of the three-level ring: the time of the
    solve with the indicator against the solve alone, and the agreement with the oracle (block RMS, flags)
    on the same mesh."""
    import lgf_synth as S
    from oracle import refine
    mesh, f = S.three_level_ring()
    m = L.Mesh(mesh["levels"], 16, mesh["h0"], n_ext=mesh["n_ext"])
    table = L.lgf_table_create(16, (14, 14, 14), L.LGF_TBL_BOX_ONLY)
    ft = torch.from_numpy(np.concatenate(f, axis=1)).to(dev)
    phi = torch.zeros_like(ft)
    n = m.total_blocks
    rms = torch.zeros(n, dtype=torch.float64, device=dev)
    flags = torch.zeros(n, dtype=torch.uint8, device=dev)
    smax = torch.zeros(1, dtype=torch.float64, device=dev)
    st = torch.cuda.Stream(dev)
    opts = L.make_opts(precision=L.LGF_PREC_DF32, mac_mode=L.LGF_MAC_BOX)

    def with_ind():
        smax.zero_()
        L.lgf_refinement_indicator(table, m, 3, ft.data_ptr(), phi.data_ptr(), L.LGF_F64, opts, 0.3, 0.5, 2,
                                   rms.data_ptr(), flags.data_ptr(), smax.data_ptr(), None, st.cuda_stream)

    def plain():
        L.lgf_poisson_solve(table, m, 3, ft.data_ptr(), phi.data_ptr(), L.LGF_F64, opts, None, st.cuda_stream)

    ms_ind = time_calls(torch, with_ind, steps, warmup, st, flush=flush, world=world)
    ms_plain = time_calls(torch, plain, steps, warmup, st, flush=flush, world=world)
    with torch.cuda.stream(st):
        with_ind()
    torch.cuda.synchronize()
    ref = refine.refinement_indicator(mesh, f, 0.3, 0.5, 2)
    got_rms, got_fl = rms.cpu().numpy(), flags.cpu().numpy()
    scale = max(r.max() for r in ref["rms"])
    rms_err, flag_miss, o = 0.0, 0, 0
    for k, blk in enumerate(mesh["levels"]):
        rms_err = max(rms_err, float(np.abs(got_rms[o:o + len(blk)] - ref["rms"][k]).max() / scale))
        flag_miss += int(((got_fl[o:o + len(blk)] & 1) > 0).tolist() != ref["refine"][k].tolist())
        flag_miss += int(((got_fl[o:o + len(blk)] & 2) > 0).tolist() != ref["coarsen"][k].tolist())
        o += len(blk)
    L.lgf_table_destroy(table)
    return {"workload": "three-level ring, DF32 solve + indicator (alpha = 0.3, beta = 0.5, N_l = 2)",
            "ms_solve_with_indicator": ms_ind, "ms_solve_alone": ms_plain, "overhead": ms_ind / ms_plain - 1.0,
            "rms_rel_err": rms_err, "flag_levels_differing": flag_miss,
            "refine_blocks": int(((got_fl & 1) > 0).sum()), "coarsen_blocks": int(((got_fl & 2) > 0).sum()),
            "s_max": float(smax.item())}


def cfg2_case():
    import lgf_synth as S
    case = S.single_level_ring()
    src = {tuple(b) for b in case["src_blocks"]}
    case["roles"] = np.array([2 + (1 if tuple(b) in src else 0) for b in case["blocks"]], np.uint8)
    return case


def run_gpu(args):
    import torch
    import paper_2010_13213_gb300.lgf as L

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _replicas_init(world)
    pk = peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    with ClockSampler(local) as clk:
        hb = batch_poisson(L, torch, dev, args.steps, args.warmup, world, pk)
    clocks = clk.summary()
    res = hb["res"]
    mx = max_over_ranks([res["df32"]["ms"], res["fp64"]["ms"], res["e2e_ms"], res["e2e_serial_ms"]], world, dev)
    ms_df, ms_64, ms_e2e, ms_e2e_serial = mx
    # accuracy of a seeded sample of instances against the oracle, and the oracle's own time on it (the
    # CPU baseline), both outside the timed region
    sample = batch_sample(hb["params"], hb["cells"])
    refs, cpu_s = {}, 0.0
    if rank == 0:
        for i in sample:
            t0 = time.perf_counter()
            refs[i] = oracle_instance(hb["inst"][i])
            cpu_s += time.perf_counter() - t0
    errs_df = batch_errors(res["df32"]["phis"], hb["inst"], sample, refs) if rank == 0 else {}
    errs_64 = batch_errors(res["fp64"]["phis"], hb["inst"], sample, refs) if rank == 0 else {}
    extra = {}
    if args.configs:
        import lgf_synth as S
        c1 = S.single_level_random(n=32, B=16, seed=0)
        extra["cfg1_random32"] = single_config(L, torch, dev, "cfg1", c1, args.steps, args.warmup, world, pk,
                                               [("fp64", L.LGF_PREC_FP64), ("df32", L.LGF_PREC_DF32)], (1, 1, 1),
                                               flush=flush)
        extra["cfg2_ring96"] = single_config(L, torch, dev, "cfg2", cfg2_case(), args.steps, args.warmup, world, pk,
                                             [("df32", L.LGF_PREC_DF32), ("fp64", L.LGF_PREC_FP64),
                                              ("fp32", L.LGF_PREC_FP32)], (5, 5, 2), mode=2, flush=flush, box_only=True)
        extra["cfg3_ring3level"] = multi_config(L, torch, dev, max(3, args.steps // 5), args.warmup, world, pk, flush)
        extra["cfg4_two_rings"] = single_config(L, torch, dev, "cfg4", S.two_ring_single_level(),
                                                max(3, args.steps // 2), args.warmup, world, pk,
                                                [("df32", L.LGF_PREC_DF32), ("fp64", L.LGF_PREC_FP64)], (5, 5, 6),
                                                mode=2, flush=flush, slices=(5, 6), box_only=True)
        extra["batch_rk3_stage"] = batch_stage_heat(L, torch, dev, max(2, args.steps // 10), 1, world)
        extra["heat_apply"] = heat_line(L, torch, dev, 10, 3, world, pk, flush)
        extra["velocity_refresh"] = refresh_line(L, torch, dev, 10, 3, world, flush)
        extra["bump_study"] = bump_study(L, torch, dev)
        extra["stage_projection"] = projection_line(L, torch, dev, 10, 3, world, flush)
        extra["refinement_indicator"] = indicator_line(L, torch, dev, 10, 3, world, flush)
    if rank == 0:
        total = hb["total"]
        mid_ms = hb["mid_ms"]
        sample_cells = int(sum(hb["cells"][i] for i in sample))
        line = {
            "metric": METRIC, "value": replica_rate(total, ms_df, world), "unit": "Mcells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_df, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "df32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances": NINST, "blocks": hb["blocks"], "target_cells": total,
                       "ncomp": 3, "graph_nodes": res["df32"]["nodes"],
                       "autotune": {"df32": res["df32_tuning"], "fp64": res.get("fp64_tuning")},
                       "parallelism": f"replicas{world}",
                       "l2": "no flush: the 64 instances' fields (about 1.7 GB of sources, as much of results) are "
                             "larger than L2"},
            "rel_err": {"df32": max(errs_df.values()) if errs_df else None,
                        "fp64": max(errs_64.values()) if errs_64 else None,
                        "per_instance_df32": errs_df, "per_instance_fp64": errs_64,
                        "sample": "instances " + ",".join(map(str, sample)) + " (smallest of each level count, "
                                  "two of the three-level ones) against the FP64 oracle, relative L-inf over Omega_k"},
            "fp64": {"value": replica_rate(total, ms_64, world), "unit": "Mcells/s", "ms_per_step": ms_64},
            "roofline": roofline("k_box_mid<df,16,*> (fused twiddle, local 16^3 FFTs, kernel product; one launch "
                                 "per box-mode level)", hb["alg_bytes"], mid_ms, hb["mid_launches"], pk,
                                 alg_flops=hb["alg_flops"],
                                 note="the kernel's time summed over the 64 instances run one by one with the "
                                      "library's phase events; the bytes are those of the whole solves, whose "
                                      "work the kernel completes"),
            "roofline_solve": roofline("whole batched step", hb["alg_bytes"], ms_df, hb["launches"], pk,
                                       alg_flops=hb["alg_flops"], note="the step's graph time"),
            "serial_phases_ms": {"k_box_mid": mid_ms, "block_index_dft_passes": hb["pas_ms"],
                                 "all_solves_one_by_one": hb["serial_ms"]},
            "cpu_baseline": {"value": sample_cells / cpu_s / 1e6 if cpu_s else None, "unit": "Mcells/s",
                             "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"the FP64 FLGF-AMR oracle on {len(sample)} instances ({sample_cells} target "
                                       f"cells) of the workload, once",
                             "threads_used": _oracle_threads()},
            "e2e": {"value": replica_rate(total, ms_e2e, world), "unit": "Mcells/s",
                    "h2d_bytes_per_step": res["e2e_bytes"], "d2h_bytes_per_step": res["e2e_bytes"],
                    "note": "every step: all 64 sources copied in from pinned host memory and all 64 results "
                            "copied out inside one graph (lgf_batch_graph_create_io: two copy streams, each solve "
                            "waiting for its own source only, so the copies overlap the other instances' solves)",
                    "graph_nodes": res["e2e_nodes"], "results_match_device_graph": res.get("e2e_match"),
                    "serial": {"value": replica_rate(total, ms_e2e_serial, world), "unit": "Mcells/s",
                               "note": "one stream: all copies in, the device graph, all copies out"}},
            "gpu_launches": int(hb["launches"]) * args.steps,
            "table_build_s": hb["t_table"],
            "clocks": clocks,
            "peaks": {"hbm_gbs": pk["hbm_gbs"], "source": pk["source"]},
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    _replicas_done(world)


def _oracle_threads():
    try:
        import oracle
        return oracle.num_threads()
    except Exception:  # the oracle's C library is built by build(); report nothing if it is absent
        return None


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (FLGF-AMR) on a bounded sample of the same workload, rank 0
    only; each step solves the sample instances."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    params, inst, cells = batch_case()
    sample = batch_sample(params, cells)
    ncells = int(sum(cells[i] for i in sample))
    for _ in range(args.warmup):
        for i in sample:
            oracle_instance(inst[i])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for i in sample:
            oracle_instance(inst[i])
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    val = ncells / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mcells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances": NINST, "ncomp": 3},
            "cpu_baseline": {"value": val, "unit": "Mcells/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"instances {sample} ({ncells} target cells) per step: the FP64 FLGF-AMR "
                                       "oracle (dense level boxes, pocketfft convolutions)",
                             "threads_used": _oracle_threads()},
            "e2e": {"value": val, "unit": "Mcells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_one(args):
    """One named workload as its own JSON line (one replica per rank, rank 0 prints)."""
    import torch
    import lgf_synth as S
    import paper_2010_13213_gb300.lgf as L
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _replicas_init(world)
    pk = peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    w = args.workload
    with ClockSampler(local) as clk:
        if w == "ring":
            out = single_config(L, torch, dev, "cfg2", cfg2_case(), args.steps, args.warmup, world, pk,
                                [("df32", L.LGF_PREC_DF32), ("fp64", L.LGF_PREC_FP64), ("fp32", L.LGF_PREC_FP32)],
                                (5, 5, 2), mode=2, flush=flush, box_only=True)
            ms, cells, name = out["df32"]["ms_per_step"], out["cells"], "single ring 96x96x48, DF32"
        elif w == "cfg1":
            out = single_config(L, torch, dev, "cfg1", S.single_level_random(n=32, B=16, seed=0), args.steps,
                                args.warmup, world, pk, [("fp64", L.LGF_PREC_FP64), ("df32", L.LGF_PREC_DF32)],
                                (1, 1, 1), flush=flush)
            ms, cells, name = out["df32"]["ms_per_step"], out["cells"], "32^3 random sources, DF32"
        elif w == "cfg3":
            out = multi_config(L, torch, dev, args.steps, args.warmup, world, pk, flush)
            ms, cells, name = out["df32"]["ms_per_step"], out["cells"], "three-level ring, DF32"
        elif w == "cfg4":
            out = single_config(L, torch, dev, "cfg4", S.two_ring_single_level(), args.steps, args.warmup, world,
                                pk, [("df32", L.LGF_PREC_DF32), ("fp64", L.LGF_PREC_FP64)], (5, 5, 6), mode=2,
                                flush=flush, slices=(5, 6))
            ms, cells, name = out["df32"]["ms_per_step"], out["cells"], "two coaxial rings 96x96x112, DF32"
        elif w == "poisson_batch":
            out = poisson_batch_line(L, torch, dev, args.steps, args.warmup, world)
            ms, cells, name = out["ms_per_step"], out["target_cells"], "batched Poisson step, default schedule"
        elif w == "stage":
            out = batch_stage_heat(L, torch, dev, args.steps, args.warmup, world)
            ms, cells, name = out["ms_per_stage"], out["value"] * out["ms_per_stage"] * 1e3, "batched RK3 stage"
        elif w == "heat":
            out = heat_line(L, torch, dev, args.steps, args.warmup, world, pk, flush)
            ms, cells, name = out["ms_per_step"], out["target_cells"], "heat apply, three-level ring"
        else:
            out = refresh_line(L, torch, dev, args.steps, args.warmup, world, flush)
            ms, cells, name = out["ms_per_step"], out["value"] * out["ms_per_step"] * 1e3, "velocity refresh"
    ms = max_over_ranks([ms], world, dev)[0]
    if rank == 0:
        line = {"metric": f"{name}: Mcells/s", "value": replica_rate(cells, ms, world), "unit": "Mcells/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "df32",
                "data": "synthetic", "config": {"workload": name}, "detail": out, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    _replicas_done(world)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--configs", default=1, type=int,
                    help="also measure the other configurations, the heat apply, the refresh and the full stage "
                         "(0: the batched headline only)")
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "poisson_batch", "ring", "cfg1", "cfg3", "cfg4", "stage", "heat", "refresh"],
                    help="batch: the headline line; the others print one line for that workload alone")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_gpu(args)
    else:
        run_one(args)


if __name__ == "__main__":
    main()
