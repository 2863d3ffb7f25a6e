#!/usr/bin/env python
"""Benchmark of the GB300 FFTK/Tarang hot path.

Headline (one JSON line on rank 0): 512^3 decaying-turbulence Navier-Stokes
steps/s (RK2 with viscous integrating factor, 2/3 dealiasing, FP32 data and
arithmetic), with the 1024^3 FP32 R2C+C2R pair rate reported beside it.
Inputs are synthetic and resident in HBM when the timed region starts; every
field is larger than the 126 MB L2, so no explicit L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores instead (the
only other place, besides the CPU-baseline leg, where this script runs it).
Multi-GPU runs (torchrun) are independent replicas: the method is not sharded.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1024³ R2C+C2R pairs/s & 512³ NS steps/s, % HBM roofline; mixed vs FP32 at err"
N_NS = 512
NU, DT, K0, E0, SEED = 1e-3, 5e-4, 4.0, 0.5, 0
N_FFT = 1024
E2E_CHUNKS = 16  # pieces of the state in the end-to-end leg


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------- geometry ---
def ns_counts(n):
    kd = (n - 1) // 3
    kc = kd + 1
    nk = 2 * kd + 1
    A = nk * nk * kc  # kept modes of one field
    Bx = n * nk * kc  # one field after the inverse x pass
    By = n * n * kc  # one field after the inverse y pass
    M = n * n * (n // 2 + 1)
    return A, Bx, By, M


def ns_kernel_bytes(n):
    """Algorithmic bytes per launch of each fused kernel (8 bytes per complex value
    read or written; only the rows and columns the dealiased method touches)."""
    A, Bx, By, _ = ns_counts(n)
    c = 8
    return {
        "ns_invx_curl": c * (3 * A + 6 * Bx),
        "ns_invy": c * (6 * Bx + 6 * By),
        "ns_z_product": c * (6 * By + 3 * By),
        "ns_fwdy": c * (3 * By + 3 * Bx),
        "ns_fwdx_update": c * (3 * Bx + 7.5 * A),  # mean of stage 1 (6A) and stage 2 (9A)
    }


def ns_rhs_bytes_unfused(n):
    """Bytes one right-hand side moves on a 3 * 2^m grid (no fused passes): the
    six spectra cleared and filled with (u, i k x u) on the kept modes, their
    inverse x and y passes (out of place through a second workspace, the same
    bytes) and the z pass to six real fields, u x omega
    (six read, three written), the three forward transforms, and the update
    (n, u and, in stage 2, u1 read and the state written on the kept modes)."""
    A, _, _, M = ns_counts(n)
    R = n**3
    c = 8
    clear_curl = 6 * c * M + c * (3 * A + 6 * A)
    inverse = 6 * (2 * c * M + 2 * c * M) + 6 * (c * M + 4 * R)
    cross = 4 * (6 * R + 3 * R)
    forward = 3 * (4 * R + c * M) + 3 * (2 * c * M + 2 * c * M)
    update = c * (3 * A + 4.5 * A + 3 * A)
    return clear_curl + inverse + cross + forward + update


def ns_step_bytes(n):
    kb = ns_kernel_bytes(n)
    pruned = 2 * sum(kb.values())
    _, _, _, M = ns_counts(n)
    unpruned = 93 * 8 * M  # 3-pass method on full arrays, no pruning
    return pruned, unpruned


def fft_pass_bytes(n):
    R = n**3
    M = n * n * (n // 2 + 1)
    return {
        "z_r2c": 4 * R + 8 * M, "y_fwd": 16 * M, "x_fwd": 16 * M,
        "x_inv": 16 * M, "y_inv": 16 * M, "z_c2r": 8 * M + 4 * R,
    }


# --------------------------------------------------- measured DRAM traffic ---
KERNEL_SOURCES = {
    "ns": ["ns.cu", "ns_common.cuh", "fft_engine.cuh", "internal.h", "tcgen05.cuh"],
    "fft": ["fft_passes.cu", "fft_engine.cuh", "internal.h", "abi.cu"],
    "fft16": ["fft_tc.cu", "tcgen05.cuh", "fft_passes.cu", "fft_engine.cuh", "internal.h", "abi.cu"],
}


def source_hash(group: str) -> str:
    """SHA-1 over the CUDA sources a kernel group is built from."""
    import hashlib

    h = hashlib.sha1()
    for f in KERNEL_SOURCES[group]:
        with open(os.path.join(ROOT, "paper_1805_07801_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measured_traffic(kernel: str, workload: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) recorded
    in profiles/dram_traffic.txt for this kernel and workload, or None when no
    record exists or the kernel sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[1] == workload:
            group = "ns" if kernel.startswith("ns_") else ("fft16" if workload.endswith("s16") else "fft")
            if parts[3] == source_hash(group):
                return int(float(parts[2]))
    return None


# ----------------------------------------------------------------- clocks ---
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", self.gpu_id], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, n = [], None, set(), 0
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            n += 1
            for name, v in zip(self.REASONS, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": n}


# ------------------------------------------------------------ distributed ---
def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world, dev=None):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, value, dev):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- GPU arm --
def run_ours(args, world, rank, local):
    import torch

    import paper_1805_07801_gb300 as fk
    from paper_1805_07801_gb300 import build as fkbuild

    fkbuild.build()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    st_obj = torch.cuda.Stream(dev)
    st = st_obj.cuda_stream
    hbm, peak_kind = peaks()
    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(local)
    uuid = getattr(props, "uuid", None)
    if uuid is not None:
        gpu_id = "GPU-" + str(uuid) if not str(uuid).startswith("GPU-") else str(uuid)

    n = N_NS
    plan = fk.fftk_plan_create(n, n, n)
    with torch.cuda.stream(st_obj):
        normals = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
        for f in range(3):
            fk.fftk_fill_normal(normals[f].data_ptr(), n**3, SEED, f, st)
        u = torch.empty((3, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        fk.tarang_ic_random(plan, normals.data_ptr(), u.data_ptr(), K0, E0, st)
    del normals
    prm = fk.make_params(NU, DT)
    for _ in range(args.warmup):
        fk.tarang_ns_step(plan, u.data_ptr(), prm, 1, False, st)
    torch.cuda.synchronize(dev)

    fk.fftk_profile_enable(plan, True)
    clocks = Clocks(gpu_id)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    c0 = fk.fftk_launch_count(plan)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st_obj)
    for _ in range(args.steps):
        fk.tarang_ns_step(plan, u.data_ptr(), prm, 1, False, st)
    e1.record(st_obj)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    launches = fk.fftk_launch_count(plan) - c0
    t_ms = e0.elapsed_time(e1)
    t_ms = max_over_ranks(world, t_ms, dev)
    kern = {}
    for k in range(fk.fftk_kernel_kinds()):
        ms, cnt = fk.fftk_profile_read(plan, k)
        if cnt:
            kern[fk.fftk_kernel_name(k)] = (ms, cnt)
    fk.fftk_profile_enable(plan, False)
    E, eps, _ = fk.tarang_diag(plan, u.data_ptr(), NU, st)

    kb = ns_kernel_bytes(n)
    kernels = {}
    for name, (ms, cnt) in kern.items():
        avg = ms / cnt
        row = {"launches": cnt, "ms_avg": round(avg, 5), "share": round(ms / sum(v[0] for v in kern.values()), 4)}
        if name in kb:
            row["GBps"] = round(kb[name] / (avg * 1e-3) / 1e9, 1)
        kernels[name] = row
    dom = max(kern.items(), key=lambda kv: kv[1][0])[0]
    dom_avg = kern[dom][0] / kern[dom][1]
    achieved = kb[dom] / (dom_avg * 1e-3) / 1e9
    pruned, unpruned = ns_step_bytes(n)
    ms_step = t_ms / args.steps
    value = world * args.steps / (t_ms * 1e-3)

    # end to end through the C ABI with host buffers, as a host-driven run:
    # every step's input state comes from pinned host memory (H2D), the step
    # runs, its diagnostics (E, eps, E(K)) are reduced, and the stepped state
    # and the diagnostics go back to pinned host memory (D2H); the next step
    # starts from the state the host got back.  The state travels in E2E_CHUNKS
    # pieces: piece i of step k's result goes D2H on the step's stream, and
    # once it has landed in host memory a second stream copies that host piece
    # H2D into the other device buffer for step k + 1, so the two directions
    # of the link run at the same time.  The first H2D and the last D2H are
    # whole.  The host waits once, at the end of the region.
    k_e2e = min(args.steps, 20)
    host_u = torch.empty(u.shape, dtype=torch.float32, pin_memory=True)
    host_u.copy_(u)
    bufs = [torch.empty_like(u), torch.empty_like(u)]
    kmax = fk.tarang_diag_kmax(plan)
    diag_dev = torch.empty((2 + kmax + 1,), dtype=torch.float64, device=dev)
    diag_host = torch.empty((k_e2e, 2 + kmax + 1), dtype=torch.float64, pin_memory=True)
    fk.tarang_diag_noalloc(n, u.data_ptr(), NU, diag_dev.data_ptr(), st)  # first call: device setup
    up_obj = torch.cuda.Stream(device=dev)
    h_pieces = host_u.view(-1).chunk(E2E_CHUNKS)
    d_pieces = [b.view(-1).chunk(E2E_CHUNKS) for b in bufs]
    torch.cuda.synchronize(dev)
    barrier(world)
    t0 = time.perf_counter()
    with torch.cuda.stream(st_obj):
        bufs[0].copy_(host_u, non_blocking=True)
        for k in range(k_e2e):
            cur, nxt = k % 2, (k + 1) % 2
            fk.tarang_ns_step(plan, bufs[cur].data_ptr(), prm, 1, False, st)
            fk.tarang_diag_noalloc(n, bufs[cur].data_ptr(), NU, diag_dev.data_ptr(), st)
            diag_host[k].copy_(diag_dev, non_blocking=True)
            if k + 1 == k_e2e:
                host_u.copy_(bufs[cur], non_blocking=True)
                break
            up_obj.wait_stream(st_obj)  # the next buffer is free once the step before has run
            for i in range(E2E_CHUNKS):
                h_pieces[i].copy_(d_pieces[cur][i], non_blocking=True)
                landed = torch.cuda.Event()
                landed.record(st_obj)
                up_obj.wait_event(landed)
                with torch.cuda.stream(up_obj):
                    d_pieces[nxt][i].copy_(h_pieces[i], non_blocking=True)
            st_obj.wait_stream(up_obj)
    torch.cuda.synchronize(dev)
    t_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(world, t_e2e, dev)
    fk.fftk_sync(plan, st)
    if not bool(torch.isfinite(diag_host[:, :2]).all()):
        raise RuntimeError("end-to-end diagnostics not finite")
    e2e = {"value": round(world * k_e2e / t_e2e, 3), "unit": "steps/s", "steps": k_e2e,
           "h2d_bytes_per_step": int(u.numel() * 4),
           "d2h_bytes_per_step": int(u.numel() * 4 + (2 + kmax + 1) * 8),
           "overlap": f"each step's input is the state copied back by the step before; the state moves in "
                      f"{E2E_CHUNKS} pieces, and piece i goes H2D for the next step once its D2H has landed, "
                      "so the two link directions overlap; no copy overlaps a step",
           "E_last": float(diag_host[-1, 0])}
    del bufs, d_pieces, h_pieces, host_u, diag_dev, diag_host

    fft = None
    if not args.no_fft:
        fft = bench_fft(fk, torch, dev, st_obj, args, hbm, peak_kind)
    fk.fftk_plan_destroy(plan)

    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic: random-phase solenoidal field from the library's SplitMix64 normals, seed 0",
        "config": {
            "workload": "512^3 decaying turbulence, pseudo-spectral NS, RK2 + viscous integrating factor, "
                        "2/3 dealiasing, nu=1e-3, dt=5e-4, E(k)~k^4 exp(-2(k/4)^2), E=0.5",
            "n": n, "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            "l2": "no flush: every field (539 MB) exceeds the 126 MB L2",
        },
        "roofline": {
            "bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": measured_traffic(dom, f"ns{n}"),
            "peak_kind": peak_kind, "bytes_per_launch": int(kb[dom]),
        },
        "step_roofline": {
            "pruned_bytes": int(pruned), "unpruned_bytes": int(unpruned),
            "frac_pruned": round(pruned / (ms_step * 1e-3) / 1e9 / hbm, 4),
            "frac_unpruned": round(unpruned / (ms_step * 1e-3) / 1e9 / hbm, 4),
            "peak_kind": peak_kind,
        },
        "kernels": kernels,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "clocks": clk,
        "state_after": {"E": E, "eps": eps},
    }
    if fft is not None:
        line["fft_pair_1024"] = fft
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    return line


def _time_pairs(fk, torch, dev, st_obj, plan, x, F, y, warm, kp):
    st = st_obj.cuda_stream
    for _ in range(warm):
        fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, st)
        fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), 1, st)
    torch.cuda.synchronize(dev)
    fk.fftk_profile_enable(plan, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st_obj)
    for _ in range(kp):
        fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, st)
        fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), 1, st)
    e1.record(st_obj)
    torch.cuda.synchronize(dev)
    fk.fftk_sync(plan, st)
    ms = e0.elapsed_time(e1) / kp
    times = {}
    for k in range(fk.fftk_kernel_kinds()):
        t, cnt = fk.fftk_profile_read(plan, k)
        if cnt:
            times[fk.fftk_kernel_name(k)] = (t, cnt)
    fk.fftk_profile_enable(plan, False)
    return ms, times


def bench_fft(fk, torch, dev, st_obj, args, hbm, peak_kind):
    """1024^3 pair in FP32 and in split-FP16 (tensor-core radix-16 stages)."""
    n = N_FFT
    st = st_obj.cuda_stream
    pb = fft_pass_bytes(n)
    pair = sum(pb.values())
    with torch.cuda.stream(st_obj):
        x = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        fk.fftk_fill_normal(x.data_ptr(), n**3, SEED, 0, st)
        F = torch.empty((n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        y = torch.empty_like(x)
    res = {}
    F32 = None
    for dtype, key in [(fk.FFTK_R32, "fp32"), (fk.FFTK_R32_SPLIT16, "split16")]:
        plan = fk.fftk_plan_create(n, n, n, dtype)
        try:
            ms, times = _time_pairs(fk, torch, dev, st_obj, plan, x, F, y, max(3, args.warmup), 20)
            rt = (torch.linalg.vector_norm((y - x).double()) / torch.linalg.vector_norm(x.double())).item()
            kern = {}
            for name, (t, cnt) in times.items():
                avg = t / cnt
                kern[name] = {"launches": cnt, "ms_avg": round(avg, 5),
                              "GBps": round(pb[name] / (avg * 1e-3) / 1e9, 1) if name in pb else None}
            dom = max(kern.items(), key=lambda kv: kv[1]["ms_avg"] * kv[1]["launches"])[0]
            r = {
                "value": round(1e3 / ms, 3), "unit": "pairs/s", "ms_per_pair": round(ms, 4),
                "frac_pair": round(pair / (ms * 1e-3) / 1e9 / hbm, 4),
                "roofline": {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["GBps"], "peak": hbm,
                             "unit": "GB/s", "frac": round(kern[dom]["GBps"] / hbm, 4),
                             "traffic": measured_traffic(dom, f"fft{n}" if key == "fp32" else f"fft{n}s16"),
                             "peak_kind": peak_kind},
                "kernels": kern,
                "round_trip_rel_l2": rt,
            }
            fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, st)
            torch.cuda.synchronize(dev)
            if key == "fp32":
                F32 = F.clone()
            else:
                r["rel_l2_vs_fp32_spectrum"] = (torch.linalg.vector_norm((F - F32).double()) /
                                                torch.linalg.vector_norm(F32.double())).item()
            res[key] = r
        finally:
            fk.fftk_plan_destroy(plan)
    del F32
    out = dict(res["fp32"])
    out.update({
        "config": "1024^3 FP32 real field, normal(0,1) seed 0, batch 1",
        "pair_bytes": int(pair),
        "nominal_gflops": round(2 * 5 * n**3 * 3 * 10 / (out["ms_per_pair"] * 1e-3) / 1e9, 1),
        "split16": res["split16"],
        "split16_speedup": round(res["split16"]["value"] / res["fp32"]["value"], 4),
    })
    return out


# ------------------------------------------------------ CPU oracle timing ---
def _oracle_state(n):
    import numpy as np

    import oracle
    import synth

    u = oracle.ic_random(synth.normal_fields(SEED, 3, (n, n, n)), k0=K0, E0=E0)
    return u.astype(np.complex64).astype(np.complex128)


def cpu_baseline():
    """One RK2-IF step of the 512^3 workload by the FP64 oracle on the host cores."""
    import oracle

    u = _oracle_state(N_NS)
    t0 = time.perf_counter()
    oracle.ns_step(u, NU, DT, 1)
    t = time.perf_counter() - t0
    return {"value": round(1.0 / t, 5), "unit": "steps/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"one full RK2-IF step of the 512^3 workload (FP64 oracle, OpenMP over lines), {t:.1f} s"}


def oracle_beside(label, n, work, units):
    """The FP64 oracle timed on the host cores beside a GPU measurement: one
    run of work(), a bounded sample of the same kind of work at n^3 (no
    warm-up run, to keep it short).  Returns the seconds, the rate in `units`
    and the threads used."""
    import oracle

    t0 = time.perf_counter()
    work()
    t = time.perf_counter() - t0
    return {"sample": f"{label}, n = {n}", "seconds": round(t, 3), "rate": round(1.0 / t, 4), "unit": units,
            "grid_points_per_s": round(n**3 / t, 1), "cores": oracle.threads(), "kind": "oracle"}


def run_reference(args, world, rank):
    """The oracle as the reference arm: W untimed, then K timed steps of the
    512^3 workload, each one whole RK2-IF step (both right-hand sides with
    their 18 transforms, products, projection and update) by the FP64 oracle
    on the host cores, advancing the state; steps/s = K / total time."""
    import oracle

    u = _oracle_state(N_NS)
    n = N_NS
    for _ in range(args.warmup):
        u = oracle.ns_step(u, NU, DT, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = oracle.ns_step(u, NU, DT, 1)
    t = time.perf_counter() - t0
    value = args.steps / t
    sample = (f"{args.steps} whole RK2-IF steps of the 512^3 workload (after {args.warmup} untimed), "
              f"FP64 oracle with OpenMP over lines, {t:.1f} s; no work skipped")
    return {
        "metric": METRIC, "value": round(value, 6), "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t / max(args.steps, 1) * 1e3, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (oracle's own initial field)",
        "config": {"workload": "512^3 decaying turbulence, pseudo-spectral NS, RK2 + viscous integrating factor, "
                               "2/3 dealiasing, nu=1e-3, dt=5e-4, E(k)~k^4 exp(-2(k/4)^2), E=0.5", "n": n},
        "impl": "reference",
        "cpu_baseline": {"value": round(value, 6), "unit": "steps/s", "cores": oracle.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_case(case: str):
    """One small invocation for profiler captures (no timing, no output line):
    'ns:<n>' = random-phase field + one NS step; 'fft:<nx>,<ny>,<nz>' = two pairs
    ('fft16:' in the split-FP16 mode); 'mlp:<batch>' = two training steps;
    'sgs:<n>' = two unforced steps with the learned subgrid force;
    'transfer:<n>' = random-phase field + one energy transfer spectrum;
    'bases:<nx>,<ny>,<nz>' = one SFF and one CCS forward + inverse pair;
    'rbc:<n>' / 'rbcsff:<n>' = two RK4 convection steps on the cube / between plates."""
    import torch

    import paper_1805_07801_gb300 as fk
    from paper_1805_07801_gb300 import build as fkbuild

    fkbuild.build()
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream(dev).cuda_stream
    kind, arg = case.split(":")
    if kind == "ns":
        n = int(arg)
        plan = fk.fftk_plan_create(n, n, n)
        nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
        for f in range(3):
            fk.fftk_fill_normal(nr[f].data_ptr(), n**3, SEED, f, st)
        u = torch.empty((3, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        fk.tarang_ic_random(plan, nr.data_ptr(), u.data_ptr(), K0, E0, st)
        del nr
        fk.tarang_ns_step(plan, u.data_ptr(), fk.make_params(NU, DT), 1, False, st)
    elif kind == "bases":
        nx, ny, nz = (int(v) for v in arg.split(","))
        plan = fk.fftk_plan_create(nx, ny, nz)
        x = torch.empty((nx, ny, nz), dtype=torch.float32, device=dev)
        fk.fftk_fill_normal(x.data_ptr(), x.numel(), SEED, 0, st)
        F = torch.empty((nx, ny, nz // 2 + 1, 2), dtype=torch.float32, device=dev)
        y = torch.empty_like(x)
        for basis in ("SFF", "CCS"):
            fk.fftk_forward(plan, basis, x.data_ptr(), F.data_ptr(), 1, st)
            fk.fftk_inverse(plan, basis, F.data_ptr(), y.data_ptr(), 1, st)
    elif kind in ("rbc", "rbcsff"):  # two RK4 convection steps (periodic cube or plates)
        n = int(arg)
        plan = fk.fftk_plan_create(n, n, n)
        nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
        for f in range(3):
            fk.fftk_fill_normal(nr[f].data_ptr(), n**3, SEED, f, st)
        s4 = torch.empty((4, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        fk.tarang_ic_random(plan, nr.data_ptr(), s4.data_ptr(), K0, E0, st)
        del nr
        s4[3].copy_(s4[2])
        basis = fk.TARANG_RBC_SFF if kind == "rbcsff" else fk.TARANG_RBC_FFF
        if basis == fk.TARANG_RBC_SFF:
            s4[:, (2 * n - 1) // 3:] = 0
        fk.tarang_rbc_step(plan, s4.data_ptr(), 1e8, 1.0, 1e-3, 2, fk.TARANG_RK4, st, basis=basis)
    elif kind == "transfer":
        n = int(arg)
        plan = fk.fftk_plan_create(n, n, n)
        nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
        for f in range(3):
            fk.fftk_fill_normal(nr[f].data_ptr(), n**3, SEED, f, st)
        u = torch.empty((3, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        fk.tarang_ic_random(plan, nr.data_ptr(), u.data_ptr(), K0, E0, st)
        del nr
        fk.tarang_transfer(plan, u.data_ptr(), None, st)
    elif kind == "fft3":  # a grid with 3 * 2^m axes, same as fft
        nx, ny, nz = (int(v) for v in arg.split(","))
        plan = fk.fftk_plan_create(nx, ny, nz)
        x = torch.empty((nx, ny, nz), dtype=torch.float32, device=dev)
        fk.fftk_fill_normal(x.data_ptr(), x.numel(), SEED, 0, st)
        F = torch.empty((nx, ny, nz // 2 + 1, 2), dtype=torch.float32, device=dev)
        y = torch.empty_like(x)
        for _ in range(2):
            fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, st)
            fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), 1, st)
    elif kind in ("fft", "fft16"):
        nx, ny, nz = (int(v) for v in arg.split(","))
        plan = fk.fftk_plan_create(nx, ny, nz, fk.FFTK_R32_SPLIT16 if kind == "fft16" else fk.FFTK_R32)
        x = torch.empty((nx, ny, nz), dtype=torch.float32, device=dev)
        fk.fftk_fill_normal(x.data_ptr(), x.numel(), SEED, 0, st)
        F = torch.empty((nx, ny, nz // 2 + 1, 2), dtype=torch.float32, device=dev)
        y = torch.empty_like(x)
        for _ in range(2):
            fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, st)
            fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), 1, st)
    elif kind == "mlp":
        import numpy as np

        from paper_1805_07801_gb300 import les

        B = int(arg)
        plan = None
        rng = np.random.default_rng(SEED)
        x = torch.from_numpy(rng.standard_normal((B, 5)).astype(np.float32)).to(dev)
        t = torch.from_numpy(rng.standard_normal((B, 6)).astype(np.float32)).to(dev)
        p = torch.from_numpy(les.init_params(SEED)).to(dev)
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        ctx = fk.tarang_mlp_create(B)
        for step in (1, 2):
            fk.tarang_mlp_train_step(ctx, p.data_ptr(), m.data_ptr(), v.data_ptr(), step, x.data_ptr(),
                                     t.data_ptr(), B, 1e-3, 0, st)
        torch.cuda.synchronize(dev)
        fk.tarang_mlp_destroy(ctx)
    elif kind == "sgs":
        import numpy as np

        from paper_1805_07801_gb300 import les

        n = int(arg)
        plan = fk.fftk_plan_create(n, n, n)
        nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
        for f in range(3):
            fk.fftk_fill_normal(nr[f].data_ptr(), n**3, SEED, f, st)
        u = torch.empty((3, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        fk.tarang_ic_random(plan, nr.data_ptr(), u.data_ptr(), 2.0, E0, st)
        p = torch.from_numpy(les.init_params(SEED)).to(dev)
        model = fk.make_sgs_model(p.data_ptr(), np.zeros(5), np.ones(5), np.full(6, 1e-3))
        fk.tarang_ns_step(plan, u.data_ptr(), fk.make_params(NU, DT, sgs_model=model), 2, False, st)
    else:
        raise SystemExit(f"unknown case {case}")
    torch.cuda.synchronize(dev)
    if plan is not None:
        fk.fftk_plan_destroy(plan)


def run_forced(n: int, steps: int):
    """Forced turbulence (k0 = 2, constant power 0.1 on 1 <= |k| <= 2,
    nu = 4e-4, dt = 2.5e-4) from the same seeded field, once with an FP32
    plan (fused step) and once with a split-FP16 plan (unfused step, radix-16
    stages on the tensor cores); energy and dissipation reduced in FP64 every
    50 steps.  Prints one JSON line: steps/s of each run, their histories and
    the per-shell relative difference of the final spectra."""
    import numpy as np
    import torch

    import paper_1805_07801_gb300 as fk
    from paper_1805_07801_gb300 import build as fkbuild

    fkbuild.build()
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream(dev).cuda_stream
    runs = {}
    for key, dtype in (("fp32", fk.FFTK_R32), ("split16", fk.FFTK_R32_SPLIT16)):
        plan = fk.fftk_plan_create(n, n, n, dtype)
        nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
        for f in range(3):
            fk.fftk_fill_normal(nr[f].data_ptr(), n**3, SEED, f, st)
        u = torch.empty((3, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        fk.tarang_ic_random(plan, nr.data_ptr(), u.data_ptr(), 2.0, E0, st)
        del nr
        prm = fk.make_params(4e-4, 2.5e-4, 0.1, (1, 4))
        hist = []
        secs = 0.0
        done = 0
        while done < steps:
            k = min(50, steps - done)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fk.tarang_ns_step(plan, u.data_ptr(), prm, k, False, st)
            b.record()
            b.synchronize()
            secs += a.elapsed_time(b) * 1e-3
            done += k
            E, eps, EK = fk.tarang_diag(plan, u.data_ptr(), 4e-4, st)
            hist.append({"step": done, "E": E, "eps": eps})
        fk.fftk_sync(plan, st)
        fk.fftk_plan_destroy(plan)
        del u
        torch.cuda.empty_cache()
        runs[key] = {"steps_per_s": round(steps / secs, 3), "ms_per_step": round(1e3 * secs / steps, 3),
                     "history": hist, "EK": np.asarray(EK)}
    ek32, ek16 = runs["fp32"].pop("EK"), runs["split16"].pop("EK")
    res = ek32 >= 1e-8 * ek32.max()
    rel = np.abs(ek16[res] - ek32[res]) / ek32[res]
    f32, f16 = runs["fp32"]["history"][-1], runs["split16"]["history"][-1]
    print(json.dumps({"workload": f"{n}^3 forced turbulence, k0=2, eps=0.1 on 1<=|k|<=2, nu=4e-4, dt=2.5e-4, "
                                  f"RK2-IF, 2/3 dealiasing, seed {SEED}, {steps} steps",
                      "fp32": runs["fp32"], "split16": runs["split16"],
                      "split16_vs_fp32": {"dE_over_E": abs(f16["E"] - f32["E"]) / f32["E"],
                                          "deps_over_eps": abs(f16["eps"] - f32["eps"]) / f32["eps"],
                                          "max_shell_rel_diff": float(rel.max()),
                                          "shells_compared": int(res.sum()),
                                          "cutoff_shell": int(np.nonzero(res)[0].max())}}), flush=True)


def run_transfer(n: int):
    """Energy transfer spectrum and flux of the 512^3 decaying workload's field
    after 50 steps: tarang_transfer (right-hand side + FP64 per-shell
    reduction + host flux) against tarang_ns_rhs alone, CUDA events over 10
    calls after 3, and the flux it reports; then the shell-to-shell matrix
    over octave shells (tarang_shell_transfer, 3 calls after 3).  Prints one
    JSON line."""
    import numpy as np
    import torch

    import paper_1805_07801_gb300 as fk
    from paper_1805_07801_gb300 import build as fkbuild

    fkbuild.build()
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream(dev).cuda_stream
    plan = fk.fftk_plan_create(n, n, n)
    nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
    for f in range(3):
        fk.fftk_fill_normal(nr[f].data_ptr(), n**3, SEED, f, st)
    u = torch.empty((3, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
    fk.tarang_ic_random(plan, nr.data_ptr(), u.data_ptr(), K0, E0, st)
    del nr
    fk.tarang_ns_step(plan, u.data_ptr(), fk.make_params(NU, DT), 50, False, st)
    nh = torch.empty_like(u)
    prm = fk.make_params(NU, DT)

    def timed(fn, k=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        t = []
        for _ in range(k):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            t.append(a.elapsed_time(b))
        return float(np.median(t))

    ms_transfer = timed(lambda: fk.tarang_transfer(plan, u.data_ptr(), None, st))
    ms_rhs = timed(lambda: fk.tarang_ns_rhs(plan, u.data_ptr(), nh.data_ptr(), prm, st))
    tot, T, Pi = fk.tarang_transfer(plan, u.data_ptr(), None, st)
    kmax = fk.tarang_diag_kmax(plan)
    bounds = [0] + [1 << i for i in range(int(np.log2(n)))] + [kmax + 1]
    ms_shell = timed(lambda: fk.tarang_shell_transfer(plan, u.data_ptr(), bounds, st), k=3)
    S = np.array(fk.tarang_shell_transfer(plan, u.data_ptr(), bounds, st))
    fk.fftk_plan_destroy(plan)
    T, Pi = np.array(T), np.array(Pi)
    kd = (n - 1) // 3
    kept = (2 * kd + 1) ** 2 * (kd + 1)
    import oracle

    uo = _oracle_state(256)
    ocpu = oracle_beside("oracle right-hand side + T(K) of the decaying field's initial state", 256,
                         lambda: oracle.transfer_spectrum(uo, oracle.ns_rhs(uo)), "calls/s")
    u128 = _oracle_state(128)
    ocpu_shell = oracle_beside("oracle shell-to-shell matrix, octave shells", 128,
                               lambda: oracle.shell_transfer(u128, [0, 1, 2, 4, 8, 16, 32, 64, 112]),
                               "calls/s")
    print(json.dumps({"workload": f"{n}^3 decaying field (k0={K0}, E={E0}, seed {SEED}) after 50 steps "
                                  f"nu={NU}, dt={DT}",
                      "ms_transfer": round(ms_transfer, 4), "ms_rhs": round(ms_rhs, 4),
                      "ms_reduction_and_copy": round(ms_transfer - ms_rhs, 4),
                      "reduction_bytes": 2 * 3 * 8 * kept,
                      "sum_T_over_sum_absT": tot / float(np.sum(np.abs(T))),
                      "flux_max": float(Pi.max()), "flux_argmax": int(Pi.argmax()),
                      "flux_K_0_to_63": [float(v) for v in Pi[:64]],
                      "oracle_cpu": ocpu, "oracle_cpu_shell_transfer": ocpu_shell,
                      "shell_bounds": bounds, "ms_shell_transfer": round(ms_shell, 3),
                      "shell_antisymmetry": float(np.max(np.abs(S + S.T)) / np.max(np.abs(S))),
                      "shell_transfer": [[float(v) for v in row] for row in S]}), flush=True)


def run_schemes(n: int, steps: int):
    """The n^3 decaying workload (random-phase field, k0 = 4, E = 0.5, seed 0,
    nu = 1e-3, dt = 5e-4) stepped with RK2 and with the paper's RK4 (four
    fused right-hand sides per step), CUDA events over `steps` steps after 3.
    Prints one JSON line with steps/s, the per-step bytes of each scheme and
    the energies reached."""
    import torch

    import paper_1805_07801_gb300 as fk
    from paper_1805_07801_gb300 import build as fkbuild

    fkbuild.build()
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream(dev).cuda_stream
    hbm, peak_kind = peaks()
    plan = fk.fftk_plan_create(n, n, n)
    nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
    for f in range(3):
        fk.fftk_fill_normal(nr[f].data_ptr(), n**3, SEED, f, st)
    u0 = torch.empty((3, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
    fk.tarang_ic_random(plan, nr.data_ptr(), u0.data_ptr(), K0, E0, st)
    del nr
    fused = n & (n - 1) == 0
    pruned = ns_step_bytes(n)[0] if fused else 2 * ns_rhs_bytes_unfused(n)
    out = {"path": "fused passes restricted to the 2/3 set" if fused else
           "unfused: the plan's radix-3 transforms, u x omega in real space, the fused path's update"}
    for name, scheme in (("rk2", fk.TARANG_RK2), ("rk4", fk.TARANG_RK4)):
        u = u0.clone()
        prm = fk.make_params(NU, DT, scheme=scheme)
        fk.tarang_ns_step(plan, u.data_ptr(), prm, 3, False, st)
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fk.tarang_ns_step(plan, u.data_ptr(), prm, steps, False, st)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        E, eps, _ = fk.tarang_diag(plan, u.data_ptr(), NU, st)
        # RK4: four right-hand sides of about half an RK2 step's bytes each, plus the accumulator
        step_bytes = pruned if scheme == fk.TARANG_RK2 else 2 * pruned
        out[name] = {"steps_per_s": round(1e3 / ms, 3), "ms_per_step": round(ms, 4),
                     "approx_step_bytes": step_bytes, "frac": round(step_bytes / (ms * 1e-3) / 1e9 / hbm, 4),
                     "E": E, "eps": eps, "steps": steps + 3}
    fk.fftk_sync(plan, st)
    fk.fftk_plan_destroy(plan)
    import oracle

    no = 128 if fused else 96
    uo = _oracle_state(no)
    out["oracle_cpu"] = oracle_beside("oracle RK4 step", no, lambda: oracle.ns_step_rk4(uo, NU, DT, 1), "steps/s")
    print(json.dumps({"workload": f"{n}^3 decaying turbulence, nu={NU}, dt={DT}, seed {SEED}",
                      "peak_GBps": hbm, "peak_kind": peak_kind, **out}), flush=True)


def run_rbc(n: int, steps: int):
    """Rayleigh-Benard convection at n^3 (Ra = 1e8, Pr = 1, dt = 1e-3): the
    random-phase velocity of the decaying workload with theta = u_z, stepped
    on the periodic cube with RK4 (the paper's scheme: 52 transforms per step)
    and RK2, and between free-slip plates (the same coefficients read in the
    plates' bases) with RK4; CUDA events over `steps` steps after 3.  Prints
    one JSON line with steps/s and the time per transform."""
    import numpy as np
    import torch

    import paper_1805_07801_gb300 as fk
    from paper_1805_07801_gb300 import build as fkbuild

    fkbuild.build()
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream(dev).cuda_stream
    plan = fk.fftk_plan_create(n, n, n)
    nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
    for f in range(3):
        fk.fftk_fill_normal(nr[f].data_ptr(), n**3, SEED, f, st)
    s0 = torch.empty((4, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
    fk.tarang_ic_random(plan, nr.data_ptr(), s0.data_ptr(), K0, E0, st)
    s0[3].copy_(s0[2])
    del nr
    out = {}
    cases = [("rk4", fk.TARANG_RK4, 52, fk.TARANG_RBC_FFF), ("rk2", fk.TARANG_RK2, 26, fk.TARANG_RBC_FFF)]
    if n & (n - 1) == 0:  # the plates' sine/cosine passes need power-of-two axes
        cases.append(("sff_rk4", fk.TARANG_RK4, 52, fk.TARANG_RBC_SFF))
    for name, scheme, ntr, basis in cases:
        s = s0.clone()
        if basis == fk.TARANG_RBC_SFF:  # the same coefficients read in the plates' bases, truncated to them
            s[:, (2 * n - 1) // 3:] = 0
        fk.tarang_rbc_step(plan, s.data_ptr(), 1e8, 1.0, 1e-3, 3, scheme, st, basis=basis)
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        fk.fftk_profile_enable(plan, True)
        a.record()
        fk.tarang_rbc_step(plan, s.data_ptr(), 1e8, 1.0, 1e-3, steps, scheme, st, basis=basis)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        kern = {}
        for k in range(fk.fftk_kernel_kinds()):
            kms, cnt = fk.fftk_profile_read(plan, k)
            if cnt:
                kern[fk.fftk_kernel_name(k)] = {"launches": cnt, "ms_per_step": round(kms / steps, 4)}
        fk.fftk_profile_enable(plan, False)
        fin = bool(torch.isfinite(s).all())
        out[name] = {"steps_per_s": round(1e3 / ms, 3), "ms_per_step": round(ms, 4), "transforms_per_step": ntr,
                     "ms_per_transform_incl_pointwise": round(ms / ntr, 4), "finite": fin, "kernels": kern}
        if name == "rk4":  # kinetic and thermal fluxes of the state reached (Sec. 7)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            (tu, Tu, Pu), (tt, Tt, Pt) = fk.tarang_rbc_transfer(plan, s.data_ptr(), st)
            b.record()
            b.synchronize()
            out["flux"] = {"ms": round(a.elapsed_time(b), 3), "sum_Tu_over_sum_absTu": tu / sum(abs(v) for v in Tu),
                           "sum_Ttheta_over_sum_absTtheta": tt / sum(abs(v) for v in Tt),
                           "Pi_u_K_0_to_31": [float(v) for v in Pu[:32]],
                           "Pi_theta_K_0_to_31": [float(v) for v in Pt[:32]]}
    fk.fftk_sync(plan, st)
    fk.fftk_plan_destroy(plan)
    import oracle

    so = np.concatenate([_oracle_state(128), _oracle_state(128)[2:3]])
    out["oracle_cpu"] = oracle_beside("oracle RK4 convection step (cube)", 128,
                                      lambda: oracle.rbc_step(so, 1e8, 1.0, 1e-3, 1, 1), "steps/s")
    print(json.dumps({"workload": f"{n}^3 Rayleigh-Benard (FFF), Ra=1e8, Pr=1, dt=1e-3, random-phase u (k0={K0}), "
                                  f"theta = u_z, seed {SEED}", **out}), flush=True)


def run_radix3():
    """R2C + C2R pairs on the paper's 3 * 2^m grids (768^3 and 1536^3; 3072^3
    needs 348 GB for input, spectrum and inverse workspace and is left out)
    beside 512^3 and 1024^3, normal(0,1), seed 0, CUDA events over 10 pairs
    after 3, against the pair roofline 8R + 80M.  Prints one JSON line."""
    import numpy as np
    import torch

    import paper_1805_07801_gb300 as fk
    from paper_1805_07801_gb300 import build as fkbuild

    fkbuild.build()
    dev = torch.device("cuda:0")
    st_obj = torch.cuda.Stream(dev)
    st = st_obj.cuda_stream
    hbm, peak_kind = peaks()
    rows = []
    for n in (512, 768, 1024, 1536):
        R, M = n**3, n * n * (n // 2 + 1)
        pair = 8 * R + 80 * M
        plan = fk.fftk_plan_create(n, n, n)
        with torch.cuda.stream(st_obj):
            x = torch.empty((n, n, n), dtype=torch.float32, device=dev)
            fk.fftk_fill_normal(x.data_ptr(), R, SEED, 0, st)
            F = torch.empty((n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
            y = torch.empty_like(x)
        for _ in range(3):
            fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, st)
            fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), 1, st)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        kp = 10
        e0.record(st_obj)
        for _ in range(kp):
            fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, st)
            fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), 1, st)
        e1.record(st_obj)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / kp
        err = float(torch.linalg.vector_norm((y - x).double()) / torch.linalg.vector_norm(x.double()))
        rows.append({"n": n, "pairs_s": round(1e3 / ms, 3), "ms_per_pair": round(ms, 4), "pair_bytes": pair,
                     "frac_pair": round(pair / (ms * 1e-3) / 1e9 / hbm, 4), "round_trip_rel_l2": err,
                     "gflops_paper_model": round(2 * 5 * R * np.log2(R) / (ms * 1e-3) / 1e9, 1)})
        fk.fftk_plan_destroy(plan)
        del x, F, y
        torch.cuda.empty_cache()
    import oracle
    import synth

    f192 = synth.normal(SEED, 0, (192, 192, 192)).astype(np.float64)
    ocpu = oracle_beside("oracle R2C + C2R pair, lines of 3*2^m by the DFT's definition", 192,
                         lambda: oracle.irfft3(oracle.rfft3(f192), 192), "pairs/s")
    print(json.dumps({"workload": "R2C+C2R pairs of normal(0,1), seed 0, 2^m and 3*2^m cubes", "peak_GBps": hbm,
                      "peak_kind": peak_kind, "sizes": rows, "oracle_cpu": ocpu}), flush=True)


def run_bases(n: int):
    """Forward + inverse pairs of an n^3 normal(0,1) field (seed 0) in the
    paper's bases FFF, SFF, SSF and SSS (sine on x, y and z in turn; cosine
    on the other S axes: {S,F,F}, {S,C,F}, {C,C,S}), CUDA events over 20
    pairs after 3, against the pair roofline: every pass reads and writes its
    field once (8R + 80M bytes with a Fourier z axis, 48R for SSS).  Prints
    one JSON line."""
    import numpy as np
    import torch

    import paper_1805_07801_gb300 as fk
    from paper_1805_07801_gb300 import build as fkbuild

    fkbuild.build()
    dev = torch.device("cuda:0")
    st_obj = torch.cuda.Stream(dev)
    st = st_obj.cuda_stream
    hbm, peak_kind = peaks()
    R, M = n**3, n * n * (n // 2 + 1)
    plan = fk.fftk_plan_create(n, n, n)
    x = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    with torch.cuda.stream(st_obj):
        fk.fftk_fill_normal(x.data_ptr(), R, SEED, 0, st)
        spec = torch.empty((n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        y = torch.empty_like(x)
    rows = []
    for name, basis in (("FFF", "FFF"), ("SFF", "SFF"), ("SSF", "SCF"), ("SSS", "CCS")):
        pair = 48 * R if basis[2] != "F" else 8 * R + 80 * M
        for _ in range(3):
            fk.fftk_forward(plan, basis, x.data_ptr(), spec.data_ptr(), 1, st)
            fk.fftk_inverse(plan, basis, spec.data_ptr(), y.data_ptr(), 1, st)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        kp = 20
        e0.record(st_obj)
        for _ in range(kp):
            fk.fftk_forward(plan, basis, x.data_ptr(), spec.data_ptr(), 1, st)
            fk.fftk_inverse(plan, basis, spec.data_ptr(), y.data_ptr(), 1, st)
        e1.record(st_obj)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / kp
        err = float(torch.linalg.vector_norm((y - x).double()) / torch.linalg.vector_norm(x.double()))
        rows.append({"basis": name, "axes": basis, "pairs_s": round(1e3 / ms, 3), "ms_per_pair": round(ms, 4),
                     "pair_bytes": pair, "frac_pair": round(pair / (ms * 1e-3) / 1e9 / hbm, 4),
                     "round_trip_rel_l2": err})
    fk.fftk_plan_destroy(plan)
    import oracle
    import synth

    f128 = synth.normal(SEED, 0, (128, 128, 128)).astype(np.float64)
    ocpu = oracle_beside("oracle SFF forward + inverse pair (sine axis by its definition, O(n^4))", 128,
                         lambda: oracle.itransform3(oracle.transform3(f128, "SFF"), 128, "SFF"), "pairs/s")
    print(json.dumps({"workload": f"{n}^3 forward + inverse pairs of normal(0,1), seed {SEED}, mixed bases",
                      "peak_GBps": hbm, "peak_kind": peak_kind, "bases": rows, "oracle_cpu": ocpu}), flush=True)


def run_fft_sweep(args):
    """Batched R2C + C2R pairs with B * N^3 = 2^30 reals: 256^3 x 64, 512^3 x 8,
    1024^3 and 2048^3, each in FP32 and in split-FP16.  Pairs/s (CUDA events,
    20 pairs after 3), the fraction of the pair roofline (8R + 80M bytes per
    field) of measured HBM, the round-trip error, and the split-FP16 spectrum
    against the FP32 GPU spectrum (the comparison prescribed at 2048^3; parity
    with the oracle up to 1024^3 is the tests').  Prints one JSON line."""
    import torch

    import paper_1805_07801_gb300 as fk
    from paper_1805_07801_gb300 import build as fkbuild

    fkbuild.build()
    dev = torch.device("cuda:0")
    st_obj = torch.cuda.Stream(dev)
    st = st_obj.cuda_stream
    hbm, peak_kind = peaks()

    def rel_l2(a, b):  # ||a - b|| / ||b||, FP64 sums over slices (no full-size temporaries)
        a2, b2 = a.reshape(-1, a.shape[-1]), b.reshape(-1, b.shape[-1])
        num = den = 0.0
        for i in range(0, a2.shape[0], 1 << 16):
            d = (a2[i:i + (1 << 16)].double() - b2[i:i + (1 << 16)].double())
            num += float((d * d).sum())
            den += float((b2[i:i + (1 << 16)].double() ** 2).sum())
        return (num / den) ** 0.5

    out = []
    for n, B in ((256, 64), (512, 8), (1024, 1), (2048, 1)):
        R, M = n**3, n * n * (n // 2 + 1)
        pair = B * (8 * R + 80 * M)
        with torch.cuda.stream(st_obj):
            x = torch.empty((B, n, n, n), dtype=torch.float32, device=dev)
            fk.fftk_fill_normal(x.data_ptr(), B * R, SEED, 0, st)
            F = torch.empty((B, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
            y = torch.empty_like(x)
        row = {"n": n, "batch": B, "pair_bytes": pair}
        F32 = None
        for dtype, key in ((fk.FFTK_R32, "fp32"), (fk.FFTK_R32_SPLIT16, "split16")):
            plan = fk.fftk_plan_create(n, n, n, dtype)
            try:
                for _ in range(3):
                    fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), B, st)
                    fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), B, st)
                torch.cuda.synchronize(dev)
                kp = 20
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st_obj)
                for _ in range(kp):
                    fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), B, st)
                    fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), B, st)
                e1.record(st_obj)
                torch.cuda.synchronize(dev)
                fk.fftk_sync(plan, st)
                ms = e0.elapsed_time(e1) / kp
                rt = rel_l2(y, x)
                r = {"pairs_s": round(B * 1e3 / ms, 3), "ms_per_batch": round(ms, 4),
                     "frac_pair": round(pair / (ms * 1e-3) / 1e9 / hbm, 4), "round_trip_rel_l2": rt}
                fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), B, st)
                torch.cuda.synchronize(dev)
                if key == "fp32":
                    F32 = F.clone()
                else:
                    r["rel_l2_vs_fp32_spectrum"] = rel_l2(F, F32)
                row[key] = r
            finally:
                fk.fftk_plan_destroy(plan)
        row["split16_speedup"] = round(row["split16"]["pairs_s"] / row["fp32"]["pairs_s"], 4)
        out.append(row)
        del x, F, y, F32
        torch.cuda.empty_cache()
    print(json.dumps({"workload": "batched R2C+C2R pairs of normal(0,1) fields, seed 0, B*N^3 = 2^30",
                      "peak_GBps": hbm, "peak_kind": peak_kind, "sizes": out}), flush=True)


def run_closure(which: str, out_path: str, flux_weights=None, targets=None, seeded_runs=0):
    """The learned-closure workflow (resolved snapshots -> filtered data ->
    training -> coarse runs with and without the model); prints one JSON line
    and writes the full results to out_path."""
    from paper_1805_07801_gb300 import build as fkbuild

    fkbuild.build()
    from paper_1805_07801_gb300 import les

    cfg = les.ClosureConfig() if which == "full" else les.ClosureConfig.small()
    if flux_weights:
        cfg = dataclasses.replace(cfg, flux_weights=tuple(flux_weights))
    if targets:
        cfg = dataclasses.replace(cfg, targets=tuple(targets))
    if seeded_runs:
        cfg = dataclasses.replace(cfg, seeded_runs=int(seeded_runs))
    res = les.run(cfg, log=lambda s: print(s, file=sys.stderr, flush=True))
    if out_path:
        os.makedirs(os.path.dirname(os.path.abspath(out_path)), exist_ok=True)
        with open(out_path, "w") as fh:
            json.dump(res, fh, indent=1)
    keys = ("resolved_seconds", "resolved_steps_per_s", "ref_samples", "train_seconds", "train_samples_per_s",
            "heldout_loss", "heldout_loss_zero_model", "coarse_steps_per_s", "coarse_steps_per_s_no_model",
            "speedup")
    line = {k: res.get(k) for k in keys}
    for name in ("model", "no_model"):
        r = res[name]
        line[name] = {"finite": r["finite"]}
        for w in ("stated", "long"):
            if w in r:
                line[name][w] = {k: r[w][k] for k in ("max_rel_err", "mean_rel_err", "shells_within_5pct")}
    if "variants" in res:
        line["variants"] = [{"data": v.get("data"), "target": v["target"], "flux_weight": v["flux_weight"],
                             "heldout_loss": v.get("heldout_loss"),
                             "heldout_loss_zero_model": v.get("heldout_loss_zero_model"),
                             "stated": {k: v["model"]["stated"][k] for k in ("mean_rel_err", "max_rel_err",
                                                                           "shells_within_5pct")},
                             "long": {k: v["model"]["long"][k] for k in ("mean_rel_err", "max_rel_err",
                                                                       "shells_within_5pct")}}
                            for v in res["variants"] if v["model"]["finite"]]
    line["workload"] = f"closure {which}: {cfg.n}^3 -> {cfg.m}^3"
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 100; 3 for --impl reference, whose steps take seconds each)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fft", action="store_true")
    ap.add_argument("--case", default=None,
                    help="profiler case: ns:<n>, transfer:<n>, bases:<nx>,<ny>,<nz>, fft:<nx>,<ny>,<nz>, "
                         "fft16:<nx>,<ny>,<nz>, mlp:<batch> "
                         "or sgs:<n>")
    ap.add_argument("--closure", choices=["full", "small"], default=None,
                    help="run the learned-closure workflow instead of the benchmark")
    ap.add_argument("--closure-out", default="", help="JSON file for the closure workflow's results")
    ap.add_argument("--flux-weights", type=float, nargs="*", default=None,
                    help="closure: loss weights of the frame stress's diagonal components, one model each")
    ap.add_argument("--targets", nargs="*", choices=["les", "box", "box_coarse", "blend"], default=None,
                    help="closure: training data sets, one model each (default all four)")
    ap.add_argument("--seeded-runs", type=int, default=0, metavar="K",
                    help="closure: also train on one snapshot from each of K separately seeded runs")
    ap.add_argument("--fft-sweep", action="store_true", help="batched pair sweep 256^3 x 64 ... 2048^3")
    ap.add_argument("--forced", type=int, default=0, metavar="N",
                    help="run N^3 forced turbulence for --steps steps and print its JSON line")
    ap.add_argument("--transfer", type=int, default=0, metavar="N",
                    help="time the energy transfer spectrum and flux of an N^3 field")
    ap.add_argument("--schemes", type=int, default=0, metavar="N",
                    help="time N^3 NS steps with RK2 and with RK4 for --steps steps")
    ap.add_argument("--rbc", type=int, default=0, metavar="N",
                    help="time N^3 Rayleigh-Benard steps (RK4 and RK2) for --steps steps")
    ap.add_argument("--radix3", action="store_true", help="time pairs at 512^3, 768^3, 1024^3 and 1536^3")
    ap.add_argument("--bases", type=int, default=0, metavar="N",
                    help="time N^3 transform pairs in the FFF, SFF, SSF and SSS bases")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 100 if args.impl == "ours" else 3
    if args.case:
        run_case(args.case)
        return
    if args.closure:
        run_closure(args.closure, args.closure_out, args.flux_weights, args.targets, args.seeded_runs)
        return
    if args.forced:
        run_forced(args.forced, args.steps)
        return
    if args.fft_sweep:
        run_fft_sweep(args)
        return
    if args.transfer:
        run_transfer(args.transfer)
        return
    if args.bases:
        run_bases(args.bases)
        return
    if args.radix3:
        run_radix3()
        return
    if args.schemes:
        run_schemes(args.schemes, args.steps)
        return
    if args.rbc:
        run_rbc(args.rbc, args.steps)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, world, rank)), flush=True)
        return
    line = run_ours(args, world, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
