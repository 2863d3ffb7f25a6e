"""Learned subgrid closure workflow: a coarse run with a trained network
standing in for a filtered resolved simulation.

Steps (each one a call into the library; this module only orchestrates and
keeps small host-side statistics):

1. Resolved run.  A seeded random-phase solenoidal field (spectrum
   K^4 exp(-2 (K/k0)^2), energy 0.5) is advanced with constant-power forcing
   on the shells 1 <= |k| <= 2 through a spin-up, then through a window in
   which closure-data snapshots are taken at a fixed interval.  The forced
   flow has a slow cycle (several large-eddy times) that moves energy between
   the lowest shells, so single snapshots are poor spectra: the reference is
   the filtered spectrum averaged over many samples of the whole window.
2. Closure data.  Each snapshot is box-filtered to the coarse grid
   (tarang_box_filter: ubar and tau_ij = <u_i u_j> - ubar_i ubar_j); the
   coarse gradient's five invariants, the strain eigenframe Q and the stress
   in that frame Q^T tau Q come from tarang_closure_features.  The "les"
   target instead takes the stress the coarse solver misses as it computes,
   T[tau_ij + ubar_i ubar_j - (T ubar)_i (T ubar)_j] with T the 2/3
   truncation (tarang_les_stress), and the features of the coarse state
   P T ubar that the model sees at run time.
3. Training.  The 5 -> 64 -> 64 -> 64 -> 6 tanh network maps normalised
   invariants to the normalised frame stress (MSE, Adam), through
   tarang_sgs_train; the last snapshot is held out.
4. Coarse run.  The coarse solver steps the first filtered snapshot with the
   model's subgrid force P[-i k_j tau_ij] fused into its right-hand side; the
   same run without the model is the baseline.  Their time-averaged spectra
   are compared shell by shell to the reference (filtered fields are
   2/3-truncated and projected like any coarse state).

The coarse point I of the box filter is the mean over the fine cells
[f I, f I + f) in each direction; every coarse field shares that offset.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import (FFTKError, fftk_c2r, fftk_fill_normal, fftk_plan_create, fftk_plan_destroy, fftk_r2c, make_params,
               make_sgs_model, tarang_box_filter, tarang_closure_features, tarang_dealias_project, tarang_diag,
               tarang_ic_random, tarang_les_stress, tarang_mlp_create, tarang_mlp_destroy, tarang_mlp_loss_grad,
               tarang_ns_step, tarang_sgs_train)

NPARAMS = 9094
DIMS = (5, 64, 64, 64, 6)
DEV = "cuda:0"


@dataclasses.dataclass
class ClosureConfig:
    n: int = 512               # resolved grid
    m: int = 64                # coarse grid
    seed: int = 0              # initial field of the resolved run
    nu: float = 1e-3
    force_eps: float = 0.1     # injected power on 1 <= |k| <= 2
    k0: float = 2.0
    dt: float = 5e-4           # resolved time step
    spinup_time: float = 5.0   # before the first snapshot
    snapshots: int = 8         # closure-data snapshots, the last one held out
    snapshot_every: float = 2.5
    ref_every: float = 0.25    # filtered spectra averaged into the reference
    train_steps: int = 20000
    batch: int = 65536
    lr: float = 1e-3
    les_dt: float = 4e-3
    les_steps: int = 2000      # the stated coarse run; spectrum averaged over its second half
    les_long_steps: int = 10000  # the same run continued; spectrum averaged over its last 80 %
    les_sample_every: int = 10
    kcmp: int = 20             # shells 1..kcmp are compared
    init_seed: int = 0         # network initialisation and batch order
    # loss weight of the frame stress's diagonal components (the ones that
    # carry the local energy flux -tau_ij S_ij in the strain eigenframe); one
    # model is trained per value, on the same data, and the first is reported
    # as "model"
    flux_weights: tuple = (1.0,)
    # training data per model: "les" = the stress the coarse solver misses
    # as it computes (tarang_les_stress) with features of the coarse state
    # P T ubar; "box" = the box-filter stress tau with features of ubar;
    # "box_coarse" = tau with features of P T ubar (the state the model sees
    # at run time); "blend" = (1 - blend) box_coarse + blend les, frame by
    # frame (both share the features).  One model per (target, flux weight);
    # the first is reported as "model"
    targets: tuple = ("box", "box_coarse", "les", "blend")
    blend: float = 0.5
    # a second training set: one snapshot from each of `seeded_runs` runs of
    # their own (seeds seed + 1, ...), each after the same spin-up; the last
    # is held out.  Models for `seeded_targets` are trained on it and
    # evaluated like the others (0 = off)
    seeded_runs: int = 0
    seeded_targets: tuple = ("box", "blend")

    @property
    def factor(self) -> int:
        return self.n // self.m

    @classmethod
    def small(cls) -> "ClosureConfig":
        """256^3 resolved / 32^3 coarse (the same factor 8), shorter window
        and training: the workflow end to end in about a minute."""
        return cls(n=256, m=32, dt=1e-3, snapshot_every=1.25, ref_every=0.25, train_steps=3000, batch=16384,
                   lr=2e-3, les_steps=2000, les_long_steps=5000, kcmp=10, targets=("box",))


def _dev_empty(shape, dtype=torch.float32):
    return torch.empty(shape, dtype=dtype, device=DEV)


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _half(n):
    return n // 2 + 1


def initial_state(plan: int, n: int, cfg: ClosureConfig):
    """Seeded random-phase solenoidal field, energy 0.5, peak wavenumber k0."""
    normals = _dev_empty((3, n, n, n))
    for f in range(3):
        fftk_fill_normal(normals[f].data_ptr(), n ** 3, cfg.seed, f, _stream())
    uhat = _dev_empty((3, n, n, _half(n), 2))
    tarang_ic_random(plan, normals.data_ptr(), uhat.data_ptr(), cfg.k0, 0.5, _stream())
    return uhat


def advance(plan: int, uhat, prm, steps: int) -> float:
    """Advance `steps` steps; returns the seconds they took (CUDA events)."""
    if steps <= 0:
        return 0.0
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    tarang_ns_step(plan, uhat.data_ptr(), prm, steps, False, _stream())
    b.record()
    b.synchronize()
    return a.elapsed_time(b) * 1e-3


def filtered_state(plan_n: int, plan_m: int, uhat, cfg: ClosureConfig, features: bool):
    """Box filter of a resolved state onto the coarse grid: the coarse solver
    state (2/3-truncated, projected), its spectrum and, with `features`, the
    closure data per training target (invariants and frame stress, host
    copies)."""
    m = cfg.m
    R = m ** 3
    ubar = _dev_empty((3, m, m, m))
    tau = _dev_empty((6, m, m, m))
    tarang_box_filter(plan_n, uhat.data_ptr(), cfg.factor, ubar.data_ptr(), tau.data_ptr(), _stream())
    uc = _dev_empty((3, m, m, _half(m), 2))
    fftk_r2c(plan_m, ubar.data_ptr(), uc.data_ptr(), 3, _stream())
    tarang_dealias_project(plan_m, uc.data_ptr(), _stream())
    out = {}
    if features:
        def closure_data(u, t):
            inv = _dev_empty((5, R))
            frame = _dev_empty((9, R))
            taup = _dev_empty((6, R))
            tarang_closure_features(plan_m, u.data_ptr(), t.data_ptr(), inv.data_ptr(), frame.data_ptr(),
                                    taup.data_ptr(), _stream())
            return dict(inv=inv.cpu().numpy(), taup=taup.cpu().numpy())

        ucoarse = None
        wanted = list(cfg.targets)
        if "blend" in wanted:
            wanted = [t for t in wanted if t != "blend"] + ["les", "box_coarse", "blend"]
        for target in dict.fromkeys(wanted):
            if target in ("les", "box_coarse") and ucoarse is None:
                ucoarse = _dev_empty((3, m, m, m))
                fftk_c2r(plan_m, uc.data_ptr(), ucoarse.data_ptr(), 3, _stream())
            if target == "box":
                out[target] = closure_data(ubar, tau)
            elif target == "box_coarse":
                out[target] = closure_data(ucoarse, tau)
            elif target == "les":
                tles = _dev_empty((6, m, m, m))
                tarang_les_stress(plan_m, ubar.data_ptr(), tau.data_ptr(), tles.data_ptr(), _stream())
                out[target] = closure_data(ucoarse, tles)
            elif target == "blend":
                out[target] = dict(inv=out["les"]["inv"],
                                   taup=(1.0 - cfg.blend) * out["box_coarse"]["taup"] + cfg.blend * out["les"]["taup"])
            else:
                raise ValueError(f"unknown closure target {target!r}")
    E, eps, EK = tarang_diag(plan_m, uc.data_ptr(), cfg.nu, _stream())
    out.update(uc=uc, E=E, EK=np.asarray(EK))
    return out


def resolved_run(plan_n: int, plan_m: int, cfg: ClosureConfig, log=None):
    """The forced resolved run: spin-up, then a window of `snapshots` x
    `snapshot_every` time units in which the closure data are taken every
    snapshot_every and the filtered spectrum every ref_every."""
    n = cfg.n
    uhat = initial_state(plan_n, n, cfg)
    prm = make_params(cfg.nu, cfg.dt, cfg.force_eps, (1, 4))
    secs = 0.0
    steps = 0
    spin = int(round(cfg.spinup_time / cfg.dt))
    chunk = max(1, int(round(0.5 / cfg.dt)))
    done = 0
    while done < spin:
        k = min(chunk, spin - done)
        secs += advance(plan_n, uhat, prm, k)
        done += k
        steps += k
        if log:
            E, eps, _ = tarang_diag(plan_n, uhat.data_ptr(), cfg.nu, _stream())
            log(f"  resolved t={done * cfg.dt:6.2f}: E={E:.5f} eps={eps:.5f}")
    ref_steps = max(1, int(round(cfg.ref_every / cfg.dt)))
    per_snap = max(1, int(round(cfg.snapshot_every / cfg.ref_every)))
    snaps, spectra = [], []
    for i in range(cfg.snapshots * per_snap):
        feat = i % per_snap == 0
        f = filtered_state(plan_n, plan_m, uhat, cfg, feat)
        spectra.append(f["EK"])
        if feat:
            snaps.append(f)
            if log:
                log(f"  snapshot {len(snaps)} at t={(spin + i * ref_steps) * cfg.dt:6.2f}: filtered E={f['E']:.5f}")
        secs += advance(plan_n, uhat, prm, ref_steps)
        steps += ref_steps
    return snaps, np.mean(spectra, axis=0), len(spectra), steps / secs


def seeded_snapshots(plan_n: int, plan_m: int, cfg: ClosureConfig, log=None):
    """One filtered snapshot (with closure data) from each of cfg.seeded_runs
    forced runs seeded seed + 1, seed + 2, ..., each after the spin-up."""
    prm = make_params(cfg.nu, cfg.dt, cfg.force_eps, (1, 4))
    spin = int(round(cfg.spinup_time / cfg.dt))
    chunk = max(1, int(round(0.5 / cfg.dt)))
    out = []
    for i in range(cfg.seeded_runs):
        uhat = initial_state(plan_n, cfg.n, dataclasses.replace(cfg, seed=cfg.seed + 1 + i))
        done = 0
        while done < spin:
            k = min(chunk, spin - done)
            advance(plan_n, uhat, prm, k)
            done += k
        f = filtered_state(plan_n, plan_m, uhat, cfg, True)
        del f["uc"]
        out.append(f)
        if log:
            log(f"  seeded run {i + 1} (seed {cfg.seed + 1 + i}): filtered E={f['E']:.5f}")
        del uhat
    return out


def normalisation(inv: np.ndarray, taup: np.ndarray, flux_weight: float = 1.0):
    """Input shift/scale (mean, 1/std of each invariant) and output scale (RMS
    of each frame-stress component) over the training set.  A flux weight w
    divides the scale of the diagonal components (xx, yy, zz of the frame
    stress) by sqrt(w): their normalised targets, and so their squared errors
    in the loss, grow by w, while the model's outputs are scaled back the
    same way at inference."""
    shift = inv.mean(axis=1)
    scale = 1.0 / np.maximum(inv.std(axis=1), 1e-30)
    out_scale = np.sqrt(np.mean(taup.astype(np.float64) ** 2, axis=1))
    out_scale = np.maximum(out_scale, 1e-30)
    out_scale[:3] /= np.sqrt(flux_weight)
    return shift, scale, out_scale


def init_params(seed: int) -> np.ndarray:
    """Weights N(0, 1/fan_in), biases 0, in the library's parameter layout."""
    rng = np.random.default_rng(seed)
    out = []
    for l in range(4):
        fi, fo = DIMS[l], DIMS[l + 1]
        out.append(rng.standard_normal((fo, fi)) / np.sqrt(fi))
        out.append(np.zeros(fo))
    p = np.concatenate([a.ravel() for a in out]).astype(np.float32)
    assert p.size == NPARAMS
    return p


def train(x: np.ndarray, t: np.ndarray, cfg: ClosureConfig, log=None):
    """Train on x [S][5], t [S][6] (normalised) with tarang_sgs_train: one
    shuffle of the set, then batches that are windows at SplitMix64 offsets.
    Returns (params on the device, loss history, seconds, samples/s)."""
    S = x.shape[0]
    B = min(cfg.batch, S)
    rng = np.random.default_rng(cfg.init_seed + 1)
    perm = rng.permutation(S)
    xd = torch.from_numpy(np.ascontiguousarray(x[perm], dtype=np.float32)).to(DEV)
    td = torch.from_numpy(np.ascontiguousarray(t[perm], dtype=np.float32)).to(DEV)
    p = torch.from_numpy(init_params(cfg.init_seed)).to(DEV)
    mom = torch.zeros(NPARAMS, dtype=torch.float32, device=DEV)
    var = torch.zeros_like(mom)
    every = max(1, cfg.train_steps // 20)
    nlog = cfg.train_steps // every
    losses = torch.zeros(max(nlog, 1), dtype=torch.float64, device=DEV)
    ctx = tarang_mlp_create(B)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tarang_sgs_train(ctx, p.data_ptr(), mom.data_ptr(), var.data_ptr(), 1, cfg.train_steps, xd.data_ptr(),
                         td.data_ptr(), S, B, cfg.lr, cfg.init_seed + 2, losses.data_ptr(), every, _stream())
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
    finally:
        tarang_mlp_destroy(ctx)
    hist = [((i + 1) * every, float(v)) for i, v in enumerate(losses.cpu().numpy()[:nlog])]
    if log:
        for step, v in hist:
            log(f"  train step {step}: loss {v:.5f}")
    return p, hist, secs, cfg.train_steps * B / secs


def eval_loss(p, x: np.ndarray, t: np.ndarray) -> float:
    """Mean-squared error of the network on a held-out set, reduced by the
    library (the loss of tarang_mlp_loss_grad; its gradient is discarded)."""
    B = x.shape[0]
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(DEV)
    td = torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32)).to(DEV)
    g = torch.empty(NPARAMS, dtype=torch.float32, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    ctx = tarang_mlp_create(B)
    try:
        tarang_mlp_loss_grad(ctx, p.data_ptr(), xd.data_ptr(), td.data_ptr(), B, g.data_ptr(), loss.data_ptr(),
                             _stream())
        return float(loss.item())
    finally:
        tarang_mlp_destroy(ctx)


def coarse_run(plan_m: int, u0, cfg: ClosureConfig, model=None, log=None):
    """Forced coarse run from u0 (copied) for les_long_steps; the spectrum is
    sampled every les_sample_every steps.  Returns the averages over the second
    half of the first les_steps (the stated run) and over the last 80 % of the
    whole run, the final energy, and whether the run stayed finite."""
    u = u0.clone()
    prm = make_params(cfg.nu, cfg.les_dt, cfg.force_eps, (1, 4), sgs_model=model)
    every = cfg.les_sample_every
    samples = []
    done = 0
    E = float("nan")
    try:
        while done < cfg.les_long_steps:
            k = min(every, cfg.les_long_steps - done)
            E, eps, EK = tarang_ns_step(plan_m, u.data_ptr(), prm, k, True, _stream())
            done += k
            samples.append((done, np.asarray(EK)))
            if log and done % (cfg.les_long_steps // 10) == 0:
                log(f"  coarse step {done}: E={E:.5f} eps={eps:.5f}")
    except FFTKError as e:
        return dict(finite=False, error=str(e), steps=done)

    def window(lo, hi):
        sel = [EK for (st, EK) in samples if lo < st <= hi]
        return np.mean(sel, axis=0)

    return dict(finite=True, E=E, steps=done, EK_stated=window(cfg.les_steps // 2, cfg.les_steps),
                EK_long=window(cfg.les_long_steps // 5, cfg.les_long_steps))


def timed_coarse_steps(plan_m: int, u0, cfg: ClosureConfig, model, steps: int = 500) -> float:
    """Coarse steps/s without diagnostics (CUDA events on the current stream)."""
    u = u0.clone()
    prm = make_params(cfg.nu, cfg.les_dt, cfg.force_eps, (1, 4), sgs_model=model)
    advance(plan_m, u, prm, 3)
    return steps / advance(plan_m, u, prm, steps)


def shell_errors(EK, ref, kcmp: int):
    """Per-shell relative error |E(K) - E_ref(K)| / E_ref(K), K = 1..kcmp."""
    EK = np.asarray(EK)[1:kcmp + 1]
    ref = np.asarray(ref)[1:kcmp + 1]
    return np.abs(EK - ref) / ref


def _compare(EK, ref, kcmp):
    err = shell_errors(EK, ref, kcmp)
    return dict(EK=np.asarray(EK)[:kcmp + 1].tolist(), shell_rel_err=err.tolist(), max_rel_err=float(err.max()),
                mean_rel_err=float(err.mean()), shells_within_5pct=int(np.sum(err <= 0.05)))


def run(cfg: ClosureConfig, log=print):
    """The whole workflow; returns a dict of results (JSON-serialisable)."""
    res = dict(config=dataclasses.asdict(cfg))
    plan_n = fftk_plan_create(cfg.n, cfg.n, cfg.n)
    plan_m = fftk_plan_create(cfg.m, cfg.m, cfg.m)
    try:
        t0 = time.perf_counter()
        snaps, ref, nref, rate = resolved_run(plan_n, plan_m, cfg, log)
        res["resolved_seconds"] = time.perf_counter() - t0
        res["resolved_steps_per_s"] = rate
        res["ref_samples"] = nref
        res["ref_EK"] = ref[:cfg.kcmp + 1].tolist()

        # training set: every snapshot but the last, which is held out
        hold = snaps[-1] if len(snaps) > 1 else None
        tr = snaps[:-1] if len(snaps) > 1 else snaps
        u0 = snaps[0]["uc"]

        def evaluate(mdl):
            r = coarse_run(plan_m, u0, cfg, mdl, log)
            out = dict(finite=r["finite"], steps=r["steps"])
            if r["finite"]:
                out["E"] = r["E"]
                out["stated"] = _compare(r["EK_stated"], ref, cfg.kcmp)
                out["long"] = _compare(r["EK_long"], ref, cfg.kcmp)
            else:
                out["error"] = r["error"]
            return out

        variants = []
        first = None

        def train_variants(tr, hold, targets, data):
            nonlocal first
            for target, w in [(tg, w) for tg in targets for w in cfg.flux_weights]:
                inv = np.concatenate([s[target]["inv"] for s in tr], axis=1)
                taup = np.concatenate([s[target]["taup"] for s in tr], axis=1)
                shift, scale, out_scale = normalisation(inv, taup, w)
                x = ((inv.T - shift) * scale).astype(np.float32)
                t = (taup.T / out_scale).astype(np.float32)
                del inv, taup
                p, hist, secs, sps = train(x, t, cfg, log)
                v = dict(data=data, target=target, flux_weight=w, train_seconds=secs, train_samples_per_s=sps,
                         loss_history=hist, train_set=int(x.shape[0]),
                         normalisation=dict(in_shift=shift.tolist(), in_scale=scale.tolist(),
                                            out_scale=out_scale.tolist()))
                if hold is not None:
                    xh = ((hold[target]["inv"].T - shift) * scale)
                    th = hold[target]["taup"].T / out_scale
                    v["heldout_loss"] = eval_loss(p, xh, th)
                    v["heldout_loss_zero_model"] = float(np.mean(th ** 2))
                model = make_sgs_model(p.data_ptr(), shift, scale, out_scale)
                v["model"] = evaluate(model)
                variants.append(v)
                if first is None:
                    first = (p, model, v)

        train_variants(tr, hold, cfg.targets, "time-sampled")
        if cfg.seeded_runs > 1:
            sn = seeded_snapshots(plan_n, plan_m, dataclasses.replace(cfg, targets=tuple(cfg.seeded_targets)), log)
            train_variants(sn[:-1], sn[-1], cfg.seeded_targets, "seeded")
            del sn
        p, model, v = first
        for k in ("train_seconds", "train_samples_per_s", "loss_history", "train_set", "heldout_loss",
                  "heldout_loss_zero_model", "normalisation"):
            if k in v:
                res[k] = v[k]
        res["model"] = v["model"]
        res["flux_weight"] = v["flux_weight"]
        res["target"] = v["target"]
        if len(variants) > 1:
            res["variants"] = [{k: x[k] for k in x if k not in ("loss_history", "normalisation")} for x in variants]
        res["no_model"] = evaluate(None)
        res["coarse_steps_per_s"] = timed_coarse_steps(plan_m, u0, cfg, model)
        res["coarse_steps_per_s_no_model"] = timed_coarse_steps(plan_m, u0, cfg, None)
        # wall-clock per unit of simulated time, resolved over coarse
        res["speedup"] = (res["coarse_steps_per_s"] * cfg.les_dt) / (rate * cfg.dt)
        res["params_checksum"] = float(np.abs(p.cpu().numpy().astype(np.float64)).sum())
    finally:
        fftk_plan_destroy(plan_m)
        fftk_plan_destroy(plan_n)
    return res
