"""Write ns512_decay_100steps.json: the FP64 oracle's energy spectrum after
100 RK2 integrating-factor steps of 512^3 decaying turbulence.

Workload: random-phase solenoidal initial field with E(K) ~ K^4 exp(-2 (K/4)^2),
total energy 0.5, seed 0 (SplitMix64 normals), nu = 1e-3, dt = 5e-4, 2/3
dealiasing.  The initial field is the oracle's FP64 field rounded to
complex64; the oracle then evolves that rounded field in FP64.  This script
calls only oracle/ and synth/ (no GPU code).  Runtime: about an hour on 8 cores.

Usage: python tests/golden/make_ns512_golden.py [n]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def config(n=512):
    return dict(n=n, seed=0, k0=4.0, E0=0.5, nu=1e-3, dt=5e-4, steps=100)


def initial_field(cfg):
    n = cfg["n"]
    u = oracle.ic_random(synth.normal_fields(cfg["seed"], 3, (n, n, n)), k0=cfg["k0"], E0=cfg["E0"])
    return u.astype(np.complex64)


def checksum(u64: np.ndarray) -> float:
    return float(np.sum(np.abs(u64.astype(np.complex128)) ** 2 * np.arange(1, u64.shape[-1] + 1)))


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 512
    cfg = config(n)
    t0 = time.time()
    u64 = initial_field(cfg)
    E0, eps0, EK0 = oracle.diag(u64.astype(np.complex128), cfg["nu"])
    u = oracle.ns_step(u64.astype(np.complex128), cfg["nu"], cfg["dt"], cfg["steps"])
    E, eps, EK = oracle.diag(u, cfg["nu"])
    out = dict(
        description=f"FP64 oracle, {n}^3 decaying turbulence after {cfg['steps']} RK2-IF steps; "
        "written by make_ns512_golden.py from oracle/ only",
        config=cfg,
        ic_checksum=checksum(u64),
        ic=dict(E=E0, eps=eps0, EK=EK0.tolist()),
        final=dict(E=E, eps=eps, EK=EK.tolist()),
        oracle_seconds=time.time() - t0,
    )
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"ns{n}_decay_{cfg['steps']}steps.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path, out["oracle_seconds"])


if __name__ == "__main__":
    main()
