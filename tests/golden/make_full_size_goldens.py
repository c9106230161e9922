"""Writes the oracle's whole-run results on a full-size workload to a golden
file that the GPU parity tests compare against.

Calls only the oracle (oracle/) and the seeded input recipes (inputs.py, no
method arithmetic).  Run once per workload; a whole run of the oracle on the
differentiation workload (N = 2^18, d = 54) takes about 20 minutes on 8 cores
and about 20 GB of memory, on the scale workload (N = 2^20, d = 28) about an
hour on 16 cores and about 60 GB:

    python tests/golden/make_full_size_goldens.py differentiation
    python tests/golden/make_full_size_goldens.py scale [--out DIR]

The file records, for the workload's seeded data:
  * every node's rank and a 64-bit FNV-1a hash of its skeleton list (tree
    positions in pivot order), so that a test can first check that the GPU
    approximates the same K~ (Algorithm 1) before comparing solutions;
  * the oracle's solution x = (lambda I + K~)^-1 b (Algorithm 3) and the
    gradient dL/db of L = ||x - y||^2 at 2,000 seeded point indices, with
    ||x||, L, dL/dlambda, dL/dh and the oracle's own relative residual
    (Eq. e:errors) of x (the scale workload has no loss and no gradient);
  * scale workload: also the oracle's direct solution refined by the
    oracle's own steps x += (lambda I + K~)^-1 (b - (lambda I + K~) x) until
    the residual stops falling (its K~ is ill-conditioned: the direct solve
    alone reaches eps_r ~ 1e-8), at the same indices, with its residual.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1701_02324_gb300 import inputs  # noqa: E402

N_SAMPLED = 2000


def fnv1a64(values) -> int:
    """64-bit FNV-1a over the little-endian bytes of int64 values."""
    h = 0xCBF29CE484222325
    for v in values:
        for byte in int(v).to_bytes(8, "little", signed=True):
            h ^= byte
            h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def golden_path(name: str) -> str:
    return os.path.join(HERE, f"{name}_oracle.json")


def make(name: str) -> dict:
    if name == "differentiation":
        p = inputs.differentiation()
        y = p.extra["y"]
    elif name == "scale":
        p = inputs.scale()
        y = None
    else:
        raise SystemExit(f"unknown workload {name}")
    b = p.B[:, 0]
    t0 = time.time()
    o = oracle.Oracle(p.X, p.m)
    o.skeletonize(p.h, p.tau, p.s_max, n_samp=p.n_samp, seed=p.seed)
    st = o.factorize(p.lam)
    t1 = time.time()
    x = o.solve(b)
    eps = o.residual(b, x)
    idx = np.sort(np.random.default_rng(20260 + p.N).choice(p.N, size=N_SAMPLED, replace=False))
    nodes = range(2, o.nnodes + 1)
    res = {
        "workload": p.name, "N": p.N, "d": p.d, "h": p.h, "lambda": p.lam, "m": p.m, "s_max": p.s_max,
        "tau": p.tau, "n_samp": p.n_samp, "seed": p.seed, "depth": o.D, "factorize_status": int(st),
        "ranks": [o.rank(a) for a in nodes],
        "skel_fnv1a64": [format(fnv1a64(o.skel(a)), "016x") for a in nodes],
        "index": idx.tolist(),
        "x": [repr(float(v)) for v in x[idx]],
        "x_norm": float(np.linalg.norm(x)), "eps_r": float(eps),
    }
    if y is not None:
        dldb, dldl, dldh = o.grad(x, 2.0 * (x - y))
        res.update({"dL_db": [repr(float(v)) for v in dldb[idx]], "loss": float(np.sum((x - y) ** 2)),
                    "dL_dlambda": float(dldl), "dL_dh": float(dldh)})
    else:
        xr, er, steps = x.copy(), eps, 0
        while steps < 8:
            cand = xr + o.solve(b - o.matvec(xr))
            ec = o.residual(b, cand)
            if not ec < 0.5 * er:
                break
            xr, er, steps = cand, ec, steps + 1
        res.update({"x_refined": [repr(float(v)) for v in xr[idx]], "x_refined_norm": float(np.linalg.norm(xr)),
                    "eps_r_refined": float(er), "refine_steps": steps})
    res["oracle_seconds"] = round(time.time() - t0, 1)
    res["factorize_seconds"] = round(t1 - t0, 1)
    return res


if __name__ == "__main__":
    args = sys.argv[1:]
    out_dir = HERE
    if "--out" in args:
        i = args.index("--out")
        out_dir = args[i + 1]
        del args[i:i + 2]
    for name in args or ["differentiation"]:
        res = make(name)
        path = os.path.join(out_dir, f"{name}_oracle.json")
        with open(path, "w") as fh:
            json.dump(res, fh, indent=0)
        print(name, "written:", path, f"({res['oracle_seconds']} s)")
