"""Write the FP64 oracle's results for the 64x64 RGB parity workload.

Workload: 64x64x3 synthetic Voronoi image (4 regions, noise sigma 0.05, no ramp), window
radius 2, T = 20 Euler steps, 30 DAL iterations per multiplier step, 10 multiplier steps,
paper constants otherwise (dt 0.25, E = [2, 1100]^2, eps0 = 57, rho = gamma = 1e-2,
Armijo sigma0 = 1, b = 1/2, c = 1e-4).  Fidelity alpha = 3000 (the paper's ADMM runs)
and alpha = 100 (strong clustering on a 64x64 grid).  Seeds 0, 1, 2.

The input image is cast to float32 and back (the CUDA path's storage) before the oracle
runs in float64.  Every stored value is computed by ``oracle/`` alone.

    python tests/golden/make_oracle_parity.py
"""
import os
import sys
from multiprocessing import get_context

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

RADIUS, NSTEPS, K_IN, K_OUT = 2, 20, 30, 10
ALPHAS = (3000.0, 100.0)


def run(job) -> str:
    alpha, seed = job
    from oracle import Params, SolveOpts, admm_solve, cluster_labels
    from synth import make_image, PARITY_64_RGB
    c0 = make_image(PARITY_64_RGB, seed).astype(np.float32).astype(np.float64)
    p = Params(radius=RADIUS, nsteps=NSTEPS, alpha=alpha)
    o = SolveOpts(k_out=K_OUT, k_in=K_IN)
    res = admm_solve(c0, p, o)
    labels, count = cluster_labels(res["c"])
    inner = res["inner"]
    out = os.path.join(HERE, f"oracle_parity64_a{int(alpha)}_seed{seed}.npz")
    np.savez_compressed(
        out, c=res["c"], eps=res["eps"], v=res["v"], mu=res["mu"], labels=labels,
        count=count,
        trials=np.array([i.trials for i in inner]),
        tau=np.array([i.tau for i in inner]),
        L0=np.array([i.L0 for i in inner]),
        L=np.array([i.L for i in inner]),
        stalled=np.array([i.stalled for i in inner]),
        stationary=np.array([i.stationary for i in inner]),
        gnorm2=np.array([i.gnorm2 for i in inner]),
        gap=np.array([s["gap"] for s in res["outer"]]),
        Ltilde=np.array([s["Ltilde"] for s in res["outer"]]),
        params=np.array([RADIUS, NSTEPS, K_IN, K_OUT, alpha]))
    return out


if __name__ == "__main__":
    jobs = [(a, s) for a in ALPHAS for s in (0, 1, 2)]
    with get_context("spawn").Pool(len(jobs)) as pool:
        for path in pool.map(run, jobs):
            print("wrote", path)
