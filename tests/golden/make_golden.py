"""Writes the stored oracle values that the GPU tests compare with, for cases
whose oracle run takes minutes (so that the GPU suite does not repeat it).
Every number comes from oracle/ (FP64, CPU) on inputs from the seeded
generators; nothing here calls the CUDA path.

  python tests/golden/make_golden.py rangefinder   # D=5, chi=44 truncated-SVD case
  python tests/golden/make_golden.py lbfgs         # plain (5) and preconditioned (3) L-BFGS iterations
  python tests/golden/make_golden.py lbfgs_bp      # mean-field (chi = 1) preconditioned L-BFGS iteration
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from oracle import ctmrg as OC  # noqa: E402
from oracle import gradient as OG  # noqa: E402
from oracle import models as OM  # noqa: E402
from oracle import optimize as OO  # noqa: E402
from paper_2511_09546_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _write(name, rec):
    rec["threads"] = torch.get_num_threads()
    with open(os.path.join(HERE, name), "w") as fh:
        json.dump(rec, fh, indent=1)
    print("wrote", name, flush=True)


def rangefinder():
    """Heisenberg 1x1 (rotated), random D=5 tensor (uniform seed 3), chi=44: the
    four-corner product is 1100 x 1100, beyond the size where the GPU path cold
    starts its projector SVD from a random range finder, and its cut is
    resolvable (relative gap (s_chi - s_chi+1) / s_1 about 1.8e-8)."""
    D, chi, seed, tol = 5, 44, 3, 1e-11
    cell = inputs.uniform_cell(1, 1, 2, D, seed)
    t0 = time.time()
    E, g, info = OG.energy_and_gradient(cell, OM.heisenberg(True), chi, tol=tol, maxit=800, return_info=True)
    gap = min(OC.cut_gaps(1, 1, OC.as_torch_cell(cell), info["env"], chi))
    _write(f"rangefinder_d{D}_chi{chi}.json",
           {"case": f"uniform_cell(1, 1, 2, {D}, seed={seed}), Heisenberg rotated", "D": D, "chi": chi,
            "seed": seed, "ctm_tol": tol, "E": E, "grad": g[0][0].ravel().tolist(), "min_cut_gap": gap,
            "ctm_iters": info["ctm_iters"], "adjoint_residual": info["adjoint_residual"],
            "seconds": time.time() - t0})


def lbfgs():
    """Oracle L-BFGS iterates at D=2, chi=16: 5 plain iterations from the seeded
    Neel-like start (the D=1 Neel state embedded in D=2 plus 1e-2 noise) and 3
    preconditioned iterations from the seeded random start of the survey's first
    configuration.  (From the random start the plain method's line searches run
    their whole 40-evaluation budget at every iteration; from the Neel-like start
    the preconditioned method's do from its second iteration on, because the
    near-product state's local metric is nearly singular and delta = |g|^2 is
    tiny: both too long for the GPU suite.)"""
    out = {}
    for name, pre, iters, wname in (("plain", False, 5, "heis_d2_chi16_neel"),
                                    ("preconditioned", True, 3, "heis_d2_chi16")):
        w = inputs.WORKLOADS[wname]
        t0 = time.time()
        cell = w["gen"]()

        def cb(rec):
            print(name, rec, flush=True)

        _, _, log = OO.optimize(cell, OM.heisenberg(True), w["chi"], precond=pre, maxiter=iters, tol=1e-11,
                                ctm_maxit=150, callback=cb)
        out[name] = {"workload": wname, "iterations": iters,
                     "log": [{k: (float(v) if k != "k" else int(v)) for k, v in r.items()} for r in log],
                     "seconds": time.time() - t0}
    _write("lbfgs_heis_d2_chi16.json", {"ctm_tol": 1e-11, "ctm_maxit": 150, **out})


def lbfgs_bp():
    """The first oracle L-BFGS iteration with the mean-field (chi = 1) metric
    preconditioner (Sec. III.B, App. A) from the seeded Neel-like D=2 start,
    chi = 16.  (Its second line search runs the whole 40-evaluation budget.)"""
    w = inputs.WORKLOADS["heis_d2_chi16_neel"]
    t0 = time.time()

    def cb(rec):
        print("bp", rec, flush=True)

    _, _, log = OO.optimize(w["gen"](), OM.heisenberg(True), w["chi"], precond="bp", maxiter=1, tol=1e-11,
                            ctm_maxit=150, callback=cb)
    _write("lbfgs_bp_heis_d2_chi16.json",
           {"ctm_tol": 1e-11, "ctm_maxit": 150, "bp_tol": 1e-12, "bp_maxit": 1000,
            "workload": "heis_d2_chi16_neel", "iterations": 1,
            "log": [{k: (float(v) if k != "k" else int(v)) for k, v in r.items()} for r in log],
            "seconds": time.time() - t0})


if __name__ == "__main__":
    {"rangefinder": rangefinder, "lbfgs": lbfgs, "lbfgs_bp": lbfgs_bp}[sys.argv[1]]()
