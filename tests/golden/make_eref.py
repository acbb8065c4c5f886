"""Writes eref_heis_d4_chi64.json: the reference energy E_ref of the Heisenberg
1x1, d=2, D=4, chi=64 workload (Neel-like seed plus noise, seed 0), used by the
time-to-|dE| <= 1e-7 measurement (|dE| = E_k - E_ref).

E_ref is the lowest energy of a long FP64 run of the oracle's local-metric
preconditioned L-BFGS (Sec. II, III, IV.A: GMRES(30) preconditioner, m = 200,
Hager-Zhang line search; CTMRG to 1e-10 with at most 120 iterations per
evaluation, as on the GPU path, a trial point without a converged CTMRG
counting as beyond the minimiser), stopped when the energy has changed by less
than 1e-11 over 5 iterations or after maxiter.  Calls only oracle/ and the
seeded input generators; runs for about an hour on 8 host cores.

    python tests/golden/make_eref.py [maxiter]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

from oracle import models as M  # noqa: E402
from oracle import optimize as O  # noqa: E402
from paper_2511_09546_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "eref_heis_d4_chi64.json")


def main():
    maxiter = int(sys.argv[1]) if len(sys.argv) > 1 else 300
    w = inputs.WORKLOADS["heis_d4_chi64"]
    cell = w["gen"]()
    hist = []
    t0 = time.time()
    inner = O.energy_and_gradient

    def timed(*a, **k):
        t = time.time()
        out = inner(*a, **k)
        print(f"  eval E {out[0]:.12f} conv {out[2]['converged']} {time.time() - t:.1f} s", flush=True)
        return out

    O.energy_and_gradient = timed

    def cb(rec):
        if not rec.get("failed"):
            hist.append(float(rec["f"]))
            print(f"iter {rec['k']} E {rec['f']:.14f} |g| {rec.get('gnorm', float('nan')):.3e} "
                  f"{time.time() - t0:.0f} s", flush=True)

    def stop(k, f, g):
        return len(hist) > 5 and abs(hist[-6] - hist[-1]) < 1e-11

    _, f, log = O.optimize(cell, M.heisenberg(True), w["chi"], precond=True, maxiter=maxiter, tol=1e-10,
                           callback=cb, stop=stop, ctm_maxit=120)
    E = [r["f"] for r in log if not r.get("failed") and r["f"] < float("inf")]
    rec = {"workload": "heis_d4_chi64", "model": "Heisenberg 1x1, sublattice-rotated bond", "chi": w["chi"],
           "E_ref": min(E), "iterations": len(hist), "ctm_tol": 1e-10, "ctm_maxit": 120,
           "energy_history": E, "cpu_seconds": time.time() - t0, "threads": torch.get_num_threads(),
           "source": "oracle/optimize.py, preconditioned L-BFGS, FP64, CPU"}
    with open(OUT, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(f"E_ref = {rec['E_ref']:.14f} after {rec['iterations']} iterations -> {OUT}")


if __name__ == "__main__":
    main()
