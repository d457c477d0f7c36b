"""Runs the oracle's four solves of the 512^2 + 64-layer workload (kh = 0.5, Gaussian-bump k,
Gaussian source): {Bi-CGSTAB, IDR(4)} x {CSG theta_beta = 0.3, CSL shift 1 + 0.5i}, damped
Jacobi (omega 0.5) V(1,1), tol 1e-6, and writes their matvec counts and times to
oracle/workload_counts.json.  The benchmark's CPU-baseline leg uses these counts to turn the
oracle's measured time per preconditioned matvec into solves/s.  Test infrastructure: calls
only the oracle and the seeded input generators.

Usage: python -m oracle.workload_counts
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import helm_inputs as hi  # noqa: E402
from oracle import Oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_counts.json")


def main():
    p = hi.workload_2d_512()
    out = {"workload": p.name, "n": p.n, "solves": []}
    sh = hi.shadow_space(p.n, 4)
    for name, pc in (("csg", hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)),
                     ("csl", hi.Precond(kind=hi.PC_CSL, shift=1 + 0.5j, smoother=hi.SM_JACOBI, omega=0.5))):
        o = Oracle(p, pc)
        for mname, method in (("bicgstab", hi.BICGSTAB), ("idr4", hi.IDR)):
            t = time.time()
            x, info = o.solve(p.b, hi.SolveOpts(method=method, s=4, tol=1e-6, maxmv=4000), shadow=sh)
            dt = time.time() - t
            rec = dict(precond=name, method=mname, seconds=dt, **info)
            out["solves"].append(rec)
            print(rec, flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
