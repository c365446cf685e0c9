"""Write oracle_fp64_iterations.json: the iteration counts of the FP64 CPU
oracle's even-odd BiCGstab (and CG on the normal equations) solves of the
24^3 x 64 workload (links exp(0.3 i H), gauge seed 1001, Gaussian source seed
2001, tol 1e-12).  Calls only oracle/ and the input generators.  The counts
scale the bounded CPU-baseline sample of bench.py to a full solve."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import lattice_inputs as li  # noqa: E402
import oracle  # noqa: E402


def main():
    dims = (24, 24, 24, 64)
    U = li.gauge(dims, 0.3, 1001)
    b = li.gaussian_spinor(dims, 2001)
    out = {"lattice": "24x24x24x64", "eps": 0.3, "gauge_seed": 1001, "source_seed": 2001, "tol": 1e-12,
           "bicgstab_schur": {}, "cgnr_schur": {}}
    solvers = sys.argv[1:] or ["bicgstab"]
    for solver in solvers:
        for kappa in (0.12, 0.124):
            t0 = time.time()
            x, st, iters, rel = oracle.solve(b, U, dims, kappa, tol=1e-12, maxiter=20000, solver=solver)
            out[f"{solver}_schur"][f"{kappa:.3f}"] = {"iterations": iters, "status": st, "true_rel_residual": rel,
                                                      "cpu_seconds": round(time.time() - t0, 1)}
            print(solver, kappa, iters, st, rel, flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_fp64_iterations.json")
    old = json.load(open(path)) if os.path.exists(path) else {}
    for k in ("bicgstab_schur", "cgnr_schur"):
        old.setdefault(k, {}).update(out[k])
    out.update({k: old[k] for k in ("bicgstab_schur", "cgnr_schur")})
    json.dump(out, open(path, "w"), indent=1)


if __name__ == "__main__":
    main()
