"""Write octet<N>_rho0.10.json: the FP64 oracle's mean stress of the N^3
octet-truss cell at relative density 0.10 (the section 4.1 cell with the 4^3
Voigt sub-sampling of section 3.3), rotated frequencies of eq. (freqrot),
solved to a relative residual of 1e-10 for unit macro strains.

Only the oracle and the seeded geometry generator run here; the GPU tests and
the benchmark read the stored numbers, because the oracle needs about 15
minutes per load case at 128^3 and about two hours at 256^3 on eight cores.

    python tests/golden/make_octet_golden.py 128 0 3    # E11 and E23
    python tests/golden/make_octet_golden.py 256 0      # E11 (the headline cell)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import rve_inputs as ri  # noqa: E402

RHO, E, NU, DERIV, TOL = 0.10, 110e9, 0.3, 1, 1e-10


def main(n, cases):
    phi, radius = ri.octet(n, RHO)
    phi = phi.astype(np.float64)
    out = {"grid": [n, n, n], "relative_density": RHO, "radius": float(radius), "E": E, "nu": NU,
           "derivative": "rotated", "tol": TOL, "phi_mean": float(phi.mean()), "cases": []}
    path = os.path.join(HERE, f"octet{n}_rho0.10.json")
    for J in cases:
        Eb = np.eye(6)[J]
        t = time.time()
        r = oracle.solve(phi, E, NU, DERIV, Eb, tol=TOL, max_it=20000)
        out["cases"].append({"macro_strain": Eb.tolist(), "sigma_mean": [float(v) for v in r["sigma_mean"]],
                             "iterations": int(r["iterations"]), "true_residual": float(r["true_residual"]),
                             "seconds": round(time.time() - t, 1), "threads": oracle.num_threads()})
        print(J, out["cases"][-1], flush=True)
        with open(path, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(int(sys.argv[1]), [int(a) for a in sys.argv[2:]] or [0])
