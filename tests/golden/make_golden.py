"""Write the stored expected values used by the GPU tests. Calls only the CPU oracle.

    python tests/golden/make_golden.py

c1_lu_receivers.json: the 16^3 @0.5 m, 100 kHz, three-VTI-layer workload (seed 0): total H at the
three coaxial receivers from the exact discrete solution of eq. 8 (dense LU of I - G dsigma,
``oracle.solve.forward(method="lu")``), the FP64 relative residual of that solution (eq. 9), and how
far the oracle's own restarted GMRES(30) at tol 1e-8 lands from it (the scale of the difference a
1e-8-residual solution may legitimately show).
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import solve  # noqa: E402
from paper_2306_17537_gb300 import inputs  # noqa: E402


def c1(seed=0):
    wl = inputs.config1(seed)
    H_lu, info = solve.forward(wl.grid, wl.sigma6, wl.sigma0, wl.freq, wl.sources, wl.receivers, method="lu")
    H_gm, ginfo = solve.forward(wl.grid, wl.sigma6, wl.sigma0, wl.freq, wl.sources, wl.receivers,
                                method="gmres", tol=1e-8, restart=30, max_inner=20000)
    diff = float(np.max(np.abs(H_gm - H_lu)) / np.max(np.abs(H_lu)))
    return {
        "workload": wl.name, "seed": seed, "method": "oracle dense LU of eq. 8",
        "receivers": wl.receivers.tolist(),
        "H_re": H_lu.real.tolist(), "H_im": H_lu.imag.tolist(),
        "lu_rel_residual": info.rel_residual,
        "oracle_gmres30_iterations": ginfo.gmres_iters, "oracle_gmres30_rel_residual": ginfo.rel_residual,
        "oracle_gmres30_vs_lu_max_rel": diff,
    }


if __name__ == "__main__":
    out = c1(0)
    with open(os.path.join(HERE, "c1_lu_receivers.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if not k.startswith("H_")}, indent=1))
