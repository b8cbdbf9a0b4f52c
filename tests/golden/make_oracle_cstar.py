"""Writes oracle_cstar.json: effective tensors C* of seeded sphere packings on
grids with radix-3 lengths, computed by the FP64 CPU oracle alone (oracle/,
CG to relative residual 1e-13).  The GPU tests compare the library's C* with
these values instead of re-running the oracle's direct DFTs (minutes of host
time per 48^3 solve).

Run from the repository root:  python tests/golden/make_oracle_cstar.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1411_0330_gb300 import microstructures as ms  # noqa: E402

# (E, nu) -> (bulk, shear), matrix E=1 nu=0.3, inclusions E=10 nu=0.2
EL = [[1.0 / (3.0 * 0.4), 1.0 / 2.6], [10.0 / (3.0 * 0.6), 10.0 / 2.4]]

# name: (grid n, radius in voxels, volume fraction, seed, green)
CASES = {
    "spheres48_f25_s148_filtered": (48, 6.0, 0.25, 148, oracle.FILTERED),
    "spheres48_f15_s1_r3_filtered": (48, 3.0, 0.15, 1, oracle.FILTERED),
    "spheres48_f30_s2_r3_filtered": (48, 3.0, 0.30, 2, oracle.FILTERED),
}


def main():
    oracle.build()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_cstar.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for name, (n, r, f, seed, green) in CASES.items():
        if name in out:
            continue
        ph, _, _ = ms.sphere_microstructure(n, r, f, seed=seed)
        A, infos = oracle.effective(oracle.Problem(ph, np.array(EL), physics=oracle.ELASTIC, green=green), tol=1e-13)
        out[name] = {"n": n, "radius": r, "fraction": f, "seed": seed, "green": int(green),
                     "realised_fraction": float(ph.mean()), "moduli_K_mu": EL, "tol": 1e-13,
                     "cstar_mandel": np.asarray(A).tolist()}
        print(name, float(A[0, 0]), flush=True)
        with open(path, "w") as fh:  # after every case: a long run keeps what it finished
            json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
