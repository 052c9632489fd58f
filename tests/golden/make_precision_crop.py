"""Write the FP64 oracle reference of the precision workload's 64^3 crop.

    python tests/golden/make_precision_crop.py [--steps 5000] [--every 500]

The precision workload is the 256^3 periodic Gaussian-random-field box (shell
|k| = 12 +- 1, porosity 0.5, seed 3; tau = 1, sigma = 0.01, beta = 0.7,
contact angle 60 degrees, k = 1e-3, D = 0.05, liquid start with C = 1).  Its
FP16- and FP32-storage runs are compared with the FP64 oracle on the crop
x, y, z < 64 of that mask, run as a periodic box of its own.  This script calls
only the oracle (and the seeded mask generator) and writes
``precision_crop64_fp64.txt``: the observables every ``every`` steps, and at the
last step the velocity u = (sum c f^m) / rho^m of 4096 fluid nodes drawn with a
fixed seed.  It takes about an hour of one CPU core.
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import cglbm as O  # noqa: E402
from paper_2608_15781_b300 import synth  # noqa: E402

OUT = os.path.join(HERE, "precision_crop64_fp64.txt")
CROP = 64
SAMPLE = 4096
SAMPLE_SEED = 64


def crop_mask():
    return synth.grf_mask((256, 256, 256), 12, 0.5, 3, periodic_z=True)[:CROP, :CROP, :CROP].copy()


def params():
    return O.Params(tau=1.0, sigma=0.01, beta=0.7, theta_deg=60.0, k_rate=1e-3, diffusivity=0.05, c_init=1.0)


def sample_nodes(solid):
    """(z, y, x) of SAMPLE fluid nodes, drawn without replacement with a fixed seed."""
    fl = np.argwhere(~solid)
    idx = np.random.default_rng(SAMPLE_SEED).choice(len(fl), size=SAMPLE, replace=False)
    return fl[np.sort(idx)]


def velocity(f, solid):
    fm = f[0:19] + f[19:38]
    rho = np.where(solid, 1.0, fm.sum(axis=0))
    return np.stack([np.tensordot(O.C19[:, a].astype(np.float64), fm, axes=(0, 0)) for a in range(3)]) / rho


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--every", type=int, default=500)
    args = ap.parse_args()
    solid = crop_mask()
    g = O.Geometry(solid=solid, bc_z=0)
    p = params()
    st = O.init_state(g, p)
    rows = []
    t0 = time.time()
    for k in range(1, args.steps + 1):
        st = O.step(st, g, p)
        if k % args.every == 0:
            ob = O.observables(st, g, p)
            rows.append((k, ob["conversion"], ob["gas_saturation"], ob["mass_r"], ob["mass_p"], ob["mass_c"]))
            print(f"step {k}: conversion {ob['conversion']:.10f}, gas saturation {ob['gas_saturation']:.10f} "
                  f"({time.time() - t0:.0f} s)", flush=True)
    u = velocity(st.f, solid)
    nodes = sample_nodes(solid)
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle reference of the precision workload's 64^3 crop (x, y, z < 64 of the 256^3 periodic\n")
        fh.write("# GRF mask: shell |k| = 12 +- 1, porosity 0.5, seed 3), run periodic from the liquid start (rho^r = 1,\n")
        fh.write("# C = 1): tau = 1, sigma = 0.01, beta = 0.7, theta = 60 deg, k = 1e-3, D = 0.05.  Written by\n")
        fh.write("# tests/golden/make_precision_crop.py, which calls only the oracle.\n")
        fh.write(f"# fluid nodes {int((~solid).sum())}, steps {args.steps}\n")
        fh.write("[observables] step conversion gas_saturation mass_r mass_p mass_c\n")
        for r in rows:
            fh.write(f"{r[0]} " + " ".join(f"{v:.17g}" for v in r[1:]) + "\n")
        fh.write(f"[velocity] z y x ux uy uz at step {args.steps}, {SAMPLE} fluid nodes (seed {SAMPLE_SEED})\n")
        for z, y, x in nodes:
            fh.write(f"{z} {y} {x} " + " ".join(f"{u[a, z, y, x]:.17g}" for a in range(3)) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
