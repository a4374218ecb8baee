#!/usr/bin/env python
"""Write the FP64 oracle's whole-fit results at full size for the end-to-end
parity tests (tests/test_gpu_fullsize_fit.py).

The inputs are tests/cases.py's full-size recipe (the 1 mm or 0.8 mm volume,
the 3-contrast 8/8/6-echo protocol, seeded phantom and Rician noise, float32
images, or their bfloat16 values with --echo bf16).  The fit is the headline
schedule: constant initial maps, 20 Newton updates of 30 PCG iterations,
lambda = 10, eps = 1e-3, then the posterior variance.  Everything stored is
computed by the oracle (its threaded build, bit-identical to the serial one):

  F, nll, jtv      objective and its parts before every update and at the end
  cg_rel           |r_end| / |r_0| of every solve
  idx, y, var      maps and posterior variances at seeded sample voxels
                   (uniform over the volume plus voxels on its faces)
  y_blocks         per-map means over 16^3 blocks (whole-volume summary)

  python tests/golden/make_fullsize.py --config 1mm --echo f32 [--threads N]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, os.path.dirname(HERE)):
    if p not in sys.path:
        sys.path.insert(0, p)

import oracle as orc  # noqa: E402
from cases import FULLSIZE_FIT, block_means, fullsize_case, sample_voxels  # noqa: E402


def golden_path(config: str, echo: str) -> str:
    return os.path.join(HERE, f"fullsize_fit_{config}_{echo}.npz")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", choices=["1mm", "0.8mm"], default="1mm")
    ap.add_argument("--echo", choices=["f32", "bf16"], default="f32")
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0: all cores)")
    a = ap.parse_args(argv)
    threads = orc.use_threads(a.threads)
    t0 = time.time()
    d = fullsize_case(a.config, a.echo)
    shape, vx = d["shape"], d["vx"]
    f = FULLSIZE_FIT
    p = orc.make_problem(d["prot"], shape, vx=vx, lam=f["lam"], eps=f["eps"])
    t1 = time.time()
    r = orc.fit(p, d["x"], None, d["b1p"], d["b1m"], gn_iters=f["gn_iters"],
                cg_iters=f["cg_iters"])
    assert r["iters"] == f["gn_iters"], r["iters"]
    nll, g, h = orc.grad_hess(p, d["x"], r["y"], d["b1p"], d["b1m"])
    _, w = orc.jtv(p, r["y"])
    var, _, _, st = orc.uncertainty(p, h, w)
    assert st == 0
    t2 = time.time()
    idx = sample_voxels(shape)
    out = golden_path(a.config, a.echo)
    np.savez_compressed(
        out, shape=np.array(shape), vx=np.array(vx), echo=a.echo,
        gn_iters=f["gn_iters"], cg_iters=f["cg_iters"], lam=f["lam"], eps=f["eps"],
        seed=f["seed"], F=r["F"], nll=r["nll"], jtv=r["jtv"], cg_rel=r["cg_rel"], idx=idx,
        y=r["y"][:, idx], var=var[:, idx], y_blocks=block_means(r["y"], shape))
    print(f"{out}: inputs {t1 - t0:.0f} s, oracle fit + variance {t2 - t1:.0f} s on "
          f"{threads} threads; F {r['F'][0]:.6e} -> {r['F'][-1]:.6e}")


if __name__ == "__main__":
    main()
