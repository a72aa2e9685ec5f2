"""Writes tests/golden/tiny_tod.txt: the oracle's TOD for a tiny seeded case.

It calls only the CPU oracle (``oracle``) and the seeded generators
(``workloads``); it is a regression fixture for the oracle itself (the paper
prints no worked numeric example to store instead).  Run from the repo root:
``python -m tests.golden.make_golden``.
"""
import os

import numpy as np


def case():
    import workloads as W
    L, K = 8, 2
    ell = np.arange(L + 1, dtype=float)
    return dict(sky=W.sky_gaussian(L, [(ell + 1) ** -2], seed=0),
                beam=W.beam_gaussian_taper(L, K, 4.0, seed=1),
                ring_theta=W.healpix_ring_theta(4), nphi=16,
                **dict(zip(("theta", "phi", "psi"), W.pointings_uniform(40, seed=2))))


if __name__ == "__main__":
    import oracle
    g = case()
    tod = oracle.tod(g["sky"], g["beam"], g["ring_theta"], g["nphi"], g["theta"], g["phi"], g["psi"])
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_tod.txt")
    np.savetxt(out, tod, fmt="%.17e",
               header="oracle TOD, L=8 K=2, Nside=4 HEALPix-like rings, nphi=16, 40 uniform "
                      "pointings (seeds 0/1/2); written by tests/golden/make_golden.py")
