"""Writes the stored expected values under tests/golden/ from the FP64 oracle
(and from nothing else).  Run from the repository root:

    python tests/golden/make_golden.py

The fixtures pin the oracle against unintended changes: a change of its
arithmetic must name, in its commit message, the passage of the paper (or the
reading of it) that justifies the new values.
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_2602_01057_gb300 import synth  # noqa: E402


def cases():
    """Small seeded cases: (name, geometry, Gaussians, header)."""
    G = synth.gaussians_uniform(12, 101, half_box=0.6, log_sigma=math.log(0.15))
    yield ("parallel", synth.geom_parallel(2, 6, 7, 0.2, 0.2, -0.5, 0.7), G,
           "parallel-beam CT, 2 views x 6 x 7, pitch 0.2, segment [-0.5, 0.7]")
    G = synth.gaussians_uniform(12, 102, half_box=0.6, log_sigma=math.log(0.15))
    yield ("cone", synth.geom_cone(2, 6, 7, 0.3, 0.3, 3.0, 4.5), G,
           "cone-beam CT, 2 views x 6 x 7, pitch 0.3, source-origin 3, source-detector 4.5")
    G = synth.gaussians_uniform(12, 103, half_box=40.0, log_sigma=math.log(8.0))
    G["mu"][:, 2] *= 0.1
    yield ("pet", synth.geom_pet(3, 9, 3, 400.0, 576, 2.0), G,
           "PET ring radius 400, 576 crystals, arc-corrected, 3 angles x 9 radial x 3 planes")


def write(name, gd, G, header):
    fwd = oracle.forward(gd, G)
    w = synth.random_weights(synth.num_rays(gd), 7)
    bwd = oracle.backward(gd, G, w)
    path = os.path.join(HERE, f"oracle_{name}.txt")
    with open(path, "w") as f:
        f.write(f"# FP64 oracle outputs, {header}; 12 seeded Gaussians (synth.gaussians_uniform).\n")
        f.write("# Forward: Eqs. 4, 7-12 with the segment erf factor and the m <= 9 cut.\n")
        f.write("# Adjoint: derivatives of Eqs. 7-11 chained through Eq. 2, weights synth.random_weights(R, 7).\n")
        f.write("# Written by tests/golden/make_golden.py (oracle only).\n")
        for i, v in enumerate(fwd["I"]):
            f.write(f"I {i} {float(v)!r}\n")
        for k in ("mu", "ls", "q", "rho"):
            for i, v in enumerate(np.asarray(bwd[k]).reshape(-1)):
                f.write(f"g_{k} {i} {float(v)!r}\n")


if __name__ == "__main__":
    oracle.build()
    for c in cases():
        write(*c)
