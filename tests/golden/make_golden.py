"""Writes the stored expected values under tests/golden/ (calls only the
oracle and the seeded input generators).

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def small_gaussian():
    """50 x 40 x 30 Gaussian workload: stratified samples of iteration 0 with
    seed 3001, p = q = 1000, the sampled loss and per-mode gradient norms."""
    w = synth.workload_small_gaussian()
    idx, x, wts, att = oracle.stratified_samples(3001, 0, w["p"], w["q"], w["dims"], w["coords"], w["vals"])
    F, G = oracle.sampled_loss_grad(w["dims"], w["factors"], w["loss"], idx, x, wts)
    Ffull, Gfull = oracle.full_loss_grad(w["dims"], w["factors"], w["loss"],
                                         oracle.densify(w["dims"], w["coords"], w["vals"]))
    return {
        "workload": "50x40x30, 2000 uniform nonzeros 1+Poisson(2), rank 4, Gaussian, seed 3001, t 0, p=q=1000",
        "first_samples": idx[:8].tolist() + idx[1000:1008].tolist(),
        "zero_attempts": att,
        "sampled_loss": F,
        "sampled_grad_fro": [float(np.linalg.norm(g)) for g in G],
        "full_loss": Ffull,
        "full_grad_fro": [float(np.linalg.norm(g)) for g in Gfull],
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "small_gaussian.json"), "w") as f:
        json.dump(small_gaussian(), f, indent=1)
