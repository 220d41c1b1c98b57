"""One Adam step used as a readout of the gradient it consumed.

The training step (gcp_step) and the batched local step fold the hot-row
replicas into the gradient and apply Adam in one epilogue, so the folded
gradient is never written out.  With beta1 = beta2 = 0, the first step of
Algorithm 1 moves every factor entry by -lr g / sqrt(g^2 + eps): both bias
corrections are 1, the moments are g and g^2.  That is a one-to-one function
of g, so the factors before and after one step give g back exactly:

    u = (a0 - a1) / lr,    g = u sqrt(eps) / sqrt(1 - u^2).

Unlike a comparison of factors after an ordinary Adam step (about
-lr sign(g), blind to any rescaling of g), this checks the gradient's
values.  eps = (4 max|g|)^2 keeps |u| below 0.25, so the inversion is well
conditioned; lr = 1e6 makes each step large against factors of order one,
so the FP32 rounding of a1 costs about 1e-7 of the step.  No lower bound
applies (lower = -inf).
"""
import math

import numpy as np


def readout_params(gcp, g_max):
    """Adam hyperparameters of the readout step for gradients up to g_max."""
    eps = float(np.float32((4.0 * float(g_max)) ** 2))  # exact in the kernels' FP32
    return gcp.AdamParams(lr=1e6, beta1=0.0, beta2=0.0, eps=eps, lower=-math.inf)


def recover_gradient(a0, a1, prm):
    """The gradient one readout step consumed, from the factors before (a0)
    and after (a1) it, in FP64."""
    u = (np.asarray(a0, np.float32).astype(np.float64) - np.asarray(a1, np.float32).astype(np.float64)) / prm.lr
    assert np.all(np.abs(u) < 0.5), float(np.abs(u).max())
    return u * math.sqrt(prm.eps) / np.sqrt(1.0 - u * u)


def flat(factors):
    return np.concatenate([np.asarray(a).ravel() for a in factors])
