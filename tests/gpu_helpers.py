"""Shared helpers of the GPU tests: weight files and error metrics."""

import os
import tempfile

import numpy as np

import synth

_TMP = tempfile.mkdtemp(prefix="dpa1w_")


def weight_file(cfg, weights, tag: str) -> str:
    path = os.path.join(_TMP, f"{tag}.bin")
    if not os.path.exists(path):
        synth.write_weights(path, cfg, weights)
    return path


def force_rmse(a, b) -> float:
    d = np.asarray(a) - np.asarray(b)
    return float(np.sqrt(np.mean(d * d)))


# Tolerances against the FP64 oracle (force RMS of the default model on the
# water box is 1.0 eV/A by construction of its output scale).
FP32_FORCE_RMSE = 1e-5      # eV/A
BF16_FORCE_RMSE = 5e-3      # eV/A
BF16_ATOM_ENERGY = 1e-3     # eV, max over atoms
