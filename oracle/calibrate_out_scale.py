"""Compute the fitting-net output scale of the default model.

The random-weight model has no physical energy scale, so its absolute
force tolerances would mean nothing.  The output scale is fixed once so
that the FP64 oracle's force RMS on the 192-atom water box (seed 0) with
seed-0 weights is 1.0 eV/A; forces are linear in the scale, so one
evaluation at scale 1 gives it.  Run ``python -m oracle.calibrate_out_scale``
and copy the printed value into ``synth.model.ModelConfig.out_scale``.
Test infrastructure: only the oracle is called.
"""

import dataclasses

import numpy as np

import synth
from oracle import OracleModel, energy_force_virial


def main() -> float:
    cfg = dataclasses.replace(synth.DEFAULT_CONFIG, out_scale=1.0)
    w = synth.make_weights(cfg, seed=0)
    coord, atype, box = synth.water_box(seed=0)
    _, _, f, _ = energy_force_virial(OracleModel.from_numpy(cfg, w), coord, box, atype)
    scale = 1.0 / float(np.sqrt(np.mean(f * f)))
    print(repr(scale))
    return scale


if __name__ == "__main__":
    main()
