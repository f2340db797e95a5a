"""The stored output scales of the seeded models reproduce what they were
calibrated to: the FP64 oracle's force RMS on the 192-atom water box (seed 0)
is 1.0 eV/A with seed-0 weights.  The values were written by
``oracle/calibrate_out_scale.py``; this keeps them in step with the oracle."""

import numpy as np
import pytest

import synth
from oracle import OracleModel, energy_force_virial


@pytest.mark.parametrize("cfg", [synth.DEFAULT_CONFIG, synth.PAPER_SIZE_CONFIG], ids=["default", "paper-size"])
def test_output_scale_gives_unit_force_rms(cfg):
    coord, atype, box = synth.water_box(seed=0)
    w = synth.make_weights(cfg, seed=0)
    _, _, f, _ = energy_force_virial(OracleModel.from_numpy(cfg, w), coord, box, atype)
    assert abs(float(np.sqrt(np.mean(f * f))) - 1.0) < 1e-9
