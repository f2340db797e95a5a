"""Compute the fitting-net output scales of the default model, of the
paper-size model and of the distillation teacher's base (the student
family).

The random-weight models have no physical energy scale, so absolute force
tolerances and thresholds would mean nothing.  Each output scale is fixed
once so that the FP64 oracle's force RMS on the 192-atom water box (seed 0)
is 1.0 eV/A; forces are linear in the scale, so one evaluation at scale 1
gives it.  Run ``python -m oracle.calibrate_out_scale`` and copy the printed
values into ``synth.model`` (``DEFAULT_CONFIG.out_scale``,
``PAPER_SIZE_CONFIG.out_scale`` and ``TEACHER_BASE_OUT_SCALE``).  Test infrastructure: only the oracle is called.
"""

import dataclasses

import numpy as np

import synth
from oracle import OracleModel, energy_force_virial


def _scale(cfg, w) -> float:
    w = dict(w)
    w["out_scale"] = np.array(1.0)
    coord, atype, box = synth.water_box(seed=0)
    _, _, f, _ = energy_force_virial(OracleModel.from_numpy(cfg, w), coord, box, atype)
    return 1.0 / float(np.sqrt(np.mean(f * f)))


def main() -> float:
    cfg = dataclasses.replace(synth.DEFAULT_CONFIG, out_scale=1.0)
    scale = _scale(cfg, synth.make_weights(cfg, seed=0))
    print("default model:", repr(scale))
    pcfg = dataclasses.replace(synth.PAPER_SIZE_CONFIG, out_scale=1.0)
    print("paper-size model:", repr(_scale(pcfg, synth.make_weights(pcfg, seed=0))))
    scfg, base = synth.teacher_base_weights()
    print("distillation teacher base:", repr(_scale(scfg, base)))
    return scale


if __name__ == "__main__":
    main()
