"""Parity of the concat type-embedding mode (the embedding net reads
[s, T_j, T_i]; the library folds the type rows of the first layer into a
bias per (centre, neighbour) type) with the FP64 oracle, on the FP32 path
(SIMT embedding net) and the 16-bit path (tensor-core embedding net)."""

import numpy as np
import pytest

import synth
from oracle import energy_force_virial

from gpu_helpers import weight_file, force_rmse, FP32_FORCE_RMSE, BF16_FORCE_RMSE

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp16x"])
@pytest.mark.parametrize("system", ["water", "lattice"])
def test_concat_mode(concat_model, water, precision, system):
    import paper_2604_07276_gb300 as p

    cfg, w, om = concat_model
    coord, atype, box = water if system == "water" else synth.lattice_system(700, seed=29)
    m = p.DPA1(weight_file(cfg, w, "concat"), precision=precision)
    E, F, W, e = m.compute(coord, box, atype, atom_energy=True)
    m.close()
    rE, re, rF, rW = energy_force_virial(om, coord, box, atype)
    frms = float(np.sqrt(np.mean(rF * rF)))
    assert frms > 0.1  # the types matter: forces of a real size
    if precision == "fp32":
        assert force_rmse(F, rF) <= FP32_FORCE_RMSE, force_rmse(F, rF)
        assert np.abs(e - re).max() <= 1e-5
    else:
        # as for the model with non-zero biases in the 16-bit tests: rounding
        # the weights to FP16 shifts atomic energies by up to a few 1e-3 eV
        assert force_rmse(F, rF) <= BF16_FORCE_RMSE, force_rmse(F, rF)
        assert np.abs(e - re).max() <= 2.5e-3
    assert np.abs(W - rW).max() <= 5e-3 * max(1.0, np.abs(rW).max())


def test_concat_mode_rejects_training():
    """The training calls support strip mode only; they refuse a concat
    model instead of training the wrong parameters."""
    import dataclasses

    import torch

    import paper_2604_07276_gb300 as p

    cfg = dataclasses.replace(synth.STUDENT_CONFIG, tebd_input_mode="concat")
    w = synth.make_weights(cfg, seed=3)
    m = p.DPA1(weight_file(cfg, w, "concat_student"), precision="fp32")
    coord, atype, box = synth.water_box(seed=0)
    dev = torch.device("cuda", 0)
    c = torch.tensor(coord, dtype=torch.float64, device=dev)
    t = torch.tensor(atype, dtype=torch.int32, device=dev)
    b = torch.tensor(p.box9(box), dtype=torch.float64, device=dev)
    f = torch.zeros_like(c)
    loss = torch.zeros(3, dtype=torch.float64, device=dev)
    with pytest.raises(p.DPError):
        m.train_frame(c, b, t, 0.0, f, loss)
    m.close()
