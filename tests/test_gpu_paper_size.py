"""The paper's own DPA-1 size (three gated attention layers of width 256,
embedding net [32, 64, 128], fitting net [256, 256, 256]) on the FP32 path,
against the FP64 oracle.  The 16-bit paths have no kernels for an attention
width of 256 and refuse the model at dp_init."""

import dataclasses

import numpy as np
import pytest

import synth
from oracle import OracleModel, energy_force_virial

from gpu_helpers import weight_file, force_rmse

pytestmark = pytest.mark.gpu

PAPER_SIZE = dataclasses.replace(synth.DEFAULT_CONFIG, embed=(32, 64, 128), attn_layers=3, attn_dim=256,
                                 fitting=(256, 256, 256), out_scale=10.0)


@pytest.fixture(scope="module")
def paper_model():
    w = synth.make_weights(PAPER_SIZE, seed=13, bias_scale=0.05)
    return PAPER_SIZE, w, OracleModel.from_numpy(PAPER_SIZE, w)


def test_paper_size_fp32(paper_model, water):
    import paper_2604_07276_gb300 as p

    cfg, w, om = paper_model
    coord, atype, box = water
    m = p.DPA1(weight_file(cfg, w, "paper_size"), precision="fp32")
    E, F, W, e = m.compute(coord, box, atype, atom_energy=True)
    m.close()
    rE, re, rF, rW = energy_force_virial(om, coord, box, atype)
    frms = float(np.sqrt(np.mean(rF * rF)))
    assert frms > 0.05
    assert force_rmse(F, rF) <= 1e-5 * max(1.0, frms), (force_rmse(F, rF), frms)
    assert np.abs(e - re).max() <= 1e-5 * max(1.0, np.abs(re).max())
    assert np.abs(W - rW).max() <= 1e-4 * max(1.0, np.abs(rW).max())


@pytest.mark.parametrize("precision", ["fp16x", "bf16"])
def test_paper_size_16bit_refused(paper_model, precision):
    import paper_2604_07276_gb300 as p

    cfg, w, _ = paper_model
    with pytest.raises(p.DPError):
        p.DPA1(weight_file(cfg, w, "paper_size"), precision=precision)
