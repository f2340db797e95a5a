"""The paper's own DPA-1 size (Sec. IV-B: three gated attention layers of
width 256, embedding net [32, 64, 128], fitting net [256, 256, 256]) against
the FP64 oracle: on the FP32 path, and in bf16x, whose attention cores take
the 256 features in two halves of 128 on the tensor cores.  The fused 16-bit
layer kernels (fp16x, bf16) hold a layer's weights in shared memory, which a
width of 256 does not fit; they refuse the model at dp_init."""

import numpy as np
import pytest

import synth
from oracle import OracleModel, energy_force_virial

from gpu_helpers import weight_file, force_rmse, BF16_FORCE_RMSE, BF16_ATOM_ENERGY

pytestmark = pytest.mark.gpu

PAPER_SIZE = synth.PAPER_SIZE_CONFIG


@pytest.fixture(scope="module")
def paper_model():
    """Seed-0 weights (the measured ones; force RMS 1 eV/A on the water box by
    the output scale's calibration)."""
    w = synth.make_weights(PAPER_SIZE, seed=0)
    return PAPER_SIZE, w, OracleModel.from_numpy(PAPER_SIZE, w)


@pytest.fixture(scope="module")
def paper_model_rich():
    """Seed-13 weights with biases and descriptor statistics (davg, dstd)."""
    w = synth.make_weights(PAPER_SIZE, seed=13, bias_scale=0.05, stats=True)
    return PAPER_SIZE, w, OracleModel.from_numpy(PAPER_SIZE, w)


@pytest.fixture(scope="module")
def ragged():
    return synth.lattice_system(700, seed=3)


def _check(m, om, system, force_tol, e_tol, w_rel):
    coord, atype, box = system
    E, F, W, e = m.compute(coord, box, atype, atom_energy=True)
    rE, re, rF, rW = energy_force_virial(om, coord, box, atype)
    frms = float(np.sqrt(np.mean(rF * rF)))
    assert frms > 0.05
    err = force_rmse(F, rF)
    assert err <= force_tol, (err, frms)
    assert np.abs(e - re).max() <= e_tol, np.abs(e - re).max()
    assert np.abs(W - rW).max() <= w_rel * max(1.0, np.abs(rW).max())
    return err


@pytest.mark.parametrize("weights", ["default", "rich"])
def test_paper_size_fp32(paper_model, paper_model_rich, water, weights):
    import paper_2604_07276_gb300 as p

    cfg, w, om = paper_model if weights == "default" else paper_model_rich
    m = p.DPA1(weight_file(cfg, w, f"paper_size_{weights}"), precision="fp32")
    try:
        _check(m, om, water, 1e-5, 1e-5, 1e-4)
    finally:
        m.close()


@pytest.mark.parametrize("weights", ["default", "rich"])
def test_paper_size_bf16x(paper_model, paper_model_rich, water, ragged, weights):
    import paper_2604_07276_gb300 as p

    cfg, w, om = paper_model if weights == "default" else paper_model_rich
    m = p.DPA1(weight_file(cfg, w, f"paper_size_{weights}"), precision="bf16x")
    try:
        for system in (water, ragged):
            _check(m, om, system, BF16_FORCE_RMSE, BF16_ATOM_ENERGY, 1e-3)
    finally:
        m.close()


def test_paper_size_bf16x_concat(water):
    """The concat type-embedding form (the embedding net reads [s, T_j, T_i])
    at the paper's size, on the tensor-core embedding net."""
    import dataclasses

    import paper_2604_07276_gb300 as p

    cfg = dataclasses.replace(PAPER_SIZE, tebd_input_mode="concat")
    w = synth.make_weights(cfg, seed=19, bias_scale=0.05)
    om = OracleModel.from_numpy(cfg, w)
    m = p.DPA1(weight_file(cfg, w, "paper_size_concat"), precision="bf16x")
    try:
        _check(m, om, water, BF16_FORCE_RMSE, BF16_ATOM_ENERGY, 1e-3)
    finally:
        m.close()


def test_paper_size_bf16x_deterministic(paper_model, ragged):
    import paper_2604_07276_gb300 as p

    cfg, w, _ = paper_model
    coord, atype, box = ragged
    m = p.DPA1(weight_file(cfg, w, "paper_size_default"), precision="bf16x")
    try:
        a = m.compute(coord, box, atype, atom_energy=True)
        b = m.compute(coord, box, atype, atom_energy=True)
    finally:
        m.close()
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("precision", ["fp16x", "bf16"])
def test_paper_size_fused_16bit_refused(paper_model, precision):
    import paper_2604_07276_gb300 as p

    cfg, w, _ = paper_model
    with pytest.raises(p.DPError):
        p.DPA1(weight_file(cfg, w, "paper_size_default"), precision=precision)
