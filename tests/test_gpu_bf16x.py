"""Parity of the BF16-operand precision mode ("bf16x") with the FP64 oracle,
at the bounds stated for the BF16 path: force RMSE <= 5e-3 eV/A and every
atomic energy within 1e-3 eV.  Every product of the attention layers and of
the fitting net runs on tcgen05 with BF16 operands (both split in two
terms) and FP32 accumulation.  The whole 15,668-atom box is compared in
test_gpu_fullbox.py, the intermediates stage by stage in test_gpu_stages.py."""

import numpy as np
import pytest

import synth
from oracle import OracleModel, energy_force_virial

from gpu_helpers import weight_file, force_rmse, BF16_FORCE_RMSE, BF16_ATOM_ENERGY

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2604_07276_gb300 as p

    return p


@pytest.fixture(scope="module")
def bf16x_model(lib, default_model):
    cfg, w, _ = default_model
    m = lib.DPA1(weight_file(cfg, w, "default"), precision="bf16x")
    yield m
    m.close()


def _check(m, om, coord, atype, box, tag=""):
    E, F, W, e = m.compute(coord, box, atype, atom_energy=True)
    rE, re, rF, rW = energy_force_virial(om, coord, box, atype)
    frmse = force_rmse(F, rF)
    emax = float(np.abs(e - re).max()) if len(e) else 0.0
    print(f"\nbf16x {tag}: force rmse {frmse:.2e}, max |de_i| {emax:.2e}")
    assert frmse <= BF16_FORCE_RMSE, frmse
    assert emax <= BF16_ATOM_ENERGY, emax
    assert np.abs(W - rW).max() <= 5e-3 * max(1.0, np.abs(rW).max())
    return frmse, emax


def test_bf16x_water(bf16x_model, default_model, water):
    cfg, w, om = default_model
    _check(bf16x_model, om, *water, tag="water")


def test_bf16x_rich_weights(lib, rich_model, water):
    """Non-zero biases, LayerNorm gains and davg / dstd."""
    cfg, w, om = rich_model
    m = lib.DPA1(weight_file(cfg, w, "rich"), precision="bf16x")
    _check(m, om, *water, tag="rich water")
    m.close()


def test_bf16x_concat_mode(lib, concat_model, water):
    cfg, w, om = concat_model
    m = lib.DPA1(weight_file(cfg, w, "concat"), precision="bf16x")
    _check(m, om, *water, tag="concat water")
    m.close()


def test_bf16x_lattice_ragged(bf16x_model, default_model):
    cfg, w, om = default_model
    coord, atype, box = synth.lattice_system(1123, seed=31)
    _check(bf16x_model, om, coord, atype, box, tag="lattice 1123")


def test_bf16x_edge_cases(bf16x_model, default_model):
    cfg, w, om = default_model
    box = np.array([30.0, 30.0, 30.0])
    E, F, W, e = bf16x_model.compute(np.zeros((0, 3)), box, np.zeros(0, np.int32), atom_energy=True)
    assert E == 0.0 and F.shape == (0, 3)
    for coord, atype in ((np.array([[3.0, 4.0, 5.0]]), np.array([2], np.int32)),
                         (np.array([[1.0, 1.0, 1.0], [15.0, 15.0, 15.0]]), np.array([0, 4], np.int32)),
                         (np.array([[10.0, 10.0, 10.0], [11.2, 10.3, 9.9], [20.0, 20.0, 20.0], [21.0, 20.2, 20.0],
                                    [20.1, 21.1, 19.5]]), np.array([3, 0, 1, 2, 3], np.int32))):
        _check(bf16x_model, om, coord, atype, box, tag=f"{len(coord)} atoms")


def test_bf16x_deterministic_and_batch(bf16x_model, water):
    """Repeated calls are bitwise equal, and so is a packed batch of frames
    to frame-by-frame calls (every product works on one atom's rows)."""
    coord, atype, box = water
    a = bf16x_model.compute(coord, box, atype, atom_energy=True)
    b = bf16x_model.compute(coord, box, atype, atom_energy=True)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    frames = synth.frame_batch(seed=2, nframes=3, lo=200, hi=500)
    E, F, W = bf16x_model.compute_batch(frames)
    for k, (c, t, bx) in enumerate(frames):
        Ek, Fk, Wk, _ = bf16x_model.compute(c, bx, t)
        assert E[k] == Ek and np.array_equal(F[k], Fk) and np.array_equal(W[k], Wk)


def test_bf16x_without_attention(lib, water):
    """No attention layer: only the fitting net's products are BF16-split
    tensor-core GEMMs (the embedding net is FP32), whose ~2^-16 relative
    error stays far inside the BF16 bounds."""
    cfg = synth.ModelConfig(attn_layers=0, out_scale=synth.DEFAULT_CONFIG.out_scale)
    w = synth.make_weights(cfg, seed=6, bias_scale=0.1, stats=True)
    om = OracleModel.from_numpy(cfg, w)
    m = lib.DPA1(weight_file(cfg, w, "noattn"), precision="bf16x")
    frmse, emax = _check(m, om, *water, tag="no attention")
    assert frmse <= 1e-3
    m.close()



@pytest.mark.parametrize("shape", ["width256_m1_100", "width128_m1_128"])
def test_bf16x_mixed_widths(lib, water, shape):
    """The cores' two branches on the other embedding widths: attention width
    256 over M1 = 100 (two feature halves; the row-sum column inside the MMA
    width) and width 128 over M1 = 128 (one half; [P G, rowsum P] reaching
    past 128 columns), each with biases and descriptor statistics."""
    import dataclasses

    if shape == "width256_m1_100":
        cfg = dataclasses.replace(synth.DEFAULT_CONFIG, attn_layers=2, attn_dim=256)
    else:
        cfg = dataclasses.replace(synth.PAPER_SIZE_CONFIG, attn_layers=2, attn_dim=128)
    w = synth.make_weights(cfg, seed=23, bias_scale=0.05, stats=True)
    om = OracleModel.from_numpy(cfg, w)
    m = lib.DPA1(weight_file(cfg, w, shape), precision="bf16x")
    try:
        _check(m, om, *water, tag=shape)
        coord, atype, box = synth.lattice_system(400, seed=29)
        _check(m, om, coord, atype, box, tag=shape + " lattice")
    finally:
        m.close()
