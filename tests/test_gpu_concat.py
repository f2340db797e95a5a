"""Parity of the concat type-embedding mode (the embedding net reads
[s, T_j, T_i]; the library folds the type rows of the first layer into a
bias per (centre, neighbour) type) with the FP64 oracle, on the FP32 path
(SIMT embedding net) and the 16-bit path (tensor-core embedding net)."""

import numpy as np
import pytest

import synth
from oracle import energy_force_virial

from gpu_helpers import weight_file, force_rmse, FP32_FORCE_RMSE, BF16_FORCE_RMSE, BF16_ATOM_ENERGY

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
        assert force_rmse(F, rF) <= BF16_FORCE_RMSE, force_rmse(F, rF)
        assert np.abs(e - re).max() <= BF16_ATOM_ENERGY, np.abs(e - re).max()
    assert np.abs(W - rW).max() <= 5e-3 * max(1.0, np.abs(rW).max())


@pytest.mark.parametrize("pe,pf", [(1.0, 0.0), (0.0, 1.0)])
def test_concat_training_gradient(default_model, pe, pf):
    """Training in concat mode: the loss gradient against the FP64 oracle's
    double backward.  The type rows of em_W0 are not trained (they stay fixed
    with the type embedding), so the oracle's gradient for them is dropped."""
    import dataclasses

    import torch

    import paper_2604_07276_gb300 as p
    from oracle import OracleModel
    from oracle.student import loss_and_grad

    _, _, om_t = default_model
    coord, atype, box = synth.water_box(seed=0)
    E_ref, _, F_ref, _ = energy_force_virial(om_t, coord, box, atype)
    cfg = dataclasses.replace(synth.STUDENT_CONFIG, tebd_input_mode="concat")
    w = synth.make_weights(cfg, seed=3, bias_scale=0.1)
    m = p.DPA1(weight_file(cfg, w, "concat_student"), precision="fp32")
    L, lE, lF, g_ref = loss_and_grad(OracleModel.from_numpy(cfg, w), coord, box, atype, E_ref, F_ref, pe=pe, pf=pf)
    e0, td = cfg.embed[0], cfg.tebd_dim
    g_ref = np.concatenate([g_ref[:e0], g_ref[(1 + 2 * td) * e0:]])
    dev = torch.device("cuda", 0)
    c = torch.tensor(coord, dtype=torch.float64, device=dev)
    t = torch.tensor(atype, dtype=torch.int32, device=dev)
    b = torch.tensor(p.box9(box), dtype=torch.float64, device=dev)
    fr = torch.tensor(F_ref, device=dev)
    loss = torch.zeros(3, dtype=torch.float64, device=dev)
    m.zero_grad()
    m.train_frame(c, b, t, E_ref, fr, loss, pe=pe, pf=pf)
    torch.cuda.synchronize()
    m.status()
    g = m.get_grad().astype(np.float64)
    assert g.shape == g_ref.shape
    lo = loss.cpu().numpy()
    assert abs(lo[0] - L) < 1e-5 * max(1.0, L)
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    print(f"concat pe={pe} pf={pf}: relative error {rel:.3e}")
    assert rel < 1e-5, rel
    m.close()


def test_concat_bias_update_reaches_the_type_pair_table():
    """set_params on em_b0 moves the folded per-type-pair bias: the energy
    after the update matches the oracle with the updated em_b0."""
    import dataclasses

    import paper_2604_07276_gb300 as p
    from oracle import OracleModel

    cfg = dataclasses.replace(synth.STUDENT_CONFIG, tebd_input_mode="concat")
    w = synth.make_weights(cfg, seed=3, bias_scale=0.1)
    m = p.DPA1(weight_file(cfg, w, "concat_student"), precision="fp32")
    coord, atype, box = synth.water_box(seed=0)
    e0 = cfg.embed[0]
    theta = m.get_params()
    theta[e0:2 * e0] += np.float32(0.25)
    m.set_params(theta)
    E, F, _, _ = m.compute(coord, box, atype)
    w2 = dict(w)
    w2["em_b0"] = theta[e0:2 * e0].astype(np.float64)
    w2["em_W0"] = np.array(w["em_W0"], dtype=np.float64)
    w2["em_W0"].reshape(-1)[:e0] = theta[:e0]
    rE, _, rF, _ = energy_force_virial(OracleModel.from_numpy(cfg, w2), coord, box, atype)
    rE0, _, _, _ = energy_force_virial(OracleModel.from_numpy(cfg, w), coord, box, atype)
    assert abs(rE - rE0) > 1e-2  # the update matters
    assert abs(E - rE) < 1e-4 * max(1.0, abs(rE)), (E, rE)
    assert force_rmse(F, rF) <= FP32_FORCE_RMSE
    m.close()
