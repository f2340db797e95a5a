"""Dense boxes (0.17 atoms/A^3, ~150 candidates per centre) where the
nearest-sel cap applies to nearly every centre, on both paths and with
sel = 128 (every row of an atom's 128-row tile in use).  Energies, atomic
energies, forces and the virial against the FP64 oracle, over all 1,500
atoms."""

import dataclasses
import functools

import numpy as np
import pytest

import synth
from oracle import OracleModel, energy_force_virial, neighbor_list

from gpu_helpers import weight_file, force_rmse, FP32_FORCE_RMSE, BF16_FORCE_RMSE, BF16_ATOM_ENERGY

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _reference(sel):
    cfg = dataclasses.replace(synth.DEFAULT_CONFIG, sel=sel)
    w = synth.make_weights(cfg, seed=0)
    coord, atype, box = synth.lattice_system(1500, seed=17, density=0.17)
    _, _, ncand = neighbor_list(coord, box, cfg.rcut, cfg.sel)
    ref = energy_force_virial(OracleModel.from_numpy(cfg, w), coord, box, atype)
    return cfg, w, (coord, atype, box), ncand, ref


@pytest.mark.parametrize("precision", ["fp32", "fp16x"])
@pytest.mark.parametrize("sel", [120, 128])
def test_dense_box_with_sel_cap(precision, sel):
    import paper_2604_07276_gb300 as p

    cfg, w, (coord, atype, box), ncand, (rE, re, rF, rW) = _reference(sel)
    assert (ncand > sel).mean() > 0.9  # the cap is active for nearly every centre
    m = p.DPA1(weight_file(cfg, w, f"dense_sel{sel}"), precision=precision)
    m.reserve(len(coord))
    E, F, W, e = m.compute(coord, box, atype, atom_energy=True)
    mx, ntrunc = m.stats()
    m.close()
    assert mx == sel and ntrunc == int((ncand > sel).sum())
    frmse = force_rmse(F, rF)
    print(f"dense sel {sel} {precision}: force rmse {frmse:.2e}, max |de_i| {np.abs(e - re).max():.2e}")
    if precision == "fp32":
        assert frmse <= FP32_FORCE_RMSE, frmse
        assert np.abs(e - re).max() <= 1e-5
    else:
        assert frmse <= BF16_FORCE_RMSE, frmse
        assert np.abs(e - re).max() <= BF16_ATOM_ENERGY
    assert np.abs(W - rW).max() <= 5e-3 * max(1.0, np.abs(rW).max())
