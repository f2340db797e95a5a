"""Parity on sparse boxes, whose neighbour counts put the end of an atom's
neighbour rows inside the first, second and third 32-row lane quadrants and
column quarters of the layer kernels' 128-row tiles, so that every skip of
work past the last neighbour (dead quarters, dead 16-key halves, dead lane
quadrants) runs against the FP64 oracle in both the tensor-core and the FP32
paths."""

import numpy as np
import pytest

import synth
from oracle import energy_force_virial, neighbor_list

from gpu_helpers import weight_file, force_rmse, FP32_FORCE_RMSE, BF16_FORCE_RMSE, BF16_ATOM_ENERGY

pytestmark = pytest.mark.gpu

# lattice densities (atoms / A^3) and seeds: 600 atoms with 5-16, 26-44 and
# 51-69 neighbours (rcut 6 A)
CASES = [(0.012, 41), (0.04, 42), (0.065, 43)]


@pytest.mark.parametrize("precision", ["fp16x", "bf16x", "fp32"])
@pytest.mark.parametrize("density,seed", CASES)
def test_sparse_box(default_model, precision, density, seed):
    import paper_2604_07276_gb300 as p

    cfg, w, om = default_model
    coord, atype, box = synth.lattice_system(600, seed=seed, density=density)
    _, nn, _ = neighbor_list(coord, box, cfg.rcut, cfg.sel)
    assert nn.min() < nn.max()  # a spread of counts within the case
    m = p.DPA1(weight_file(cfg, w, "default"), precision=precision)
    E, F, W, e = m.compute(coord, box, atype, atom_energy=True)
    m.close()
    rE, re, rF, rW = energy_force_virial(om, coord, box, atype)
    if precision == "fp32":
        assert force_rmse(F, rF) <= FP32_FORCE_RMSE, force_rmse(F, rF)
        assert np.abs(e - re).max() <= 1e-5
    else:
        assert force_rmse(F, rF) <= BF16_FORCE_RMSE, force_rmse(F, rF)
        assert np.abs(e - re).max() <= BF16_ATOM_ENERGY
    assert np.abs(W - rW).max() <= 5e-3 * max(1.0, np.abs(rW).max())
