"""Local and ghost atoms through dp_compute_local (Eq. eq_forcesLocalGhost):
a periodic box split into two x slabs with their rcut halos, each slab
against the oracle's evaluation of the same slab (local centres only), and
the slabs reassembled against the whole box on the same path."""

import numpy as np
import pytest

import synth
from oracle import energy_force_virial

from gpu_helpers import weight_file, force_rmse, FP32_FORCE_RMSE, BF16_FORCE_RMSE

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp16x"])
def test_local_ghost_slabs(default_model, precision):
    import paper_2604_07276_gb300 as p

    cfg, w, om = default_model
    tol = FP32_FORCE_RMSE if precision == "fp32" else BF16_FORCE_RMSE
    coord, atype, box = synth.lattice_system(1200, seed=23)
    m = p.DPA1(weight_file(cfg, w, "default"), precision=precision)
    E, F, W, _ = m.compute(coord, box, atype)
    Es, Fs, Ws = 0.0, np.zeros_like(F), np.zeros((3, 3))
    for c, t, b, nloc, owner in synth.slab_subdomains(coord, atype, box, 2, cfg.rcut):
        e, f, wv, ae = m.compute(c, b, t, atom_energy=True, nlocal=nloc)
        assert np.all(ae[nloc:] == 0.0) and np.any(ae[:nloc] != 0.0)
        rE, _, rF, rW = energy_force_virial(om, c, b, t, centres=np.arange(nloc))
        assert force_rmse(f, rF) <= tol, force_rmse(f, rF)
        assert abs(e - rE) <= (1e-5 if precision == "fp32" else 1e-3) * nloc ** 0.5
        assert np.abs(wv - rW).max() <= 5e-3 * max(1.0, np.abs(rW).max())
        Es += e
        Ws += wv
        np.add.at(Fs, owner, f)
    assert abs(Es - E) <= (1e-5 if precision == "fp32" else 1e-3) * len(coord) ** 0.5
    assert force_rmse(Fs, F) <= tol
    assert np.abs(Ws - W).max() <= 5e-3 * max(1.0, np.abs(W).max())
    # every atom local: the same as dp_compute
    e2, f2, w2, _ = m.compute(coord, box, atype, nlocal=len(coord))
    assert e2 == E and np.array_equal(f2, F) and np.array_equal(w2, W)
    # no local atom: nothing counts
    e0, f0, w0, _ = m.compute(coord, box, atype, nlocal=0)
    assert e0 == 0.0 and not np.any(f0) and not np.any(w0)
    with pytest.raises(p.DPError):
        m.compute(coord, box, atype, nlocal=len(coord) + 1)
    m.close()
