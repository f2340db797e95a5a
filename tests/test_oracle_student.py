"""Pin of the oracle's student-loss gradient (double backward through the
forces) against central finite differences of the loss in weight space."""

import dataclasses

import numpy as np
import pytest

import synth
import oracle
from oracle import OracleModel
from oracle.student import loss_and_grad, trainable_names


@pytest.mark.parametrize("mode", ["strip", "concat"])
def test_student_loss_gradient_matches_weight_space_differences(mode):
    cfg = dataclasses.replace(synth.STUDENT_CONFIG, tebd_input_mode=mode)
    w = synth.make_weights(cfg, seed=3, bias_scale=0.1)
    coord, atype, box = synth.isolated_cluster(seed=9, natoms=10)
    rng = np.random.default_rng(0)
    f_ref = rng.normal(size=coord.shape) * 0.05
    e_ref = 0.3
    m = OracleModel.from_numpy(cfg, w)
    L, lE, lF, g = loss_and_grad(m, coord, box, atype, e_ref, f_ref, pe=1.0, pf=1.0)
    assert abs(L - (lE + lF)) < 1e-15
    names = trainable_names(cfg)
    sizes = [w[k].size for k in names]
    assert g.size == sum(sizes)
    h = 1e-5
    for trial in range(3):
        d = rng.normal(size=g.size)
        def loss_at(sign):
            ww = dict(w)
            off = 0
            for k, sz in zip(names, sizes):
                ww[k] = np.asarray(w[k]) + sign * h * d[off:off + sz].reshape(np.shape(w[k]))
                off += sz
            return loss_and_grad(OracleModel.from_numpy(cfg, ww), coord, box, atype, e_ref, f_ref)[0]
        fd = (loss_at(1) - loss_at(-1)) / (2 * h)
        assert abs(fd - g @ d) < 1e-6 * max(1.0, abs(fd)), (fd, g @ d)
