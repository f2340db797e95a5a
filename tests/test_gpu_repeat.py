"""Bitwise repeatability under load: every precision evaluates a 2,000-atom box
several times (through the host and the device entry points) and must give
the same bits each time.  The sums of the library run in fixed orders, so any
difference means a race between threads, blocks or phases of a kernel (a
staging block reused before every thread had read it was found this way).
The paper-size model covers the attention cores' two-half branch."""

import numpy as np
import pytest

import synth

from gpu_helpers import weight_file

pytestmark = pytest.mark.gpu

REPEATS = 5


def _repeat(m, coord, atype, box):
    import torch

    import paper_2604_07276_gb300 as p

    ref = m.compute(coord, box, atype, atom_energy=True)
    for _ in range(REPEATS - 1):
        got = m.compute(coord, box, atype, atom_energy=True)
        for x, y in zip(ref, got):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    # the device entry point, repeated: the same bits
    n = len(coord)
    dev = torch.device("cuda", 0)
    c = torch.tensor(coord, dtype=torch.float64, device=dev)
    t = torch.tensor(atype, dtype=torch.int32, device=dev)
    b = torch.tensor(p.box9(box), dtype=torch.float64, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    W = torch.zeros(9, dtype=torch.float64, device=dev)
    runs = []
    for _ in range(3):
        m.compute_device(c, b, t, E, F, W)
        torch.cuda.synchronize()
        runs.append((float(E.item()), F.cpu().numpy().copy(), W.cpu().numpy().copy()))
    for e_, f_, w_ in runs[1:]:
        assert e_ == runs[0][0] and np.array_equal(f_, runs[0][1]) and np.array_equal(w_, runs[0][2])


@pytest.mark.parametrize("precision", ["fp32", "fp16x", "bf16x", "bf16"])
def test_repeatable_default_model(default_model, precision):
    import paper_2604_07276_gb300 as p

    cfg, w, _ = default_model
    coord, atype, box = synth.lattice_system(2000, seed=41)
    m = p.DPA1(weight_file(cfg, w, "default"), precision=precision)
    try:
        _repeat(m, coord, atype, box)
    finally:
        m.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16x"])
def test_repeatable_paper_size(precision):
    import paper_2604_07276_gb300 as p

    cfg = synth.PAPER_SIZE_CONFIG
    w = synth.make_weights(cfg, seed=0)
    coord, atype, box = synth.lattice_system(2000, seed=43)
    m = p.DPA1(weight_file(cfg, w, "paper_size_default"), precision=precision)
    try:
        _repeat(m, coord, atype, box)
    finally:
        m.close()
