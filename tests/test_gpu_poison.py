"""Independence from stale workspace contents.  After dp_debug_poison fills a
model's whole workspace with NaN / -1 bit patterns, every precision gives the
same bits as before, on a 2,000-atom box and on the water box evaluated after
it, whose rows past each atom's last neighbour then hold the poison or the
larger box's data.  The 16-bit paths read and write only an atom's live rows
of their per-row blocks, and no path may depend on memory it does not write in
the call."""

import numpy as np
import pytest

import synth

from gpu_helpers import weight_file

pytestmark = pytest.mark.gpu


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def _check(m, big, small):
    m.reserve(len(big[0]))
    ref_big = m.compute(big[0], big[2], big[1], atom_energy=True)
    ref_small = m.compute(small[0], small[2], small[1], atom_energy=True)
    m.debug_poison()
    _same(m.compute(small[0], small[2], small[1], atom_energy=True), ref_small)
    m.debug_poison()
    _same(m.compute(big[0], big[2], big[1], atom_energy=True), ref_big)
    # the small box right after the big one: its dead rows hold the big box's data
    _same(m.compute(small[0], small[2], small[1], atom_energy=True), ref_small)


@pytest.mark.parametrize("precision", ["fp32", "fp16x", "bf16x", "bf16"])
def test_results_do_not_depend_on_stale_workspace(default_model, precision):
    import paper_2604_07276_gb300 as p

    cfg, w, _ = default_model
    m = p.DPA1(weight_file(cfg, w, "default"), precision=precision)
    try:
        _check(m, synth.lattice_system(2000, seed=41), synth.water_box(0))
    finally:
        m.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16x"])
def test_paper_size_does_not_depend_on_stale_workspace(precision):
    import paper_2604_07276_gb300 as p

    cfg = synth.PAPER_SIZE_CONFIG
    w = synth.make_weights(cfg, seed=0)
    m = p.DPA1(weight_file(cfg, w, "paper_size_default"), precision=precision)
    try:
        _check(m, synth.lattice_system(2000, seed=43), synth.water_box(0))
    finally:
        m.close()
