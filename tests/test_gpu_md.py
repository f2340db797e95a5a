"""Velocity-Verlet MD on the device (dp_md_run): CUDA-graph replay equals the
eager loop bit for bit, and the total energy is conserved."""

import numpy as np
import pytest

import synth

from gpu_helpers import weight_file

pytestmark = pytest.mark.gpu


def _state(p, torch, seed=0):
    from paper_2604_07276_gb300 import md

    coord, atype, box = synth.water_box(seed)
    vel = synth.maxwell_boltzmann(atype, 300.0, seed=11)
    mass = synth.MASSES[atype]
    return md.MDState(coord, vel, mass, box, atype)


@pytest.mark.parametrize("precision", ["fp32", "fp16x"])
def test_graph_replay_matches_eager(default_model, precision):
    import torch
    import paper_2604_07276_gb300 as p
    from paper_2604_07276_gb300 import md

    cfg, w, _ = default_model
    m = p.DPA1(weight_file(cfg, w, "default"), precision=precision)
    a = _state(p, torch)
    b = _state(p, torch)
    ta = md.run(m, a, dt=0.5, nsteps=20, graph=False)
    tb = md.run(m, b, dt=0.5, nsteps=20, graph=True)
    torch.cuda.synchronize()
    m.status()
    assert torch.equal(a.coord, b.coord) and torch.equal(a.vel, b.vel)
    assert torch.equal(ta, tb)
    # a second replay of the cached graph continues the trajectory identically
    tc = md.run(m, b, dt=0.5, nsteps=20, graph=True)
    td = md.run(m, a, dt=0.5, nsteps=20, graph=False)
    torch.cuda.synchronize()
    assert torch.equal(tc, td) and torch.equal(a.coord, b.coord)
    m.close()


def test_nve_energy_conservation(default_model):
    """10 fs from 100 K on the 192-atom water box (FP32 path), at dt = 0.5 fs
    and at 0.25 fs.  Velocity Verlet with exact forces conserves the energy
    up to O(dt^2): the drift must be small against the kinetic-energy change
    and shrink about fourfold when dt halves.  (A random-weight model has no
    short-range repulsion, so long trajectories collapse atoms onto each
    other; the window here ends well before that.)"""
    import torch
    import paper_2604_07276_gb300 as p
    from paper_2604_07276_gb300 import md

    cfg, w, _ = default_model
    m = p.DPA1(weight_file(cfg, w, "default"), precision="fp32")
    coord, atype, box = synth.water_box(0)
    drift = {}
    for dt, steps in ((0.5, 20), (0.25, 40)):
        s = md.MDState(coord, synth.maxwell_boltzmann(atype, 100.0, seed=11), synth.MASSES[atype], box, atype)
        th = md.run(m, s, dt=dt, nsteps=steps, graph=True).cpu().numpy()
        m.status()
        n = len(atype)
        drift[dt] = np.abs(th[:, 2] - th[0, 2]).max() / n
        ke_change = (th[:, 1].max() - th[:, 1].min()) / n
        assert ke_change > 20 * drift[dt], (dt, ke_change, drift[dt])
    assert drift[0.25] < 1e-3
    assert drift[0.5] / drift[0.25] > 2.5, drift
    m.close()
