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


@pytest.mark.parametrize("precision", ["fp32", "fp16x", "bf16x"])
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


@pytest.mark.parametrize("precision,x_tol", [("fp32", 2e-6), ("fp16x", 1e-3)])
def test_md_matches_fp64_oracle_verlet(default_model, precision, x_tol):
    """Five velocity-Verlet steps of dp_md_run against the FP64 host
    integrator (oracle/md.py) driven by the FP64 oracle's forces, from the
    same start on the water box.  The FP32 path's largest force error on this
    box (~2e-4 eV/A on one atom, an ill-conditioned row of the attention
    layer; RMSE ~1e-6) moves that atom by ~4e-7 A in 2.5 fs (measured; at
    most a t^2 / 2 ~ 6e-6 A with a = dF / m for hydrogen); a wrong half kick,
    unit or mass would move the atoms by ~1e-2 A."""
    import torch
    import paper_2604_07276_gb300 as p
    from paper_2604_07276_gb300 import md
    from oracle import energy_force_virial
    from oracle.md import velocity_verlet

    cfg, w, om = default_model
    coord, atype, box = synth.water_box(0)
    vel = synth.maxwell_boltzmann(atype, 300.0, seed=11)
    mass = synth.MASSES[atype]

    def force(x):
        E, _, F, _ = energy_force_virial(om, x, box, atype)
        return E, F

    xr, vr, fr, thr = velocity_verlet(coord, vel, mass, force, 0.5, 5)
    m = p.DPA1(weight_file(cfg, w, "default"), precision=precision)
    s = md.MDState(coord, vel, mass, box, atype)
    th = md.run(m, s, dt=0.5, nsteps=5, graph=False).cpu().numpy()
    m.status()
    m.close()
    dx = np.abs(s.coord.cpu().numpy() - xr).max()
    dv = np.abs(s.vel.cpu().numpy() - vr).max()
    df = np.abs(s.force.cpu().numpy() - fr).max()
    print(f"\n{precision}: max |dx| {dx:.2e} A, |dv| {dv:.2e} A/fs, |dF| {df:.2e} eV/A, "
          f"|dE_pot| {np.abs(th[:, 0] - thr[:, 0]).max():.2e} eV, |dE_kin| {np.abs(th[:, 1] - thr[:, 1]).max():.2e} eV")
    assert dx <= x_tol and dv <= x_tol
    # energies: potential within the per-atom bound of the mode, kinetic to the
    # velocity difference
    e_tol = 1e-5 if precision == "fp32" else 1e-3
    assert np.abs(th[:, 0] - thr[:, 0]).max() <= e_tol * len(atype)
    assert np.abs(th[:, 1] - thr[:, 1]).max() <= 1e-6 * len(atype) + 100 * x_tol
