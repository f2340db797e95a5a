"""Pins of the FP64 velocity-Verlet oracle (oracle/md.py) against facts that
do not come from it: the closed-form harmonic oscillator, the second-order
convergence of the scheme, its exact time reversibility and the unit
conversion from SI constants.  CPU only."""

import math

import numpy as np

from oracle.md import acceleration_unit, kinetic_energy, velocity_verlet


def test_acceleration_unit_from_si():
    # 1 eV / (A amu) = e N_A / (1e-10 m * 1e-3 kg) = F * 1e13 m/s^2 with the
    # Faraday constant F = e N_A (the molar mass constant is 1 g/mol to 1e-9),
    # i.e. F * 1e-7 A/fs^2
    faraday = 96485.33212  # C/mol
    assert abs(acceleration_unit() / (faraday * 1e-7) - 1.0) < 1e-8


def _harmonic(k, mass):
    def force(x):
        return 0.5 * k * float(np.sum(x * x)), -k * x
    omega = math.sqrt(k * acceleration_unit() / mass)
    return force, omega


def test_harmonic_oscillator_converges_at_second_order():
    """x(t) = x0 cos(wt) + v0/w sin(wt) for F = -k x; velocity Verlet is
    second order, so halving dt divides the error at fixed t by ~4."""
    k, mass = 2.5, 3.0
    force, w = _harmonic(k, mass)
    x0 = np.array([[0.3, -0.2, 0.1]])
    v0 = np.array([[0.01, 0.02, -0.005]])
    T = 40.0
    errs = []
    for dt in (0.4, 0.2, 0.1):
        n = int(round(T / dt))
        x, v, f, th = velocity_verlet(x0, v0, np.array([mass]), force, dt, n)
        xe = x0 * math.cos(w * T) + v0 / w * math.sin(w * T)
        errs.append(np.abs(x - xe).max())
    assert errs[2] < 1e-3 * np.abs(x0).max()
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_energy_is_conserved_and_reported():
    k, mass = 2.5, 3.0
    force, w = _harmonic(k, mass)
    x0 = np.array([[0.3, -0.2, 0.1], [0.0, 0.1, 0.0]])
    v0 = np.array([[0.01, 0.02, -0.005], [0.0, 0.0, 0.03]])
    masses = np.array([mass, mass])
    x, v, f, th = velocity_verlet(x0, v0, masses, force, 0.05, 200)
    e0 = force(x0)[0] + kinetic_energy(v0, masses)
    assert np.abs(th[:, 2] - e0).max() < 1e-3 * e0
    assert abs(th[-1, 0] - force(x)[0]) < 1e-15 and abs(th[-1, 1] - kinetic_energy(v, masses)) < 1e-15


def test_time_reversible():
    """Integrate forward, flip the velocities, integrate back: velocity
    Verlet returns to the start up to rounding (an anharmonic force)."""
    def force(x):
        r2 = np.sum(x * x, axis=1, keepdims=True)
        return float(np.sum(r2 * r2)), -4.0 * r2 * x
    rng = np.random.default_rng(0)
    x0 = rng.normal(size=(5, 3))
    v0 = 0.05 * rng.normal(size=(5, 3))
    m = rng.uniform(1.0, 16.0, size=5)
    x1, v1, _, _ = velocity_verlet(x0, v0, m, force, 0.05, 100)
    x2, v2, _, _ = velocity_verlet(x1, -v1, m, force, 0.05, 100)
    assert np.abs(x2 - x0).max() < 1e-10 and np.abs(v2 + v0).max() < 1e-10
