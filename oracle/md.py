"""FP64 velocity-Verlet integration driven by oracle forces, for checking the
device MD loop.  Test infrastructure only (see the package docstring).

The paper couples the model's forces F = -dE/dx (Eq. eq_forceGradE) to the
MD engine's integration of Newton's equations (Sec. II-A).  One step of the
velocity-Verlet scheme with time step dt:

    v <- v + (dt / 2) a(x),   x <- x + dt v,   v <- v + (dt / 2) a(x_new),

with a = F / m.  Units: A, fs, amu, eV.  The conversion of an acceleration
of 1 eV / (A amu) to A / fs^2 is derived here from the SI values of the
elementary charge and the atomic mass constant (exact / CODATA 2018).

Parity status: ``acceleration_unit`` and ``velocity_verlet`` are pinned by
the closed-form harmonic oscillator (second-order convergence), exact time
reversibility and the SI derivation of the unit (tests/test_oracle_md.py).
"""

from __future__ import annotations

from typing import Callable, List, Tuple

import numpy as np

ELEMENTARY_CHARGE_C = 1.602176634e-19  # exact (SI 2019)
ATOMIC_MASS_KG = 1.66053906660e-27     # CODATA 2018


def acceleration_unit() -> float:
    """A / fs^2 per eV / (A amu): (e J / (1e-10 m * u kg)) in m / s^2,
    times 1e10 A / m and (1e-15 s / fs)^2."""
    si = ELEMENTARY_CHARGE_C / (1e-10 * ATOMIC_MASS_KG)  # m / s^2
    return si * 1e10 * 1e-30


def kinetic_energy(v: np.ndarray, mass: np.ndarray) -> float:
    """sum_k m_k |v_k|^2 / 2 in eV (v in A / fs, m in amu)."""
    return float(0.5 * np.sum(mass[:, None] * v * v) / acceleration_unit())


def velocity_verlet(x: np.ndarray, v: np.ndarray, mass: np.ndarray,
                    force: Callable[[np.ndarray], Tuple[float, np.ndarray]], dt: float,
                    nsteps: int):
    """Advance (x, v) by ``nsteps`` steps.  ``force(x)`` returns
    (potential energy eV, forces [N, 3] eV/A).  Returns the final x, v,
    forces and the per-step (potential, kinetic, total) energies after
    each step."""
    acc = acceleration_unit()
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    m = np.asarray(mass, dtype=np.float64)[:, None]
    epot, f = force(x)
    thermo: List[Tuple[float, float, float]] = []
    for _ in range(nsteps):
        v = v + 0.5 * dt * f / m * acc
        x = x + dt * v
        epot, f = force(x)
        v = v + 0.5 * dt * f / m * acc
        ek = kinetic_energy(v, m[:, 0])
        thermo.append((epot, ek, epot + ek))
    return x, v, f, np.array(thermo)
