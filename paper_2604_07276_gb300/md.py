"""Velocity-Verlet molecular dynamics on the GPU through ``dp_md_run``.

PyTorch only holds the device arrays; every step (drift, neighbour list,
energy / forces, kick, FP64 kinetic energy) runs in the library, replayed
from one CUDA graph when ``graph`` is true.
"""

from __future__ import annotations

from typing import Optional

import numpy as np

from .binding import DPA1, _check, box9

MASSES = {"H": 1.008, "C": 12.011, "N": 14.007, "O": 15.999, "S": 32.06}


class MDState:
    """Device arrays of one trajectory (A, fs, amu)."""

    def __init__(self, coord, vel, mass, box, atype, device="cuda"):
        import torch

        self.coord = torch.tensor(np.asarray(coord, dtype=np.float64), device=device)
        self.vel = torch.tensor(np.asarray(vel, dtype=np.float64), device=device)
        self.mass = torch.tensor(np.asarray(mass, dtype=np.float64), device=device)
        self.box = torch.tensor(box9(box), device=device)
        self.atype = torch.tensor(np.asarray(atype, dtype=np.int32), device=device)
        n = self.coord.shape[0]
        self.force = torch.zeros((n, 3), dtype=torch.float64, device=device)
        self.energy = torch.zeros(1, dtype=torch.float64, device=device)
        self.virial = torch.zeros(9, dtype=torch.float64, device=device)


def run(model: DPA1, state: MDState, dt: float, nsteps: int, graph: bool = True, stream: Optional[int] = None):
    """Advance ``state`` by ``nsteps`` steps of ``dt`` fs; returns the
    per-step (potential, kinetic, total) energies as a CUDA tensor."""
    import torch

    n = int(state.coord.shape[0])
    model.reserve(n)
    thermo = torch.zeros((max(nsteps, 1), 3), dtype=torch.float64, device=state.coord.device)
    st = stream if stream is not None else torch.cuda.current_stream(state.coord.device).cuda_stream
    _check(model.lib.dp_md_run(model.h, n, state.coord.data_ptr(), state.vel.data_ptr(), state.mass.data_ptr(),
                               state.box.data_ptr(), state.atype.data_ptr(), float(dt), int(nsteps),
                               state.force.data_ptr(), state.energy.data_ptr(), state.virial.data_ptr(),
                               thermo.data_ptr(), 1 if graph else 0, st))
    return thermo[:nsteps]
