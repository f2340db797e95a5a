"""Distilled student potential: data from the full model, training with the
library's own kernels, and MD with a full-model check and fallback.

The student is the same descriptor family with no attention layer and
smaller nets (embedding [16, 32, 64], axis 8, fitting [128, 128]); it is
trained on energies and forces that the full DPA-1 model computes along
its own short MD trajectories.  Every gradient comes from dp_train_frame and
every update from dp_adam_step; PyTorch only holds the device arrays.
"""

from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from .binding import DPA1, box9
from . import md as dmd


@dataclass
class Frame:
    coord: object   # CUDA float64 [N, 3]
    box: object     # CUDA float64 [9]
    atype: object   # CUDA int32 [N]
    energy: float
    force: object   # CUDA float64 [N, 3]


def teacher_frames(teacher: DPA1, systems, masses_of, n_traj: int, steps: int, every: int, dt: float = 0.5,
                   temperature: float = 300.0, seed: int = 0) -> List[Frame]:
    """Frames along teacher MD trajectories: for each system and each of
    n_traj Maxwell-Boltzmann velocity draws, run ``steps`` velocity-Verlet
    steps and keep every ``every``-th configuration with its energy and
    forces."""
    import torch

    rng = np.random.default_rng(seed)
    frames: List[Frame] = []
    for coord, atype, box in systems:
        for _ in range(n_traj):
            v = _maxwell(atype, masses_of, temperature, rng)
            st = dmd.MDState(coord, v, masses_of[atype], box, atype)
            for _k in range(steps // every):
                dmd.run(teacher, st, dt=dt, nsteps=every, graph=False)
                torch.cuda.synchronize()
                frames.append(Frame(st.coord.clone(), st.box.clone(), st.atype.clone(), float(st.energy.item()),
                                    st.force.clone()))
    return frames


def _maxwell(atype, masses_of, temperature, rng):
    m = masses_of[np.asarray(atype)]
    sigma = np.sqrt(8.617333262e-5 * temperature / m * 9.648533212e-3)
    v = rng.normal(size=(len(m), 3)) * sigma[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    return v


def train(student: DPA1, frames: Sequence[Frame], epochs: int, batch: int = 16, lr0: float = 1e-3,
          lr_end: float = 1e-5, pe: float = 1.0, pf: float = 1.0, seed: int = 0):
    """Adam on mini-batches of frames (gradient = mean over the batch); the
    learning rate decays exponentially from lr0 to lr_end.  Returns the mean
    loss of every batch."""
    import torch

    rng = np.random.default_rng(seed)
    nb = max(1, math.ceil(len(frames) / batch))
    total = max(1, epochs * nb)
    loss = torch.zeros(3, dtype=torch.float64, device="cuda")
    acc = torch.zeros(3, dtype=torch.float64, device="cuda")
    history = []
    step = 0
    student.reserve(max(int(f.coord.shape[0]) for f in frames))
    for _ in range(epochs):
        order = rng.permutation(len(frames))
        for b in range(nb):
            idx = order[b * batch:(b + 1) * batch]
            acc.zero_()
            student.zero_grad()
            for i in idx:
                f = frames[i]
                student.train_frame(f.coord, f.box, f.atype, f.energy, f.force, loss, pe=pe, pf=pf,
                                    stream=torch.cuda.current_stream().cuda_stream)
                acc += loss
            # mean over the batch: scale the learning rate (Adam is invariant to
            # a constant gradient scale, so only the loss history is divided)
            lr = lr0 * (lr_end / lr0) ** (step / max(1, total - 1))
            student.adam_step(lr, stream=torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            history.append((acc / len(idx)).cpu().numpy())
            step += 1
    return np.array(history)


def force_rmse(model: DPA1, frames: Sequence[Frame]) -> float:
    import torch

    se, cnt = 0.0, 0
    for f in frames:
        n = int(f.coord.shape[0])
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        W = torch.zeros(9, dtype=torch.float64, device="cuda")
        model.reserve(n)
        model.compute_device(f.coord, f.box, f.atype, e, F, W)
        se += float(((F - f.force) ** 2).sum().item())
        cnt += 3 * n
    return math.sqrt(se / max(1, cnt))


def md_with_fallback(student: DPA1, teacher: DPA1, state: dmd.MDState, nsteps: int, dt: float = 0.5,
                     check_every: int = 10, threshold: float = 0.05):
    """Student MD checked against the full model every ``check_every`` steps.
    When the student's force RMSE against the full model at a check exceeds
    ``threshold`` (eV/A), the state returns to the last passed check and the
    next ``check_every`` steps run with the full model; then the student is
    tried again.  Returns (student segments, fallback segments, RMSE of
    every check)."""
    import torch

    n = int(state.coord.shape[0])
    F_t = torch.zeros((n, 3), dtype=torch.float64, device=state.coord.device)
    e = torch.zeros(1, dtype=torch.float64, device=state.coord.device)
    W = torch.zeros(9, dtype=torch.float64, device=state.coord.device)
    done, used_student, used_teacher, checks = 0, 0, 0, []
    while done < nsteps:
        k = min(check_every, nsteps - done)
        saved = (state.coord.clone(), state.vel.clone())
        dmd.run(student, state, dt=dt, nsteps=k, graph=True)
        teacher.compute_device(state.coord, state.box, state.atype, e, F_t, W)
        torch.cuda.synchronize()
        rmse = float(torch.sqrt(((state.force - F_t) ** 2).mean()).item())
        checks.append(rmse)
        if rmse > threshold:
            state.coord.copy_(saved[0])
            state.vel.copy_(saved[1])
            dmd.run(teacher, state, dt=dt, nsteps=k, graph=True)
            used_teacher += 1
        else:
            used_student += 1
        done += k
    torch.cuda.synchronize()
    return used_student, used_teacher, checks
