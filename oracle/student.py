"""Exact gradient of the student's training loss, for checking the CUDA
training kernels.  Test infrastructure only (see the package docstring).

Loss of one frame (the reading used for the distilled student; the paper's
own model is trained on energies and forces, Sec. IV-B):

    L = pe ((E - E_ref) / N)^2 + pf mean_k,a (F_ka - F_ref,ka)^2,

with F = -dE/dx (Eq. eq_forceGradE).  The gradient with respect to the
trainable weights is taken by reverse-mode differentiation through the
force (a second derivative of E), in float64.
"""

from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np
import torch

from .dpa1 import F64, OracleModel, _displacements, atomic_energies, neighbor_list


def trainable_names(cfg) -> List[str]:
    """Trainable tensors in the order of the flat parameter vector."""
    names = []
    for l in range(len(cfg.embed)):
        names += [f"em_W{l}", f"em_b{l}"]
    for l in range(len(cfg.fitting) + 1):
        names += [f"fit_W{l}", f"fit_b{l}"]
    names.append("ebias")
    return names


def flat(model: OracleModel, names: Sequence[str]) -> np.ndarray:
    return np.concatenate([model.t[k].detach().numpy().ravel() for k in names])


def loss_and_grad(model: OracleModel, coord, box, atype, e_ref: float, f_ref, pe: float = 1.0, pf: float = 1.0):
    """(L, L_E, L_F, flat gradient) for one frame."""
    cfg = model.cfg
    names = trainable_names(cfg)
    leaves = {k: model.t[k].detach().clone().requires_grad_(True) for k in names}
    t = dict(model.t)
    t.update(leaves)
    m = OracleModel(cfg, t)
    coord = np.asarray(coord, dtype=np.float64)
    n = coord.shape[0]
    nl, _, _ = neighbor_list(coord, box, cfg.rcut, cfg.sel)
    x = torch.tensor(coord, dtype=F64, requires_grad=True)
    rij = _displacements(x, box, np.arange(n), nl, None)
    E = atomic_energies(m, rij, nl, np.asarray(atype), np.asarray(atype)).sum()
    (gx,) = torch.autograd.grad(E, x, create_graph=True)
    F = -gx
    fr = torch.as_tensor(np.asarray(f_ref, dtype=np.float64))
    lE = pe * ((E - e_ref) / n) ** 2
    lF = pf * ((F - fr) ** 2).mean()
    L = lE + lF
    grads = torch.autograd.grad(L, [leaves[k] for k in names])
    g = np.concatenate([gi.detach().numpy().ravel() for gi in grads])
    return float(L.detach()), float(lE.detach()), float(lF.detach()), g
