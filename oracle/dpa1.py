"""Plain FP64 definition of the DPA-1 (se_atten, smooth gated attention)
energy, forces and virial.  Test infrastructure only (see package doc).

Every step follows the paper's description of the descriptor + fitting
architecture (Sec. II-B) in the order it is stated there, with the
details the paper leaves open fixed by one reading each:

1. full neighbour list within rcut, nearest ``sel`` kept (Sec. II-C);
2. smooth environment matrix R with a C2 switch (Sec. II-B, DP-SE);
3. type embedding Z and the strip-mode type-pair table (Sec. II-B, DPA-1);
4. embedding net G (Sec. II-B, DP-SE);
5. ``l_a`` gated self-attention blocks within each neighbour set, the
   gate carrying the angular correlation R R^T (Sec. II-B, DPA-1);
6. descriptor D = G^T R R^T G_< (Sec. II-B, DP-SE);
7. fitting net e_i = Phi(D_i), E = sum_i e_i (Sec. II-B, Eq. eq_totE_singleAtomE);
8. F = -dE/dr (Eq. eq_forceGradE) and the virial W = -dE/d(strain)^T,
   both obtained by reverse-mode differentiation of this FP64 forward.

All arithmetic is float64 on the CPU, written with plain torch tensor
operations (gather, matmul, tanh, softmax) and numpy for the neighbour
search.  Nothing here is blocked, fused or reordered for speed.
"""

from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np
import torch

F64 = torch.float64


# ---------------------------------------------------------------------------
# 1. Neighbour list (Sec. II-C: full lists are required by DP models; the
#    cutoff list of Sec. II-A).  Reading: candidates are all j != i with
#    |mic(r_j - r_i)| < rcut; keep the ``sel`` nearest, ties broken by the
#    lower index j.  Orthorhombic box with every edge > 2 rcut.
# ---------------------------------------------------------------------------

def minimum_image(d: np.ndarray, box: np.ndarray) -> np.ndarray:
    """d - L * rint(d / L), per axis (round half to even)."""
    return d - box * np.rint(d / box)


def squared_distance(d: np.ndarray) -> np.ndarray:
    """(dx*dx + dy*dy) + dz*dz, evaluated in this order in float64."""
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def neighbor_list(coord, box, rcut: float, sel: int, centres: Optional[Sequence[int]] = None,
                  chunk: int = 128):
    """Brute-force O(N^2) full neighbour list.

    Returns ``(nlist [C, sel] int64 padded with -1, nnei [C], ncand [C])``
    where C = len(centres) (all atoms by default), ``nlist[c]`` lists
    the kept neighbours of centre ``centres[c]`` sorted by (d^2, j) and
    ``ncand`` is the number of candidates before the ``sel`` cap.
    """
    coord = np.asarray(coord, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64).reshape(3)
    if np.any(box <= 2.0 * rcut):
        raise ValueError("every box edge must exceed 2*rcut")
    n = coord.shape[0]
    centres = np.arange(n) if centres is None else np.asarray(centres, dtype=np.int64)
    rc2 = rcut * rcut
    nlist = np.full((len(centres), sel), -1, dtype=np.int64)
    nnei = np.zeros(len(centres), dtype=np.int64)
    ncand = np.zeros(len(centres), dtype=np.int64)
    for start in range(0, len(centres), chunk):
        ci = centres[start:start + chunk]
        d = minimum_image(coord[None, :, :] - coord[ci, None, :], box)
        d2 = squared_distance(d)
        for a, i in enumerate(ci):
            row = d2[a]
            cand = np.nonzero(row < rc2)[0]
            cand = cand[cand != i]
            order = np.lexsort((cand, row[cand]))
            keep = cand[order][:sel]
            nlist[start + a, :len(keep)] = keep
            nnei[start + a] = len(keep)
            ncand[start + a] = len(cand)
    return nlist, nnei, ncand


def reverse_centres(coord, box, rcut: float, sel: int, atoms: Iterable[int]) -> np.ndarray:
    """All centres i whose atomic energy e_i depends on the position of
    any atom k in ``atoms``: k itself and every i with k in N(i)."""
    atoms = np.unique(np.asarray(list(atoms), dtype=np.int64))
    cand_l, _, _ = neighbor_list(coord, box, rcut, len(coord), centres=atoms)
    cands = np.unique(cand_l[cand_l >= 0])
    out = set(int(k) for k in atoms)
    if len(cands):
        nl, _, _ = neighbor_list(coord, box, rcut, sel, centres=cands)
        aset = set(int(k) for k in atoms)
        for c, i in enumerate(cands):
            if aset.intersection(int(j) for j in nl[c] if j >= 0):
                out.add(int(i))
    return np.array(sorted(out), dtype=np.int64)


# ---------------------------------------------------------------------------
# 2. Smooth environment matrix (Sec. II-B, DP-SE: R^i in invariant
#    coordinates).  Reading: s(r) = w(r)/r with the C2 switch
#    w = 1 (r < rcs), u^3(-6u^2 + 15u - 10) + 1 (rcs <= r < rc), 0 beyond,
#    u = (r - rcs)/(rc - rcs); a row of R is (s, s x/r, s y/r, s z/r),
#    normalised per centre type and column by (R - davg)/dstd; padding
#    rows are zero.
# ---------------------------------------------------------------------------

def switch(r: torch.Tensor, rcs: float, rc: float) -> torch.Tensor:
    u = (r - rcs) / (rc - rcs)
    poly = u * u * u * (-6.0 * u * u + 15.0 * u - 10.0) + 1.0
    one = torch.ones_like(r)
    zero = torch.zeros_like(r)
    return torch.where(r < rcs, one, torch.where(r < rc, poly, zero))


def env_matrix(rij: torch.Tensor, mask: torch.Tensor, tcentre: torch.Tensor,
               davg: torch.Tensor, dstd: torch.Tensor, rcs: float, rc: float):
    """rij [C,S,3] (padding rows arbitrary, non-zero), mask [C,S] bool.

    Returns R [C,S,4] normalised, w [C,S] switch weights, rhat [C,S,3]."""
    m = mask.to(F64)
    r = torch.sqrt((rij * rij).sum(-1))
    w = switch(r, rcs, rc) * m
    s = w / r
    rhat = rij / r[..., None]
    raw = torch.cat([s[..., None], s[..., None] * rhat], dim=-1)
    R = (raw - davg[tcentre][:, None, :]) / dstd[tcentre][:, None, :]
    R = R * m[..., None]
    rhat = rhat * m[..., None]
    return R, w, rhat


# ---------------------------------------------------------------------------
# 3.-4. Type embedding Z and embedding net (Sec. II-B, DPA-1 adds the type
#    embedding into G).  Reading (strip mode): Z[t] = tanh(onehot(t) W + b);
#    type-pair table Gt[a, b] = net_t([Z[b], Z[a]]) (neighbour type first,
#    centre type second); G0_ij = net_s(R_ij,0) * (1 + Gt[t_i, t_j]).
#    Reading (concat mode, the original DPA-1 form): the embedding net reads
#    the row [R_ij,0, Z[t_j], Z[t_i]] and G0_ij is its output.
#    Both nets: dense + tanh layers with the residual rule y = x + f(x)
#    when the width is kept, y = [x, x] + f(x) when it doubles, else f(x).
# ---------------------------------------------------------------------------

def embedding_net(x: torch.Tensor, layers: Sequence[Tuple[torch.Tensor, torch.Tensor]]) -> torch.Tensor:
    for W, b in layers:
        y = torch.tanh(x @ W + b)
        if W.shape[1] == W.shape[0]:
            x = x + y
        elif W.shape[1] == 2 * W.shape[0]:
            x = torch.cat([x, x], dim=-1) + y
        else:
            x = y
    return x


def type_embedding(te_W: torch.Tensor, te_b: torch.Tensor) -> torch.Tensor:
    nt = te_W.shape[0]
    onehot = torch.eye(nt, dtype=F64)
    return torch.tanh(onehot @ te_W + te_b)


def type_pair_table(tebd: torch.Tensor, layers) -> torch.Tensor:
    nt, td = tebd.shape
    nb = tebd[None, :, :].expand(nt, nt, td)  # [a, b] -> Z[b]
    ce = tebd[:, None, :].expand(nt, nt, td)  # [a, b] -> Z[a]
    return embedding_net(torch.cat([nb, ce], dim=-1), layers)


# ---------------------------------------------------------------------------
# 5. Gated self-attention within the neighbour set (Sec. II-B, DPA-1).
#    Reading (one head, smooth form):
#      Q, K, V = G Wq + bq, G Wk + bk, G Wv + bv
#      l_jk  = Q_j . K_k / sqrt(d_attn)
#      l'_jk = (l_jk + S) w_j w_k - S                (S = attention shift)
#      A_jk  = softmax over valid k of l'_jk
#      P_jk  = A_jk w_j w_k (rhat_j . rhat_k)        (gate: angular R R^T)
#      O     = P V
#      G    <- G + LayerNorm(O Wo + bo)              (over the M1 features)
# ---------------------------------------------------------------------------

def layer_norm(y: torch.Tensor, g: torch.Tensor, b: torch.Tensor, eps: float) -> torch.Tensor:
    mu = y.mean(dim=-1, keepdim=True)
    var = ((y - mu) * (y - mu)).mean(dim=-1, keepdim=True)
    return (y - mu) / torch.sqrt(var + eps) * g + b


def gated_attention(G: torch.Tensor, w: torch.Tensor, rhat: torch.Tensor, mask: torch.Tensor,
                    p: Dict[str, torch.Tensor], shift: float, eps: float) -> torch.Tensor:
    d_attn = p["Wq"].shape[1]
    Q = G @ p["Wq"] + p["bq"]
    K = G @ p["Wk"] + p["bk"]
    V = G @ p["Wv"] + p["bv"]
    logits = Q @ K.transpose(-1, -2) / math.sqrt(d_attn)
    ww = w[:, :, None] * w[:, None, :]
    lp = (logits + shift) * ww - shift
    # softmax over the valid keys k only (padding keys get probability 0)
    lp = lp.masked_fill(~mask[:, None, :], -1e30)
    A = torch.softmax(lp, dim=-1)
    gate = rhat @ rhat.transpose(-1, -2)
    P = A * ww * gate
    O = P @ V
    Y = O @ p["Wo"] + p["bo"]
    Z = layer_norm(Y, p["ln_g"], p["ln_b"], eps)
    return G + Z * mask.to(F64)[..., None]


# ---------------------------------------------------------------------------
# 6. Descriptor D = G^T R R^T G_< (Sec. II-B, DP-SE).  Reading: T = R^T G / sel
#    (4 x M1), D = T^T T[:, :axis] (M1 x axis, row-major), and the fitting
#    input is [D, Z[t_i]].
# ---------------------------------------------------------------------------

def descriptor(R: torch.Tensor, G: torch.Tensor, sel: int, axis: int):
    T = R.transpose(-1, -2) @ G / sel
    D = T.transpose(-1, -2) @ T[:, :, :axis]
    return D.reshape(D.shape[0], -1), T


# ---------------------------------------------------------------------------
# 7. Fitting net e_i = Phi(D_i) (Sec. II-B), E = sum_i e_i
#    (Eq. eq_totE_singleAtomE).  Reading: hidden layers with the same
#    residual rule as the embedding net, a linear output, scaled by
#    out_scale, plus a per-type energy bias.
# ---------------------------------------------------------------------------

def fitting(x: torch.Tensor, layers, out_scale: float, ebias_t: torch.Tensor) -> torch.Tensor:
    h = embedding_net(x, layers[:-1])
    W, b = layers[-1]
    return out_scale * (h @ W + b)[..., 0] + ebias_t


@dataclass
class OracleModel:
    """Weights as float64 torch tensors plus the hyper-parameters."""
    cfg: object
    t: Dict[str, torch.Tensor]

    @classmethod
    def from_numpy(cls, cfg, weights: Dict[str, np.ndarray]) -> "OracleModel":
        return cls(cfg, {k: torch.as_tensor(np.asarray(v), dtype=F64) for k, v in weights.items()})

    def layers(self, prefix: str, n: int):
        return [(self.t[f"{prefix}_W{l}"], self.t[f"{prefix}_b{l}"]) for l in range(n)]

    def attn(self, l: int) -> Dict[str, torch.Tensor]:
        keys = ["Wq", "bq", "Wk", "bk", "Wv", "bv", "Wo", "bo", "ln_g", "ln_b"]
        return {k: self.t[f"at{l}_{k}"] for k in keys}


def atomic_energies(model: OracleModel, rij: torch.Tensor, nlist: np.ndarray, atype_c: np.ndarray,
                    atype_all: np.ndarray, stages: Optional[dict] = None) -> torch.Tensor:
    """e_i for centres with displacement rows ``rij`` [C,S,3] (rows of
    padding slots arbitrary but non-zero), neighbour ids ``nlist`` [C,S]
    (-1 = padding) and centre types ``atype_c``."""
    cfg = model.cfg
    t = model.t
    mask = torch.as_tensor(nlist >= 0)
    tc = torch.as_tensor(np.asarray(atype_c, dtype=np.int64))
    tn = torch.as_tensor(np.where(nlist >= 0, np.asarray(atype_all)[np.maximum(nlist, 0)], 0).astype(np.int64))
    R, w, rhat = env_matrix(rij, mask, tc, t["davg"], t["dstd"], cfg.rcut_smth, cfg.rcut)
    tebd = type_embedding(t["te_W"], t["te_b"])
    if getattr(cfg, "tebd_input_mode", "strip") == "concat":
        # concat mode: the embedding net reads [s, T_j, T_i]
        Gt = None
        tj = tebd[tn]
        ti = tebd[tc][:, None, :].expand_as(tj)
        Gs = embedding_net(torch.cat([R[..., 0:1], tj, ti], dim=-1), model.layers("em", len(cfg.embed)))
        G = Gs * mask.to(F64)[..., None]
    else:
        Gt = type_pair_table(tebd, model.layers("tt", len(cfg.embed)))
        Gs = embedding_net(R[..., 0:1], model.layers("em", len(cfg.embed)))
        G = Gs * (1.0 + Gt[tc[:, None], tn]) * mask.to(F64)[..., None]
    if stages is not None:
        stages.update(R=R, w=w, rhat=rhat, G0=G, tebd=tebd)
        if Gt is not None:
            stages["Gt"] = Gt
    for l in range(cfg.attn_layers):
        G = gated_attention(G, w, rhat, mask, model.attn(l), cfg.attn_shift, cfg.ln_eps)
        if stages is not None:
            stages[f"G{l + 1}"] = G
    D, T = descriptor(R, G, cfg.sel, cfg.axis)
    x = torch.cat([D, tebd[tc]], dim=-1)
    nfit = len(cfg.fitting)
    e = fitting(x, model.layers("fit", nfit + 1), float(t["out_scale"]), t["ebias"][tc])
    if stages is not None:
        stages.update(T=T, D=D, e=e)
    return e


def _displacements(x: torch.Tensor, box: np.ndarray, centres: np.ndarray, nlist: np.ndarray,
                   strain: Optional[torch.Tensor]) -> torch.Tensor:
    idx = torch.as_tensor(np.maximum(nlist, 0))
    ci = torch.as_tensor(centres)
    raw = x[idx] - x[ci][:, None, :]
    L = torch.as_tensor(np.asarray(box, dtype=np.float64).reshape(3))
    shift = -(L * torch.round(raw.detach() / L))  # torch.round: half to even
    rij = raw + shift
    # padding rows: a harmless non-zero vector beyond the cutoff
    pad = torch.zeros_like(rij)
    pad[..., 0] = 1.0
    rij = torch.where(torch.as_tensor(nlist >= 0)[..., None], rij, pad)
    if strain is not None:
        rij = rij @ (torch.eye(3, dtype=F64) + strain).T
    return rij


def energy_force_virial(model: OracleModel, coord, box, atype, nlist=None, chunk: int = 256,
                        centres: Optional[np.ndarray] = None, stages: Optional[dict] = None):
    """Total energy, per-atom energies, forces and virial.

    F = -dE/dx (Eq. eq_forceGradE); W_ab = -sum_ij r_ij,a dE/dr_ij,b,
    obtained as the transposed negative derivative of E with respect to
    a homogeneous strain of every displacement.  With ``centres`` given,
    E is the sum of e_i over those centres only (used to get exact
    forces on a few atoms of a large system, see ``forces_on``).
    """
    cfg = model.cfg
    coord = np.asarray(coord, dtype=np.float64)
    atype = np.asarray(atype)
    n = coord.shape[0]
    centres = np.arange(n) if centres is None else np.asarray(centres, dtype=np.int64)
    if nlist is None:
        nlist, _, _ = neighbor_list(coord, box, cfg.rcut, cfg.sel, centres=centres)
    x = torch.tensor(coord, dtype=F64, requires_grad=True)
    strain = torch.zeros(3, 3, dtype=F64, requires_grad=True)
    e_all = np.zeros(len(centres))
    E = 0.0
    for s0 in range(0, len(centres), chunk):
        sl = slice(s0, s0 + chunk)
        rij = _displacements(x, box, centres[sl], nlist[sl], strain)
        st = {} if (stages is not None and s0 == 0 and len(centres) <= chunk) else None
        e = atomic_energies(model, rij, nlist[sl], atype[centres[sl]], atype, stages=st)
        if st is not None:
            stages.update({k: v.detach() for k, v in st.items()})
        e.sum().backward()
        e_all[sl] = e.detach().numpy()
        E += float(e.detach().sum())
    force = -x.grad.numpy().copy() if x.grad is not None else np.zeros_like(coord)
    virial = -strain.grad.numpy().T.copy() if strain.grad is not None else np.zeros((3, 3))
    return E, e_all, force, virial


def forces_on(model: OracleModel, coord, box, atype, atoms: Sequence[int]) -> np.ndarray:
    """Exact forces on ``atoms`` of a (possibly large) system, computed from
    the atomic energies of the centres that depend on them only."""
    cfg = model.cfg
    atoms = np.asarray(atoms, dtype=np.int64)
    cs = reverse_centres(coord, box, cfg.rcut, cfg.sel, atoms)
    _, _, f, _ = energy_force_virial(model, coord, box, atype, centres=cs)
    return f[atoms]
