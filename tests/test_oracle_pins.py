"""Pins of the FP64 oracle against facts that do not come from the oracle
itself: library routines, closed forms, symmetries the paper states
(Sec. II-B: translational, rotational and same-species permutational
invariance; forces are exact energy gradients, Eq. eq_forceGradE) and
finite differences.  CPU only."""

import math

import numpy as np
import pytest
import torch
import torch.nn.functional as tF

import synth
import oracle
from oracle import OracleModel, energy_force_virial
from oracle.dpa1 import gated_attention, switch, embedding_net, type_embedding, type_pair_table

F64 = torch.float64


# --------------------------------------------------------------------- switch

def test_switch_end_values_and_smoothness():
    rcs, rc = 0.5, 6.0
    assert float(switch(torch.tensor(rcs, dtype=F64), rcs, rc)) == 1.0
    assert float(switch(torch.tensor(rc, dtype=F64), rcs, rc)) == 0.0
    assert float(switch(torch.tensor(0.2, dtype=F64), rcs, rc)) == 1.0
    assert float(switch(torch.tensor(7.0, dtype=F64), rcs, rc)) == 0.0
    # first and second derivatives vanish at both ends of the switch region
    for r0 in (rcs + 1e-9, rc - 1e-9):
        r = torch.tensor(r0, dtype=F64, requires_grad=True)
        (d1,) = torch.autograd.grad(switch(r, rcs, rc), r, create_graph=True)
        (d2,) = torch.autograd.grad(d1, r)
        assert abs(float(d1)) < 1e-12
        assert abs(float(d2)) < 1e-6
    # monotone decreasing in between, and value 1/2 at the midpoint (symmetry of the quintic)
    r = torch.linspace(rcs, rc, 1001, dtype=F64)
    v = switch(r, rcs, rc)
    assert torch.all(v[1:] <= v[:-1])
    assert abs(float(switch(torch.tensor((rcs + rc) / 2, dtype=F64), rcs, rc)) - 0.5) < 1e-15


# ----------------------------------------------------------------- neighbours

def test_neighbors_match_periodic_kdtree():
    from scipy.spatial import cKDTree

    coord, atype, box = synth.lattice_system(900, seed=7)
    rc = 6.0
    nl, nn, nc = oracle.neighbor_list(coord, box, rc, 500)
    tree = cKDTree(coord, boxsize=box)
    ref = tree.query_ball_point(coord, r=rc)
    for i in range(len(coord)):
        want = set(ref[i]) - {i}
        got = set(int(j) for j in nl[i] if j >= 0)
        assert got == want
        assert nn[i] == nc[i] == len(want)


def test_neighbor_sel_truncation_keeps_nearest():
    from scipy.spatial import cKDTree

    coord, atype, box = synth.lattice_system(900, seed=8)
    rc, sel = 6.0, 40
    nl, nn, nc = oracle.neighbor_list(coord, box, rc, sel)
    tree = cKDTree(coord, boxsize=box)
    d, idx = tree.query(coord, k=sel + 1)
    for i in range(len(coord)):
        assert nc[i] > sel
        want = [int(j) for j in idx[i][1:]]
        assert [int(j) for j in nl[i]] == want  # sorted by distance
    assert np.all(nn == sel)


# ------------------------------------------------------- forces = -dE/dx (FD)

def test_forces_central_difference(default_model, water, water_ref):
    """The neighbour list is held fixed: E is then a smooth function of the
    coordinates and F must be its exact negative gradient."""
    cfg, w, m = default_model
    coord, atype, box = water
    E, e, F, W = water_ref
    nl, _, _ = oracle.neighbor_list(coord, box, cfg.rcut, cfg.sel)
    rng = np.random.default_rng(0)
    h = 1e-4

    def en(a, k, t):
        c = coord.copy(); c[a, k] += t
        return energy_force_virial(m, c, box, atype, nlist=nl)[0]

    for a in rng.choice(len(coord), size=6, replace=False):
        for k in range(3):
            # central difference, and its fourth-order (five-point) refinement
            fd2 = -(en(a, k, h) - en(a, k, -h)) / (2 * h)
            fd4 = -(-en(a, k, 2 * h) + 8 * en(a, k, h) - 8 * en(a, k, -h) + en(a, k, -2 * h)) / (12 * h)
            assert abs(fd2 - F[a, k]) < 1e-4 * max(1.0, abs(F[a, k])), (a, k, fd2, F[a, k])
            assert abs(fd4 - F[a, k]) < 1e-8 * max(1.0, abs(F[a, k])), (a, k, fd4, F[a, k])


def test_sum_of_forces_is_zero(water_ref):
    E, e, F, W = water_ref
    assert np.abs(F.sum(axis=0)).max() < 1e-11
    assert abs(E - e.sum()) < 1e-10


def test_virial_diagonal_strain_difference(default_model, water, water_ref):
    cfg, w, m = default_model
    coord, atype, box = water
    W = water_ref[3]
    nl, _, _ = oracle.neighbor_list(coord, box, cfg.rcut, cfg.sel)
    h = 1e-5
    for a in range(3):
        s = np.ones(3); s[a] += h
        Ep = energy_force_virial(m, coord * s, box * s, atype, nlist=nl)[0]
        s = np.ones(3); s[a] -= h
        Em = energy_force_virial(m, coord * s, box * s, atype, nlist=nl)[0]
        assert abs(-(Ep - Em) / (2 * h) - W[a, a]) < 1e-6


def test_virial_symmetric(water_ref):
    W = water_ref[3]
    assert np.abs(W - W.T).max() < 1e-11


def test_virial_equals_position_force_moment_for_cluster(default_model):
    cfg, w, m = default_model
    coord, atype, box = synth.isolated_cluster(seed=3, natoms=14)
    E, e, F, W = energy_force_virial(m, coord, box, atype)
    ref = coord.T @ F  # sum_i x_i (x) F_i
    assert np.abs(W - ref).max() < 1e-10


# ------------------------------------------------------------- invariances

def test_translation_invariance(default_model, water, water_ref):
    cfg, w, m = default_model
    coord, atype, box = water
    E, e, F, W = water_ref
    E2, e2, F2, W2 = energy_force_virial(m, coord + np.array([3.3, -7.1, 0.37]), box, atype)
    assert abs(E2 - E) < 1e-10
    assert np.abs(F2 - F).max() < 1e-10


def test_periodic_cube_symmetries(default_model, water, water_ref):
    cfg, w, m = default_model
    coord, atype, box = water
    E, e, F, W = water_ref
    perm = [1, 2, 0]
    E2, _, F2, _ = energy_force_virial(m, coord[:, perm], box, atype)
    assert abs(E2 - E) < 1e-10
    assert np.abs(F2 - F[:, perm]).max() < 1e-10
    refl = coord.copy(); refl[:, 0] = box[0] - refl[:, 0]
    E3, _, F3, _ = energy_force_virial(m, refl, box, atype)
    assert abs(E3 - E) < 1e-10
    assert np.abs(F3[:, 0] + F[:, 0]).max() < 1e-10
    assert np.abs(F3[:, 1:] - F[:, 1:]).max() < 1e-10


def test_rotation_invariance_of_cluster(default_model):
    cfg, w, m = default_model
    coord, atype, box = synth.isolated_cluster(seed=4, natoms=14)
    E, e, F, W = energy_force_virial(m, coord, box, atype)
    rot = torch.linalg.matrix_exp(torch.tensor([[0, -0.3, 0.8], [0.3, 0, -0.5], [-0.8, 0.5, 0]], dtype=F64)).numpy()
    c0 = coord.mean(axis=0)
    rc = (coord - c0) @ rot.T + c0
    E2, e2, F2, W2 = energy_force_virial(m, rc, box, atype)
    assert abs(E2 - E) < 1e-10
    assert np.abs(F2 - F @ rot.T).max() < 1e-10
    assert np.abs(W2 - rot @ W @ rot.T).max() < 1e-10


def test_same_type_permutation_invariance(default_model, water, water_ref):
    cfg, w, m = default_model
    coord, atype, box = water
    E, e, F, W = water_ref
    perm = np.random.default_rng(1).permutation(len(coord))
    E2, e2, F2, W2 = energy_force_virial(m, coord[perm], box, atype[perm])
    assert abs(E2 - E) < 1e-10
    assert np.abs(e2 - e[perm]).max() < 1e-10
    assert np.abs(F2 - F[perm]).max() < 1e-10


def test_replication_is_extensive(default_model, water, water_ref):
    cfg, w, m = default_model
    coord, atype, box = water
    E, e, F, W = water_ref
    shifts = np.array([[i, j, k] for i in range(2) for j in range(2) for k in range(2)], dtype=float)
    big = np.concatenate([coord + s * box for s in shifts])
    E8, e8, F8, W8 = energy_force_virial(m, big, 2 * box, np.tile(atype, 8))
    assert abs(E8 - 8 * E) < 1e-8
    assert np.abs(e8 - np.tile(e, 8)).max() < 1e-10
    assert np.abs(F8 - np.tile(F, (8, 1))).max() < 1e-10
    assert np.abs(W8 - 8 * W).max() < 1e-8


def test_locality(default_model, water, water_ref):
    cfg, w, m = default_model
    coord, atype, box = water
    E, e, F, W = water_ref
    k = 17
    moved = coord.copy(); moved[k] += np.array([0.05, -0.03, 0.02])
    _, e2, _, _ = energy_force_virial(m, moved, box, atype)
    d = coord - coord[k]
    d -= box * np.rint(d / box)
    far = np.sqrt((d * d).sum(1)) > cfg.rcut + 0.1
    assert far.sum() > 10
    assert np.abs(e2[far] - e[far]).max() < 1e-12
    assert np.abs(e2[~far] - e[~far]).max() > 1e-6


def test_energy_continuous_across_cutoff(default_model):
    """With no attention layer (the DP-SE reduction) the switch makes E
    continuous as a neighbour crosses rcut.  With the smooth attention the
    entering key still adds exp(-S) to each softmax normaliser, so E jumps
    by a small amount (relative size exp(-S)/Z per row)."""
    import dataclasses

    cfg, w, _ = default_model
    box = np.array([40.0, 40.0, 40.0])
    base = np.array([[20.0, 20.0, 20.0], [21.1, 20.4, 19.8], [20.3, 21.0, 20.2]])
    atype = np.array([3, 0, 1, 0], dtype=np.int32)
    se_cfg = dataclasses.replace(cfg, attn_layers=0)
    for c, bound in ((se_cfg, 1e-12), (cfg, 1e-3)):
        m = OracleModel.from_numpy(c, w)
        out = []
        for dr in (-1e-9, 1e-9):
            xyz = np.vstack([base, [20.0 + c.rcut + dr, 20.0, 20.0]])
            out.append(energy_force_virial(m, xyz, box, atype)[0])
        assert abs(out[0] - out[1]) < bound, (c.attn_layers, out[0] - out[1])


# ------------------------------------------------------------ special cases

@pytest.mark.parametrize("stats", [False, True])
def test_two_atom_closed_form(rich_model, stats):
    """One neighbour each: softmax over one key is 1 and the gate is 1, so a
    layer is G <- G + LN((w^2 (G Wv + bv)) Wo + bo), and with the single row
    R_j = ((s - davg_0)/dstd_0, (s x/r - davg_1)/dstd_1, ...) of the centre's
    type (Sec. II-B: R in invariant coordinates, normalised per centre type)
    D = |R_j|^2 G (x) G_< / sel^2, where G's input is the normalised R_j0.
    With ``stats`` the rich model's davg/dstd (non-zero, non-unit, different
    for the two centre types) are kept; the pair lies along (1, 1, 1), so
    the two centres see displacement components of opposite sign and a
    wrong sign, scale, column or type index in the normalisation changes e."""
    cfg, w0, _ = rich_model
    w = dict(w0)
    if not stats:
        w["davg"] = np.zeros_like(w["davg"]); w["dstd"] = np.ones_like(w["dstd"])
    else:
        # the pin needs every column's mean and spread to differ between types
        assert np.all(np.abs(w["davg"][3] - w["davg"][1]) > 1e-3)
        assert np.all(np.abs(w["dstd"][[1, 3]] - 1.0) > 1e-2)
    m = OracleModel.from_numpy(cfg, w)
    box = np.array([40.0, 40.0, 40.0])
    ta, tb = 3, 1
    r = 3.7
    coord = np.array([[20.0, 20.0, 20.0], [20.0 + r / math.sqrt(3)] * 3])
    atype = np.array([ta, tb], dtype=np.int32)
    E, e, F, W = energy_force_virial(m, coord, box, atype)

    rcs, rc = cfg.rcut_smth, cfg.rcut
    u = (r - rcs) / (rc - rcs)
    sw = u ** 3 * (-6 * u * u + 15 * u - 10) + 1
    s = sw / r

    def net(x, pre):
        for l in range(3):
            Wl, bl = w[f"{pre}_W{l}"], w[f"{pre}_b{l}"]
            y = np.tanh(x @ Wl + bl)
            x = y if Wl.shape[0] * 2 != Wl.shape[1] and Wl.shape[0] != Wl.shape[1] else (
                x + y if Wl.shape[0] == Wl.shape[1] else np.concatenate([x, x]) + y)
        return x

    z = np.tanh(w["te_W"] + w["te_b"])
    for centre, other, sign in ((ta, tb, 1.0), (tb, ta, -1.0)):
        raw = np.array([s, sign * s / math.sqrt(3), sign * s / math.sqrt(3), sign * s / math.sqrt(3)])
        Rj = (raw - w["davg"][centre]) / w["dstd"][centre]
        G = net(np.array([Rj[0]]), "em") * (1 + net(np.concatenate([z[other], z[centre]]), "tt"))
        for l in range(cfg.attn_layers):
            y = (sw * sw * (G @ w[f"at{l}_Wv"] + w[f"at{l}_bv"])) @ w[f"at{l}_Wo"] + w[f"at{l}_bo"]
            zz = (y - y.mean()) / math.sqrt(y.var() + cfg.ln_eps)
            G = G + zz * w[f"at{l}_ln_g"] + w[f"at{l}_ln_b"]
        D = float(Rj @ Rj) * np.outer(G, G[: cfg.axis]) / cfg.sel ** 2
        x = np.concatenate([D.ravel(), z[centre]])
        h = np.tanh(x @ w["fit_W0"] + w["fit_b0"])
        for l in (1, 2):
            h = h + np.tanh(h @ w[f"fit_W{l}"] + w[f"fit_b{l}"])
        e_ref = cfg.out_scale * (h @ w["fit_W3"] + w["fit_b3"])[0] + w["ebias"][centre]
        idx = 0 if centre == ta else 1
        assert abs(e[idx] - e_ref) < 1e-12 * max(1.0, abs(e_ref))
    # Newton's third law (translation invariance) always; a central force
    # only without the per-column shift, which is not rotation invariant
    assert np.abs(F[0] + F[1]).max() < 1e-12
    if not stats:
        rhat = (coord[1] - coord[0]) / r
        assert np.abs(F[0] - np.dot(F[0], rhat) * rhat).max() < 1e-12


def test_gated_attention_reduces_to_sdpa_and_layer_norm(rich_model):
    """With Q' = w Q, K' = w K and the additive mask S (w_j w_k - 1), the
    smooth logits are exactly the scaled dot-product logits, and since the
    gate rhat_j . rhat_k splits into three rank-one terms,
    O_j = w_j sum_a rhat_ja SDPA(Q', K', w rhat_a V)_j."""
    cfg, w, m = rich_model
    p = m.attn(0)
    g = torch.Generator().manual_seed(0)
    C, S, M1 = 5, 24, cfg.m1
    G = torch.randn(C, S, M1, generator=g, dtype=F64)
    nvalid = torch.tensor([24, 17, 1, 9, 3])
    mask = torch.arange(S)[None, :] < nvalid[:, None]
    wsw = torch.rand(C, S, generator=g, dtype=F64) * mask
    rh = torch.randn(C, S, 3, generator=g, dtype=F64)
    rh = rh / rh.norm(dim=-1, keepdim=True) * mask[..., None]
    G = G * mask[..., None]
    out = gated_attention(G, wsw, rh, mask, p, cfg.attn_shift, cfg.ln_eps)

    Q = (G @ p["Wq"] + p["bq"]) * wsw[..., None]
    K = (G @ p["Wk"] + p["bk"]) * wsw[..., None]
    V = G @ p["Wv"] + p["bv"]
    add = cfg.attn_shift * (wsw[:, :, None] * wsw[:, None, :] - 1.0)
    add = add.masked_fill(~mask[:, None, :], float("-inf"))
    O = torch.zeros(C, S, V.shape[-1], dtype=F64)
    for a in range(3):
        Va = V * (wsw * rh[..., a])[..., None]
        O = O + (wsw * rh[..., a])[..., None] * tF.scaled_dot_product_attention(Q, K, Va, attn_mask=add)
    Y = O @ p["Wo"] + p["bo"]
    ref = G + tF.layer_norm(Y, (M1,), p["ln_g"], p["ln_b"], cfg.ln_eps)
    assert torch.allclose(out[mask], ref[mask], rtol=0, atol=1e-12)
    assert torch.equal(out[~mask], G[~mask])


def test_type_pair_table_orders_neighbour_then_centre(default_model):
    cfg, w, m = default_model
    tebd = type_embedding(m.t["te_W"], m.t["te_b"])
    Gt = type_pair_table(tebd, m.layers("tt", 3))
    x = torch.cat([tebd[4], tebd[2]])  # neighbour type 4, centre type 2
    assert torch.allclose(Gt[2, 4], embedding_net(x, m.layers("tt", 3)), atol=0, rtol=0)
    assert not torch.allclose(Gt[2, 4], Gt[4, 2])


def test_isolated_atoms_have_descriptor_zero(default_model):
    cfg, w, m = default_model
    box = np.array([30.0, 30.0, 30.0])
    coord = np.array([[1.0, 1.0, 1.0], [15.0, 15.0, 15.0]])
    atype = np.array([0, 4], dtype=np.int32)
    E, e, F, W = energy_force_virial(m, coord, box, atype)
    z = np.tanh(w["te_W"] + w["te_b"])
    for i, t in enumerate(atype):
        x = np.concatenate([np.zeros(cfg.desc_dim), z[t]])
        h = np.tanh(x @ w["fit_W0"] + w["fit_b0"])
        for l in (1, 2):
            h = h + np.tanh(h @ w[f"fit_W{l}"] + w[f"fit_b{l}"])
        assert abs(e[i] - (cfg.out_scale * (h @ w["fit_W3"] + w["fit_b3"])[0] + w["ebias"][t])) < 1e-12
    assert np.abs(F).max() == 0.0


# ------------------------------------------------------------- generators

def test_synthetic_systems_recipes():
    coord, atype, box = synth.lattice_system(15668, seed=1)
    assert coord.shape == (15668, 3)
    counts = np.bincount(atype, minlength=5)
    assert counts.tolist() == [9871, 1880, 470, 3290, 157]
    assert abs(box[0] - (15668 / 0.1) ** (1 / 3)) < 1e-9
    assert np.all((coord >= 0) & (coord < box))
    c, t, b = synth.water_box(0)
    assert c.shape == (192, 3) and b[0] == 12.4
    d = c[:, None] - c[None]
    d -= b * np.rint(d / b)
    r = np.sqrt((d ** 2).sum(-1)) + np.eye(192) * 10
    assert r.min() >= 0.9 - 1e-12  # inter-molecular >= 0.9 A, intra-molecular O-H 0.96 A


def test_local_ghost_decomposition_reassembles_the_box():
    """Eq. eq_forcesLocalGhost: a periodic box split into two x slabs, each
    evaluated with its ghost atoms within rcut and only its local atoms'
    energies counted, gives back the whole box: energies and virials add up,
    and the forces on local and ghost rows summed per original atom are the
    full forces."""
    import synth
    from oracle import OracleModel, energy_force_virial

    cfg = synth.DEFAULT_CONFIG
    om = OracleModel.from_numpy(cfg, synth.make_weights(cfg, seed=1))
    coord, atype, box = synth.lattice_system(420, seed=23)
    E, _, F, W = energy_force_virial(om, coord, box, atype)
    Es, Fs, Ws = 0.0, np.zeros_like(F), np.zeros((3, 3))
    for c, t, b, nloc, owner in synth.slab_subdomains(coord, atype, box, 2, cfg.rcut):
        e, _, f, w = energy_force_virial(om, c, b, t, centres=np.arange(nloc))
        Es += e
        Ws += w
        np.add.at(Fs, owner, f)
    assert abs(Es - E) < 1e-10 * max(1.0, abs(E))
    assert np.abs(Fs - F).max() < 1e-10
    assert np.abs(Ws - W).max() < 1e-9


def _one_type(cfg, mode):
    import dataclasses

    return dataclasses.replace(cfg, ntypes=1, type_map=("X",), embed=(16, 32, 64), axis=8, attn_layers=1,
                               fitting=(64, 64), tebd_input_mode=mode)


def test_concat_single_type_reduces_to_strip():
    """With one atom type the concat input [s, T, T] adds a constant to the
    first layer: concat mode equals strip mode with that constant in the
    first bias, G0 divided by strip mode's (1 + Gt[0, 0]).  The two modes
    build G0 by separate code, so this checks the concat path's input."""
    base = synth.DEFAULT_CONFIG
    cc, cs = _one_type(base, "concat"), _one_type(base, "strip")
    wc = synth.make_weights(cc, seed=11, bias_scale=0.2)
    ws = synth.make_weights(cs, seed=12, bias_scale=0.2)
    for k in wc:
        if k in ws and not k.startswith("em_W0") and not k.startswith("em_b0"):
            ws[k] = wc[k]
    td = cc.tebd_dim
    T = np.tanh(wc["te_W"][0] + wc["te_b"])
    ws["em_W0"] = wc["em_W0"][0:1]
    ws["em_b0"] = wc["em_b0"] + T @ wc["em_W0"][1:1 + td] + T @ wc["em_W0"][1 + td:]
    mc, ms = OracleModel.from_numpy(cc, wc), OracleModel.from_numpy(cs, ws)
    coord, atype, box = synth.water_box(seed=3)
    atype = np.zeros_like(atype)
    stc, sts = {}, {}
    energy_force_virial(mc, coord[:40], box, atype[:40], stages=stc)
    energy_force_virial(ms, coord[:40], box, atype[:40], stages=sts)
    gt = sts["Gt"][0, 0]
    assert torch.allclose(stc["G0"] * (1.0 + gt), sts["G0"], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("block", ["neighbour", "centre"])
def test_concat_input_orders_neighbour_then_centre(concat_model, block):
    """With only the neighbour block (columns 1..td of the input) of the
    first layer non-zero, a row of G0 depends on the neighbour's type and
    not on the centre's; with only the centre block, the other way round."""
    import dataclasses

    cfg, w, _ = concat_model
    td = cfg.tebd_dim
    w = dict(w)
    W0 = w["em_W0"].copy()
    if block == "neighbour":
        W0[1 + td:] = 0.0
    else:
        W0[1:1 + td] = 0.0
    w["em_W0"] = W0
    m = OracleModel.from_numpy(cfg, w)
    box = np.array([30.0, 30.0, 30.0])
    coord = np.array([[10.0, 10.0, 10.0], [11.5, 10.0, 10.0]])  # centre 0, neighbour 1 at 1.5 A
    g = {}
    for tc in (0, 3):
        for tn in (1, 4):
            st = {}
            energy_force_virial(m, coord, box, np.array([tc, tn], np.int32), centres=np.array([0]), stages=st)
            g[tc, tn] = st["G0"][0, 0]
    if block == "neighbour":
        assert torch.equal(g[0, 1], g[3, 1]) and not torch.allclose(g[0, 1], g[0, 4])
    else:
        assert torch.equal(g[0, 1], g[0, 4]) and not torch.allclose(g[0, 1], g[3, 1])


def test_concat_forces_central_difference(concat_model, water):
    cfg, w, m = concat_model
    coord, atype, box = water
    E, e, F, W = energy_force_virial(m, coord, box, atype)
    nl, _, _ = oracle.neighbor_list(coord, box, cfg.rcut, cfg.sel)
    h = 1e-4

    def en(a, k, t):
        c = coord.copy(); c[a, k] += t
        return energy_force_virial(m, c, box, atype, nlist=nl)[0]

    for a in (5, 77):
        for k in range(3):
            fd4 = -(-en(a, k, 2 * h) + 8 * en(a, k, h) - 8 * en(a, k, -h) + en(a, k, -2 * h)) / (12 * h)
            assert abs(fd4 - F[a, k]) < 1e-8 * max(1.0, abs(F[a, k])), (a, k, fd4, F[a, k])
