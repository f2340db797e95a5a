"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Neighbour lists must be bit-exact; energies, forces and virials must be
within the stated tolerances of the oracle."""

import dataclasses

import numpy as np
import pytest

import synth
import oracle
from oracle import OracleModel, energy_force_virial

from gpu_helpers import weight_file, force_rmse, FP32_FORCE_RMSE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2604_07276_gb300 as p

    return p


@pytest.fixture(scope="module")
def fp32_model(lib, default_model):
    cfg, w, _ = default_model
    m = lib.DPA1(weight_file(cfg, w, "default"), precision="fp32")
    yield m
    m.close()


@pytest.fixture(scope="module")
def fp32_rich(lib, rich_model):
    cfg, w, _ = rich_model
    m = lib.DPA1(weight_file(cfg, w, "rich"), precision="fp32")
    yield m
    m.close()


def _device(arrs):
    import torch

    return [torch.as_tensor(np.ascontiguousarray(a)).cuda() for a in arrs]


# ----------------------------------------------------------------- neighbours

@pytest.mark.parametrize("system", ["water", "lattice", "truncated"])
def test_neighbor_list_bit_exact(lib, default_model, system):
    import torch

    cfg, w, _ = default_model
    if system == "water":
        coord, atype, box = synth.water_box(0)
    else:
        coord, atype, box = synth.lattice_system(2500, seed=21)
    if system == "truncated":
        cfg = dataclasses.replace(cfg, sel=40)
    m = lib.DPA1(weight_file(cfg, w, f"sel{cfg.sel}"), precision="fp32")
    m.reserve(len(coord))
    c, b = _device([coord, lib.box9(box)])
    nl, nn = m.nlist_device(c, b)
    torch.cuda.synchronize()
    m.status()
    ref, rnn, rcand = oracle.neighbor_list(coord, box, cfg.rcut, cfg.sel)
    got = nl.cpu().numpy()
    assert np.array_equal(nn.cpu().numpy(), rnn)
    assert np.array_equal(got[:, :cfg.sel], ref)
    assert np.all(got[:, cfg.sel:] == -1)
    if system == "truncated":
        assert np.any(rcand > cfg.sel)
    m.close()


# ------------------------------------------------------------ FP32 vs oracle

def _compare(m, om, coord, atype, box, f_rmse, e_tol, w_tol):
    E, F, W, e = m.compute(coord, box, atype, atom_energy=True)
    rE, re, rF, rW = energy_force_virial(om, coord, box, atype)
    assert force_rmse(F, rF) <= f_rmse, force_rmse(F, rF)
    assert np.abs(e - re).max() <= e_tol, np.abs(e - re).max()
    assert abs(E - rE) <= e_tol * max(1, len(coord)) ** 0.5 + 1e-9 * abs(rE)
    assert np.abs(W - rW).max() <= w_tol * max(1.0, np.abs(rW).max()), np.abs(W - rW).max()
    return E, F, W, e


def test_fp32_water_default(fp32_model, default_model, water):
    cfg, w, om = default_model
    coord, atype, box = water
    _compare(fp32_model, om, coord, atype, box, FP32_FORCE_RMSE, 1e-4, 1e-4)


def test_fp32_water_rich_weights(fp32_rich, rich_model, water):
    cfg, w, om = rich_model
    coord, atype, box = water
    _compare(fp32_rich, om, coord, atype, box, FP32_FORCE_RMSE, 1e-4, 1e-4)


def test_fp32_fitting_widths_not_multiples_of_4(lib, water):
    """Fitting widths of 30: the FP32 GEMM's 4-byte load and store path
    (16-byte accesses need every width a multiple of 4)."""
    cfg = dataclasses.replace(synth.DEFAULT_CONFIG, fitting=(30, 30))
    w = synth.make_weights(cfg, seed=37, bias_scale=0.1, stats=True)
    om = OracleModel.from_numpy(cfg, w)
    m = lib.DPA1(weight_file(cfg, w, "fit30"), precision="fp32")
    try:
        coord, atype, box = water
        _compare(m, om, coord, atype, box, FP32_FORCE_RMSE, 1e-4, 1e-4)
    finally:
        m.close()


def test_fp32_lattice_ragged(fp32_model, default_model):
    cfg, w, om = default_model
    coord, atype, box = synth.lattice_system(1123, seed=31)
    _compare(fp32_model, om, coord, atype, box, FP32_FORCE_RMSE, 1e-4, 1e-4)


def test_fp32_edge_cases(fp32_model, default_model):
    cfg, w, om = default_model
    box = np.array([30.0, 30.0, 30.0])
    # no atoms
    E, F, W, e = fp32_model.compute(np.zeros((0, 3)), box, np.zeros(0, np.int32), atom_energy=True)
    assert E == 0.0 and np.all(W == 0.0) and F.shape == (0, 3)
    # one atom, and two far-apart atoms (empty neighbourhoods)
    for coord, atype in ((np.array([[3.0, 4.0, 5.0]]), np.array([2], np.int32)),
                         (np.array([[1.0, 1.0, 1.0], [15.0, 15.0, 15.0]]), np.array([0, 4], np.int32))):
        _compare(fp32_model, om, coord, atype, box, FP32_FORCE_RMSE, 1e-5, 1e-5)
    # a pair and a triple: one and two neighbours
    coord = np.array([[10.0, 10.0, 10.0], [11.2, 10.3, 9.9], [20.0, 20.0, 20.0], [21.0, 20.2, 20.0],
                      [20.1, 21.1, 19.5]])
    _compare(fp32_model, om, coord, np.array([3, 0, 1, 2, 3], np.int32), box, FP32_FORCE_RMSE, 1e-5, 1e-5)
    # unwrapped coordinates far outside the box give the same result as wrapped ones
    c, t, b = synth.water_box(0)
    E1, F1, _, _ = fp32_model.compute(c, b, t)
    E2, F2, _, _ = fp32_model.compute(c + np.array([3, -2, 5]) * b, b, t)
    # the shifted copy rounds its displacements differently in FP64, which FP32
    # arithmetic then carries at the 1e-7 relative level
    assert abs(E1 - E2) < 1e-6 * abs(E1) and np.abs(F1 - F2).max() < 5e-5


def test_fp32_deterministic(fp32_model, water):
    coord, atype, box = water
    a = fp32_model.compute(coord, box, atype, atom_energy=True)
    b = fp32_model.compute(coord, box, atype, atom_energy=True)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


def test_bad_box_and_types(lib, fp32_model, water):
    coord, atype, box = water
    with pytest.raises(lib.DPError) as ei:
        fp32_model.compute(coord, np.array([11.0, 12.4, 12.4]), atype)
    assert ei.value.code == -3
    with pytest.raises(lib.DPError) as ei:
        fp32_model.compute(coord, box, np.full(len(atype), 7, np.int32))
    assert ei.value.code == -1
    with pytest.raises(lib.DPError) as ei:
        bad = coord.copy(); bad[3, 1] = np.nan
        fp32_model.compute(bad, box, atype)
    assert ei.value.code == -7


def test_device_path_box_check_sets_status(lib, fp32_model, water):
    """A bad box passed to the device entry point is caught on the device and
    reported by dp_get_status, without a fault."""
    import torch

    coord, atype, box = water
    fp32_model.reserve(len(coord))
    c, t = _device([coord, atype.astype(np.int32)])
    b = torch.tensor(lib.box9([11.0, 12.4, 12.4])).cuda()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros((len(coord), 3), dtype=torch.float64, device="cuda")
    W = torch.zeros(9, dtype=torch.float64, device="cuda")
    fp32_model.compute_device(c, b, t, E, F, W)
    with pytest.raises(lib.DPError) as ei:
        fp32_model.status()
    assert ei.value.code == -3
    fp32_model.status()  # cleared


def test_fp32_batch_uneven(fp32_model, default_model):
    cfg, w, om = default_model
    frames = synth.frame_batch(seed=2, nframes=3, lo=200, hi=500)
    E, F, W = fp32_model.compute_batch(frames)
    for k, (c, t, b) in enumerate(frames):
        rE, re, rF, rW = energy_force_virial(om, c, b, t)
        assert force_rmse(F[k], rF) <= FP32_FORCE_RMSE
        assert abs(E[k] - rE) < 1e-3


def test_autograd_function(lib, fp32_model, water):
    import torch
    from paper_2604_07276_gb300.autograd import energy

    coord, atype, box = water
    c = torch.tensor(coord, device="cuda", requires_grad=True)
    b = torch.tensor(lib.box9(box), device="cuda")
    t = torch.tensor(atype, dtype=torch.int32, device="cuda")
    E = energy(c, fp32_model, b, t)
    (g,) = torch.autograd.grad(2.0 * E, c)
    _, F, _, _ = fp32_model.compute(coord, box, atype)
    assert np.allclose(g.cpu().numpy(), -2.0 * F, atol=1e-9)


def test_autograd_box_gradient(lib, fp32_model, default_model, water):
    """dE/dh from the autograd Function (h^{-T}(sum x (x) F - W) of the
    CUDA path's forces and virial) against central differences of the FP64
    oracle's energy in each box edge, coordinates held fixed (h = 1e-4 A;
    the neighbour sets do not change over that step)."""
    import torch
    from paper_2604_07276_gb300.autograd import energy

    cfg, w, om = default_model
    coord, atype, box = water
    c = torch.tensor(coord, device="cuda", requires_grad=True)
    b = torch.tensor(lib.box9(box), device="cuda", requires_grad=True)
    t = torch.tensor(atype, dtype=torch.int32, device="cuda")
    E = energy(c, fp32_model, b, t)
    gc, gb = torch.autograd.grad(E, (c, b))
    gb = gb.cpu().numpy().reshape(3, 3)
    h = 1e-4
    fd = np.zeros(3)
    for a in range(3):
        bp, bm = np.array(box, dtype=float), np.array(box, dtype=float)
        bp[a] += h
        bm[a] -= h
        fd[a] = (energy_force_virial(om, coord, bp, atype)[0] - energy_force_virial(om, coord, bm, atype)[0]) / (2 * h)
    print(f"\ndE/dL GPU {np.diag(gb)}, oracle FD {fd}")
    assert np.abs(np.diag(gb) - fd).max() <= 1e-4 * max(1.0, np.abs(fd).max())
    # an isolated cluster has no periodic images: the box gradient vanishes
    cc, ct, cb = synth.isolated_cluster(3)
    c2 = torch.tensor(cc, device="cuda")
    b2 = torch.tensor(lib.box9(cb), device="cuda", requires_grad=True)
    (g2,) = torch.autograd.grad(energy(c2, fp32_model, b2, torch.tensor(ct, dtype=torch.int32, device="cuda")), b2)
    # (FP32 forces times coordinates near 20 A cancel to ~1e-6 relative)
    assert np.abs(g2.cpu().numpy()).max() < 1e-4
