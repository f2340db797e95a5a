"""Adjoint check on a batch of uneven frames: 32 frames of U{200..3000}
atoms (same composition and density as the protein-like box, seed 2) in
one batched call.  Per frame, the forces on 2 sampled atoms (64 in all) are
compared with the FP64 oracle and with central finite differences of the
GPU energy at h = 1e-4 A (and at 2e-3 A, where FP32 noise is small)."""

import numpy as np
import pytest

import synth
import oracle

from gpu_helpers import weight_file, force_rmse, FP32_FORCE_RMSE, BF16_FORCE_RMSE

pytestmark = pytest.mark.gpu

H = 1e-4


@pytest.fixture(scope="module")
def frames():
    return synth.frame_batch(seed=2, nframes=32)


@pytest.fixture(scope="module")
def sampled(frames, default_model):
    _, _, om = default_model
    rng = np.random.default_rng(7)
    out = []
    for c, t, b in frames:
        atoms = rng.choice(len(c), size=2, replace=False)
        out.append((atoms, oracle.forces_on(om, c, b, t, atoms)))
    return out


def _near_cut(coord, box, a, rcut, h):
    """True if atom a has a partner within 2h of the cutoff (a displacement
    of h could change a neighbour list, where the smooth-attention reading
    is not continuous)."""
    d = coord - coord[a]
    L = np.asarray(box, dtype=np.float64)
    d -= L * np.rint(d / L)
    r = np.sqrt((d * d).sum(axis=1))
    return bool(np.any(np.abs(r - rcut) < 2 * h))


def test_batch_fp32_oracle_and_fd(default_model, frames, sampled):
    import paper_2604_07276_gb300 as p

    cfg, w, _ = default_model
    m = p.DPA1(weight_file(cfg, w, "default"), precision="fp32")
    m.reserve(max(len(t) for _, t, _ in frames))
    E, F, W = m.compute_batch(frames)
    got = np.concatenate([F[k][atoms] for k, (atoms, _) in enumerate(sampled)])
    ref = np.concatenate([rF for _, rF in sampled])
    assert force_rmse(got, ref) <= FP32_FORCE_RMSE  # RMSE over the 64 sampled atoms
    for k, (c, t, b) in enumerate(frames):
        Ek, Fk, Wk, _ = m.compute(c, b, t)  # a batched frame is the same frame alone
        assert Ek == E[k] and np.array_equal(Fk, F[k]) and np.array_equal(Wk, W[k])
    # Central differences of the GPU energy.  At h = 1e-4 A the quotient is
    # dominated by the FP32 rounding noise of the ~90 atomic energies a
    # displacement touches, divided by 2h (measured: error rms ~8 % of the
    # force rms); at h = 2e-3 A that noise is 20x smaller and the truncation
    # error still negligible, so the agreement there is tight.  Atoms with a
    # partner within 2h of the cutoff are skipped.
    for h, rms_bound, max_bound, min_count in ((1e-4, 0.15, 0.5, 150), (2e-3, 0.01, 0.05, 100)):
        fd_err, fscale = [], []
        for k, ((c, t, b), (atoms, _)) in enumerate(zip(frames, sampled)):
            for a in atoms:
                if _near_cut(c, b, a, cfg.rcut, h):
                    continue
                for d in range(3):
                    cp = c.copy()
                    cp[a, d] += h
                    cm = c.copy()
                    cm[a, d] -= h
                    fd = -(m.compute(cp, b, t)[0] - m.compute(cm, b, t)[0]) / (2 * h)
                    fd_err.append(fd - F[k][a, d])
                    fscale.append(F[k][a, d])
        fd_err = np.asarray(fd_err)
        rms, mx = float(np.sqrt(np.mean(fd_err ** 2))), float(np.abs(fd_err).max())
        frms = float(np.sqrt(np.mean(np.square(fscale))))
        print(f"FD h={h}: {len(fd_err)} components, error rms {rms:.3e} max {mx:.3e}, force rms {frms:.3e}")
        assert len(fd_err) >= min_count
        assert rms <= rms_bound * frms and mx <= max_bound * frms, (h, rms, mx, frms)
    m.close()


def test_batch_fp16x_oracle(default_model, frames, sampled):
    import paper_2604_07276_gb300 as p

    cfg, w, _ = default_model
    m = p.DPA1(weight_file(cfg, w, "default"), precision="fp16x")
    m.reserve(max(len(t) for _, t, _ in frames))
    E, F, W = m.compute_batch(frames)
    got = np.concatenate([F[k][atoms] for k, (atoms, _) in enumerate(sampled)])
    ref = np.concatenate([rF for _, rF in sampled])
    assert force_rmse(got, ref) <= BF16_FORCE_RMSE
    for k, (c, t, b) in enumerate(frames):
        Ek, Fk, Wk, _ = m.compute(c, b, t)  # the packed pass gives each frame's own result
        assert Ek == E[k] and np.array_equal(Fk, F[k]) and np.array_equal(Wk, W[k])
    m.close()


def _same_as_alone(m, frames):
    E, F, W = m.compute_batch(frames)
    assert len(E) == len(frames) and W.shape == (len(frames), 3, 3)
    for k, (c, t, b) in enumerate(frames):
        Ek, Fk, Wk, _ = m.compute(c, b, t)
        assert Ek == E[k] and np.array_equal(Fk, F[k]) and np.array_equal(Wk, W[k]), k


@pytest.mark.parametrize("precision", ["fp32", "fp16x"])
def test_batch_edge_frames(default_model, precision):
    """Empty frames, frames of 1, 2 and 5 atoms (padding in every force
    block), isolated atoms and a ragged lattice frame, mixed in one batch."""
    import paper_2604_07276_gb300 as p

    cfg, w, _ = default_model
    box = np.array([30.0, 30.0, 30.0])
    c2 = np.array([[1.0, 1.0, 1.0], [15.0, 15.0, 15.0]])
    c5 = np.array([[10.0, 10.0, 10.0], [11.2, 10.3, 9.9], [20.0, 20.0, 20.0], [21.0, 20.2, 20.0],
                   [20.1, 21.1, 19.5]])
    lat = synth.lattice_system(301, seed=5)
    frames = [(np.zeros((0, 3)), np.zeros(0, np.int32), box),
              (np.array([[3.0, 4.0, 5.0]]), np.array([2], np.int32), box),
              (c5, np.array([3, 0, 1, 2, 3], np.int32), box),
              (np.zeros((0, 3)), np.zeros(0, np.int32), box),
              (lat[0], lat[1], lat[2]),
              (c2, np.array([0, 4], np.int32), box * 1.5)]
    m = p.DPA1(weight_file(cfg, w, "default"), precision=precision)
    _same_as_alone(m, frames)
    E, F, W = m.compute_batch(frames[:1])  # a batch of one empty frame
    assert E[0] == 0.0 and np.all(W == 0.0) and F[0].shape == (0, 3)
    m.close()


def test_batch_several_passes(default_model):
    """Three frames of 25,001 atoms: 75,012 padded slots, more than one pass
    holds, so the batch runs as two passes (frames 0-1, then frame 2)."""
    import paper_2604_07276_gb300 as p

    cfg, w, _ = default_model
    frames = [synth.lattice_system(25001, seed=s) for s in (41, 42, 43)]
    frames = [(c, t, b) for c, t, b in frames]
    m = p.DPA1(weight_file(cfg, w, "default"), precision="fp16x")
    _same_as_alone(m, frames)
    m.close()
