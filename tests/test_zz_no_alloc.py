"""The allocation-free neighbour list (dp_nlist_noalloc) against the
workspace-backed one (dp_nlist_device), through the C ABI.

Some callers cannot allocate device memory while they run (an MD engine
that only lends its own pooled buffers, code inside a host callback or a
captured stream), so this entry point keeps its scratch in a fixed device
array.  Its list must be identical to the regular entry point's, on two
calls in a row (the shared scratch keeps the previous call's contents).

The file name makes pytest collect it last, so that a run stopping at the
first failure (-x) has run every other test before this one; the tests
depend on no order and also pass alone in a fresh process."""

import numpy as np
import pytest

import synth

from gpu_helpers import weight_file

pytestmark = pytest.mark.gpu


def _run_noalloc(p, torch, coord_t, box_t, rcut, sel):
    n = coord_t.shape[0]
    nl = torch.full((n, 128), -7, dtype=torch.int32, device="cuda")
    nn = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    p.binding.nlist_noalloc(coord_t, box_t, rcut, sel, nl, nn, status)
    torch.cuda.synchronize()
    return nl.cpu().numpy(), nn.cpu().numpy(), int(status.item())


def test_noalloc_nlist_matches_workspace_nlist(default_model):
    import torch
    import paper_2604_07276_gb300 as p

    cfg, w, _ = default_model
    model = p.DPA1(weight_file(cfg, w, "default"), precision="fp32")
    systems = [synth.water_box(0), synth.lattice_system(3000, seed=41), synth.lattice_system(700, seed=42)]
    for coord, atype, box in systems:
        model.reserve(len(coord))
        c = torch.tensor(coord, dtype=torch.float64, device="cuda")
        b = torch.tensor(p.box9(box), dtype=torch.float64, device="cuda")
        ref_nl, ref_nn = model.nlist_device(c, b)
        torch.cuda.synchronize()
        model.status()
        ref_nl, ref_nn = ref_nl.cpu().numpy(), ref_nn.cpu().numpy()
        for _ in range(2):  # two calls in a row share the scratch array
            nl, nn, status = _run_noalloc(p, torch, c, b, cfg.rcut, cfg.sel)
            assert status == 0
            assert np.array_equal(nn, ref_nn)
            assert np.array_equal(nl, ref_nl)
    model.close()


def test_noalloc_nlist_rejects_oversize():
    import torch
    import paper_2604_07276_gb300 as p

    n = 65537
    c = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    b = torch.tensor(p.box9([100.0, 100.0, 100.0]), dtype=torch.float64, device="cuda")
    nl = torch.empty((1, 128), dtype=torch.int32, device="cuda")
    nn = torch.empty((1,), dtype=torch.int32, device="cuda")
    st = torch.empty((1,), dtype=torch.int32, device="cuda")
    with pytest.raises(p.DPError) as ei:
        p.binding.nlist_noalloc(c, b, 6.0, 120, nl, nn, st)
    assert ei.value.code == -4
    assert "65536" in str(ei.value)


def test_noalloc_nlist_empty_and_device_status():
    """natoms == 0 accepts null coordinate and output pointers and leaves the
    status at 0; a box edge <= 2 rcut sets status bit 1 and a non-finite
    coordinate bit 4 (both found by the kernels, which skip the bad input)."""
    import torch
    import paper_2604_07276_gb300 as p

    st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    b = torch.tensor(p.box9([30.0, 30.0, 30.0]), dtype=torch.float64, device="cuda")
    lib = p.load_library()
    p.binding._check(lib.dp_nlist_noalloc(0, None, b.data_ptr(), 6.0, 120, None, None, st.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert int(st.item()) == 0

    coord, atype, box = synth.water_box(0)
    c = torch.tensor(coord, dtype=torch.float64, device="cuda")
    small = torch.tensor(p.box9([11.0, 12.4, 12.4]), dtype=torch.float64, device="cuda")
    _, _, status = _run_noalloc(p, torch, c, small, 6.0, 120)
    assert status & 1
    bad = coord.copy()
    bad[5, 2] = np.nan
    cb = torch.tensor(bad, dtype=torch.float64, device="cuda")
    b = torch.tensor(p.box9(box), dtype=torch.float64, device="cuda")
    nl, nn, status = _run_noalloc(p, torch, cb, b, 6.0, 120)
    assert status & 4
    assert nn[5] == 0
    # a good call afterwards starts from a cleared status
    _, _, status = _run_noalloc(p, torch, c, b, 6.0, 120)
    assert status == 0
