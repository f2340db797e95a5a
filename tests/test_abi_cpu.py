"""CPU-side checks of the C ABI library: it loads, exports every symbol that
include/dpa1.h declares, parses weight files, and reports errors without a
GPU.  No compute call is made."""

import os
import re
import tempfile

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib_or_skip():
    path = os.path.join(ROOT, "paper_2604_07276_gb300", "lib", "libdpa1.so")
    if not os.path.exists(path):
        pytest.skip("library not built (run __graft_entry__.build())")
    import paper_2604_07276_gb300 as p

    return p


def _declared():
    src = open(os.path.join(ROOT, "include", "dpa1.h")).read()
    return sorted(set(re.findall(r"DP_API\s+[\w\s\*]*?\b(dp_\w+)\s*\(", src)))


def test_header_declares_the_abi():
    names = _declared()
    assert "dp_init" in names and "dp_compute" in names and "dp_compute_device" in names
    assert len(names) >= 13


def test_library_exports_every_declared_symbol():
    p = _lib_or_skip()
    lib = p.load_library()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(p.EXPORTS) <= set(_declared())


def test_inspect_weights_roundtrip():
    p = _lib_or_skip()
    cfg = synth.DEFAULT_CONFIG
    w = synth.make_weights(cfg, 0)
    with tempfile.TemporaryDirectory() as d:
        f = os.path.join(d, "w.bin")
        synth.write_weights(f, cfg, w)
        ints, dbls = p.inspect_weights(f)
        assert list(ints[:15]) == [1, 5, 8, 120, 16, 3, 25, 50, 100, 2, 128, 3, 240, 240, 240]
        assert dbls[0] == 6.0 and dbls[1] == 0.5 and dbls[2] == 20.0 and dbls[4] == cfg.out_scale
        # truncated / wrong files are rejected with DP_ERR_IO
        with open(f, "rb") as fh:
            head = fh.read(50)
        bad = os.path.join(d, "bad.bin")
        with open(bad, "wb") as fh:
            fh.write(b"NOTDPA1!" + head[8:])
        with pytest.raises(p.DPError) as ei:
            p.inspect_weights(bad)
        assert ei.value.code == -2
        with pytest.raises(p.DPError) as ei:
            p.inspect_weights(os.path.join(d, "missing.bin"))
        assert ei.value.code == -2


def test_init_without_gpu_fails_cleanly():
    p = _lib_or_skip()
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = synth.DEFAULT_CONFIG
    with tempfile.TemporaryDirectory() as d:
        f = os.path.join(d, "w.bin")
        synth.write_weights(f, cfg, synth.make_weights(cfg, 0))
        with pytest.raises(p.DPError) as ei:
            p.DPA1(f)
        assert ei.value.code == -5


def test_weight_file_matches_generator_order():
    """The writer's layout is what the reader expects: sizes add up."""
    cfg = synth.DEFAULT_CONFIG
    w = synth.make_weights(cfg, 0)
    with tempfile.TemporaryDirectory() as d:
        f = os.path.join(d, "w.bin")
        synth.write_weights(f, cfg, w)
        n = sum(int(np.prod(s)) for _, s in synth.model.tensor_order(cfg))
        assert os.path.getsize(f) == 8 + 64 + 64 + 8 * cfg.ntypes + 8 * n
