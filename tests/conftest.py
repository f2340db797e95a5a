import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: longer CPU checks")


@pytest.fixture(scope="session")
def default_model():
    import synth
    from oracle import OracleModel

    cfg = synth.DEFAULT_CONFIG
    w = synth.make_weights(cfg, seed=0)
    return cfg, w, OracleModel.from_numpy(cfg, w)


@pytest.fixture(scope="session")
def rich_model():
    """Default sizes with non-zero biases, perturbed LayerNorm and davg/dstd,
    so that every term of the network is exercised."""
    import synth
    from oracle import OracleModel

    cfg = synth.DEFAULT_CONFIG
    w = synth.make_weights(cfg, seed=5, bias_scale=0.1, ln_scale=0.1, stats=True)
    return cfg, w, OracleModel.from_numpy(cfg, w)


@pytest.fixture(scope="session")
def concat_model():
    """Default sizes with the concat type-embedding mode (the embedding net
    reads [s, T_j, T_i]) and non-zero biases."""
    import dataclasses

    import synth
    from oracle import OracleModel

    cfg = dataclasses.replace(synth.DEFAULT_CONFIG, tebd_input_mode="concat")
    w = synth.make_weights(cfg, seed=7, bias_scale=0.1)
    return cfg, w, OracleModel.from_numpy(cfg, w)


@pytest.fixture(scope="session")
def paper_size_model():
    """The paper's model size (Sec. IV-B) with non-zero biases, perturbed
    LayerNorm and davg/dstd."""
    import synth
    from oracle import OracleModel

    cfg = synth.PAPER_SIZE_CONFIG
    w = synth.make_weights(cfg, seed=17, bias_scale=0.05, ln_scale=0.1, stats=True)
    return cfg, w, OracleModel.from_numpy(cfg, w)


@pytest.fixture(scope="session")
def water():
    import synth

    return synth.water_box(seed=0)


@pytest.fixture(scope="session")
def water_ref(default_model, water):
    from oracle import energy_force_virial

    cfg, w, m = default_model
    coord, atype, box = water
    return energy_force_virial(m, coord, box, atype)
