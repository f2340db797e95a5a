"""Stage-by-stage parity: the CUDA path's intermediates (read back through
dp_debug_copy) against the FP64 oracle's, element by element, on a ragged
lattice box.  A break in the end-to-end parity is then located at the first
stage that differs:

  env  - normalised environment matrix R (Sec. II-B, DP-SE);
  G0   - embedding net output with the type-pair factor (Sec. II-B, DPA-1);
  G<l> - output of gated attention layer l (Sec. II-B, DPA-1);
  D    - descriptor G^T R R^T G_< (flattened) and the centre type embedding;
  e    - atomic energies (Eq. eq_totE_singleAtomE).

The neighbour slots of a centre are in the same order on both sides (sorted
by distance, then index; the list is bit-exact), so rows compare directly.
Bounds are relative to the largest magnitude of each stage."""

import numpy as np
import pytest

import synth
import oracle
from oracle import energy_force_virial

from gpu_helpers import weight_file

pytestmark = pytest.mark.gpu

# largest |GPU - FP64| over a stage / largest |FP64| of that stage; "e" in eV.
# FP32 atomic energies: the output layer sums 240 products |w_k h_k| ~ 0.1
# each in FP32 and is scaled by out_scale ~17, an FP32 noise floor of
# ~6e-8 * 24 * 17 ~ 3e-5 eV.
BOUNDS = {
    "fp32": {"env": 1e-6, "G0": 1e-5, "G": 2e-5, "D": 1e-5, "e": 5e-5},
    "fp16x": {"env": 1e-6, "G0": 1e-5, "G": 5e-3, "D": 1e-3, "e": 1e-3},
    # BF16 two-term splits: ~2^-16 per product
    "bf16x": {"env": 1e-6, "G0": 1e-5, "G": 5e-4, "D": 2e-4, "e": 1e-3},
}


CASES = [(p, w) for w in ("default", "rich") for p in ("fp32", "fp16x", "bf16x")]
# the paper's model size (attention width 256, embedding net [32, 64, 128]):
# the fused 16-bit layer kernels do not take it
CASES += [("fp32", "paper_size"), ("bf16x", "paper_size")]


@pytest.mark.parametrize("precision,which", CASES)
def test_stages_match_oracle(request, precision, which):
    import paper_2604_07276_gb300 as p

    cfg, w, om = request.getfixturevalue(f"{which}_model")
    coord, atype, box = synth.lattice_system(300, seed=33)
    n = len(coord)
    m = p.DPA1(weight_file(cfg, w, which), precision=precision)
    E, F, W, e = m.compute(coord, box, atype, atom_energy=True)
    st = {}
    energy_force_virial(om, coord, box, atype, chunk=n, stages=st)
    ref_nl, ref_nn, _ = oracle.neighbor_list(coord, box, cfg.rcut, cfg.sel)
    nl = m.debug("nlist", (n, 128), np.int32)
    assert np.array_equal(nl[:, :cfg.sel], ref_nl)
    mask = ref_nl >= 0
    b = BOUNDS[precision]

    def rel(got, ref):
        return float(np.abs(got - ref).max() / max(1e-30, np.abs(ref).max()))

    report = {}
    R = m.debug("env", (n, 128, 4))[:, :cfg.sel]
    report["env"] = rel(R[mask], st["R"].numpy()[mask])
    for l in range(cfg.attn_layers + 1):
        G = m.debug(f"G{l}", (n, 128, cfg.m1))[:, :cfg.sel]
        report[f"G{l}"] = rel(G[mask], st[f"G{l}"].numpy()[mask])
    X = m.debug("D", (n, cfg.fit_in))
    report["D"] = rel(X[:, :cfg.desc_dim], st["D"].numpy())
    report["tebd"] = rel(X[:, cfg.desc_dim:], st["tebd"].numpy()[atype])
    ed = m.debug("e", (n,))
    report["e"] = float(np.abs(ed - st["e"].numpy()).max())
    m.close()
    print(f"\n{which} {precision}: " + ", ".join(f"{k} {v:.2e}" for k, v in report.items()))
    assert report["env"] <= b["env"]
    assert report["G0"] <= b["G0"]
    for l in range(1, cfg.attn_layers + 1):
        assert report[f"G{l}"] <= b["G"], (l, report[f"G{l}"])
    assert report["D"] <= b["D"]
    assert report["tebd"] <= 1e-6
    assert report["e"] <= b["e"]
