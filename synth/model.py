"""DPA-1 model hyper-parameters, seeded random weights, and the weight file.

The hyper-parameters of the default model are the ones the build is
measured on: 5 types (H, C, N, O, S), type embedding of width 8, rcut
6.0 A, rcut_smth 0.5 A, sel 120, embedding net [25, 50, 100] with tanh,
axis 16, two gated attention layers of width 128 and a fitting net
[240, 240, 240].  The paper's DPA-1 (Sec. IV-B) uses a larger network
of the same family; the paper gives no weights, so every weight here is
drawn Xavier-uniform from a seed (biases zero unless asked otherwise).

Weight file layout (little endian), read by ``dp_init``:

    char    magic[8]      = b"DPA1WTS1"
    int32   ints[16]      = version(1), ntypes, tebd_dim, sel, axis,
                            n_embed, embed[0..2], n_attn, attn_dim,
                            n_fit, fit[0..2], type-embedding mode
                            (0: strip, 1: concat)
    float64 dbls[8]       = rcut, rcut_smth, attn_shift, ln_eps,
                            out_scale, 0, 0, 0
    char    type_map[ntypes][8]
    float64 arrays in the order of ``tensor_order(cfg)``; each array is
            row-major with the shape given there ([in, out] for dense
            layers, so that y = x @ W + b).
"""

from __future__ import annotations

import dataclasses
import struct
from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np

MAGIC = b"DPA1WTS1"


@dataclass(frozen=True)
class ModelConfig:
    ntypes: int = 5
    type_map: Tuple[str, ...] = ("H", "C", "N", "O", "S")
    tebd_dim: int = 8
    rcut: float = 6.0
    rcut_smth: float = 0.5
    sel: int = 120
    embed: Tuple[int, ...] = (25, 50, 100)
    axis: int = 16
    attn_layers: int = 2
    attn_dim: int = 128
    fitting: Tuple[int, ...] = (240, 240, 240)
    attn_shift: float = 20.0
    ln_eps: float = 1e-5
    # Output scale of the fitting net (1.0 unless a calibrated value is given).
    out_scale: float = 1.0
    # How the type embedding enters the embedding net: "strip" (the paper's
    # model: G0 = net_s(s) * (1 + net_t([T_j, T_i]))) or "concat" (the
    # embedding net's input is [s, T_j, T_i]).
    tebd_input_mode: str = "strip"

    @property
    def m1(self) -> int:
        return self.embed[-1]

    @property
    def desc_dim(self) -> int:
        return self.m1 * self.axis

    @property
    def fit_in(self) -> int:
        return self.desc_dim + self.tebd_dim


# The output scale of the default model was written by
# oracle/calibrate_out_scale.py: with it, the FP64 oracle's force RMS on the
# 192-atom water box (seed 0) with seed-0 weights is 1.0 eV/A, which gives
# the absolute force tolerances (eV/A) a meaning for random weights.
DEFAULT_CONFIG = ModelConfig(out_scale=16.873387265124986)
STUDENT_CONFIG = ModelConfig(embed=(16, 32, 64), axis=8, attn_layers=0, fitting=(128, 128), out_scale=1.0)
# The paper's own model size (Sec. IV-B: embedding net [32, 64, 128], three
# gated attention layers of width 256, fitting net [256, 256, 256]); its output
# scale is calibrated the same way (seed-0 weights).
PAPER_SIZE_CONFIG = ModelConfig(embed=(32, 64, 128), attn_layers=3, attn_dim=256, fitting=(256, 256, 256),
                                out_scale=8.82029019500646)


def tensor_order(cfg: ModelConfig) -> List[Tuple[str, Tuple[int, ...]]]:
    """Names and shapes of every weight array, in file order."""
    out: List[Tuple[str, Tuple[int, ...]]] = []
    nt, td = cfg.ntypes, cfg.tebd_dim
    out += [("te_W", (nt, td)), ("te_b", (td,))]
    concat = cfg.tebd_input_mode == "concat"
    if not concat:
        fan = 2 * td
        for l, w in enumerate(cfg.embed):
            out += [(f"tt_W{l}", (fan, w)), (f"tt_b{l}", (w,))]
            fan = w
    fan = 1 + 2 * td if concat else 1
    for l, w in enumerate(cfg.embed):
        out += [(f"em_W{l}", (fan, w)), (f"em_b{l}", (w,))]
        fan = w
    out += [("davg", (nt, 4)), ("dstd", (nt, 4))]
    m1, a = cfg.m1, cfg.attn_dim
    for l in range(cfg.attn_layers):
        out += [
            (f"at{l}_Wq", (m1, a)), (f"at{l}_bq", (a,)),
            (f"at{l}_Wk", (m1, a)), (f"at{l}_bk", (a,)),
            (f"at{l}_Wv", (m1, a)), (f"at{l}_bv", (a,)),
            (f"at{l}_Wo", (a, m1)), (f"at{l}_bo", (m1,)),
            (f"at{l}_ln_g", (m1,)), (f"at{l}_ln_b", (m1,)),
        ]
    fan = cfg.fit_in
    for l, w in enumerate(cfg.fitting):
        out += [(f"fit_W{l}", (fan, w)), (f"fit_b{l}", (w,))]
        fan = w
    out += [(f"fit_W{len(cfg.fitting)}", (fan, 1)), (f"fit_b{len(cfg.fitting)}", (1,))]
    out += [("ebias", (nt,))]
    return out


def _xavier(rng: np.random.Generator, fan_in: int, fan_out: int) -> np.ndarray:
    a = np.sqrt(6.0 / (fan_in + fan_out))
    return rng.uniform(-a, a, size=(fan_in, fan_out))


def make_weights(
    cfg: ModelConfig = DEFAULT_CONFIG,
    seed: int = 0,
    bias_scale: float = 0.0,
    ln_scale: float = 0.0,
    stats: bool = False,
) -> Dict[str, np.ndarray]:
    """Seeded Xavier-uniform weights (float64).

    ``bias_scale`` > 0 draws biases N(0, bias_scale) instead of zeros,
    ``ln_scale`` > 0 perturbs the LayerNorm gain/shift away from (1, 0),
    and ``stats`` draws non-trivial davg/dstd, so that parity tests see
    every term of the network.  The default (all off) is the model the
    benchmark runs.
    """
    rng = np.random.default_rng(seed)
    w: Dict[str, np.ndarray] = {}
    for name, shape in tensor_order(cfg):
        if name in ("davg",):
            w[name] = rng.normal(0.0, 0.05, size=shape) if stats else np.zeros(shape)
        elif name in ("dstd",):
            w[name] = rng.uniform(0.7, 1.3, size=shape) if stats else np.ones(shape)
        elif name.endswith("ln_g"):
            w[name] = np.ones(shape) + (rng.normal(0.0, ln_scale, size=shape) if ln_scale > 0 else 0.0)
        elif name.endswith("ln_b"):
            w[name] = rng.normal(0.0, ln_scale, size=shape) if ln_scale > 0 else np.zeros(shape)
        elif name == "ebias":
            w[name] = rng.normal(0.0, 1.0, size=shape)
        elif len(shape) == 2:
            w[name] = _xavier(rng, shape[0], shape[1])
        else:
            w[name] = rng.normal(0.0, bias_scale, size=shape) if bias_scale > 0 else np.zeros(shape)
    w["out_scale"] = np.array(cfg.out_scale)
    return w


def write_weights(path: str, cfg: ModelConfig, weights: Dict[str, np.ndarray]) -> None:
    """Serialise ``weights`` in the layout described in the module docstring."""
    if len(cfg.embed) != 3 or len(cfg.fitting) not in (2, 3):
        raise ValueError("file format holds 3 embedding layers and 2 or 3 fitting layers")
    fit = list(cfg.fitting) + [0] * (3 - len(cfg.fitting))
    if cfg.tebd_input_mode not in ("strip", "concat"):
        raise ValueError("tebd_input_mode is strip or concat")
    ints = [1, cfg.ntypes, cfg.tebd_dim, cfg.sel, cfg.axis, len(cfg.embed), *cfg.embed,
            cfg.attn_layers, cfg.attn_dim, len(cfg.fitting), *fit, 1 if cfg.tebd_input_mode == "concat" else 0]
    assert len(ints) == 16
    out_scale = float(np.asarray(weights.get("out_scale", cfg.out_scale)))
    dbls = [cfg.rcut, cfg.rcut_smth, cfg.attn_shift, cfg.ln_eps, out_scale, 0.0, 0.0, 0.0]
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<16i", *ints))
        f.write(struct.pack("<8d", *dbls))
        for name in cfg.type_map:
            b = name.encode()[:7]
            f.write(b + b"\0" * (8 - len(b)))
        for name, shape in tensor_order(cfg):
            a = np.ascontiguousarray(weights[name], dtype="<f8")
            if a.shape != shape:
                raise ValueError(f"{name}: shape {a.shape} != {shape}")
            f.write(a.tobytes())


def with_out_scale(cfg: ModelConfig, out_scale: float) -> ModelConfig:
    return dataclasses.replace(cfg, out_scale=out_scale)


# The distillation teacher (stage a17): a DPA-1 of the student's sizes with one
# gated attention layer whose LayerNorm gain is small, so that the student
# family (no attention) can represent it to within a known floor.  Its base
# (every weight but the attention layer) is the seed-4 student model with
# biases; the output scale below was written by oracle/calibrate_out_scale.py
# (FP64 force RMS 1.0 eV/A of the base on the 192-atom water box).
TEACHER_BASE_OUT_SCALE = 536.6297988626927


def teacher_base_weights(out_scale: float = 1.0):
    """(config, weights) of the teacher's base: the student family, seed 4."""
    cfg = STUDENT_CONFIG
    w = make_weights(cfg, seed=4, bias_scale=0.1)
    w["out_scale"] = np.array(out_scale)
    return cfg, w


def teacher_weights(ln_gain: float, out_scale: float = TEACHER_BASE_OUT_SCALE):
    """(config, weights) of the distillation teacher: the base plus one
    attention layer (width 128, seed-12 weights with biases) whose LayerNorm
    gain is ``ln_gain`` and shift 0."""
    _, base = teacher_base_weights(out_scale)
    cfg = dataclasses.replace(STUDENT_CONFIG, attn_layers=1, attn_dim=128)
    att = make_weights(cfg, seed=12, bias_scale=0.1)
    w = dict(base)
    for k, v in att.items():
        if k.startswith("at0_"):
            w[k] = v
    w["at0_ln_g"] = ln_gain * np.ones_like(w["at0_ln_g"])
    w["at0_ln_b"] = np.zeros_like(w["at0_ln_b"])
    return cfg, w


def perturbed(weights: Dict[str, np.ndarray], sigma: float, seed: int) -> Dict[str, np.ndarray]:
    """A copy of the weights with every embedding and fitting matrix scaled
    elementwise by (1 + sigma N(0, 1)): the student's starting point."""
    rng = np.random.default_rng(seed)
    out = dict(weights)
    for k, v in weights.items():
        if (k.startswith("em_W") or k.startswith("fit_W")) and np.ndim(v) == 2:
            out[k] = v * (1.0 + sigma * rng.normal(size=np.shape(v)))
    return out
