"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package holds no arithmetic of the DPA-1 method.  It only draws
random numbers (model weights, atom positions, types, velocities) from
fixed seeds and serialises weights to the binary file format that
``dp_init`` reads.  Both the oracle (``oracle/``) and the GPU tests /
benchmark import it; it imports neither of them.
"""

from .model import (ModelConfig, make_weights, write_weights, STUDENT_CONFIG, DEFAULT_CONFIG, PAPER_SIZE_CONFIG,
                    TEACHER_BASE_OUT_SCALE, teacher_base_weights, teacher_weights, perturbed)
from .systems import (
    water_box,
    lattice_system,
    frame_batch,
    maxwell_boltzmann,
    isolated_cluster,
    slab_subdomains,
    MASSES,
    TYPE_MAP,
)

__all__ = [
    "ModelConfig",
    "make_weights",
    "write_weights",
    "DEFAULT_CONFIG",
    "STUDENT_CONFIG",
    "PAPER_SIZE_CONFIG",
    "TEACHER_BASE_OUT_SCALE",
    "teacher_base_weights",
    "teacher_weights",
    "perturbed",
    "water_box",
    "lattice_system",
    "frame_batch",
    "maxwell_boltzmann",
    "isolated_cluster",
    "slab_subdomains",
    "MASSES",
    "TYPE_MAP",
]
