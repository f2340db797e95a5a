"""FP64 CPU oracle for the DPA-1 energy / force / virial evaluation.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain definition
that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import it.  The product library
(``paper_2604_07276_gb300``) never imports, calls or links it, and it
shares no code with the CUDA path: both sides only share the seeded input
generators in ``synth/``.

Parity status per function (pins live in ``tests/test_oracle_*.py``):

* ``neighbor_list`` - pinned (scipy cKDTree periodic queries, brute-force
  re-derivation of the sel truncation).
* ``switch`` - pinned (closed-form end values, vanishing first and second
  derivatives at both ends).
* ``energy_force_virial`` - pinned by central finite differences of E in
  coordinates and in strain, translation / periodic-symmetry / rotation /
  same-type-permutation invariance, sum of forces = 0, virial symmetry and
  the non-periodic virial identity, 2x2x2 replication (extensivity),
  locality, continuity across rcut, the two-atom closed form and the
  reduction of the gated attention to ``torch.nn.functional``'s
  scaled-dot-product attention and layer norm.
* The readings of the paper's unstated details (switch form, attention
  shift, gate, residual and LayerNorm placement, descriptor
  normalisation, fitting input) are fixed by this code; whether they
  equal DeePMD-kit's se_atten_v2 numerically is parity unpinned (no
  implementation, weights or printed values exist to compare with).
"""

from .dpa1 import (
    neighbor_list,
    reverse_centres,
    switch,
    env_matrix,
    type_embedding,
    type_pair_table,
    embedding_net,
    gated_attention,
    descriptor,
    fitting,
    atomic_energies,
    energy_force_virial,
    forces_on,
    OracleModel,
)

__all__ = [
    "neighbor_list",
    "reverse_centres",
    "switch",
    "env_matrix",
    "type_embedding",
    "type_pair_table",
    "embedding_net",
    "gated_attention",
    "descriptor",
    "fitting",
    "atomic_energies",
    "energy_force_virial",
    "forces_on",
    "OracleModel",
]
