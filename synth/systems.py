"""Seeded synthetic atomic systems (positions, types, periodic box).

They stand in for the paper's solvated proteins (Sec. V-B: 1YRF with
582 DP atoms, 1HCI with 15,668 DP atoms), whose structure files are not
available.  Type ids index ``TYPE_MAP``.

* ``water_box``: 64 rigid water-like triples (O-H 0.96 A, H-O-H 104.5
  deg) at random positions and orientations in a 12.4 A periodic cube,
  rejection-sampled so that atoms of different molecules are >= 0.9 A
  apart (192 atoms, density 0.1007 A^-3).
* ``lattice_system``: a jittered simple-cubic lattice at 0.1 atoms/A^3
  with the elemental fractions of a solvated protein (H .63, C .12,
  N .03, O .21, S .01).  Sites are chosen without replacement from the
  smallest n^3 >= N lattice; each atom is jittered uniformly by up to
  0.25 lattice spacings per axis, so no two atoms come closer than half
  a spacing (about 1.0 A at this density).
* ``frame_batch``: frames of uneven size (uniform 200..3000 atoms) built
  with the lattice recipe.
* ``isolated_cluster``: a few atoms in a box far larger than 2*rcut, for
  tests that need a non-periodic system.
"""

from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

TYPE_MAP = ("H", "C", "N", "O", "S")
# amu, indexed by type id
MASSES = np.array([1.008, 12.011, 14.007, 15.999, 32.06])
PROTEIN_FRACTIONS = (0.63, 0.12, 0.03, 0.21, 0.01)
KB_EV = 8.617333262e-5  # Boltzmann constant, eV/K


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def water_box(seed: int = 0, nmol: int = 64, box: float = 12.4, r_oh: float = 0.96,
              angle_deg: float = 104.5, min_sep: float = 0.9) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Return (coord [3*nmol, 3] A, atype [3*nmol] int32, box [3] A)."""
    rng = np.random.default_rng(seed)
    half = np.deg2rad(angle_deg) / 2.0
    local = np.array([
        [0.0, 0.0, 0.0],
        [r_oh * np.sin(half), r_oh * np.cos(half), 0.0],
        [-r_oh * np.sin(half), r_oh * np.cos(half), 0.0],
    ])
    L = np.array([box, box, box])
    mols: List[np.ndarray] = []
    tries = 0
    while len(mols) < nmol:
        tries += 1
        if tries > 200000:
            raise RuntimeError("water_box: could not place molecules")
        cand = rng.uniform(0.0, box, size=3) + local @ _random_rotation(rng).T
        ok = True
        for m in mols:
            d = cand[:, None, :] - m[None, :, :]
            d -= L * np.rint(d / L)
            if np.min(np.sum(d * d, axis=-1)) < min_sep * min_sep:
                ok = False
                break
        if ok:
            mols.append(cand)
    coord = np.concatenate(mols, axis=0)
    coord -= L * np.floor(coord / L)
    atype = np.tile(np.array([3, 0, 0], dtype=np.int32), nmol)
    return coord, atype, L


def _type_counts(natoms: int, fractions: Sequence[float]) -> np.ndarray:
    counts = np.floor(np.asarray(fractions) * natoms + 0.5).astype(np.int64)
    counts[0] += natoms - counts.sum()
    return counts


def lattice_system(natoms: int, seed: int, density: float = 0.1,
                   fractions: Sequence[float] = PROTEIN_FRACTIONS,
                   jitter: float = 0.25) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Return (coord [N,3] A, atype [N] int32, box [3] A) for a jittered lattice."""
    rng = np.random.default_rng(seed)
    L = (natoms / density) ** (1.0 / 3.0)
    n = int(np.ceil(natoms ** (1.0 / 3.0) - 1e-9))
    while n ** 3 < natoms:
        n += 1
    a = L / n
    sites = rng.choice(n ** 3, size=natoms, replace=False)
    ijk = np.stack([sites // (n * n), (sites // n) % n, sites % n], axis=1).astype(np.float64)
    coord = (ijk + 0.5) * a + rng.uniform(-jitter, jitter, size=(natoms, 3)) * a
    coord -= L * np.floor(coord / L)
    counts = _type_counts(natoms, fractions)
    atype = np.repeat(np.arange(len(counts), dtype=np.int32), counts)
    rng.shuffle(atype)
    return coord, atype.astype(np.int32), np.array([L, L, L])


def frame_batch(seed: int = 2, nframes: int = 32, lo: int = 200, hi: int = 3000):
    """List of (coord, atype, box) frames with natoms ~ U{lo..hi}."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=nframes)
    return [lattice_system(int(n), seed=int(rng.integers(1 << 31))) for n in sizes]


def maxwell_boltzmann(atype: np.ndarray, temperature: float = 300.0, seed: int = 11) -> np.ndarray:
    """Velocities in A/fs with zero net momentum, for masses MASSES[atype]."""
    rng = np.random.default_rng(seed)
    m = MASSES[atype]
    # sqrt(kT/m) in A/fs: kT [eV] / m [amu] -> (A/fs)^2 via 1 eV/amu = 9.648533e-3 A^2/fs^2
    sigma = np.sqrt(KB_EV * temperature / m * 9.648533212e-3)
    v = rng.normal(size=(len(atype), 3)) * sigma[:, None]
    p = (m[:, None] * v).sum(axis=0)
    v -= p / m.sum()
    return v


def isolated_cluster(seed: int, natoms: int = 12, radius: float = 3.0, box: float = 40.0,
                     min_sep: float = 1.0, ntypes: int = 5):
    """A small cluster near the centre of a large periodic box (no image within rcut)."""
    rng = np.random.default_rng(seed)
    pts: List[np.ndarray] = []
    while len(pts) < natoms:
        p = rng.uniform(-radius, radius, size=3)
        if all(np.linalg.norm(p - q) >= min_sep for q in pts):
            pts.append(p)
    coord = np.array(pts) + box / 2.0
    atype = rng.integers(0, ntypes, size=natoms).astype(np.int32)
    return coord, atype, np.array([box, box, box])


def slab_subdomains(coord, atype, box, nslab: int, halo: float, pad: float = 10.0):
    """Split a periodic orthorhombic box into ``nslab`` slabs along x, each
    with the ghost atoms within ``halo`` of its faces, for local/ghost
    evaluations.  Returns a list of (coord, atype, box, nlocal, owner):
    the slab's local atoms come first, then the ghosts (periodic images in x
    written out explicitly); ``owner`` maps every row to its atom of the
    original box.  The slab boxes keep y and z periodic and stretch x so
    that no x image comes within reach."""
    coord = np.asarray(coord, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64).reshape(3)
    L = box[0]
    x = coord[:, 0] - L * np.floor(coord[:, 0] / L)
    out = []
    for s in range(nslab):
        lo, hi = s * L / nslab, (s + 1) * L / nslab
        local = np.nonzero((x >= lo) & (x < hi))[0]
        ghosts, shifts = [], []
        for t in (-1, 0, 1):
            xs = x + t * L
            sel = np.nonzero((xs >= lo - halo) & (xs < hi + halo))[0]
            for j in sel:
                if t == 0 and lo <= x[j] < hi:
                    continue
                ghosts.append(j)
                shifts.append(t)
        ghosts = np.asarray(ghosts, dtype=np.int64)
        c = np.concatenate([coord[local], coord[ghosts]])
        c[:, 0] = np.concatenate([x[local], x[ghosts] + L * np.asarray(shifts, dtype=np.float64)])
        owner = np.concatenate([local, ghosts])
        sub_box = np.array([L / nslab + 2 * halo + 2 * pad + L, box[1], box[2]])
        c[:, 0] += halo + pad - lo  # inside the stretched box, away from its x faces
        out.append((c, np.asarray(atype)[owner].astype(np.int32), sub_box, len(local), owner))
    return out
