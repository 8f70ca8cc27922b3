"""Seeded synthetic systems standing in for the paper's cycloalkane test set.

The paper (Sec. 4, Table 4, Fig. 2) runs cycloalkanes with aug-cc-pVDZ and
a GEN-A2* auxiliary set on Psi4-optimised geometries.  None of those
geometries or basis sets are available, so every workload here is a
synthetic stand-in with the same shape:

* geometry: a planar ring of n_C carbons (C-C 1.54 A) with two hydrogens
  per carbon (C-H 1.09 A, H-C-H 109.5 deg, bisecting the exterior of the
  ring), plus a seeded uniform jitter of every Cartesian coordinate; or,
  for the smallest case, four atoms on a square;
* basis: normalised s-type Gaussians centred on the atoms, with
  even-tempered exponent tables per element;
* auxiliary basis: s-type Gaussians, even-tempered, per element;
* orbitals: C = S^-1/2 Q, a seeded Haar-random rotation Q of the symmetric
  (Loewdin) orthonormalisation of the basis, so that the columns are
  orthonormal functions (C^T S C = I); the overlap S is supplied by the
  caller (the oracle's integrals in the tests, the engine's own in the
  benchmark and the drivers);
* occupations: the PNOF7 electron-pairing angles gamma, drawn uniformly.

Nothing in this module evaluates an integral or any other part of the
method: it only produces numbers that both the oracle and the GPU engine
take as inputs (the one matrix function here, S^-1/2 of a given overlap,
is the input recipe's orthonormalisation, not a step of the method).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ANGSTROM_TO_BOHR = 1.0 / 0.529177210903

# Nuclear charges of the elements used by the rings ("Gh": a ghost centre, which
# carries auxiliary functions only).
_Z = {"C": 6.0, "H": 1.0, "X": 2.0, "Gh": 0.0}


def even_tempered(alpha0: float, ratio: float, n: int) -> np.ndarray:
    """alpha_k = alpha0 * ratio**k for k = 0..n-1."""
    return alpha0 * ratio ** np.arange(n, dtype=np.float64)


@dataclass
class System:
    """Atoms plus s-type basis and auxiliary basis (all lengths in bohr)."""

    name: str
    atom_xyz: np.ndarray          # [n_atoms, 3]
    atom_charge: np.ndarray       # [n_atoms]
    bf_atom: np.ndarray           # [nbf] int32, centre of each basis function
    bf_alpha: np.ndarray          # [nbf]
    aux_atom: np.ndarray          # [naux] int32
    aux_alpha: np.ndarray         # [naux]
    n_strong: int                 # N_I (doubly-occupied-like orbitals)
    n_weak_per: int               # N_g (weak orbitals per strong orbital)

    @property
    def nbf(self) -> int:
        return int(self.bf_alpha.shape[0])

    @property
    def naux(self) -> int:
        return int(self.aux_alpha.shape[0])

    @property
    def n_atoms(self) -> int:
        return int(self.atom_xyz.shape[0])

    @property
    def n_omega(self) -> int:
        """N_Omega = N_I (1 + N_g): orbitals of the pairing space."""
        return self.n_strong * (1 + self.n_weak_per)

    @property
    def n_electrons(self) -> int:
        return int(round(float(self.atom_charge.sum())))


def _square_geometry(side_angstrom: float) -> tuple[np.ndarray, list[str]]:
    s = side_angstrom * ANGSTROM_TO_BOHR
    xyz = np.array([[0.0, 0.0, 0.0], [s, 0.0, 0.0], [s, s, 0.0], [0.0, s, 0.0]])
    return xyz, ["X"] * 4


def _ring_geometry(n_c: int, jitter_angstrom: float, rng: np.random.Generator,
                   cc: float = 1.54, ch: float = 1.09,
                   hch_deg: float = 109.5) -> tuple[np.ndarray, list[str]]:
    """Planar CnH2n ring; returns coordinates in bohr and element labels."""
    radius = cc / (2.0 * np.sin(np.pi / n_c))
    half = np.deg2rad(hch_deg) / 2.0
    xyz, elem = [], []
    for k in range(n_c):
        phi = 2.0 * np.pi * k / n_c
        radial = np.array([np.cos(phi), np.sin(phi), 0.0])
        c = radius * radial
        xyz.append(c)
        elem.append("C")
        for sgn in (+1.0, -1.0):
            d = np.cos(half) * radial + sgn * np.sin(half) * np.array([0.0, 0.0, 1.0])
            xyz.append(c + ch * d)
            elem.append("H")
    xyz = np.asarray(xyz)
    xyz = xyz + rng.uniform(-jitter_angstrom, jitter_angstrom, size=xyz.shape)
    return xyz * ANGSTROM_TO_BOHR, elem


@dataclass
class BasisTable:
    """Even-tempered s-type exponent tables per element: (alpha0, ratio, n)."""

    basis: dict
    aux: dict


# Basis and auxiliary exponent tables.  The per-element counts reproduce the
# workloads' (nbf, naux): C6H12 -> (144, 504), C10H20 -> (240, 840),
# C16H32 -> (480, 1680), C20H40 -> (720, 2520).  With Coulomb-normalised
# auxiliary functions, ratios of 2.0 (C) and 2.2 (H) from 0.3 keep the
# metric's condition number near 1e7 for every ring (ratios near 1.75 push
# it past 1e8); the smallest exponent keeps diffuse fitting functions on
# neighbouring atoms from becoming nearly linearly dependent.
_TABLES = {
    "square": BasisTable(basis={"X": (0.1, 3.0, 6)}, aux={"X": (0.05, 2.0, 20)}),
    "ring_small": BasisTable(basis={"C": (0.12, 2.5, 12), "H": (0.12, 3.0, 6)},
                             aux={"C": (0.3, 2.0, 42), "H": (0.3, 2.2, 21)}),
    "ring_c16": BasisTable(basis={"C": (0.12, 2.2, 14), "H": (0.12, 2.2, 8)},
                           aux={"C": (0.3, 2.0, 49), "H": (0.3, 2.2, 28)}),
    "ring_c20": BasisTable(basis={"C": (0.12, 2.0, 16), "H": (0.12, 1.9, 10)},
                           aux={"C": (0.3, 2.0, 56), "H": (0.3, 2.2, 35)}),
    # The small rings' basis with an auxiliary set that fits the basis products: an
    # s-type function on an atom cannot represent the product of two functions on
    # different atoms (a Gaussian centred between them), so besides the atoms'
    # own functions (0.2 upward, ratio 2, covering the products of the basis's
    # exponents) ghost centres at 1/4, 1/2 and 3/4 of the way between every two
    # atoms closer than 5 bohr carry five functions each (0.4 upward, ratio 2).
    "ring_fit": BasisTable(basis={"C": (0.12, 2.5, 12), "H": (0.12, 3.0, 6), "Gh": (1.0, 1.0, 0)},
                           aux={"C": (0.2, 2.0, 16), "H": (0.2, 2.0, 12), "Gh": (0.4, 2.0, 5)}),
}

# Ghost centres of the "ring_fit" auxiliary set.
_GHOST_CUTOFF_BOHR = 5.0
_GHOST_FRACTIONS = (0.25, 0.5, 0.75)


def _ghost_centres(xyz: np.ndarray, cutoff: float = _GHOST_CUTOFF_BOHR,
                   fractions=_GHOST_FRACTIONS) -> np.ndarray:
    """Points (1 - f) A + f B for every pair of atoms A, B closer than `cutoff`
    (bohr) and every f in `fractions`."""
    out = []
    for i in range(len(xyz)):
        for j in range(i + 1, len(xyz)):
            if np.linalg.norm(xyz[i] - xyz[j]) < cutoff:
                out.extend((1.0 - f) * xyz[i] + f * xyz[j] for f in fractions)
    return np.asarray(out, dtype=np.float64).reshape(-1, 3)


def _assemble(name: str, xyz: np.ndarray, elem: list[str], table: BasisTable,
              n_strong: int, n_weak_per: int) -> System:
    bf_atom, bf_alpha, aux_atom, aux_alpha = [], [], [], []
    for a, e in enumerate(elem):
        a0, r, n = table.basis[e]
        al = even_tempered(a0, r, n)
        bf_alpha.extend(al)
        bf_atom.extend([a] * n)
        a0, r, n = table.aux[e]
        al = even_tempered(a0, r, n)
        aux_alpha.extend(al)
        aux_atom.extend([a] * n)
    return System(
        name=name,
        atom_xyz=np.ascontiguousarray(xyz, dtype=np.float64),
        atom_charge=np.array([_Z[e] for e in elem], dtype=np.float64),
        bf_atom=np.asarray(bf_atom, dtype=np.int32),
        bf_alpha=np.asarray(bf_alpha, dtype=np.float64),
        aux_atom=np.asarray(aux_atom, dtype=np.int32),
        aux_alpha=np.asarray(aux_alpha, dtype=np.float64),
        n_strong=n_strong,
        n_weak_per=n_weak_per,
    )


def make_system(kind: str, n_c: int = 0, seed: int = 0, jitter: float = 0.02,
                n_weak_per: int = 4) -> System:
    """Build a synthetic system.

    kind = "square": four atoms (charge 2) on a 1.5 A square, 6 basis and 20
    auxiliary functions per atom, N_I = 4, N_g = 2.
    kind = "ring": CnH2n ring with n_c carbons, seeded jitter (A), N_I equal to
    half the electron count, N_g weak orbitals per strong one.
    kind = "ring_fit": the same ring (n_c <= 12) with the small rings' basis and
    an auxiliary set that includes ghost centres between the atoms (the
    "ring_fit" table), for studies that need a small fitting error.
    """
    if kind == "square":
        xyz, elem = _square_geometry(1.5)
        return _assemble("square4", xyz, elem, _TABLES["square"], 4, 2)
    if kind not in ("ring", "ring_fit"):
        raise ValueError(f"unknown system kind {kind!r}")
    rng = np.random.default_rng(seed)
    xyz, elem = _ring_geometry(n_c, jitter, rng)
    n_elec = 6 * n_c + 2 * n_c
    if kind == "ring_fit":
        if n_c > 12:
            raise ValueError("the fitted-auxiliary rings use the small rings' basis (n_c <= 12)")
        ghosts = _ghost_centres(xyz)
        xyz = np.concatenate([xyz, ghosts])
        elem = elem + ["Gh"] * len(ghosts)
        return _assemble(f"c{n_c}h{2 * n_c}fit", xyz, elem, _TABLES["ring_fit"], n_elec // 2, n_weak_per)
    if n_c <= 12:
        table = _TABLES["ring_small"]
    elif n_c <= 16:
        table = _TABLES["ring_c16"]
    else:
        table = _TABLES["ring_c20"]
    return _assemble(f"c{n_c}h{2 * n_c}", xyz, elem, table, n_elec // 2, n_weak_per)


def pairing_columns(n_strong: int, n_weak_per: int) -> tuple[np.ndarray, np.ndarray]:
    """Electron-pairing map of the N_Omega orbital columns.

    Column g (g < N_I) is the strong orbital of subspace g.  The i-th weak
    orbital (i = 0..N_g-1) of subspace g sits at column
    N_I + i*N_I + (N_I-1-g), so the highest strong orbital pairs with the
    lowest weak ones.  Returns (subspace[N_Omega], weak_rank[N_Omega]) with
    weak_rank = -1 for strong orbitals and i for the i-th weak orbital.
    """
    n_om = n_strong * (1 + n_weak_per)
    sub = np.empty(n_om, dtype=np.int32)
    rank = np.empty(n_om, dtype=np.int32)
    for g in range(n_strong):
        sub[g] = g
        rank[g] = -1
        for i in range(n_weak_per):
            col = n_strong + i * n_strong + (n_strong - 1 - g)
            sub[col] = g
            rank[col] = i
    return sub, rank


def random_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random orthogonal n x n matrix (QR of a Gaussian matrix, diag(R)>0)."""
    a = rng.standard_normal((n, n))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    return np.ascontiguousarray(q)


def draw_gamma(n_strong: int, n_weak_per: int, rng: np.random.Generator,
               lo: float = 0.05, hi: float = 0.3) -> np.ndarray:
    """Occupation angles: N_I strong angles followed by N_I*(N_g-1) weak ones."""
    return rng.uniform(lo, hi, size=n_strong * n_weak_per)


@dataclass
class Workload:
    """A system plus the orbital matrix and occupation angles evaluated on it."""

    name: str
    system: System
    C: np.ndarray            # [nbf, nbf], column p is orbital p; C^T S C = I
    gamma: np.ndarray        # [N_I * N_g]
    Q: np.ndarray = None     # the seeded rotation, C = S^-1/2 Q
    meta: dict = field(default_factory=dict)


# Named workloads (sizes as stated beside each).
WORKLOADS = {
    # 4 atoms, nbf=24, naux=80, N_Omega=12
    "square4": dict(kind="square", seed=1),
    # C6H12 ring, nbf=144, naux=504, N_Omega=120
    "c6h12": dict(kind="ring", n_c=6, seed=2),
    # C10H20 ring, nbf=240, naux=840, N_Omega=200
    "c10h20": dict(kind="ring", n_c=10, seed=3),
    # C16H32 ring, nbf=480, naux=1680, N_Omega=320
    "c16h32": dict(kind="ring", n_c=16, seed=4),
    # C20H40 ring, nbf=720, naux=2520, N_Omega=400
    "c20h40": dict(kind="ring", n_c=20, seed=5),
    # the C6H12 ring above with 180 ghost centres in its auxiliary set,
    # nbf=144, naux=1140, N_Omega=120
    "c6h12fit": dict(kind="ring_fit", n_c=6, seed=2),
}


def orthonormal_orbitals(S: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """C = S^-1/2 Q for a symmetric positive definite overlap S and an orthogonal
    Q: the symmetric (Loewdin) orthonormalisation of the basis followed by the
    rotation Q, so that C^T S C = Q^T Q = I.  S^-1/2 from the eigenvectors of S."""
    S = np.asarray(S, dtype=np.float64)
    ev, U = np.linalg.eigh(0.5 * (S + S.T))
    if not ev.min() > 0.0:
        raise ValueError("the overlap matrix is not positive definite")
    return np.ascontiguousarray((U * ev ** -0.5) @ (U.T @ Q))


def _overlap_of(overlap, system: System) -> np.ndarray:
    S = overlap(system) if callable(overlap) else overlap
    S = np.asarray(S, dtype=np.float64)
    if S.shape != (system.nbf, system.nbf):
        raise ValueError(f"overlap has shape {S.shape}, expected {(system.nbf, system.nbf)}")
    return S


def workload_system(name: str, seed: int | None = None) -> System:
    """The system of a named workload alone (the same object make_workload builds)."""
    spec = dict(WORKLOADS[name])
    kind = spec.pop("kind")
    stored = spec.pop("seed")
    return make_system(kind, seed=stored if seed is None else seed, **spec)


def make_workload(name: str, overlap, seed: int | None = None) -> Workload:
    """Build a named workload; `seed` overrides the stored seed.

    `overlap` is the basis overlap matrix S of the workload's system, or a
    callable system -> S.  The orbitals are C = S^-1/2 Q with Q Haar-random."""
    s = WORKLOADS[name]["seed"] if seed is None else seed
    system = workload_system(name, seed)
    rng = np.random.default_rng(10_000 + s)
    Q = random_orthogonal(system.nbf, rng)
    gamma = draw_gamma(system.n_strong, system.n_weak_per, rng)
    C = orthonormal_orbitals(_overlap_of(overlap, system), Q)
    return Workload(name=name, system=system, C=C, gamma=gamma, Q=Q, meta={"seed": s})


def ring_workload(n_c: int, seed: int, overlap, jitter: float = 0.05) -> Workload:
    """A CnH2n ring with its own seeded geometry and orbitals S^-1/2 Q (the
    learned-guess training and evaluation sets: rings C6-C12, jitter 0.05 A)."""
    system = make_system("ring", n_c=n_c, seed=seed, jitter=jitter)
    rng = np.random.default_rng(10_000 + seed)
    Q = random_orthogonal(system.nbf, rng)
    gamma = draw_gamma(system.n_strong, system.n_weak_per, rng)
    C = orthonormal_orbitals(_overlap_of(overlap, system), Q)
    return Workload(name=f"c{n_c}h{2 * n_c}-s{seed}", system=system, C=C, gamma=gamma, Q=Q, meta={"seed": seed})


def standard_gamma(n_strong: int, n_weak_per: int, n_strong_occ: float = 0.98) -> np.ndarray:
    """The standard starting angles of the occupation optimisation (the paper's
    calculations start from a Fermi-Dirac-like distribution of occupations; read
    here as every strong orbital at n_strong_occ and the weak share of each
    subspace split equally): cos^2 gamma_g = 2 n - 1, cos^2 w_i = 1 / (N_g - i)."""
    g0 = np.arccos(np.sqrt(2.0 * n_strong_occ - 1.0))
    w = [np.arccos(np.sqrt(1.0 / (n_weak_per - i))) for i in range(n_weak_per - 1)]
    return np.concatenate([np.full(n_strong, g0), np.tile(np.array(w, dtype=np.float64), n_strong)])



def with_near_duplicate_aux(system: System, count: int, rel: float) -> System:
    """A copy of `system` whose first `count` auxiliary functions each get a twin
    on the same centre with exponent alpha (1 + rel): an auxiliary set that is
    linearly dependent to about rel, so that its Coulomb metric is numerically
    singular (the ill-conditioned case the modified factorisation is for)."""
    import dataclasses
    idx = np.arange(count)
    return dataclasses.replace(
        system, name=f"{system.name}+dup{count}",
        aux_atom=np.concatenate([system.aux_atom, system.aux_atom[idx]]).astype(np.int32),
        aux_alpha=np.concatenate([system.aux_alpha, system.aux_alpha[idx] * (1.0 + rel)]))


def without_basis_functions(system: System, count: int, naux_drop: int = 0) -> System:
    """A copy of `system` without its last `count` basis functions (and its last
    `naux_drop` auxiliary functions): odd and otherwise ragged sizes for the
    kernels' edge paths.  N_Omega must still fit: N_I (1 + N_g) <= nbf."""
    import dataclasses
    nb = system.nbf - count
    nx = system.naux - naux_drop
    out = dataclasses.replace(system, name=f"{system.name}-{count}bf-{naux_drop}aux",
                              bf_atom=system.bf_atom[:nb].copy(), bf_alpha=system.bf_alpha[:nb].copy(),
                              aux_atom=system.aux_atom[:nx].copy(), aux_alpha=system.aux_alpha[:nx].copy())
    if out.n_omega > out.nbf:
        raise ValueError("N_Omega exceeds nbf")
    return out
