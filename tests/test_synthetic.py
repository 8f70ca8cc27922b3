"""The seeded synthetic workloads have the stated shapes and are reproducible."""
import numpy as np
import pytest

from oracle import integrals
from synthetic import orthonormal_orbitals, pairing_columns
from tests.workloads import make_workload

SHAPES = {
    "square4": (24, 80, 4, 2, 12),
    "c6h12": (144, 504, 24, 4, 120),
    "c10h20": (240, 840, 40, 4, 200),
    "c16h32": (480, 1680, 64, 4, 320),
    "c20h40": (720, 2520, 80, 4, 400),
}


@pytest.mark.parametrize("name", list(SHAPES))
def test_shapes(name):
    w = make_workload(name)
    s = w.system
    nbf, naux, ni, ng, nom = SHAPES[name]
    assert (s.nbf, s.naux, s.n_strong, s.n_weak_per, s.n_omega) == (nbf, naux, ni, ng, nom)
    assert s.n_electrons == 2 * s.n_strong
    assert w.C.shape == (nbf, nbf)
    # orthonormal functions: C^T S C = I in the overlap metric (not C^T C = I)
    S = integrals.overlap(s)
    np.testing.assert_allclose(w.C.T @ S @ w.C, np.eye(nbf), atol=1e-11)
    np.testing.assert_allclose(w.Q.T @ w.Q, np.eye(nbf), atol=1e-12)
    assert w.gamma.shape == (ni * ng,)
    assert ((w.gamma >= 0.05) & (w.gamma <= 0.3)).all()


def test_reproducible_and_seeded():
    a = make_workload("c6h12")
    b = make_workload("c6h12")
    np.testing.assert_array_equal(a.system.atom_xyz, b.system.atom_xyz)
    np.testing.assert_array_equal(a.C, b.C)
    c = make_workload("c6h12", seed=99)
    assert not np.array_equal(a.system.atom_xyz, c.system.atom_xyz)


def test_ring_geometry():
    from synthetic.systems import ANGSTROM_TO_BOHR
    w = make_workload("c6h12")
    xyz = w.system.atom_xyz / ANGSTROM_TO_BOHR
    z = w.system.atom_charge
    carbons = xyz[z == 6.0]
    d = np.linalg.norm(carbons - np.roll(carbons, -1, axis=0), axis=1)
    assert np.all(np.abs(d - 1.54) < 0.08)
    sub, rank = pairing_columns(24, 4)
    assert sub.max() == 23


def test_without_basis_functions_trims_the_tail():
    from synthetic import make_system, without_basis_functions
    s = make_system("ring", n_c=5, seed=77, jitter=0.02, n_weak_per=3)
    t = without_basis_functions(s, 3, 5)
    assert (t.nbf, t.naux) == (s.nbf - 3, s.naux - 5)
    assert (t.bf_alpha == s.bf_alpha[:-3]).all() and (t.aux_atom == s.aux_atom[:-5]).all()
    assert t.n_omega == s.n_omega and t.atom_xyz is s.atom_xyz
    with pytest.raises(ValueError):
        without_basis_functions(s, s.nbf - s.n_omega + 1)


def test_orthonormal_orbitals_is_the_inverse_square_root():
    """S^-1/2 Q: (S^-1/2)^2 S = I and S^-1/2 symmetric, on a random SPD matrix."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((9, 9))
    S = A @ A.T + 0.5 * np.eye(9)
    X = orthonormal_orbitals(S, np.eye(9))
    np.testing.assert_allclose(X, X.T, atol=1e-13)
    np.testing.assert_allclose(X @ X @ S, np.eye(9), atol=1e-12)
    with pytest.raises(ValueError):
        orthonormal_orbitals(-S, np.eye(9))


def test_ring_fit_ghost_centres():
    """c6h12fit: the c6h12 ring plus ghost centres (no charge, no basis function,
    five auxiliary functions each) at 1/4, 1/2, 3/4 between atoms closer than 5 bohr,
    all distinct from each other and from the atoms."""
    from synthetic.systems import make_system, workload_system
    s = workload_system("c6h12fit")
    r = workload_system("c6h12")
    na = r.n_atoms
    assert (s.nbf, s.naux, s.n_omega) == (144, 1140, 120)
    np.testing.assert_array_equal(s.atom_xyz[:na], r.atom_xyz)
    assert (s.atom_charge[na:] == 0.0).all() and s.n_electrons == r.n_electrons
    assert s.bf_atom.max() < na
    ghosts = np.arange(na, s.n_atoms)
    assert (np.bincount(s.aux_atom, minlength=s.n_atoms)[ghosts] == 5).all()
    d = np.linalg.norm(s.atom_xyz[:, None] - s.atom_xyz[None], axis=-1) + 1e9 * np.eye(s.n_atoms)
    assert d.min() > 0.4
    with pytest.raises(ValueError):
        make_system("ring_fit", n_c=16)
