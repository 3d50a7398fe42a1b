"""The synthetic silicon workloads: the sizes, grids and seeds every test and
the benchmark rely on, and the diamond geometry they are cut from.  (No
method arithmetic lives in the generator; these pin the input recipe.)"""
import math

import numpy as np
import pytest

import workloads as w


@pytest.mark.parametrize("name,atoms,grid,kT", [
    ("cluster64", 64, (77, 77, 77), 0.01),
    ("sphere25", 465, (147, 147, 147), 0.01),
    ("sphere40", 1963, (224, 225, 224), 0.005),
])
def test_named_systems(name, atoms, grid, kT):
    s = w.config_system(name)
    assert s.n_atoms == atoms
    assert s.n_basis == 10 * atoms                      # 4 s + 2 x 3 p per atom
    assert s.n_electrons == 4.0 * atoms
    assert tuple(int(n) for n in s.grid_n) == grid
    assert s.kT == kT and s.grid_h == 0.4
    # 6 bohr of vacuum on every side of the atoms, grid x fastest from the origin
    lo = s.xyz.min(axis=0) - 6.0
    assert np.allclose(s.grid_origin, lo)
    hi = s.grid_origin + (np.asarray(s.grid_n) - 1) * s.grid_h
    assert np.all(hi >= s.xyz.max(axis=0) + 6.0 - 1e-12)


def test_basis_per_atom():
    s = w.config_system("tiny8")
    shells = list(zip(s.shell_l[:6].tolist(), s.shell_exp[:6].tolist()))
    assert shells == [(0, 0.1), (0, 0.3), (0, 1.0), (0, 3.0), (1, 0.2), (1, 0.8)]
    assert np.all(np.bincount(s.shell_atom) == 6)


def test_diamond_geometry():
    a = w.SI_A0
    xyz = w.diamond_sphere(12.0)
    d = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=-1)
    np.fill_diagonal(d, np.inf)
    # nearest neighbours at a sqrt(3) / 4; the atom at the origin has four
    assert np.isclose(d.min(), a * math.sqrt(3) / 4)
    origin = int(np.argmin(np.linalg.norm(xyz, axis=1)))
    assert np.allclose(xyz[origin], 0.0)
    assert int(np.sum(np.isclose(d[origin], a * math.sqrt(3) / 4))) == 4
    assert np.all(np.linalg.norm(xyz, axis=1) <= 12.0 + 1e-9)
    cell = w.diamond_supercell(1)
    assert cell.shape == (8, 3)


def test_seeds_are_reproducible_and_distinct():
    a = w.config_system("cluster64", seed=0).xyz
    b = w.config_system("cluster64", seed=0).xyz
    c = w.config_system("cluster64", seed=1).xyz
    assert np.array_equal(a, b)
    assert not np.allclose(a, c)
    # the jitter is N(0, 0.05) per coordinate around the lattice sites
    dev = (a - w.diamond_supercell(2)).ravel()
    assert abs(dev.std() - 0.05) < 0.01 and abs(dev.mean()) < 0.01


@pytest.mark.parametrize("name,n,ksum,kmin,kmax", [
    ("batch64", 64, 197420, 290, 8490),
    ("batch64s", 64, 22560, 50, 870),
])
def test_batches(name, n, ksum, kmin, kmax):
    ss = w.config_batch(name)
    ks = [s.n_basis for s in ss]
    assert len(ss) == n and sum(ks) == ksum and min(ks) == kmin and max(ks) == kmax
