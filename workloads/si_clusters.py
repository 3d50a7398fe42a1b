"""Synthetic silicon clusters cut from the diamond lattice.

The paper's own geometries (H-terminated Si nanocrystals and water clusters,
Supp. D, Tables D.1-D.2) are not available, so seeded synthetic clusters stand
in for them: diamond-cubic silicon (a = 10.26 bohr), either a 2x2x2 supercell
treated as an isolated cluster or a sphere of lattice sites of radius R around
an atom at the origin, with every coordinate jittered by a seeded normal draw.

Basis per atom (uncontracted Cartesian primitives, Eq. A.1-A.3 with N_cn = 1):
four s shells with exponents 0.1, 0.3, 1.0, 3.0 and two p shells with
exponents 0.2, 0.8, i.e. 10 functions per atom.  The grid is the Cartesian
grid of Section 2 with spacing h and 6 bohr of vacuum on each side.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SI_A0 = 10.26  # bohr, diamond-cubic lattice constant

# fractional positions of the 8 atoms in the conventional diamond cell
DIAMOND_BASIS = np.array([
    [0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])

# (l, exponent) per shell, in function order on every atom; p shells expand to x, y, z
SHELL_SPEC = ((0, 0.1), (0, 0.3), (0, 1.0), (0, 3.0), (1, 0.2), (1, 0.8))

# A contracted basis with a d shell, in the style of a split-valence set with
# polarisation: (l, exponents, contraction coefficients) per shell.  Synthetic
# numbers (no basis-set tables are available here); 10 functions per atom
# with spherical d (5), 11 with Cartesian d (6).
SHELL_SPEC_D = ((0, (3.0, 1.0, 0.3), (0.15, 0.55, 0.45)), (0, (0.1,), (1.0,)),
                (1, (0.8, 0.2), (0.4, 0.7)), (2, (0.5,), (1.0,)))


def diamond_supercell(nrep: int = 2, a: float = SI_A0) -> np.ndarray:
    """All atoms of an nrep^3 supercell of the conventional diamond cell."""
    pts = []
    for i in range(nrep):
        for j in range(nrep):
            for k in range(nrep):
                for b in DIAMOND_BASIS:
                    pts.append((np.array([i, j, k]) + b) * a)
    return np.array(pts, dtype=np.float64)


def diamond_sphere(radius: float, a: float = SI_A0) -> np.ndarray:
    """Lattice sites with |R| <= radius, centred on the atom at the origin."""
    n = int(math.ceil(radius / a)) + 1
    pts = []
    for i in range(-n, n + 1):
        for j in range(-n, n + 1):
            for k in range(-n, n + 1):
                for b in DIAMOND_BASIS:
                    p = (np.array([i, j, k]) + b) * a
                    if p @ p <= radius * radius + 1e-9:
                        pts.append(p)
    pts = np.array(pts, dtype=np.float64)
    # deterministic order: by z, then y, then x (spatial locality of indices)
    order = np.lexsort((pts[:, 0], pts[:, 1], pts[:, 2]))
    return pts[order]


@dataclass
class System:
    """One synthetic cluster and everything needed to set up a calculation.

    Attributes are plain numbers and arrays; nothing here is derived from the
    method's equations.
    """
    xyz: np.ndarray                      # (n_atoms, 3) bohr
    shell_atom: np.ndarray               # (n_shells,) int32
    shell_l: np.ndarray                  # (n_shells,) int32, 0, 1 or 2
    shell_exp: np.ndarray                # (n_shells,) float64: the exponent of one-primitive shells
    grid_origin: np.ndarray              # (3,) bohr
    grid_h: float
    grid_n: np.ndarray                   # (3,) int: nx, ny, nz
    n_electrons: float
    kT: float
    name: str = ""
    meta: dict = field(default_factory=dict)
    # contracted shells (None: one primitive per shell, exponent shell_exp,
    # coefficient 1): primitives per shell, then all exponents and contraction
    # coefficients shell by shell
    shell_nprim: np.ndarray = None
    prim_exp: np.ndarray = None
    prim_coef: np.ndarray = None
    spherical: bool = False              # d shells: 5 real solid harmonics (else 6 Cartesian)

    @property
    def n_atoms(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_basis(self) -> int:
        per_l = {0: 1, 1: 3, 2: 5 if self.spherical else 6}
        return int(sum(per_l[int(l)] for l in self.shell_l))

    @property
    def n_grid(self) -> int:
        return int(np.prod(self.grid_n))


def make_system(xyz: np.ndarray, *, h: float = 0.4, pad: float = 6.0, kT: float = 0.01,
                electrons_per_atom: float = 4.0, shells=SHELL_SPEC, name: str = "",
                grid_n=None, grid_origin=None, spherical: bool = False) -> System:
    """shells: (l, exponent) per shell, or (l, exponents, coefficients) for
    contracted shells (then every shell carries its primitive list)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    sa, sl, se = [], [], []
    contracted = any(isinstance(sh[1], tuple) for sh in shells)
    npr, pe, pc = [], [], []
    for a in range(xyz.shape[0]):
        for sh in shells:
            l = sh[0]
            sa.append(a)
            sl.append(l)
            if contracted:
                exps, coefs = (sh[1], sh[2]) if isinstance(sh[1], tuple) else ((sh[1],), (1.0,))
                npr.append(len(exps))
                pe.extend(exps)
                pc.extend(coefs)
                se.append(min(exps))
            else:
                se.append(sh[1])
    lo = xyz.min(axis=0) - pad
    hi = xyz.max(axis=0) + pad
    if grid_origin is None:
        grid_origin = lo
    if grid_n is None:
        grid_n = np.array([int(math.ceil((hi[d] - lo[d]) / h)) + 1 for d in range(3)], dtype=np.int64)
    return System(xyz=xyz, shell_atom=np.array(sa, np.int32), shell_l=np.array(sl, np.int32),
                  shell_exp=np.array(se, np.float64), grid_origin=np.asarray(grid_origin, np.float64),
                  grid_h=float(h), grid_n=np.asarray(grid_n, np.int64),
                  n_electrons=float(electrons_per_atom * xyz.shape[0]), kT=float(kT), name=name,
                  shell_nprim=np.array(npr, np.int32) if contracted else None,
                  prim_exp=np.array(pe, np.float64) if contracted else None,
                  prim_coef=np.array(pc, np.float64) if contracted else None, spherical=bool(spherical))


def jitter(xyz: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return xyz + rng.normal(0.0, sigma, xyz.shape)


def batch_systems(n: int, rmin: float, rmax: float, seed: int = 0, sigma: float = 0.1, kT: float = 0.01):
    """n spheres with radii uniform in [rmin, rmax] (one seeded draw), each
    jittered with its own seed; a ragged batch of independent clusters."""
    rng = np.random.default_rng(seed)
    radii = rng.uniform(rmin, rmax, n)
    out = []
    for i, r in enumerate(radii):
        xyz = jitter(diamond_sphere(float(r)), sigma, seed * 1000 + i + 1)
        out.append(make_system(xyz, kT=kT, name=f"sphere{r:.2f}"))
    return out


def config_batch(name: str):
    """Named batches: batch64 = 64 spheres with R in [10, 30] (the full ragged
    workload), batch<n>s = n spheres with R in [6, 14] (the same recipe at a
    size one SCF step of which takes about a second)."""
    if name == "batch64":
        return batch_systems(64, 10.0, 30.0, seed=0)
    if name.startswith("batch") and name.endswith("s"):
        return batch_systems(int(name[5:-1]), 6.0, 14.0, seed=0)
    raise ValueError(f"unknown batch {name!r}")


def config_system(name: str, seed: int = 0, **kw) -> System:
    """Named workloads.

    cluster64   2x2x2 supercell, sigma 0.05, kT 0.01            (K = 640)
    sphere25    sphere R = 25 bohr, sigma 0.05, kT 0.01          (K ~ 4.6k)
    sphere40    sphere R = 40 bohr, sigma 0.1, kT 0.005          (K ~ 19.6k)
    sphereR<r>  sphere of radius r, sigma 0.1, kT 0.01
    tiny<n>     the first n atoms of the 64-atom cluster, coarse grid (tests)
    dtiny<n>    the same atoms with the contracted basis with spherical d
                shells (SHELL_SPEC_D); ctiny<n> with Cartesian d shells
    """
    if name == "cluster64":
        xyz = jitter(diamond_supercell(2), 0.05, seed)
        return make_system(xyz, kT=0.01, name=name, **kw)
    if name == "sphere25":
        xyz = jitter(diamond_sphere(25.0), 0.05, seed)
        return make_system(xyz, kT=0.01, name=name, **kw)
    if name == "sphere40":
        xyz = jitter(diamond_sphere(40.0), 0.1, seed)
        return make_system(xyz, kT=0.005, name=name, **kw)
    if name.startswith("sphereR"):
        r = float(name[len("sphereR"):])
        xyz = jitter(diamond_sphere(r), 0.1, seed)
        return make_system(xyz, kT=kw.pop("kT", 0.01), name=name, **kw)
    if name.startswith(("dtiny", "ctiny")):
        t = config_system("tiny" + name[5:], seed=seed)
        return make_system(t.xyz, h=t.grid_h, kT=t.kT, shells=SHELL_SPEC_D, name=name, grid_n=t.grid_n,
                           grid_origin=t.grid_origin, spherical=name.startswith("d"))
    if name.startswith("tiny"):
        n = int(name[4:])
        xyz = jitter(diamond_supercell(2), 0.05, seed)
        # nearest n atoms to the cluster centre, for small well-conditioned cases
        c = xyz.mean(axis=0)
        idx = np.argsort(((xyz - c) ** 2).sum(axis=1), kind="stable")[:n]
        kw.setdefault("h", 0.5)
        kw.setdefault("pad", 5.0)
        return make_system(xyz[np.sort(idx)], kT=kw.pop("kT", 0.01), name=name, **kw)
    raise ValueError(f"unknown workload {name!r}")
