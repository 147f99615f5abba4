"""Seeded synthetic geometries standing in for the paper's clusters.

The paper's water clusters (packmol) and acene crystal clusters (Mercury) live
in an external data repository that is not available, so these generators
build clusters of the same shape and size from a seed:

* water_cluster   - N rigid waters (O-H 0.957 A, H-O-H 104.5 deg) with centres
                    uniform in a sphere at 1.0 g/cm^3, O-O >= 2.6 A, random
                    orientations (uniform quaternions);
* acene           - idealised planar D2h acene (C-C 1.40 A, C-H 1.08 A);
* herringbone     - a two-molecule-per-cell herringbone crystal block of an
                    acene, orientation chosen by a deterministic grid search
                    that maximises the smallest intermolecular distance;
* jitter          - Gaussian atomic displacements.

Everything returns coordinates in angstrom; ``System`` converts to bohr.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .params import ANGSTROM


@dataclasses.dataclass
class System:
    """Geometry + fragment partition, the input of an FMO calculation.

    Z            (n_atoms,)   atomic numbers
    xyz          (n_atoms, 3) coordinates in bohr
    frag         (n_atoms,)   fragment index of every atom, 0..n_frag-1
    frag_charge  (n_frag,)    net charge of every fragment (e)
    cut_bonds    (n_cut, 2)   (BDA, BAA) atom pairs of covalent bonds cut
                              between fragments (hybrid orbital projection)
    """
    Z: np.ndarray
    xyz: np.ndarray
    frag: np.ndarray
    frag_charge: np.ndarray
    cut_bonds: np.ndarray = dataclasses.field(
        default_factory=lambda: np.zeros((0, 2), dtype=np.int32))
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return len(self.Z)

    @property
    def n_frag(self) -> int:
        return len(self.frag_charge)

    def subsystem(self, frags) -> "System":
        """Atoms of the listed fragments as a standalone system (fragment
        numbering kept in the given order)."""
        frags = list(frags)
        idx = np.concatenate([np.nonzero(self.frag == f)[0] for f in frags])
        remap = {f: i for i, f in enumerate(frags)}
        return System(Z=self.Z[idx].copy(), xyz=self.xyz[idx].copy(),
                      frag=np.array([remap[f] for f in self.frag[idx]], dtype=np.int32),
                      frag_charge=self.frag_charge[frags].copy(), name=self.name + "-sub")


def _random_rotation(rng) -> np.ndarray:
    """Rotation matrix from a uniformly distributed unit quaternion."""
    u1, u2, u3 = rng.random(3)
    q = np.array([np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
                  np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3),
                  np.sqrt(u1) * np.cos(2 * np.pi * u3)])
    x, y, z, w = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def water_molecule() -> np.ndarray:
    """O, H, H in angstrom, O at the origin, molecule in the xy plane."""
    half = np.deg2rad(104.5 / 2.0)
    r = 0.957
    return np.array([[0.0, 0.0, 0.0],
                     [r * np.sin(half), r * np.cos(half), 0.0],
                     [-r * np.sin(half), r * np.cos(half), 0.0]])


def water_cluster(n: int = 64, seed: int = 1, density_g_cm3: float = 1.0,
                  min_oo: float = 2.6) -> System:
    rng = np.random.default_rng(seed)
    vol_per_mol = 18.015 / (density_g_cm3 * 0.6022140857)      # A^3
    radius = (3.0 * n * vol_per_mol / (4.0 * np.pi)) ** (1.0 / 3.0)
    centres = []
    tries = 0
    while len(centres) < n:
        tries += 1
        if tries > 2_000_000:
            raise RuntimeError("water packing failed")
        p = rng.uniform(-radius, radius, 3)
        if p @ p > radius * radius:
            continue
        if centres and np.min(np.linalg.norm(np.asarray(centres) - p, axis=1)) < min_oo:
            continue
        centres.append(p)
    mol = water_molecule()
    xyz, Z, frag = [], [], []
    for i, c in enumerate(centres):
        R = _random_rotation(rng)
        xyz.append(mol @ R.T + c)
        Z += [8, 1, 1]
        frag += [i, i, i]
    return System(Z=np.array(Z, dtype=np.int32), xyz=np.vstack(xyz) * ANGSTROM,
                  frag=np.array(frag, dtype=np.int32),
                  frag_charge=np.zeros(n, dtype=np.int32), name=f"water{n}")


def acene(n_rings: int, cc: float = 1.40, ch: float = 1.08):
    """Planar linear acene: returns (Z, xyz[A]) with the long axis along x,
    the molecular plane xy and the centroid at the origin."""
    step = np.sqrt(3.0) * cc                       # ring-centre spacing
    centres = (np.arange(n_rings) - (n_rings - 1) / 2.0) * step
    carbons = []
    for cx in centres:
        for k in range(6):
            ang = np.deg2rad(30.0 + 60.0 * k)
            p = np.array([cx + cc * np.cos(ang), cc * np.sin(ang), 0.0])
            if not any(np.linalg.norm(p - q) < 1e-6 for q in carbons):
                carbons.append(p)
    carbons = np.array(carbons)
    hydrogens = []
    for i, p in enumerate(carbons):
        d = np.linalg.norm(carbons - p, axis=1)
        nb = np.nonzero((d > 1e-6) & (d < cc * 1.1))[0]
        if len(nb) == 2:
            v = 2 * p - carbons[nb[0]] - carbons[nb[1]]
            hydrogens.append(p + ch * v / np.linalg.norm(v))
    xyz = np.vstack([carbons, np.array(hydrogens)])
    Z = np.array([6] * len(carbons) + [1] * len(hydrogens), dtype=np.int32)
    return Z, xyz - xyz.mean(axis=0)


def cell_vectors(a, b, c, alpha, beta, gamma) -> np.ndarray:
    """Rows a, b, c: a along x, b in the xy plane (angles in degrees)."""
    al, be, ga = np.deg2rad([alpha, beta, gamma])
    va = np.array([a, 0.0, 0.0])
    vb = np.array([b * np.cos(ga), b * np.sin(ga), 0.0])
    cx = c * np.cos(be)
    cy = c * (np.cos(al) - np.cos(be) * np.cos(ga)) / np.sin(ga)
    cz = np.sqrt(c * c - cx * cx - cy * cy)
    return np.array([va, vb, np.array([cx, cy, cz])])


def _orient(axis, theta):
    """Rotation taking the molecular frame (long axis x, plane xy) to one with
    the long axis along ``axis`` and the plane rotated by theta about it."""
    u = axis / np.linalg.norm(axis)
    ref = np.array([0.0, 0.0, 1.0]) if abs(u[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    v = np.cross(ref, u)
    v /= np.linalg.norm(v)
    w = np.cross(u, v)
    vt = np.cos(theta) * v + np.sin(theta) * w
    wt = np.cross(u, vt)
    return np.stack([u, vt, wt], axis=1)          # columns: images of x, y, z


def _place(mol_xyz, cell, frac_sites, thetas, axis, ncell):
    mols = []
    for i in range(ncell[0]):
        for j in range(ncell[1]):
            for k in range(ncell[2]):
                origin = np.array([i, j, k], dtype=float) @ cell
                for site, th in zip(frac_sites, thetas):
                    R = _orient(axis, th)
                    mols.append(mol_xyz @ R.T + origin + np.asarray(site) @ cell)
    return mols


def _min_intermolecular(mol_xyz, cell, sites, thetas, axis) -> float:
    mols = _place(mol_xyz, cell, sites, thetas, axis, (3, 3, 3))
    centre = mols[13 * len(sites): 14 * len(sites)]   # the molecules of cell (1,1,1)
    best = np.inf
    for m in centre:
        for o in mols:
            if o is m:
                continue
            d = np.sqrt(((m[:, None, :] - o[None, :, :]) ** 2).sum(-1)).min()
            best = min(best, d)
    return best


def herringbone_orientation(mol_xyz, cell, sites=((0, 0, 0), (0.5, 0.5, 0))):
    """Grid search over the long-axis tilt (from c towards the ab-plane normal)
    and the herringbone angle +-theta that maximises the smallest
    intermolecular atom-atom distance.  Returns (axis, theta, min_dist)."""
    cvec = cell[2] / np.linalg.norm(cell[2])
    nrm = np.cross(cell[0], cell[1])
    nrm /= np.linalg.norm(nrm)
    if nrm @ cvec < 0:
        nrm = -nrm
    best = (None, None, -1.0)
    for t in np.linspace(0.0, 1.0, 11):
        axis = (1 - t) * cvec + t * nrm
        axis /= np.linalg.norm(axis)
        for th in np.deg2rad(np.arange(0.0, 90.0, 5.0)):
            d = _min_intermolecular(mol_xyz, cell, sites, (th, -th), axis)
            if d > best[2] + 1e-9:
                best = (axis, th, d)
    return best


def herringbone_cluster(n_rings, lattice, ncell, keep, seed, jitter=0.05, name=""):
    """Herringbone block of an acene, trimmed to the ``keep`` molecules whose
    centroids lie nearest the block centroid (ties by index), then jittered."""
    Z1, mol = acene(n_rings)
    cell = cell_vectors(*lattice)
    sites = ((0.0, 0.0, 0.0), (0.5, 0.5, 0.0))
    axis, th, dmin = herringbone_orientation(mol, cell, sites)
    mols = _place(mol, cell, sites, (th, -th), axis, ncell)
    cents = np.array([m.mean(axis=0) for m in mols])
    c0 = cents.mean(axis=0)
    order = np.argsort(np.linalg.norm(cents - c0, axis=1), kind="stable")[:keep]
    order = np.sort(order)
    rng = np.random.default_rng(seed)
    xyz = np.vstack([mols[i] for i in order])
    xyz = xyz + rng.normal(0.0, jitter, xyz.shape)
    nat = len(Z1)
    return System(Z=np.tile(Z1, keep), xyz=xyz * ANGSTROM,
                  frag=np.repeat(np.arange(keep, dtype=np.int32), nat),
                  frag_charge=np.zeros(keep, dtype=np.int32), name=name), \
        {"axis": axis.tolist(), "theta_deg": float(np.rad2deg(th)), "min_dist_A": float(dmin)}


ANTHRACENE_CELL = (8.56, 6.04, 11.16, 90.0, 124.7, 90.0)
PENTACENE_CELL = (6.27, 7.78, 14.53, 76.5, 87.7, 84.7)


def anthracene_cluster(n_mol=128, seed=2, jitter=0.05):
    """128 anthracenes = 4x4x4 monoclinic cells x 2 molecules."""
    cells = {128: (4, 4, 4)}.get(n_mol)
    if cells is None:
        k = int(np.ceil((n_mol / 2) ** (1 / 3)))
        cells = (k, k, k)
    return herringbone_cluster(3, ANTHRACENE_CELL, cells, n_mol, seed, jitter,
                               name=f"anthracene{n_mol}")


def pentacene_cluster(n_mol=660, seed=4, jitter=0.05):
    """660 pentacenes kept from a 7x7x7-cell triclinic block (686 molecules)."""
    k = 7 if n_mol > 250 else int(np.ceil((n_mol / 2) ** (1 / 3))) + 1
    return herringbone_cluster(5, PENTACENE_CELL, (k, k, k), n_mol, seed, jitter,
                               name=f"pentacene{n_mol}")


def jittered(system: System, sigma_A: float, seed: int) -> System:
    rng = np.random.default_rng(seed)
    return dataclasses.replace(system, xyz=system.xyz + rng.normal(0.0, sigma_A * ANGSTROM,
                                                                   system.xyz.shape))


def separated(system: System, distance_A: float) -> System:
    """Move fragment k by k*distance along x (fragments far apart)."""
    xyz = system.xyz.copy()
    for f in range(system.n_frag):
        xyz[system.frag == f, 0] += f * distance_A * ANGSTROM
    return dataclasses.replace(system, xyz=xyz)
