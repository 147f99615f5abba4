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
        new_of = {int(a): i for i, a in enumerate(idx)}
        cuts = [(new_of[int(a)], new_of[int(b)]) for a, b in self.cut_bonds
                if int(a) in new_of and int(b) in new_of]     # cut bonds inside the subsystem
        return System(Z=self.Z[idx].copy(), xyz=self.xyz[idx].copy(),
                      frag=np.array([remap[f] for f in self.frag[idx]], dtype=np.int32),
                      frag_charge=self.frag_charge[frags].copy(),
                      cut_bonds=np.array(cuts, dtype=np.int32).reshape(-1, 2), name=self.name + "-sub")


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


# --------------------------------------------------------------------------
# alpha-helical polyalanine with covalent fragment boundaries (C3 stand-in)


def _nerf(a, b, c, r, theta_deg, chi_deg):
    """Position of atom d bonded to c with |cd| = r, angle b-c-d = theta and
    dihedral a-b-c-d = chi (internal coordinates to Cartesian)."""
    bc = (c - b) / np.linalg.norm(c - b)
    n = np.cross(b - a, bc)
    n /= np.linalg.norm(n)
    m = np.cross(n, bc)
    th, ch = np.radians(theta_deg), np.radians(chi_deg)
    d = np.array([-r * np.cos(th), r * np.sin(th) * np.cos(ch), r * np.sin(th) * np.sin(ch)])
    return c + d[0] * bc + d[1] * m + d[2] * n


def polyalanine_helix(n_res: int, phi=-57.0, psi=-47.0, omega=180.0, seed: int | None = None,
                      frag_sizes=(1, 2, 3)):
    """H-(Ala)n-OH as an ideal helix from standard bond lengths and angles
    (N-CA 1.458, CA-C 1.525, C-N 1.329, C=O 1.231, N-H 1.01, C-H 1.09,
    CA-CB 1.53 A; N-CA-C 111.2, CA-C-N 116.2, C-N-CA 121.7 deg).

    Residue units are cut at the CA-C(O) bonds: unit i holds C(i-1), O(i-1),
    N(i), H(i), CA(i), HA(i), CB(i) and its three H; the first unit carries
    the N-terminal H, the last the C-terminal C(=O)-OH.  Consecutive units are
    joined into fragments of 1, 2 or 3 residues drawn from the seed (seed None:
    one residue per fragment); every CA-C bond between two fragments is a cut
    bond with the CA as detachment atom (BDA) and the C as attachment atom."""
    rng = np.random.default_rng(seed) if seed is not None else None
    xyz, Z, unit = [], [], []

    def add(z, p, u):
        Z.append(z)
        xyz.append(np.asarray(p, dtype=np.float64))
        unit.append(u)
        return len(Z) - 1

    # backbone N, CA, C of every residue
    N = [np.array([0.0, 0.0, 0.0])]
    CA = [np.array([1.458, 0.0, 0.0])]
    C = [_nerf(np.array([0.0, 1.0, 0.0]), N[0], CA[0], 1.525, 111.2, 0.0)]
    for i in range(1, n_res):
        N.append(_nerf(N[i - 1], CA[i - 1], C[i - 1], 1.329, 116.2, psi))
        CA.append(_nerf(CA[i - 1], C[i - 1], N[i], 1.458, 121.7, omega))
        C.append(_nerf(C[i - 1], N[i], CA[i], 1.525, 111.2, phi))
    ca_idx, c_idx = [], []
    for i in range(n_res):
        if i > 0:   # the previous residue's carbonyl belongs to this unit
            c_idx.append(add(6, C[i - 1], i))
            add(8, _nerf(N[i - 1], CA[i - 1], C[i - 1], 1.231, 120.5, psi + 180.0), i)
            add(1, _nerf(CA[i - 1], C[i - 1], N[i], 1.01, 119.5, 0.0), i)            # H on N
        else:
            add(1, _nerf(C[0], CA[0], N[0], 1.01, 109.5, 60.0), 0)                  # N-terminal H
            add(1, _nerf(C[0], CA[0], N[0], 1.01, 109.5, -60.0), 0)
        add(7, N[i], i)
        ca_idx.append(add(6, CA[i], i))
        ref = C[i - 1] if i > 0 else _nerf(C[0], CA[0], N[0], 1.0, 109.5, 180.0)
        cb = _nerf(ref, N[i], CA[i], 1.53, 110.5, phi - 120.0 if i > 0 else 180.0 - 120.0)
        add(6, cb, i)
        add(1, _nerf(ref, N[i], CA[i], 1.09, 109.5, phi + 120.0 if i > 0 else 180.0 + 120.0), i)   # HA
        for chi in (60.0, 180.0, 300.0):
            add(1, _nerf(N[i], CA[i], cb, 1.09, 109.5, chi), i)
    last = n_res - 1
    c_idx.append(add(6, C[last], last))
    add(8, _nerf(N[last], CA[last], C[last], 1.231, 120.5, psi + 180.0), last)
    ot = _nerf(N[last], CA[last], C[last], 1.34, 116.2, psi)
    add(8, ot, last)
    add(1, _nerf(CA[last], C[last], ot, 0.97, 107.0, 180.0), last)
    # fragments of 1-3 consecutive residues
    frag_of_res, f, i = [], 0, 0
    while i < n_res:
        k = 1 if rng is None else int(rng.choice(frag_sizes))
        for _ in range(min(k, n_res - i)):
            frag_of_res.append(f)
        i += k
        f += 1
    frag = np.array([frag_of_res[u] for u in unit], dtype=np.int32)
    # cut bonds CA(i)-C(i) between fragments: BDA = CA(i), BAA = C(i) (unit i+1)
    cuts = [(ca_idx[i], c_idx[i]) for i in range(n_res - 1) if frag_of_res[i] != frag_of_res[i + 1]]
    xyz = np.array(xyz) * ANGSTROM
    return System(Z=np.array(Z, dtype=np.int32), xyz=xyz, frag=frag,
                  frag_charge=np.zeros(f, dtype=np.int32),
                  cut_bonds=np.array(cuts, dtype=np.int32).reshape(-1, 2), name=f"ala{n_res}-helix")
