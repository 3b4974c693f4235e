"""Seeded synthetic molecular systems (inputs only).

This module builds positions, velocities, atom types, topology and exclusion
lists for alkane-like liquids of the kinds the paper simulates (Section 3:
propane, neopentane, alkane chains), in LAMMPS "real" units (kcal/mol,
Angstrom, fs, g/mol).  It holds geometry and random sampling only: no part
of the RelRes potential, the sum rule or the smoothing is computed here, so
both the CUDA path and the FP64 oracle may take their inputs from it.

The paper's own systems came from OPLS-UA/AMBER-UA LAMMPS data files that are
not available; these seeded stand-ins reproduce their shape: united-atom
molecules with one hybrid (CG-carrying) site per group placed on the FG atom
nearest the group's centre (Section 2.1, Fig. 3), liquid densities, and the
switching/cutting radii of the configurations below.

Systems
-------
* ``propane(n_mol=216, box=31.8)`` -- CH3-CH2-CH3, hybrid on CH2 (n = 3).
* ``neopentane(n_mol, density=0.58)`` -- C(CH3)4, hybrid on the central C
  (n = 5).  4000 molecules = 20 000 atoms; 200 000 molecules = 1 000 000 atoms.
* ``block_copolymer(n_chain=200, n_bead=100)`` -- A50-B50 united-atom chains,
  one hybrid per 5 consecutive beads on the central bead.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# physical constants used to set densities and Maxwell-Boltzmann velocities
AVOGADRO_PER_A3 = 0.602214076          # (g/cm^3) -> (g/mol)/A^3
KB_KCAL = 0.0019872042586408316        # R / 4184, kcal/mol/K
FTM2V = 4.184e-4                       # (kcal/mol)/(g/mol) -> A^2/fs^2

M_CH3, M_CH2, M_C = 15.035, 14.027, 12.011


@dataclasses.dataclass
class System:
    name: str
    pos: np.ndarray            # (N, 3) float64, wrapped into [0, L)
    vel: np.ndarray            # (N, 3) float64, A/fs
    types: np.ndarray          # (N,) int32
    mol: np.ndarray            # (N,) int32 molecule id
    box: np.ndarray            # (3,) float64
    type_names: list
    mass_by_type: np.ndarray   # (n_types,)
    eps_fg: np.ndarray         # (n_types,) kcal/mol
    sig_fg: np.ndarray         # (n_types,) A
    is_hybrid: np.ndarray      # (n_types,) int32
    group_comp: np.ndarray     # (n_types, n_types): FG composition of the group of each hybrid type
    radii: tuple               # (r_si, r_so, r_ci, r_co) = (r_s-, r_s+, r_c-, r_c+)
    mixing: str
    skin: float
    topo: dict
    excl_off: np.ndarray       # (N+1,) CSR offsets of excluded partners
    excl_idx: np.ndarray
    temperature: float
    dt: float
    seed: int

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_types(self) -> int:
        return int(len(self.eps_fg))

    @property
    def masses(self) -> np.ndarray:
        return self.mass_by_type[self.types]

    @property
    def excl(self):
        return (self.excl_off, self.excl_idx)

    @property
    def n_hybrid(self) -> int:
        return int(self.is_hybrid[self.types].sum())

    def subset_copy(self, **changes):
        return dataclasses.replace(self, **changes)


# ----------------------------------------------------------------- geometry

def random_rotations(rng, n):
    """Uniform random rotation matrices from normalised Gaussian quaternions."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _lattice_sites(n_mol, box, rng, shuffle=True):
    k = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    while k ** 3 < n_mol:
        k += 1
    g = (np.arange(k) + 0.5) / k
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3) * box
    order = rng.permutation(len(sites)) if shuffle else np.arange(len(sites))
    return sites[np.sort(order[:n_mol])] if shuffle else sites[:n_mol], k


def _place_rigid(template, sites, k, box, rng, min_dist=3.0, max_rounds=200):
    """Place a rigid template (n_site x 3, origin = anchor) at every lattice
    site with a uniform random orientation; re-draw the orientations of
    molecules that come closer than ``min_dist`` to a neighbour molecule
    (seeded retries), checking the 13 forward lattice neighbours."""
    n_mol = len(sites)
    nsite = len(template)
    R = random_rotations(rng, n_mol)
    coords = np.einsum("mij,sj->msi", R, template) + sites[:, None, :]
    # neighbour pairs: molecules on adjacent lattice sites (26-site stencil)
    spacing = box[0] / max(k, 1)
    cell = np.floor(sites / spacing).astype(np.int64) % k
    key = (cell[:, 0] * k + cell[:, 1]) * k + cell[:, 2]
    lookup = -np.ones(k ** 3, dtype=np.int64)
    lookup[key] = np.arange(n_mol)
    offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)
            if (a, b, c) > (0, 0, 0)]
    pairs = []
    for a, b, c in offs:
        nb = (((cell[:, 0] + a) % k) * k + (cell[:, 1] + b) % k) * k + (cell[:, 2] + c) % k
        partner = lookup[nb]
        ok = partner >= 0
        pairs.append(np.stack([np.arange(n_mol)[ok], partner[ok]], axis=1))
    pairs = np.concatenate(pairs)
    pairs = pairs[pairs[:, 0] != pairs[:, 1]]

    def too_close(pp):
        out = []
        for c0 in range(0, len(pp), 100_000):
            ch = pp[c0:c0 + 100_000]
            d = coords[ch[:, 0]][:, :, None, :] - coords[ch[:, 1]][:, None, :, :]
            d -= box * np.round(d / box)
            dmin2 = (d * d).sum(-1).reshape(len(ch), -1).min(1)
            out.append(ch[dmin2 < min_dist * min_dist])
        return np.concatenate(out) if out else pp[:0]

    check = pairs
    for _ in range(max_rounds):
        bad = too_close(check)
        if len(bad) == 0:
            return coords.reshape(-1, 3)
        redo = np.unique(bad.max(axis=1))
        Rn = random_rotations(rng, len(redo))
        coords[redo] = np.einsum("mij,sj->msi", Rn, template) + sites[redo][:, None, :]
        # only pairs that involve a re-drawn molecule can have changed
        moved = np.zeros(n_mol, bool)
        moved[redo] = True
        check = pairs[moved[pairs[:, 0]] | moved[pairs[:, 1]]]
    raise RuntimeError("could not remove initial overlaps")


def maxwell_boltzmann(rng, masses, temperature):
    """Velocities (A/fs) at `temperature` K with zero total momentum."""
    sd = np.sqrt(KB_KCAL * temperature / masses * FTM2V)
    v = rng.standard_normal((len(masses), 3)) * sd[:, None]
    p = (v * masses[:, None]).sum(0) / masses.sum()
    return v - p


def exclusions_from_bonds(n_atoms, bonds, max_sep):
    """CSR exclusion lists of all atom pairs within `max_sep` bonds
    (1 = 1-2, 2 = 1-3, 3 = 1-4).  Partners sorted ascending."""
    adj = [[] for _ in range(n_atoms)]
    for a, b in bonds:
        adj[a].append(b)
        adj[b].append(a)
    off = np.zeros(n_atoms + 1, dtype=np.int32)
    idx = []
    for i in range(n_atoms):
        seen = {i}
        frontier = [i]
        for _ in range(max_sep):
            nxt = []
            for a in frontier:
                for b in adj[a]:
                    if b not in seen:
                        seen.add(b)
                        nxt.append(b)
            frontier = nxt
        part = sorted(seen - {i})
        idx.extend(part)
        off[i + 1] = off[i] + len(part)
    return off, np.asarray(idx, dtype=np.int32)


def _whole_molecule_exclusions(n_mol, nsite):
    """CSR exclusions where every pair inside a molecule is excluded."""
    n = n_mol * nsite
    off = np.arange(n + 1, dtype=np.int32) * (nsite - 1)
    base = (np.arange(n) // nsite) * nsite
    local = np.arange(n) % nsite
    cols = []
    for s in range(nsite):
        cols.append(base + s)
    allm = np.stack(cols, axis=1)  # (n, nsite)
    mask = np.arange(nsite)[None, :] != local[:, None]
    idx = allm[mask].reshape(n, nsite - 1).astype(np.int32)
    return off, idx.reshape(-1)


def _empty_topo():
    return dict(bonds=np.zeros((0, 2), np.int32), bond_type=np.zeros(0, np.int32),
                bond_k=np.zeros(0), bond_r0=np.zeros(0),
                angles=np.zeros((0, 3), np.int32), angle_type=np.zeros(0, np.int32),
                angle_k=np.zeros(0), angle_theta0=np.zeros(0),
                dihedrals=np.zeros((0, 4), np.int32), dihedral_type=np.zeros(0, np.int32),
                dihedral_k=np.zeros((0, 4)))


def box_for_density(n_mol, molar_mass, density_g_cm3):
    return (n_mol * molar_mass / (density_g_cm3 * AVOGADRO_PER_A3)) ** (1.0 / 3.0)


# ----------------------------------------------------------------- systems

def propane(n_mol=216, box=31.8, temperature=230.0, seed=2104, dt=1.0, skin=2.0,
            radii=(6.0, 7.0, 13.0, 14.0)):
    """Propane-like liquid: CH3-CH2-CH3 (1.54 A bonds, 114 deg angle), hybrid on
    CH2.  Types: 0 = CH3 (ordinary), 1 = CH2 (hybrid)."""
    rng = np.random.default_rng(seed)
    L = np.full(3, float(box))
    half = math.radians(114.0) / 2.0
    b = 1.54
    tmpl = np.array([[-b * math.sin(half), b * math.cos(half), 0.0],
                     [0.0, 0.0, 0.0],
                     [b * math.sin(half), b * math.cos(half), 0.0]])
    sites, k = _lattice_sites(n_mol, box, rng, shuffle=False)
    pos = _place_rigid(tmpl, sites, k, L, rng) % L
    types = np.tile(np.array([0, 1, 0], np.int32), n_mol)
    mol = np.repeat(np.arange(n_mol, dtype=np.int32), 3)
    mass_t = np.array([M_CH3, M_CH2])
    base = np.arange(n_mol)[:, None] * 3
    topo = _empty_topo()
    topo["bonds"] = np.concatenate([base + [0, 1], base + [1, 2]]).astype(np.int32)
    topo["bond_type"] = np.zeros(2 * n_mol, np.int32)
    topo["bond_k"] = np.array([450.0])
    topo["bond_r0"] = np.array([1.54])
    topo["angles"] = (base + [0, 1, 2]).astype(np.int32)
    topo["angle_type"] = np.zeros(n_mol, np.int32)
    topo["angle_k"] = np.array([62.0])
    topo["angle_theta0"] = np.array([math.radians(114.0)])
    eo, ei = _whole_molecule_exclusions(n_mol, 3)
    vel = maxwell_boltzmann(rng, mass_t[types], temperature)
    return System("propane", pos, vel, types, mol, L, ["CH3", "CH2_h"], mass_t,
                  np.array([0.195, 0.0914]), np.array([3.75, 3.95]),
                  np.array([0, 1], np.int32), np.array([[0, 0], [2, 1]], np.int32),
                  tuple(radii), "lb", skin, topo, eo, ei, temperature, dt, seed)


def neopentane(n_mol=4000, density=0.58, temperature=260.0, seed=2104, dt=2.0, skin=2.0,
               radii=(6.0, 7.0, 13.0, 14.0)):
    """Neopentane-like liquid: central C bonded tetrahedrally (1.54 A) to four
    CH3; hybrid on the central C.  Types: 0 = C (hybrid), 1 = CH3 (ordinary)."""
    rng = np.random.default_rng(seed)
    molar = M_C + 4 * M_CH3
    box = box_for_density(n_mol, molar, density)
    L = np.full(3, box)
    t = 1.54 / math.sqrt(3.0)
    tmpl = np.array([[0, 0, 0], [t, t, t], [t, -t, -t], [-t, t, -t], [-t, -t, t]], float)
    sites, k = _lattice_sites(n_mol, box, rng, shuffle=True)
    pos = _place_rigid(tmpl, sites, k, L, rng) % L
    types = np.tile(np.array([0, 1, 1, 1, 1], np.int32), n_mol)
    mol = np.repeat(np.arange(n_mol, dtype=np.int32), 5)
    mass_t = np.array([M_C, M_CH3])
    base = np.arange(n_mol)[:, None] * 5
    topo = _empty_topo()
    topo["bonds"] = np.concatenate([base + [0, s] for s in range(1, 5)]).astype(np.int32)
    topo["bond_type"] = np.zeros(4 * n_mol, np.int32)
    topo["bond_k"] = np.array([450.0])
    topo["bond_r0"] = np.array([1.54])
    ang = [(a, 0, b) for a in range(1, 5) for b in range(a + 1, 5)]
    topo["angles"] = np.concatenate([base + list(x) for x in ang]).astype(np.int32)
    topo["angle_type"] = np.zeros(6 * n_mol, np.int32)
    topo["angle_k"] = np.array([62.0])
    topo["angle_theta0"] = np.array([math.acos(-1.0 / 3.0)])
    eo, ei = _whole_molecule_exclusions(n_mol, 5)
    vel = maxwell_boltzmann(rng, mass_t[types], temperature)
    return System("neopentane", pos, vel, types, mol, L, ["C_h", "CH3"], mass_t,
                  np.array([0.0005, 0.195]), np.array([6.4, 3.75]),
                  np.array([1, 0], np.int32), np.array([[1, 4], [0, 0]], np.int32),
                  tuple(radii), "lb", skin, topo, eo, ei, temperature, dt, seed)


def block_copolymer(n_chain=200, n_bead=100, block=50, density=0.75, temperature=400.0,
                    seed=2104, dt=2.0, skin=2.0, radii=(6.0, 7.0, 13.0, 14.0), group=5):
    """Linear A(block)-B(block) united-atom chains grown by a seeded random walk
    (1.54 A bonds, 114 deg angles, random torsions, < 3 A overlaps rejected).
    One hybrid per `group` consecutive beads, on the central bead.  Types:
    0 = A (ordinary), 1 = B (ordinary), 2 = A hybrid, 3 = B hybrid.  OPLS
    dihedral coefficients K1..K3 drawn uniform in [0, 3] kcal/mol, K4 = 0.
    Exclusions: 1-2, 1-3, 1-4."""
    rng = np.random.default_rng(seed)
    mass_t = np.array([M_CH2, M_CH3, M_CH2, M_CH3])
    bead_t = np.where(np.arange(n_bead) < block, 0, 1).astype(np.int32)
    hyb = (np.arange(n_bead) % group) == group // 2
    bead_t = np.where(hyb, bead_t + 2, bead_t).astype(np.int32)
    molar = mass_t[bead_t].sum()
    box = box_for_density(n_chain, molar, density)
    L = np.full(3, box)
    n = n_chain * n_bead
    pos = np.zeros((n, 3))
    theta = math.radians(114.0)
    # uniform grid for overlap checks
    nc = max(1, int(box // 3.0))
    cs = box / nc
    grid = {}

    def cell_of(p):
        c = np.floor(p / cs).astype(int) % nc
        return (int(c[0]), int(c[1]), int(c[2]))

    def too_close(p, skip):
        c = cell_of(p)
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                for d in (-1, 0, 1):
                    key = ((c[0] + a) % nc, (c[1] + b) % nc, (c[2] + d) % nc)
                    for j in grid.get(key, ()):
                        if j in skip:
                            continue
                        dd = p - pos[j]
                        dd -= box * np.round(dd / box)
                        if dd @ dd < 9.0:
                            return True
        return False

    for ch in range(n_chain):
        for attempt in range(1000):
            ok = True
            placed = []
            for s in range(n_bead):
                i = ch * n_bead + s
                skip = set(range(max(ch * n_bead, i - 3), i))
                for tries in range(200):
                    if s == 0:
                        p = rng.random(3) * box
                    elif s == 1:
                        u = rng.standard_normal(3)
                        u /= np.linalg.norm(u)
                        p = pos[i - 1] + 1.54 * u
                    else:
                        b1 = pos[i - 1] - pos[i - 2]
                        b1 /= np.linalg.norm(b1)
                        if s == 2:
                            ref = rng.standard_normal(3)
                        else:
                            ref = pos[i - 3] - pos[i - 2]
                        perp = ref - (ref @ b1) * b1
                        perp /= np.linalg.norm(perp)
                        phi = rng.uniform(-math.pi, math.pi)
                        w = np.cross(b1, perp)
                        dirn = (math.cos(math.pi - theta) * b1 + math.sin(math.pi - theta)
                                * (math.cos(phi) * perp + math.sin(phi) * w))
                        p = pos[i - 1] + 1.54 * dirn
                    if not too_close(p, skip):
                        break
                else:
                    ok = False
                    break
                pos[i] = p
                placed.append(i)
                grid.setdefault(cell_of(p), []).append(i)
            if ok:
                break
            for j in placed:
                grid[cell_of(pos[j])].remove(j)
        else:
            raise RuntimeError("chain growth failed")
    pos %= L
    types = np.tile(bead_t, n_chain)
    mol = np.repeat(np.arange(n_chain, dtype=np.int32), n_bead)
    base = np.arange(n_chain)[:, None] * n_bead
    topo = _empty_topo()
    topo["bonds"] = (base[:, :, None] + np.stack([np.arange(n_bead - 1), np.arange(1, n_bead)], 1)[None]).reshape(-1, 2).astype(np.int32)
    topo["bond_type"] = np.zeros(len(topo["bonds"]), np.int32)
    topo["bond_k"] = np.array([450.0])
    topo["bond_r0"] = np.array([1.54])
    a = np.arange(n_bead - 2)
    topo["angles"] = (base[:, :, None] + np.stack([a, a + 1, a + 2], 1)[None]).reshape(-1, 3).astype(np.int32)
    topo["angle_type"] = np.zeros(len(topo["angles"]), np.int32)
    topo["angle_k"] = np.array([62.0])
    topo["angle_theta0"] = np.array([theta])
    d = np.arange(n_bead - 3)
    topo["dihedrals"] = (base[:, :, None] + np.stack([d, d + 1, d + 2, d + 3], 1)[None]).reshape(-1, 4).astype(np.int32)
    topo["dihedral_type"] = np.zeros(len(topo["dihedrals"]), np.int32)
    kd = np.zeros((1, 4))
    kd[0, :3] = rng.uniform(0.0, 3.0, 3)
    topo["dihedral_k"] = kd
    eo, ei = exclusions_from_bonds(n, topo["bonds"], 3)
    vel = maxwell_boltzmann(rng, mass_t[types], temperature)
    comp = np.zeros((4, 4), np.int32)
    comp[2] = [group - 1, 0, 1, 0]
    comp[3] = [0, group - 1, 0, 1]
    return System("block_copolymer", pos, vel, types, mol, L, ["A", "B", "A_h", "B_h"], mass_t,
                  np.array([0.0914, 0.195, 0.0914, 0.195]), np.array([3.95, 3.75, 3.95, 3.75]),
                  np.array([0, 0, 1, 1], np.int32), comp, tuple(radii), "lb", skin, topo, eo, ei,
                  temperature, dt, seed)


def fg_only(system, r_inner=13.0, r_outer=14.0):
    """The same system set up as the plain FG reference of the paper (r_s -> r_c,
    no CG interaction): r_s- = r_inner, r_s+ = r_c- = r_c+ = r_outer (the
    radii must stay ordered) and every type ordinary, so only the FG LJ term,
    smoothed to zero over [r_inner, r_outer), remains."""
    return system.subset_copy(name=system.name + "_fg_only",
                              is_hybrid=np.zeros_like(system.is_hybrid),
                              radii=(r_inner, r_outer, r_outer, r_outer))
