"""Seeded synthetic inputs and workload descriptions for tests, smoke and bench.

This module holds no arithmetic of the method: it draws magnetisation
patterns from numpy's seeded generators and lists grid sizes, materials and
mechanics of the film-pair workloads.  Both the CPU oracle side and the CUDA
side of every comparison receive the arrays made here.

Patterns (reading of the workload descriptions):
  * random unit vectors: normalised Gaussian triples, default_rng(seed);
  * PMA up/down domains of ~`size` cells: random signs on a coarse grid of
    `size`-cell blocks (block boundaries shifted by a random phase), mz = +-1
    with a small seeded in-plane tilt, normalised;
  * vortex: m = normalise(-chi (y - yc), chi (x - xc), p exp(-rho^2 / rc^2))
    with random chirality chi, polarity p and core offset;
  * stripes: up/down stripes of a given width along x with a random phase
    and a small seeded in-plane tilt.
Arrays are float64, shape (3, nz, ny, nx), x fastest.
"""

from dataclasses import dataclass, field

import numpy as np


def random_unit(shape_xyz, seed):
    nx, ny, nz = shape_xyz
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((3, nz, ny, nx))
    return m / np.sqrt(np.sum(m * m, axis=0, keepdims=True))


def pma_domains(shape_xyz, seed, size=20, tilt=0.05):
    nx, ny, nz = shape_xyz
    rng = np.random.default_rng(seed)
    cx = -(-nx // size) + 1
    cy = -(-ny // size) + 1
    signs = rng.choice([-1.0, 1.0], size=(cy, cx))
    sx, sy = rng.integers(0, size, size=2)
    ix = (np.arange(nx) + sx) // size
    iy = (np.arange(ny) + sy) // size
    mz = signs[iy][:, ix]
    m = np.empty((3, nz, ny, nx))
    m[2] = mz[None]
    m[0:2] = tilt * rng.standard_normal((2, nz, ny, nx))
    return m / np.sqrt(np.sum(m * m, axis=0, keepdims=True))


def vortex(shape_xyz, seed, rc=4.0, core_jitter=8):
    nx, ny, nz = shape_xyz
    rng = np.random.default_rng(seed)
    chi = rng.choice([-1.0, 1.0])
    pol = rng.choice([-1.0, 1.0])
    xc = (nx - 1) / 2 + rng.uniform(-core_jitter, core_jitter)
    yc = (ny - 1) / 2 + rng.uniform(-core_jitter, core_jitter)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rho2 = (x - xc) ** 2 + (y - yc) ** 2
    m = np.stack([-chi * (y - yc), chi * (x - xc), pol * np.exp(-rho2 / rc ** 2)])
    return m / np.sqrt(np.sum(m * m, axis=0, keepdims=True))


@dataclass
class Material:
    Ms: float
    Aex: float = 0.0
    Ku: float = 0.0
    ku_axis: tuple = (0.0, 0.0, 1.0)
    alpha: float = 0.5

    def as_dict(self):
        return dict(Ms=self.Ms, Aex=self.Aex, Ku=self.Ku, ku_axis=self.ku_axis, alpha=self.alpha)


@dataclass
class Mechanics:
    mass: float = 2.5e-18       # kg
    k: float = 1e-3             # N/m
    v_drive: float = 1.0        # m/s
    gamma_v: float = 4e7        # 1/s  (critical damping 2 sqrt(k/mass))
    dir: tuple = (1.0, 0.0, 0.0)
    x0_spring: float = 0.0      # m, spring end ahead of the slider at t = 0

    def as_dict(self):
        return dict(mass=self.mass, k=self.k, v_drive=self.v_drive, gamma_v=self.gamma_v,
                    dir=self.dir, x0_spring=self.x0_spring)


@dataclass
class FilmPair:
    """Two magnets: base at the origin, slider `gap` cells beyond it along
    `stack_axis` (z for films, x for side-by-side cubes), shifted by `lateral`
    cells along the two other axes."""
    name: str
    n_base: tuple
    n_slider: tuple
    cell: tuple
    gap: int
    mat_base: Material
    mat_slider: Material
    mech: Mechanics = field(default_factory=Mechanics)
    u0: tuple = (0.0, 0.0, 0.0)
    H_ext: tuple = (0.0, 0.0, 0.0)
    lateral: tuple = (0, 0)      # slider lattice offset along the other two axes (cells)
    stack_axis: int = 2

    @property
    def offsets(self):
        o = [0, 0, 0]
        others = [a for a in range(3) if a != self.stack_axis]
        o[others[0]], o[others[1]] = self.lateral
        o[self.stack_axis] = self.n_base[self.stack_axis] + self.gap
        return [(0, 0, 0), tuple(o)]

    def cells(self):
        return int(np.prod(self.n_base)) + int(np.prod(self.n_slider))


def film_pair_plain(n=(64, 64, 1), gap=1, seed=0):
    """Two random-unit films of 4 nm cells, Ms = 8e5 A/m (plain stray-field sweep)."""
    mat = Material(Ms=8e5, Aex=1.3e-11, Ku=0.0, alpha=0.5)
    fp = FilmPair("film_pair_%dx%dx%d_gap%d" % (n + (gap,)), n, n, (4e-9, 4e-9, 4e-9), gap,
                  mat, mat)
    return fp, random_unit(n, seed), random_unit(n, seed + 1)


def film_pair_stick_slip(n=(1024, 256, 2), gap=5, seed=0):
    """Spring-pulled PMA films, 4 nm cells, Ms=1.1e6, Aex=1.5e-11, Ku=1e6 (z), alpha=0.5."""
    mat = Material(Ms=1.1e6, Aex=1.5e-11, Ku=1.0e6, ku_axis=(0.0, 0.0, 1.0), alpha=0.5)
    mech = Mechanics(mass=2.5e-18, k=1e-3, v_drive=1.0, gamma_v=4e7, dir=(1.0, 0.0, 0.0))
    fp = FilmPair("stick_slip_%dx%dx%d_gap%d" % (n + (gap,)), n, n, (4e-9, 4e-9, 4e-9), gap,
                  mat, mat, mech)
    return fp, pma_domains(n, seed), pma_domains(n, seed + 1)


def stripes(shape_xyz, seed, width=20, tilt=0.05):
    """Up/down stripe domains of `width` cells along x (stripes run along y),
    phase drawn at random, mz = +-1 with a small seeded in-plane tilt, normalised."""
    nx, ny, nz = shape_xyz
    rng = np.random.default_rng(seed)
    phase = int(rng.integers(0, 2 * width))
    mz = np.where(((np.arange(nx) + phase) // width) % 2 == 0, 1.0, -1.0)
    m = np.empty((3, nz, ny, nx))
    m[2] = mz[None, None, :]
    m[0:2] = tilt * rng.standard_normal((2, nz, ny, nx))
    return m / np.sqrt(np.sum(m * m, axis=0, keepdims=True))


def film_pair_friction(n=(256, 256, 5), gap=5, seed=0, pbc_images=2):
    """The friction films of Sec. IV.B: 1024 x 1024 x 20 nm (256 x 256 x 5 cells
    of 4 nm), 20 nm apart, periodic in the film plane, CoCrPt (Ku = 1.225e5 J/m^3
    along z, Ms = 3.5e5 A/m, Aex = 5e-12 J/m, alpha = 0.05), ~80 nm (20-cell)
    stripe domains, spring k = 0.005 N/m pulled at 2 m/s with the spring 80 nm
    ahead of the slider.  Mass and viscous damping: critically damped, the
    viscous force at v_d a tenth of a 0.7 nN magnetic force (the order of
    Sec. IV.B's friction), so gamma_v m = 3.5e-11 kg/s, m = (gamma_v m)^2 / 4k.
    Grain disorder is not modelled (uniform easy axis)."""
    mat = Material(Ms=3.5e5, Aex=5e-12, Ku=1.225e5, ku_axis=(0.0, 0.0, 1.0), alpha=0.05)
    gm = 3.5e-11
    k = 0.005
    mass = gm * gm / (4.0 * k)
    mech = Mechanics(mass=mass, k=k, v_drive=2.0, gamma_v=gm / mass, dir=(1.0, 0.0, 0.0), x0_spring=80e-9)
    fp = FilmPair("friction_%dx%dx%d_gap%d_pbc" % (n + (gap,)), n, n, (4e-9, 4e-9, 4e-9), gap, mat, mat, mech)
    fp.periodic = 3
    fp.pbc_images = pbc_images
    return fp, stripes(n, seed), stripes(n, seed + 1)


def cube_pair(n=(64, 64, 64), gap=3, seed=0):
    """Two vortex-seeded cubes of 2 nm cells side by side along x, `gap` cells
    apart; Ms=8e5 A/m, Aex=1.3e-11 J/m, no anisotropy, alpha=0.5."""
    mat = Material(Ms=8e5, Aex=1.3e-11, Ku=0.0, alpha=0.5)
    fp = FilmPair("cube_pair_%dx%dx%d_gap%d" % (n + (gap,)), n, n, (2e-9, 2e-9, 2e-9), gap, mat, mat,
                  stack_axis=0)
    return fp, vortex(n, seed), vortex(n, seed + 1)


def batch_pairs(npairs=256, seed=0, nx=(64, 512), ny=(64, 256), nz=(1, 4), u_max=50.0,
                v_drive=(0.1, 10.0)):
    """Independent spring-pulled PMA film pairs of uneven sizes (the stick-slip
    pair's materials, mechanics and gap): per pair the two films share a size
    drawn uniformly from the integer ranges nx x ny x nz, the slider is displaced
    along x by u ~ U[0, u_max) cells and pulled at v_drive ~ U[v0, v1] m/s.
    Returns FilmPair descriptions only; pair i's domain patterns come from
    `batch_patterns(fp)` (pma_domains with the seeds stored on the pair), so
    a large batch need not hold all patterns on the host at once."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(npairs):
        n = (int(rng.integers(nx[0], nx[1] + 1)), int(rng.integers(ny[0], ny[1] + 1)),
             int(rng.integers(nz[0], nz[1] + 1)))
        u = float(rng.uniform(0.0, u_max))
        vd = float(rng.uniform(v_drive[0], v_drive[1]))
        mat = Material(Ms=1.1e6, Aex=1.5e-11, Ku=1.0e6, ku_axis=(0.0, 0.0, 1.0), alpha=0.5)
        mech = Mechanics(mass=2.5e-18, k=1e-3, v_drive=vd, gamma_v=4e7, dir=(1.0, 0.0, 0.0))
        fp = FilmPair("batch_pair_%d_%dx%dx%d" % ((i,) + n), n, n, (4e-9, 4e-9, 4e-9), 5, mat, mat, mech,
                      u0=(u, 0.0, 0.0))
        fp.pattern_seeds = (1000003 * seed + 2 * i, 1000003 * seed + 2 * i + 1)
        out.append(fp)
    return out


def batch_patterns(fp):
    """The seeded ~20-cell up/down domain patterns of both films of a batch pair."""
    return pma_domains(fp.n_base, fp.pattern_seeds[0]), pma_domains(fp.n_slider, fp.pattern_seeds[1])
