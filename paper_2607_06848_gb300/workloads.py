"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module draws random numbers and builds geometries; it holds none of the
method's arithmetic.  Everything here is a plain function of a seed.

Workloads (shaped like the paper's Sec. IV systems; the paper's geometries and
pseudopotentials are not available, so seeded stand-ins are used):
  dimer      2 atoms 2.2 bohr apart at the centre of a 16-bohr cube, Z = 4,
             8^3 cells of degree 4, 8 states, filter degree 20.
  atom       1 atom on the centre node of the dimer's mesh (partially filled
             p shell at 500 K).
  cluster64  64 atoms (Z = 4) placed uniformly at random in [6, 34]^3 with
             pairwise distance >= 4.2 bohr, 40-bohr cube, 24^3 cells of
             degree 6, 154 states, filter degree 30.
  cluster512 512 atoms in an 80-bohr cube, 40^3 cells of degree 5, 1230 states.
"""
import numpy as np


def place_atoms(n_atoms, lo, hi, min_dist, seed, max_tries=2_000_000):
    """Rejection-sample n_atoms positions uniform in [lo, hi]^3, pairwise >= min_dist."""
    rng = np.random.default_rng(seed)
    pos = np.empty((0, 3))
    tries = 0
    while len(pos) < n_atoms:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place atoms")
        p = rng.uniform(lo, hi, size=3)
        if len(pos) == 0 or np.min(np.sum((pos - p) ** 2, axis=1)) >= min_dist ** 2:
            pos = np.vstack([pos, p])
    return pos


def projector_strengths(n_atoms, seed):
    """h_{I,l} for l = s, p drawn uniformly from [-2, 2] Ha: shape (n_atoms, 2)."""
    return np.random.default_rng(seed).uniform(-2.0, 2.0, size=(n_atoms, 2))


def random_block(rows, cols, seed):
    """Seeded N(0, 1) block of shape (rows, cols), row-major float64."""
    return np.random.default_rng(seed).standard_normal((rows, cols))


def dimer(seed=0):
    """The 2-atom workload (8^3 cells, degree 4)."""
    L = 16.0
    atoms = np.array([[L / 2 - 1.1, L / 2, L / 2], [L / 2 + 1.1, L / 2, L / 2]])
    return dict(name="dimer", h=2.0, ncell=(8, 8, 8), p=4, atoms=atoms,
                Z=np.full(2, 4.0), hproj=projector_strengths(2, seed), nstates=8,
                cheb_degree=20)


def single_atom(seed=0):
    """One atom (Z = 4) on the centre node of the dimer's mesh (8^3 cells of
    degree 4 in a 16-bohr cube).  The mesh, the enrichment and the projectors
    are symmetric under the cube's rotations about that node, so the p level
    is 3-fold degenerate and holds 2 of the 4 electrons: the Fermi level
    falls inside the shell and every p state is occupied 1/3 (F != E)."""
    L = 16.0
    return dict(name="atom", h=2.0, ncell=(8, 8, 8), p=4, atoms=np.array([[L / 2, L / 2, L / 2]]),
                Z=np.full(1, 4.0), hproj=projector_strengths(1, seed), nstates=8, cheb_degree=20)


def cluster(n_atoms, side, ncell, p, nstates, cheb_degree, seed=0, margin=6.0,
            min_dist=4.2, name=None):
    atoms = place_atoms(n_atoms, margin, side - margin, min_dist, seed)
    return dict(name=name or f"cluster{n_atoms}", h=side / ncell, ncell=(ncell,) * 3, p=p,
                atoms=atoms, Z=np.full(n_atoms, 4.0),
                hproj=projector_strengths(n_atoms, seed + 1), nstates=nstates,
                cheb_degree=cheb_degree)


def cluster64(seed=0):
    return cluster(64, 40.0, 24, 6, 154, 30, seed=seed, name="cluster64")


def cluster64_species(seed=0):
    """cluster64 with one element's projector strengths on every atom (the paper's
    clusters are of one element); its SCF converges, while random strengths per atom
    make a disordered system whose density sloshes between the atoms."""
    w = cluster64(seed)
    w["hproj"] = species_strengths(64)
    w["name"] = "cluster64_species"
    return w


def cluster512(seed=0):
    return cluster(512, 80.0, 40, 5, 1230, 30, seed=seed, name="cluster512")


def small_cluster(n_atoms, seed, h=2.0, p=4, pad=7.0, min_dist=4.2):
    """8-32 atom training clusters: box = extent + 2*pad rounded up to a multiple of h."""
    side0 = 4.2 * (n_atoms ** (1.0 / 3.0)) * 1.3
    rel = place_atoms(n_atoms, 0.0, side0, min_dist, seed)
    ext = rel.max(axis=0) - rel.min(axis=0)
    ncell = tuple(int(np.ceil((e + 2 * pad) / h)) for e in ext)
    box = np.array(ncell) * h
    atoms = rel - rel.min(axis=0) + (box - ext) / 2.0
    return dict(name=f"small{n_atoms}_{seed}", h=h, ncell=ncell, p=p, atoms=atoms,
                Z=np.full(n_atoms, 4.0), hproj=projector_strengths(n_atoms, seed + 1),
                nstates=int(np.ceil(1.2 * 2 * n_atoms)), cheb_degree=20)


def quad_points(h, ncell, nq):
    """Gauss points of every cell in the library's order (cell-major, then q), shape (n, 3)."""
    xq, _ = np.polynomial.legendre.leggauss(nq)
    t = h * (xq + 1.0) / 2.0
    nx, ny, nz = ncell
    QZ, QY, QX = np.meshgrid(t, t, t, indexing="ij")
    loc = np.stack([QX.ravel(), QY.ravel(), QZ.ravel()], axis=1)          # (nq^3, 3)
    c = np.arange(nx * ny * nz)
    org = np.stack([c % nx, (c // nx) % ny, c // (nx * ny)], axis=1) * h   # (ncell, 3)
    return (org[:, None, :] + loc[None, :, :]).reshape(-1, 3)


def soft_coulomb_potential(points, atoms, depth=3.0, soft=0.5):
    """A smooth seeded stand-in potential: -sum_I depth / sqrt(soft + |x - R_I|^2)."""
    v = np.zeros(len(points))
    for a in atoms:
        v -= depth / np.sqrt(soft + np.sum((points - a) ** 2, axis=1))
    return v


def cluster8(seed=0):
    """A small case with the 64-atom cluster's discretisation (h = 40/24, p = 6,
    154 vectors): 8 atoms in a 20-bohr cube, 12^3 cells -- inputs above the L2
    size but only a few GB on the device (profiling captures)."""
    return cluster(8, 20.0, 12, 6, 154, 30, seed=seed, name="cluster8")


# learned warm start: parameter vector layout of the 32 -> 128 -> 128 -> 128 -> 8 network
MLP_LAYERS = ((128, 32), (128, 128), (128, 128), (8, 128))
MLP_N_TRAIN = sum(m * n + m for m, n in MLP_LAYERS)          # 38,280
MLP_N_PARAMS = MLP_N_TRAIN + 2 * 32 + 2 * 8                 # + x_mean, x_std, y_mean, y_std


def mlp_init(seed):
    """Seeded initial parameters: weights and biases U(-1/sqrt(fan_in), 1/sqrt(fan_in)),
    layer by layer ([out][in] row-major weights, then biases); normalisation
    x_mean = y_mean = 0, x_std = y_std = 1."""
    rng = np.random.default_rng(seed)
    parts = []
    for m, n in MLP_LAYERS:
        s = 1.0 / np.sqrt(n)
        parts.append(rng.uniform(-s, s, size=m * n))
        parts.append(rng.uniform(-s, s, size=m))
    parts += [np.zeros(32), np.ones(32), np.zeros(8), np.ones(8)]
    return np.concatenate(parts)


def species_strengths(n_atoms, seed=7):
    """One element: the same seeded s and p projector strengths on every atom, (n_atoms, 2)."""
    return np.tile(projector_strengths(1, seed), (n_atoms, 1))


def ws_cluster(n_atoms, seed, h=2.0, p=4, pad=7.0):
    """Clusters of the learned warm start: small_cluster's geometry and mesh (2-bohr cells
    of degree 4, box = extent + 14 bohr) with one element's projector strengths on every
    atom.  Training clusters use seeds 1000-1299, held-out ones 2000-2019."""
    w = small_cluster(n_atoms, seed, h=h, p=p, pad=pad)
    w["hproj"] = species_strengths(n_atoms)
    w["name"] = f"ws{n_atoms}_{seed}"
    return w
