"""Seeded particle sets and interaction lists shaped like the paper's workloads.

Every generator takes an explicit seed and draws from numpy's PCG64, so the
CUDA path and the FP64 oracle see bit-identical inputs. Positions are FP64,
C-contiguous ``(n, 3)`` arrays; masses are FP64 ``(n,)`` arrays.

The shapes follow the paper: Plummer spheres for the Newton accuracy and
performance runs (Section 4.1, Section 5.1), log-spaced pair separations for
the tabulated-force accuracy run (Section 4.2), and tree-style groups that
share one interaction list (Section 5.1, the Ni/Nj study). The larger sets
are the benchmark workloads: a Plummer sphere mixed with a uniform cube, a
clustered periodic box, and tree-style groups with particle and monopole
lists. Nothing here computes a force, a table or a distance bin.
"""

from __future__ import annotations

import numpy as np

# Seed of the synthetic input for each workload (1000 + workload number).
CONFIG_SEEDS = {1: 1001, 2: 1002, 3: 1003, 4: 1004, 5: 1005}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """n random unit vectors, uniform on the sphere."""
    mu = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    return np.stack([st * np.cos(ph), st * np.sin(ph), mu], axis=1)


def unit_vectors(n: int, seed: int) -> np.ndarray:
    """n isotropic unit 3-vectors (the loss weights w_i of the gradient runs)."""
    return np.ascontiguousarray(_isotropic(_rng(seed), n))


def plummer(n: int, seed: int, a: float = 1.0, total_mass: float = 1.0,
            xmax: float = 0.999):
    """Plummer sphere by inverse-CDF sampling of the enclosed mass.

    The enclosed-mass fraction X is drawn from (0, xmax] and inverted as
    r = a / sqrt(X^(-2/3) - 1); the cap xmax = 0.999 drops the far tail
    (r above about 38.7 a). Directions are isotropic and masses equal.
    """
    rng = _rng(seed)
    X = xmax * (1.0 - rng.random(n))  # (0, xmax]
    r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    x = r[:, None] * _isotropic(rng, n)
    m = np.full(n, total_mass / n)
    return np.ascontiguousarray(x), m


def _king_density(W):
    """King (1966) density in units of its value at W = 1 scale: zero for
    W <= 0, else e^W erf(sqrt W) - sqrt(4 W / pi) (1 + 2 W / 3)."""
    from scipy.special import erf
    W = np.maximum(np.asarray(W, dtype=np.float64), 0.0)
    return np.exp(W) * erf(np.sqrt(W)) - np.sqrt(4.0 * W / np.pi) * (1.0 + 2.0 * W / 3.0)


def king_profile(W0: float = 9.0, npts: int = 4000):
    """The King model's radial structure in King radii r0 (with
    r0^2 = 9 sigma^2 / (4 pi G rho0)): integrates Poisson's equation
    W'' + 2 W' / xi = -9 rho(W) / rho(W0) from W(0) = W0, W'(0) = 0 out to
    the tidal radius where W = 0, with the enclosed mass alongside.
    Returns (xi, W, mass fraction) on a grid from near 0 to xi_t."""
    from scipy.integrate import solve_ivp
    rho0 = float(_king_density(W0))

    def rhs(xi, y):
        W, dW, _ = y
        rho = float(_king_density(W)) / rho0
        return [dW, -9.0 * rho - 2.0 * dW / xi, xi * xi * rho]

    def tidal(xi, y):
        return y[0]
    tidal.terminal = True
    tidal.direction = -1
    xi0 = 1e-6          # series start: W = W0 - 1.5 xi^2, M = xi^3 / 3
    sol = solve_ivp(rhs, (xi0, 1e6), [W0 - 1.5 * xi0 ** 2, -3.0 * xi0, xi0 ** 3 / 3.0],
                    events=tidal, dense_output=True, rtol=1e-10, atol=1e-13)
    xt = float(sol.t_events[0][0])
    xi = np.concatenate([[0.0], np.geomspace(xi0, xt, npts)])
    y = sol.sol(np.maximum(xi, xi0))
    mass = np.concatenate([[0.0], y[2, 1:]])
    mass[-1] = max(mass[-1], mass[-2])
    return xi, np.maximum(y[0], 0.0), mass / mass[-1]


def king(n: int, seed: int, W0: float = 9.0, total_mass: float = 1.0):
    """King (1966) model of central depth W0 (positions only): radii by
    inverse-CDF sampling of the enclosed mass, in King radii, out to the
    tidal radius; isotropic directions; equal masses."""
    rng = _rng(seed)
    xi, _, frac = king_profile(W0)
    keep = np.concatenate([[True], np.diff(frac) > 0])
    r = np.interp(rng.random(n), frac[keep], xi[keep])
    x = r[:, None] * _isotropic(rng, n)
    return np.ascontiguousarray(x), np.full(n, total_mass / n)


def uniform_sphere(n: int, seed: int, radius: float = 1.0, total_mass: float = 1.0):
    """Uniform-density ball of the given radius, equal masses."""
    rng = _rng(seed)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    x = r[:, None] * _isotropic(rng, n)
    return np.ascontiguousarray(x), np.full(n, total_mass / n)


def plummer_cube_mix(n: int, seed: int, side: float = 4.0,
                     mlo: float = 1e-7, mhi: float = 1e-5):
    """Half a Plummer sphere, half uniform in a cube of the given side.

    The cube is centred on the origin. Masses are log-uniform in [mlo, mhi]
    and renormalised to sum to 1. The two halves are shuffled together, so
    the array order carries no spatial coherence.
    """
    rng = _rng(seed)
    nh = n // 2
    xp, _ = plummer(nh, seed + 7919)
    xc = rng.uniform(-0.5 * side, 0.5 * side, (n - nh, 3))
    x = np.concatenate([xp, xc])
    m = np.exp(rng.uniform(np.log(mlo), np.log(mhi), n))
    m /= m.sum()
    perm = rng.permutation(n)
    return np.ascontiguousarray(x[perm]), np.ascontiguousarray(m[perm])


def clustered_box(n: int, seed: int, clump_frac: float = 0.3, nclump: int = 200,
                  sigma: float = 0.005, periodic: bool = True):
    """Unit box: a uniform background plus Gaussian clumps.

    (1 - clump_frac) of the particles are uniform in [0, 1)^3. The rest are
    split as evenly as possible among ``nclump`` centres drawn uniformly in
    the box, with per-axis Gaussian offsets of width ``sigma``. With
    ``periodic`` the clump particles are wrapped back into the box. Masses
    are equal (1/n). The array is shuffled.
    """
    rng = _rng(seed)
    nc = int(round(clump_frac * n))
    nu = n - nc
    xu = rng.random((nu, 3))
    centres = rng.random((nclump, 3))
    owner = np.arange(nc) % nclump
    xc = centres[owner] + sigma * rng.standard_normal((nc, 3))
    if periodic:
        xc = np.mod(xc, 1.0)
    x = np.concatenate([xu, xc])
    perm = rng.permutation(n)
    return np.ascontiguousarray(x[perm]), np.full(n, 1.0 / n)


def _spread_bits21(v: np.ndarray) -> np.ndarray:
    """Insert two zero bits between each of the low 21 bits of v (uint64)."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_order(x: np.ndarray) -> np.ndarray:
    """Permutation that sorts points along a 63-bit Morton curve of their box."""
    lo = x.min(axis=0)
    span = max(float((x.max(axis=0) - lo).max()), 1e-300)
    q = np.clip(((x - lo) / span) * (2**21 - 1), 0, 2**21 - 1).astype(np.uint64)
    key = (_spread_bits21(q[:, 0]) << np.uint64(2)) | \
          (_spread_bits21(q[:, 1]) << np.uint64(1)) | _spread_bits21(q[:, 2])
    return np.argsort(key, kind="stable")


def _log_uniform_int(rng, lo: int, hi: int, size: int) -> np.ndarray:
    v = np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


def tree_groups(seed: int, n: int = 1 << 22, ngroups: int = 20000,
                ni_range=(16, 512), nj_range=(1024, 16384),
                particle_frac: float = 0.7, n_monopoles: int = 1 << 20):
    """Tree-style batched work: i-groups that each carry their own j-list.

    A clustered, non-periodic set of ``n`` particles is put in Morton order.
    A pool of ``n_monopoles`` pseudo-particles is built, each at the
    mass-weighted centre of a random Morton-contiguous run of 8-64 particles
    and carrying the run's summed mass. Each group takes a log-uniform number
    of i-particles from a Morton-contiguous run (groups are spread along the
    curve), and a log-uniform j-list length. A fraction ``particle_frac`` of
    the list is a Morton window of particles around the group (including the
    group itself); the rest are monopoles sampled with an even stride over
    the pool. The j array is particles followed by monopoles, and ``jlist``
    indexes into it.

    Returns a dict with xj, mj (the j array), xi (the concatenated i-groups),
    i_src (index of each i-particle in the particle array), i_off, j_off
    (CSR offsets, int64) and jlist (int32).
    """
    rng = _rng(seed)
    xp, mp = clustered_box(n, seed + 104729, periodic=False)
    order = morton_order(xp)
    xp = np.ascontiguousarray(xp[order])
    mp = np.ascontiguousarray(mp[order])

    # monopole pool
    run = rng.integers(8, 65, n_monopoles)
    start = rng.integers(0, n - 64, n_monopoles)
    cm = np.concatenate([[0.0], np.cumsum(mp)])
    cmx = np.concatenate([np.zeros((1, 3)), np.cumsum(mp[:, None] * xp, axis=0)])
    msum = cm[start + run] - cm[start]
    xmono = (cmx[start + run] - cmx[start]) / msum[:, None]
    mo = np.argsort(start, kind="stable")
    xmono, msum = xmono[mo], msum[mo]

    xj = np.ascontiguousarray(np.concatenate([xp, xmono]))
    mj = np.ascontiguousarray(np.concatenate([mp, msum]))

    ni = _log_uniform_int(rng, ni_range[0], ni_range[1], ngroups)
    nj = _log_uniform_int(rng, nj_range[0], nj_range[1], ngroups)
    gstart = (np.arange(ngroups, dtype=np.int64) * (n - ni_range[1])) // ngroups
    i_off = np.zeros(ngroups + 1, dtype=np.int64)
    i_off[1:] = np.cumsum(ni)
    i_src = np.concatenate([np.arange(s, s + k) for s, k in zip(gstart, ni)])
    xi = np.ascontiguousarray(xp[i_src])

    npart = np.rint(particle_frac * nj).astype(np.int64)
    nmono = nj - npart
    phase = rng.integers(0, n_monopoles, ngroups)
    lists = []
    for g in range(ngroups):
        c = gstart[g] + ni[g] // 2
        w0 = int(np.clip(c - npart[g] // 2, 0, n - npart[g]))
        pl = np.arange(w0, w0 + npart[g], dtype=np.int64)
        ml = n + (phase[g] + (np.arange(nmono[g], dtype=np.int64) * n_monopoles) // max(nmono[g], 1)) % n_monopoles
        lists.append(pl)
        lists.append(ml)
    jlist = np.concatenate(lists).astype(np.int32)
    j_off = np.zeros(ngroups + 1, dtype=np.int64)
    j_off[1:] = np.cumsum(nj)
    return dict(xj=xj, mj=mj, xi=xi, i_src=i_src, i_off=i_off, j_off=j_off,
                jlist=jlist, ni=ni, nj=nj)


def log_pairs(npairs: int, seed: int, lo: float = 5e-3, hi: float = 1.0):
    """Pair separation vectors with |d| / r_cut log-uniform in (lo, hi).

    Returned in units of r_cut; directions are isotropic (Section 4.2 setup).
    """
    rng = _rng(seed)
    r = np.exp(rng.uniform(np.log(lo), np.log(hi), npairs))
    return np.ascontiguousarray(r[:, None] * _isotropic(rng, npairs))


def sample_indices(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct indices out of n, sorted (the subsample the oracle checks)."""
    return np.sort(_rng(seed).choice(n, size=min(k, n), replace=False)).astype(np.int64)
