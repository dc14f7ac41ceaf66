"""FP64 oracle of the particle-mesh (PM) long-range force of the PPPM and
TreePM methods whose short-range (PP) part the paper's arbitrary-shape force
loop evaluates (Section 4.2): PP with f(r) = R(r, eps) - R(r, r_cut) plus PM
with R(r, r_cut) together give the full softened force; the Gaussian split
of the tabulated workloads pairs the same way.

TEST INFRASTRUCTURE: only the tests, the smoke check and the CPU baseline
of the bench use it. It shares no code with the CUDA library.

Units: G = 1, a periodic cube of side L, k = 2 pi n / L. The long-range
potential of a unit mass is phi(r) = -(4 pi / L^3) sum_{k != 0} D(k) / k^2
e^{i k . r} (a neutralising background, no k = 0 term), with the split
factor D:
  - "gauss": D(k) = exp(-k^2 r_s^2), the long range of the erf split whose
    short range is the tabulated Gaussian-split shape;
  - "s2": D(k) = S(k a)^2, S the form factor of Hockney and Eastwood's S2
    cloud of diameter a, S(q) = 12 (2 - 2 cos(q/2) - (q/2) sin(q/2)) / (q/2)^4:
    the force between two S2 clouds is R(r, a), the paper's S2 profile.

Two functions:
  - kspace_forces: the definition, a direct sum over k (small problems);
  - mesh_forces: the PM method, step by step: TSC mass assignment to an
    N^3 mesh (points at j h, h = L / N; weights 1/2 (1/2 - d)^2, 3/4 - d^2,
    1/2 (1/2 + d)^2 around the nearest point, d the offset in cells), FFT,
    multiply by -4 pi D(k) / (k^2 W(k)^2) (W the TSC window sinc^3(k_a h / 2)
    per axis, divided out once for the assignment and once for the
    interpolation; the k = 0 mode and the Nyquist planes dropped), spectral
    gradient (a_k = -i k phi_k), inverse FFTs, TSC interpolation.
"""

import numpy as np

SPLITS = ("gauss", "s2")


def split_factor(k, split, scale):
    """D(k) for |k| = k (array), the split's scale (r_s or the S2 diameter a)."""
    k = np.asarray(k, dtype=np.float64)
    if split == "gauss":
        return np.exp(-(k * scale) ** 2)
    if split == "s2":
        q = 0.5 * k * scale
        out = np.ones_like(q)
        big = q > 0.1     # below, the closed form cancels (2 - 2 cos q ~ q sin q)
        qb = q[big]
        out[big] = 12.0 * (2.0 - 2.0 * np.cos(qb) - qb * np.sin(qb)) / qb ** 4
        qs = q[~big]      # its series: 1 - q^2/15 + q^4/560 - q^6/37800
        out[~big] = 1.0 - qs ** 2 / 15.0 + qs ** 4 / 560.0 - qs ** 6 / 37800.0
        return out ** 2
    raise ValueError("split must be 'gauss' or 's2'")


def kspace_forces(x, m, L, split, scale, nmax, targets=None):
    """Long-range acceleration and potential at targets (default: the
    particles) by the direct sum over k = 2 pi n / L, 0 < |n_a| <= nmax:
    a(t) = -(4 pi / L^3) sum_j m_j sum_k D(k) k sin(k . (t - x_j)) / k^2,
    phi(t) = -(4 pi / L^3) sum_j m_j sum_k D(k) cos(k . (t - x_j)) / k^2,
    through the structure factor S(k) = sum_j m_j e^{-i k . x_j}, in chunks
    of k."""
    x = np.asarray(x, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    t = x if targets is None else np.asarray(targets, dtype=np.float64)
    n1 = np.arange(-nmax, nmax + 1)
    nv = np.stack(np.meshgrid(n1, n1, n1, indexing="ij"), -1).reshape(-1, 3)
    nv = nv[np.any(nv != 0, axis=1)]
    acc = np.zeros((len(t), 3))
    pot = np.zeros(len(t))
    c = -4.0 * np.pi / L ** 3
    for s in range(0, len(nv), 8192):
        kv = 2.0 * np.pi / L * nv[s:s + 8192]
        k2 = np.sum(kv * kv, axis=1)
        w = split_factor(np.sqrt(k2), split, scale) / k2        # D(k) / k^2
        S = np.exp(-1j * (x @ kv.T)).T @ m                       # (K,)
        e = np.exp(1j * (t @ kv.T)) * (w * S)[None, :]           # (T, K)
        acc += c * (e.imag @ kv)
        pot += c * e.real.sum(axis=1)
    return acc, pot


def _tsc(u):
    """Nearest mesh point and the three TSC weights of grid coordinate u."""
    j0 = np.floor(u + 0.5)
    d = u - j0
    w = np.stack([0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2], axis=-1)
    return j0.astype(np.int64), w


def _stencil(x, L, N):
    """Per particle: the 27 mesh indices (flattened) and weights of TSC."""
    u = np.mod(np.asarray(x, dtype=np.float64), L) * (N / L)
    j0, w = _tsc(u)                                            # (n, 3), (n, 3, 3)
    idx = np.zeros((len(u), 27), dtype=np.int64)
    wt = np.ones((len(u), 27))
    c = 0
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            for e in (-1, 0, 1):
                ix = (j0[:, 0] + a) % N
                iy = (j0[:, 1] + b) % N
                iz = (j0[:, 2] + e) % N
                idx[:, c] = (ix * N + iy) * N + iz
                wt[:, c] = w[:, 0, a + 1] * w[:, 1, b + 1] * w[:, 2, e + 1]
                c += 1
    return idx, wt


def tsc_window(N):
    """W(k)^2 on the rfft grid: prod_a sinc(k_a h / 2)^6 (TSC, twice)."""
    f = np.fft.fftfreq(N) * N            # integer n for the full axes
    fr = np.arange(N // 2 + 1)           # the halved last axis
    def s6(n):
        x = np.pi * n / N                # k h / 2
        out = np.ones_like(x, dtype=np.float64)
        nz = x != 0
        out[nz] = (np.sin(x[nz]) / x[nz]) ** 6
        return out
    return s6(f)[:, None, None] * s6(f)[None, :, None] * s6(fr)[None, None, :]


def deposit(x, m, L, N):
    """Step 1: the TSC density mesh (N, N, N) of particles x, m (mass per
    cell volume)."""
    x = np.asarray(x, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    h = L / N
    idx, wt = _stencil(x, L, N)
    rho = np.zeros(N ** 3)
    np.add.at(rho, idx.ravel(), (wt * m[:, None]).ravel())
    return rho.reshape(N, N, N) / h ** 3


def solve(rho, t, L, N, split, scale):
    """Steps 2-5: from a density mesh to the acceleration (n, 3) and
    potential (n,) at the points t."""
    rk = np.fft.rfftn(rho)
    n = np.fft.fftfreq(N) * N
    nr = np.arange(N // 2 + 1)
    kx = (2.0 * np.pi / L) * n[:, None, None]
    ky = (2.0 * np.pi / L) * n[None, :, None]
    kz = (2.0 * np.pi / L) * nr[None, None, :]
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2s = np.where(k2 > 0, k2, 1.0)
    green = np.where(k2 > 0, -4.0 * np.pi * split_factor(np.sqrt(k2), split, scale) / k2s, 0.0)
    # the Nyquist planes carry no derivative (its imaginary factor would
    # break the Hermitian symmetry there): dropped
    nyq = (np.abs(n) == N // 2)
    green = np.where(nyq[:, None, None] | nyq[None, :, None] | (nr == N // 2)[None, None, :], 0.0, green)
    phik = rk * green / tsc_window(N)
    fields = [np.fft.irfftn(-1j * kk * phik, s=(N, N, N), axes=(0, 1, 2)) for kk in (kx, ky, kz)]
    fields.append(np.fft.irfftn(phik, s=(N, N, N), axes=(0, 1, 2)))
    idx, wt = _stencil(t, L, N)
    out = [np.sum(f.ravel()[idx] * wt, axis=1) for f in fields]
    return np.stack(out[:3], axis=1), out[3]


def mesh_forces(x, m, L, N, split, scale):
    """The PM long-range acceleration (n, 3) and potential (n,) of every
    particle, FP64, by the steps listed in the module docstring."""
    return solve(deposit(x, m, L, N), x, L, N, split, scale)
