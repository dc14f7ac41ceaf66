"""Python binding of the pg C ABI (include/pg.h): the GB300 pairwise-force
library for the force loop of Phantom-GRAPE (Tanikawa et al., arXiv:1203.4037).

Every ``pg_*`` function here has the name and argument order of the C entry
point and does argument marshalling only; all the work runs in the CUDA
library ``libpg.so`` built in-tree by :func:`build`. If that library is
missing the import of any entry point raises: there is no CPU fallback.

``Context`` is a small convenience wrapper that accepts numpy arrays (host
entry points) or CUDA torch tensors (``*_dev`` entry points).
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

PG_OK, PG_EINVAL, PG_ESTATE, PG_ENOMEM, PG_ECUDA, PG_ETIMEOUT = 0, -1, -2, -3, -4, -5
PG_NEWTON, PG_TABLE = 0, 1
PG_PATH_AUTO, PG_PATH_TILED, PG_PATH_NARROW = 0, 1, 2
PG_SPLIT_GAUSS, PG_SPLIT_S2 = 0, 1
PG_DIFF_AUTO, PG_DIFF_SINGLE, PG_DIFF_DOUBLE = 0, 1, 2
PG_TREE_WALK_AUTO, PG_TREE_WALK_LEVEL, PG_TREE_WALK_QUEUE = 0, 1, 512
PG_FFT_AUTO, PG_FFT_LIBRARY = 0, 1

STATUS_NAMES = {0: "PG_OK", -1: "PG_EINVAL", -2: "PG_ESTATE", -3: "PG_ENOMEM", -4: "PG_ECUDA",
                -5: "PG_ETIMEOUT"}

LIB_PATH = _build.LIB
HEADER = os.path.join(_build.INCLUDE, "pg.h")

_P = C.c_void_p
_LL = C.c_longlong
_D = C.c_double
_I = C.c_int
GFUNC = C.CFUNCTYPE(C.c_double, C.c_double, C.c_void_p)

# C signatures, in the order of include/pg.h
SIGNATURES = {
    "pg_create": (_I, [C.POINTER(_P), _I]),
    "pg_destroy": (None, [_P]),
    "pg_set_stream": (_I, [_P, _P]),
    "pg_set_eps": (_I, [_P, _D]),
    "pg_set_mode": (_I, [_P, _I]),
    "pg_set_table": (_I, [_P, GFUNC, _P, _D, _I, _I]),
    "pg_set_table_values": (_I, [_P, _P, _LL, _D, _I, _I]),
    "pg_set_table_values_dev": (_I, [_P, _P, _LL, _D, _I, _I]),
    "pg_get_table": (_I, [_P, _P, _P, _LL]),
    "pg_set_n": (_I, [_P, _LL]),
    "pg_set_j": (_I, [_P, _LL, _LL, _P, _P]),
    "pg_set_j_dev": (_I, [_P, _LL, _LL, _P, _P]),
    "pg_set_i": (_I, [_P, _LL, _P]),
    "pg_set_i_dev": (_I, [_P, _LL, _P]),
    "pg_set_self": (_I, [_P, _I]),
    "pg_set_self_offset": (_I, [_P, _LL]),
    "pg_set_j_rec_dev": (_I, [_P, _LL, _LL, _P]),
    "pg_set_groups": (_I, [_P, _LL, _P, _P, _P]),
    "pg_clear_groups": (_I, [_P]),
    "pg_set_periodic": (_I, [_P, _D]),
    "pg_run": (_I, [_P]),
    "pg_get_force": (_I, [_P, _P, _P, _LL]),
    "pg_run_dev": (_I, [_P, _P, _P]),
    "pg_backward_dev": (_I, [_P, _P, _P, _P, _P]),
    "pg_sync": (_I, [_P]),
    "pg_set_graph": (_I, [_P, _I]),
    "pg_tune": (_I, [_P]),
    "pg_set_shape": (_I, [_P, _I, _I, _I]),
    "pg_set_split": (_I, [_P, _I]),
    "pg_set_differencing": (_I, [_P, _I]),
    "pg_set_groups_tile": (_I, [_P, _I, _I]),
    "pg_selftest_wait": (_I, [_P, _D]),
    "pg_set_allpairs_path": (_I, [_P, _I]),
    "pg_set_eps_i": (_I, [_P, _P, _LL]),
    "pg_set_eps_i_dev": (_I, [_P, _P, _LL]),
    "pg_set_table_pot": (_I, [_P, GFUNC, _P]),
    "pg_set_table_pot_values": (_I, [_P, _P, _LL]),
    "pg_set_tree": (_I, [_P, _D, _I, _I]),
    "pg_set_tree_quadrupole": (_I, [_P, _I]),
    "pg_set_tree_walk": (_I, [_P, _I]),
    "pg_set_pm_fft": (_I, [_P, _I]),
    "pg_get_pm_fft": (_I, [_P, _P]),
    "pg_get_tree_stats": (_I, [_P, _P, _I]),
    "pg_get_tree_pseudo": (_I, [_P, _P]),
    "pg_set_pm": (_I, [_P, _I, _I, _D]),
    "pg_pm_forces": (_I, [_P, _P, _P, _LL, _P, _P]),
    "pg_pm_forces_dev": (_I, [_P, _P, _P, _LL, _P, _P]),
    "pg_pm_deposit_dev": (_I, [_P, _P, _P, _LL, _P]),
    "pg_pm_solve_dev": (_I, [_P, _P, _P, _LL, _P, _P]),
    "pg_get_tree": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "pg_set_timing": (_I, [_P, _I]),
    "pg_kernel_time": (_I, [_P, C.POINTER(_D)]),
    "pg_info": (_I, [_P, C.POINTER(_LL), _I]),
    "pg_microbench": (_I, [_I, C.POINTER(_D), C.POINTER(_D)]),
    "pg_newton_allpairs_noalloc": (_I, [_P, _P, _LL, _D, _P, _P, _P]),
    "pg_last_error": (C.c_char_p, [_P]),
    "pg_version": (C.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


class PGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile libpg.so for sm_103a (nvcc) unless it is up to date."""
    return _build.build(force=force)


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"pg CUDA library missing at {LIB_PATH}: run "
                                   "paper_1203_4037_gb300.build() (there is no CPU fallback)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    """Address of a numpy array, a torch tensor, an int, or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _check(ctx, rc):
    if rc != PG_OK:
        msg = lib().pg_last_error(ctx)
        raise PGError(rc, msg.decode() if msg else "")
    return rc


# ----------------------------------------------------------- C entry points

def pg_create(device: int = 0):
    h = _P()
    rc = lib().pg_create(C.byref(h), device)
    if rc != PG_OK:
        raise PGError(rc, lib().pg_last_error(None).decode())
    return h


def pg_destroy(ctx):
    lib().pg_destroy(ctx)


def pg_set_stream(ctx, stream):
    return _check(ctx, lib().pg_set_stream(ctx, _ptr(stream)))


def pg_set_eps(ctx, eps):
    return _check(ctx, lib().pg_set_eps(ctx, float(eps)))


def pg_set_mode(ctx, mode):
    return _check(ctx, lib().pg_set_mode(ctx, int(mode)))


def pg_set_table(ctx, g, r_cut, E, F, user=None):
    """g(r) -> f(r)/r, a Python callable evaluated at the table's knots."""
    cb = GFUNC(lambda r, _u: float(g(r)))
    return _check(ctx, lib().pg_set_table(ctx, cb, user, float(r_cut), int(E), int(F)))


def pg_set_table_values(ctx, v, r_cut, E, F):
    v = np.ascontiguousarray(v, dtype=np.float32)
    return _check(ctx, lib().pg_set_table_values(ctx, _ptr(v), len(v), float(r_cut), int(E), int(F)))


def pg_set_table_values_dev(ctx, v, n, r_cut, E, F):
    return _check(ctx, lib().pg_set_table_values_dev(ctx, _ptr(v), int(n), float(r_cut), int(E),
                                                     int(F)))


def pg_set_table_pot(ctx, p, user=None):
    """p(r) -> psi(r), the potential shape, at the force table's knots;
    None drops the potential."""
    cb = GFUNC(lambda r, _u: float(p(r))) if p is not None else GFUNC()
    return _check(ctx, lib().pg_set_table_pot(ctx, cb, user))


def pg_set_table_pot_values(ctx, v):
    v = np.ascontiguousarray(v, dtype=np.float32)
    return _check(ctx, lib().pg_set_table_pot_values(ctx, _ptr(v), len(v)))


def pg_set_tree(ctx, theta, ncrit=64, nleaf=8):
    return _check(ctx, lib().pg_set_tree(ctx, float(theta), int(ncrit), int(nleaf)))


def pg_set_tree_quadrupole(ctx, on):
    return _check(ctx, lib().pg_set_tree_quadrupole(ctx, int(bool(on))))


def pg_set_tree_walk(ctx, mode):
    return _check(ctx, lib().pg_set_tree_walk(ctx, int(mode)))


def pg_get_tree_stats(ctx):
    """The last tree run's execution: walk (1 group, 2 level), exact (1 if
    counts were read back between stages), queue_peak, reads."""
    out = np.zeros(4, dtype=np.int64)
    _check(ctx, lib().pg_get_tree_stats(ctx, _ptr(out), 4))
    return dict(walk=int(out[0]), exact=int(out[1]), queue_peak=int(out[2]), reads=int(out[3]))


def pg_get_tree(ctx):
    """The last tree run: dict of sizes, perm, g_i0, g_ni, j_off, jlist."""
    sizes = np.zeros(6, dtype=np.int64)
    _check(ctx, lib().pg_get_tree(ctx, _ptr(sizes), None, None, None, None, None))
    n, nnodes, ng, nl, nitems, npseudo = (int(v) for v in sizes)
    out = dict(n=n, nnodes=nnodes, ngroups=ng, nlist=nl, nitems=nitems, npseudo=npseudo,
               perm=np.empty(n, np.int64), g_i0=np.empty(ng, np.int64),
               g_ni=np.empty(ng, np.int64), j_off=np.empty(ng + 1, np.int64),
               jlist=np.empty(max(nl, 1), np.int64))
    _check(ctx, lib().pg_get_tree(ctx, _ptr(sizes), _ptr(out["perm"]), _ptr(out["g_i0"]),
                                  _ptr(out["g_ni"]), _ptr(out["j_off"]), _ptr(out["jlist"])))
    out["jlist"] = out["jlist"][:nl]
    return out


def pg_get_tree_pseudo(ctx, nnodes, npseudo):
    """The last tree run's pseudo-particles, (nnodes * npseudo, 4): x, y, z, m."""
    out = np.empty((max(nnodes * npseudo, 1), 4))
    _check(ctx, lib().pg_get_tree_pseudo(ctx, _ptr(out)))
    return out[:nnodes * npseudo]


def pg_set_pm(ctx, ngrid, split=PG_SPLIT_GAUSS, scale=0.0):
    return _check(ctx, lib().pg_set_pm(ctx, int(ngrid), int(split), float(scale)))


def pg_set_pm_fft(ctx, mode):
    return _check(ctx, lib().pg_set_pm_fft(ctx, int(mode)))


def pg_get_pm_fft(ctx):
    """Which FFT the last PM solve used: 1 hand-written, 2 cuFFT, 0 none."""
    k = C.c_int(0)
    _check(ctx, lib().pg_get_pm_fft(ctx, C.byref(k)))
    return int(k.value)


def pg_pm_forces(ctx, x, m):
    """The PM long-range acceleration (n, 3) and potential (n,) of host arrays."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    m = np.ascontiguousarray(m, dtype=np.float64)
    a = np.empty_like(x)
    p = np.empty(len(x))
    _check(ctx, lib().pg_pm_forces(ctx, _ptr(x), _ptr(m), len(x), _ptr(a), _ptr(p)))
    return a, p


def pg_pm_forces_dev(ctx, x, m, n, a, p=None):
    return _check(ctx, lib().pg_pm_forces_dev(ctx, _ptr(x), _ptr(m), int(n), _ptr(a),
                                              _ptr(p) if p is not None else None))


def pg_pm_deposit_dev(ctx, x, m, n, rho):
    return _check(ctx, lib().pg_pm_deposit_dev(ctx, _ptr(x), _ptr(m), int(n), _ptr(rho)))


def pg_pm_solve_dev(ctx, rho, x, n, a, p=None):
    return _check(ctx, lib().pg_pm_solve_dev(ctx, _ptr(rho), _ptr(x), int(n), _ptr(a),
                                             _ptr(p) if p is not None else None))


def pg_set_eps_i(ctx, eps):
    """Softening per i-particle (host array), or None for the global eps."""
    if eps is None:
        return _check(ctx, lib().pg_set_eps_i(ctx, None, 0))
    e = np.ascontiguousarray(eps, dtype=np.float64)
    return _check(ctx, lib().pg_set_eps_i(ctx, _ptr(e), len(e)))


def pg_set_eps_i_dev(ctx, eps, n):
    return _check(ctx, lib().pg_set_eps_i_dev(ctx, _ptr(eps), int(n)))


def pg_get_table(ctx, n):
    G0 = np.empty(n, dtype=np.float32)
    G1 = np.empty(n, dtype=np.float32)
    _check(ctx, lib().pg_get_table(ctx, _ptr(G0), _ptr(G1), int(n)))
    return G0, G1


def pg_set_n(ctx, nj):
    return _check(ctx, lib().pg_set_n(ctx, int(nj)))


def _host_f64(a, cols=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def pg_set_j(ctx, adr, x, m):
    x = _host_f64(x, 3)
    m = _host_f64(m)
    assert len(m) == len(x)
    return _check(ctx, lib().pg_set_j(ctx, int(adr), len(x), _ptr(x), _ptr(m)))


def pg_set_j_dev(ctx, adr, nj, x, m):
    return _check(ctx, lib().pg_set_j_dev(ctx, int(adr), int(nj), _ptr(x), _ptr(m)))


def pg_set_j_rec_dev(ctx, adr, nj, rec):
    return _check(ctx, lib().pg_set_j_rec_dev(ctx, int(adr), int(nj), _ptr(rec)))


def pg_set_self_offset(ctx, lo):
    return _check(ctx, lib().pg_set_self_offset(ctx, int(lo)))


def pg_set_i(ctx, x):
    x = _host_f64(x, 3)
    return _check(ctx, lib().pg_set_i(ctx, len(x), _ptr(x)))


def pg_set_i_dev(ctx, ni, x):
    return _check(ctx, lib().pg_set_i_dev(ctx, int(ni), _ptr(x)))


def pg_set_self(ctx, on):
    return _check(ctx, lib().pg_set_self(ctx, int(bool(on))))


def pg_set_groups(ctx, i_off, j_off, jlist):
    i_off = np.ascontiguousarray(i_off, dtype=np.int64)
    j_off = np.ascontiguousarray(j_off, dtype=np.int64)
    jlist = np.ascontiguousarray(jlist, dtype=np.int32)
    return _check(ctx, lib().pg_set_groups(ctx, len(i_off) - 1, _ptr(i_off), _ptr(j_off),
                                           _ptr(jlist)))


def pg_clear_groups(ctx):
    return _check(ctx, lib().pg_clear_groups(ctx))


def pg_set_periodic(ctx, box):
    return _check(ctx, lib().pg_set_periodic(ctx, float(box)))


def pg_run(ctx):
    return _check(ctx, lib().pg_run(ctx))


def pg_get_force(ctx, ni, want_phi=True, out=None):
    """The last results as (a, phi) numpy arrays; out = (a, phi) writes into
    the caller's arrays (contiguous float64; phi may be None), which may be
    page-locked, as from torch's pin_memory(), for a direct copy."""
    if out is not None:
        a, phi = out
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                and a.shape == (ni, 3)):
            raise ValueError("out[0] must be a contiguous float64 array of shape (ni, 3)")
        if phi is not None and not (isinstance(phi, np.ndarray) and phi.dtype == np.float64
                                    and phi.flags.c_contiguous and phi.shape == (ni,)):
            raise ValueError("out[1] must be a contiguous float64 array of shape (ni,) or None")
    else:
        a = np.empty((ni, 3), dtype=np.float64)
        phi = np.empty(ni, dtype=np.float64) if want_phi else None
    _check(ctx, lib().pg_get_force(ctx, _ptr(a), _ptr(phi), int(ni)))
    return a, phi


def pg_run_dev(ctx, a, phi=None):
    return _check(ctx, lib().pg_run_dev(ctx, _ptr(a), _ptr(phi)))


def pg_backward_dev(ctx, w, dx, dm, dv=None):
    return _check(ctx, lib().pg_backward_dev(ctx, _ptr(w), _ptr(dx), _ptr(dm), _ptr(dv)))


def pg_sync(ctx):
    return _check(ctx, lib().pg_sync(ctx))


def pg_set_graph(ctx, on):
    return _check(ctx, lib().pg_set_graph(ctx, int(bool(on))))


def pg_tune(ctx):
    return _check(ctx, lib().pg_tune(ctx))


def pg_set_allpairs_path(ctx, path):
    return _check(ctx, lib().pg_set_allpairs_path(ctx, int(path)))


def pg_set_shape(ctx, np_, ctas_per_sm=0, packed=-1):
    return _check(ctx, lib().pg_set_shape(ctx, int(np_), int(ctas_per_sm), int(packed)))


def pg_set_timing(ctx, on):
    return _check(ctx, lib().pg_set_timing(ctx, int(bool(on))))


def pg_kernel_time(ctx):
    ms = C.c_double()
    _check(ctx, lib().pg_kernel_time(ctx, C.byref(ms)))
    return ms.value


def pg_selftest_wait(ctx, limit_ms):
    return _check(ctx, lib().pg_selftest_wait(ctx, float(limit_ms)))


def pg_set_split(ctx, items_per_warp):
    return _check(ctx, lib().pg_set_split(ctx, int(items_per_warp)))


def pg_set_differencing(ctx, mode):
    return _check(ctx, lib().pg_set_differencing(ctx, int(mode)))


def pg_set_groups_tile(ctx, tj, nt):
    return _check(ctx, lib().pg_set_groups_tile(ctx, int(tj), int(nt)))


def pg_info(ctx):
    out = (_LL * 10)()
    n = lib().pg_info(ctx, out, 10)
    keys = ["pairs", "launches", "i_per_thread", "grid", "slots", "packed", "split", "df",
            "j_tile", "block_threads"]
    return dict(zip(keys[:n], list(out)[:n]))


def pg_microbench(kind):
    """(rate per SM per clock, rate per second) of: 0 FFMA, 1 FFMA2 lane ops,
    2 MUFU rsqrt, 3 Newton pair-term interactions with register operands,
    4 random 8-byte gathers from a 4096-entry shared-memory table, 5 the
    same from four interleaved shared copies, 6 the same through the
    read-only global path."""
    a, b = C.c_double(), C.c_double()
    rc = lib().pg_microbench(int(kind), C.byref(a), C.byref(b))
    if rc != PG_OK:
        raise PGError(rc, "microbenchmark failed")
    return a.value, b.value


PG_NOALLOC_MAX_N = 16384


def pg_newton_allpairs_noalloc(x, m, n, eps, a, phi=None, stream=None):
    """All-pairs Newton through the entry point that allocates nothing (for
    callers that cannot allocate device memory when they need forces).
    x, m, a, phi: CUDA tensors (or device addresses); n <= PG_NOALLOC_MAX_N."""
    rc = lib().pg_newton_allpairs_noalloc(_ptr(x), _ptr(m), int(n), float(eps), _ptr(a), _ptr(phi),
                                          _ptr(stream))
    if rc != PG_OK:
        why = (f"n = {n} exceeds PG_NOALLOC_MAX_N = {PG_NOALLOC_MAX_N}" if n > PG_NOALLOC_MAX_N
               else "bad argument or CUDA launch failure")
        raise PGError(rc, why)
    return rc


def pg_last_error(ctx):
    s = lib().pg_last_error(ctx)
    return s.decode() if s else ""


def pg_version():
    return lib().pg_version().decode()


# ----------------------------------------------------------- convenience

class Context:
    """Owns one pg context; host arrays are numpy, device arrays torch CUDA."""

    def __init__(self, device: int = 0):
        self.h = pg_create(device)
        self._keep = []

    def close(self):
        if self.h:
            pg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # thin forwards
    def set_stream(self, stream):
        pg_set_stream(self.h, stream)

    def set_eps(self, eps):
        pg_set_eps(self.h, eps)

    def set_mode(self, mode):
        pg_set_mode(self.h, mode)

    def set_table(self, g, r_cut, E, F):
        pg_set_table(self.h, g, r_cut, E, F)

    def set_table_pot(self, p):
        pg_set_table_pot(self.h, p)

    def set_table_pot_values(self, v):
        pg_set_table_pot_values(self.h, v)

    def set_eps_i(self, eps):
        pg_set_eps_i(self.h, eps)

    def set_tree(self, theta, ncrit=64, nleaf=8, quadrupole=False):
        pg_set_tree(self.h, theta, ncrit, nleaf)
        pg_set_tree_quadrupole(self.h, quadrupole)

    def set_tree_walk(self, mode):
        pg_set_tree_walk(self.h, mode)

    def tree_stats(self):
        return pg_get_tree_stats(self.h)

    def get_tree(self):
        t = pg_get_tree(self.h)
        t["pseudo"] = pg_get_tree_pseudo(self.h, t["nnodes"], t["npseudo"])
        return t

    def set_eps_i_dev(self, eps):
        _require_dev(eps)
        pg_set_eps_i_dev(self.h, eps, eps.shape[0])

    def set_table_values(self, v, r_cut, E, F):
        pg_set_table_values(self.h, v, r_cut, E, F)

    def set_table_values_dev(self, v, r_cut, E, F):
        pg_set_table_values_dev(self.h, v, v.numel(), r_cut, E, F)

    def get_table(self, n):
        return pg_get_table(self.h, n)

    def set_n(self, nj):
        pg_set_n(self.h, nj)

    def set_j(self, x, m, adr=0):
        pg_set_j(self.h, adr, x, m)

    def set_j_dev(self, x, m, adr=0):
        _require_dev(x, m)
        pg_set_j_dev(self.h, adr, x.shape[0], x, m)

    def set_i(self, x):
        pg_set_i(self.h, x)

    def set_i_dev(self, x):
        _require_dev(x)
        pg_set_i_dev(self.h, x.shape[0], x)

    def set_self(self, on=True):
        pg_set_self(self.h, on)

    def set_self_offset(self, lo):
        pg_set_self_offset(self.h, lo)

    def set_j_rec_dev(self, rec, adr=0):
        """j records as a CUDA float64 tensor (n, 4): x, y, z, m."""
        _require_dev(rec)
        if str(rec.dtype) != "torch.float64" or rec.dim() != 2 or rec.shape[1] != 4:
            raise ValueError("rec must be a contiguous float64 (n, 4) tensor")
        pg_set_j_rec_dev(self.h, adr, rec.shape[0], rec)

    def set_groups(self, i_off, j_off, jlist):
        pg_set_groups(self.h, i_off, j_off, jlist)

    def clear_groups(self):
        pg_clear_groups(self.h)

    def set_periodic(self, box):
        pg_set_periodic(self.h, box)

    def set_pm(self, ngrid, split=PG_SPLIT_GAUSS, scale=0.0):
        pg_set_pm(self.h, ngrid, split, scale)

    def set_pm_fft(self, mode):
        pg_set_pm_fft(self.h, mode)

    def pm_fft(self):
        return pg_get_pm_fft(self.h)

    def pm_forces(self, x, m):
        return pg_pm_forces(self.h, x, m)

    def pm_forces_dev(self, x, m, a, p=None):
        _require_dev(x, m, a, *([p] if p is not None else []))
        pg_pm_forces_dev(self.h, x, m, x.shape[0], a, p)

    def pm_deposit_dev(self, x, m, rho):
        """Density mesh (ngrid^3 FP32 CUDA tensor) of these particles."""
        _require_dev(x, m)
        pg_pm_deposit_dev(self.h, x, m, x.shape[0], rho)

    def pm_solve_dev(self, rho, x, a, p=None):
        """Mesh forces at x from a density mesh (summed over ranks)."""
        _require_dev(x, a, *([p] if p is not None else []))
        pg_pm_solve_dev(self.h, rho, x, x.shape[0], a, p)

    def pm_forces_sharded(self, x, m, ngrid, group=None):
        """Mesh forces of this rank's particles (CUDA tensors) when the
        particles are split across the ranks of torch.distributed: the
        density meshes are summed with one all-reduce."""
        import torch
        import torch.distributed as dist
        from .multirank import mesh_forces_sharded

        def deposit(xl, ml):
            rho = torch.empty(ngrid ** 3, dtype=torch.float32, device=xl.device)
            self.pm_deposit_dev(xl, ml, rho)
            return rho

        def solve(rho, xl):
            a = torch.empty_like(xl)
            p = torch.empty(xl.shape[0], dtype=xl.dtype, device=xl.device)
            self.pm_solve_dev(rho, xl, a, p)
            return a, p

        def all_reduce(rho):
            if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
                dist.all_reduce(rho, group=group)

        return mesh_forces_sharded(deposit, solve, all_reduce, x, m)

    def set_graph(self, on=True):
        pg_set_graph(self.h, on)

    def set_allpairs_path(self, path):
        pg_set_allpairs_path(self.h, path)

    def set_shape(self, np_, ctas_per_sm=0, packed=-1):
        pg_set_shape(self.h, np_, ctas_per_sm, packed)

    def set_split(self, items_per_warp):
        pg_set_split(self.h, items_per_warp)

    def set_differencing(self, mode):
        pg_set_differencing(self.h, mode)

    def set_groups_tile(self, tj, nt):
        pg_set_groups_tile(self.h, tj, nt)

    def selftest_wait(self, limit_ms):
        pg_selftest_wait(self.h, limit_ms)

    def set_timing(self, on=True):
        pg_set_timing(self.h, on)

    def kernel_time(self):
        return pg_kernel_time(self.h)

    def tune(self):
        pg_tune(self.h)

    def info(self):
        return pg_info(self.h)

    def run(self):
        pg_run(self.h)

    def get_force(self, ni, want_phi=True, out=None):
        return pg_get_force(self.h, ni, want_phi, out)

    def run_dev(self, a, phi=None):
        _require_dev(a, *([phi] if phi is not None else []))
        pg_run_dev(self.h, a, phi)

    def backward_dev(self, w, dx, dm, dv=None):
        pg_backward_dev(self.h, w, dx, dm, dv)

    def sync(self):
        pg_sync(self.h)

    # one call: host in, host out (the GRAPE-5 style sequence of Section 3.6)
    def forces(self, xi, xj=None, mj=None):
        if xj is not None:
            self.set_j(xj, mj)
        self.set_i(xi)
        self.run()
        return self.get_force(len(np.asarray(xi).reshape(-1, 3)))


def _require_dev(*ts):
    for t in ts:
        if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
            raise ValueError("device entry points take contiguous CUDA tensors")
        if t.dtype.is_floating_point and t.element_size() == 4:
            continue
        if str(t.dtype) not in ("torch.float64", "torch.float32"):
            raise ValueError(f"unexpected dtype {t.dtype}")


def exported_symbols():
    """Names of the entry points declared in include/pg.h."""
    import re
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(pg_[a-z_]+)\s*\(", txt)))
