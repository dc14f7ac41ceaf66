"""FP64 CPU oracle for the Phantom-GRAPE pairwise force loop.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It wraps the plain C
files ``pg_oracle.c`` (the force loops, tables and gradients) and
``pg_tree.c`` (the grouped tree of the tree usage), built with gcc into
``liborc.so`` beside them, and the numpy module ``pm`` (the particle-mesh
long-range force); it shares no code with the CUDA library in
``paper_1203_4037_gb300``.

Every function takes and returns numpy FP64 arrays: positions ``(n, 3)``,
masses ``(n,)``. ``d_ij = x_j - x_i`` and G = 1 throughout.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))

# PG_ORACLE_PM names another copy of pm.py (the mutation tests plant
# mistakes in one), like PG_ORACLE_LIB for the compiled part
if os.environ.get("PG_ORACLE_PM"):
    import importlib.util as _ilu
    import sys as _sys

    _spec = _ilu.spec_from_file_location(__name__ + ".pm", os.environ["PG_ORACLE_PM"])
    pm = _ilu.module_from_spec(_spec)
    _sys.modules[__name__ + ".pm"] = pm
    _spec.loader.exec_module(pm)
_SRC = os.path.join(_HERE, "pg_oracle.c")
_SRC_TREE = os.path.join(_HERE, "pg_tree.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

SHAPE_NEWTON, SHAPE_GAUSS_SPLIT, SHAPE_S2PP, SHAPE_LINEAR, SHAPE_NEWTON_POT = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile pg_oracle.c and pg_tree.c into liborc.so (plain gcc, -O2, no
    fast-math, no contraction of multiply-add: every FP64 operation rounds
    on its own)."""
    srcs = [_SRC, _SRC_TREE]
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f)
                                               for f in srcs):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, *srcs,
                        "-lm", "-lpthread"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def nthreads() -> int:
    return max(1, os.cpu_count() or 1)


_P = C.c_void_p
_LL = C.c_longlong
_D = C.c_double
_I = C.c_int

_SIGS = {
    "orc_newton": (_I, [_LL, _P, _P, _LL, _P, _P, _D, _P, _P, _I]),
    "orc_newton_groups": (_I, [_LL, _P, _P, _P, _P, _P, _P, _D, _P, _P, _I]),
    "orc_s_max": (_D, [_I, _I]),
    "orc_table_size": (_LL, [_I, _I]),
    "orc_knot": (_D, [_I, _I, _LL]),
    "orc_bin": (_LL, [_I, _I, _D]),
    "orc_scale2": (_D, [_I, _I, _D]),
    "orc_s2_profile": (_D, [_D, _D]),
    "orc_shape": (_D, [_I, _P, _D]),
    "orc_table_from_values": (_I, [_I, _I, _P, _P, _P]),
    "orc_table_values": (_I, [_I, _I, _D, _I, _P, _P]),
    "orc_table_build": (_I, [_I, _I, _D, _I, _P, _P, _P]),
    "orc_table_eval": (_D, [_I, _I, _D, _P, _P, _D]),
    "orc_table_forces": (_I, [_LL, _P, _P, _LL, _P, _P, _I, _I, _D, _P, _P, _D, _D, _P, _P, _I]),
    "orc_table_potential": (_I, [_LL, _P, _P, _LL, _P, _P, _I, _I, _D, _P, _P, _D, _D, _P, _P, _I]),
    "orc_newton_epsi": (_I, [_LL, _P, _P, _P, _LL, _P, _P, _P, _P, _I]),
    "orc_tree_build": (_P, [_LL, _P, _P, _D, _I, _I, _I]),
    "orc_tree_free": (None, [_P]),
    "orc_tree_sizes": (None, [_P, _P]),
    "orc_tree_get": (None, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "orc_tree_get_nodes": (None, [_P, _P, _P, _P, _P]),
    "orc_tree_forces": (_I, [_P, _D, _P, _P]),
    "orc_shape_forces": (_I, [_LL, _P, _P, _LL, _P, _P, _I, _P, _D, _D, _D, _P, _P, _P, _I]),
    "orc_grad_newton": (_I, [_LL, _P, _P, _P, _D, _P, _P, _P, _I]),
    "orc_grad_newton_at": (_I, [_LL, _P, _P, _P, _D, _LL, _P, _P, _P, _I]),
    "orc_grad_table": (_I, [_LL, _P, _P, _P, _D, _I, _I, _D, _P, _P, _P, _P, _I]),
    "orc_grad_table_at": (_I, [_LL, _P, _P, _P, _D, _I, _I, _D, _P, _LL, _P, _P, _P, _I]),
    "orc_grad_table_v": (_I, [_LL, _P, _P, _P, _D, _I, _I, _D, _P, _P, _I]),
    "orc_fd_newton": (_I, [_LL, _P, _P, _P, _D, _LL, _I, _D, _P]),
    "orc_fd_table": (_I, [_LL, _P, _P, _P, _D, _I, _I, _D, _P, _LL, _I, _D, _P, _P]),
    "orc_fd_table_v": (_I, [_LL, _P, _P, _P, _D, _I, _I, _D, _P, _LL, _P, _D, _P, _I]),
}


def lib():
    """The compiled oracle. PG_ORACLE_LIB names another build of pg_oracle.c
    (the mutation test loads deliberately broken copies this way)."""
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(os.environ.get("PG_ORACLE_LIB") or build())
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _chk(rc):
    if rc != 0:
        raise ValueError(f"oracle call failed with code {rc}")


# ---------------------------------------------------------------- Newton

def newton(xi, xj, mj, eps, skip=None, nthreads_=None):
    """Eq. (1): acceleration (ni, 3) and potential (ni,) of i from all j.

    ``skip[i]`` names one j that i leaves out (-1: none).
    """
    xi = _f64(xi, (-1, 3)); xj = _f64(xj, (-1, 3)); mj = _f64(mj)
    ni, nj = len(xi), len(xj)
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.int64)
    acc = np.empty((ni, 3)); pot = np.empty(ni)
    _chk(lib().orc_newton(ni, _ptr(xi), _ptr(sk), nj, _ptr(xj), _ptr(mj), float(eps),
                          _ptr(acc), _ptr(pot), nthreads_ or nthreads()))
    return acc, pot


def newton_epsi(xi, eps_i, xj, mj, skip=None, nthreads_=None):
    """Eq. (1) with each i-particle's own softening eps_i (Section 3.1)."""
    xi = _f64(xi, (-1, 3)); xj = _f64(xj, (-1, 3)); mj = _f64(mj); ei = _f64(eps_i)
    ni, nj = len(xi), len(xj)
    if len(ei) != ni:
        raise ValueError("eps_i needs one value per i-particle")
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.int64)
    acc = np.empty((ni, 3)); pot = np.empty(ni)
    _chk(lib().orc_newton_epsi(ni, _ptr(xi), _ptr(ei), _ptr(sk), nj, _ptr(xj), _ptr(mj),
                               _ptr(acc), _ptr(pot), nthreads_ or nthreads()))
    return acc, pot


def newton_allpairs(x, m, eps, nthreads_=None):
    """All-pairs Newton with j = i left out (the double-precision reference
    of Section 4.1)."""
    n = len(x)
    return newton(x, x, m, eps, skip=np.arange(n, dtype=np.int64), nthreads_=nthreads_)


def newton_subset(x, m, eps, idx, nthreads_=None):
    """Newton on the subsample x[idx] from all particles, self left out."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    return newton(np.asarray(x)[idx], x, m, eps, skip=idx, nthreads_=nthreads_)


def newton_groups(i_off, j_off, jlist, xi, xj, mj, eps, nthreads_=None):
    """List mode: each group's i sum exactly the listed j (self included if listed)."""
    i_off = np.ascontiguousarray(i_off, dtype=np.int64)
    j_off = np.ascontiguousarray(j_off, dtype=np.int64)
    jlist = np.ascontiguousarray(jlist, dtype=np.int32)
    xi = _f64(xi, (-1, 3)); xj = _f64(xj, (-1, 3)); mj = _f64(mj)
    ni = len(xi)
    acc = np.empty((ni, 3)); pot = np.empty(ni)
    _chk(lib().orc_newton_groups(len(i_off) - 1, _ptr(i_off), _ptr(j_off), _ptr(jlist),
                                 _ptr(xi), _ptr(xj), _ptr(mj), float(eps), _ptr(acc),
                                 _ptr(pot), nthreads_ or nthreads()))
    return acc, pot


# ---------------------------------------------------------------- table

def s_max(E, F):
    return lib().orc_s_max(E, F)


def table_size(E, F):
    return lib().orc_table_size(E, F)


def knot(E, F, k):
    return lib().orc_knot(E, F, int(k))


def bin_index(E, F, s):
    return lib().orc_bin(E, F, float(s))


def scale2(E, F, r_cut):
    return lib().orc_scale2(E, F, float(r_cut))


def s2_profile(r, a):
    return lib().orc_s2_profile(float(r), float(a))


def shape(shape_id, par, r):
    par = _f64(par)
    return lib().orc_shape(int(shape_id), _ptr(par), float(r))


def table_values(E, F, r_cut, shape_id, par):
    """Knot values v_k = fp32(g(r_k)), k = 0 .. 2^(E+F) - 1 (v at r_cut last)."""
    par = _f64(par)
    v = np.empty(table_size(E, F), dtype=np.float32)
    _chk(lib().orc_table_values(E, F, float(r_cut), int(shape_id), _ptr(par), _ptr(v)))
    return v


def table_from_values(E, F, v):
    v = np.ascontiguousarray(v, dtype=np.float32)
    n = table_size(E, F)
    assert v.shape == (n,)
    G0 = np.empty(n, dtype=np.float32); G1 = np.empty(n, dtype=np.float32)
    _chk(lib().orc_table_from_values(E, F, _ptr(v), _ptr(G0), _ptr(G1)))
    return G0, G1


def table_build(E, F, r_cut, shape_id, par):
    """(G0, G1) FP32 arrays of length 2^(E+F) for a closed-form shape."""
    par = _f64(par)
    n = table_size(E, F)
    G0 = np.empty(n, dtype=np.float32); G1 = np.empty(n, dtype=np.float32)
    _chk(lib().orc_table_build(E, F, float(r_cut), int(shape_id), _ptr(par), _ptr(G0), _ptr(G1)))
    return G0, G1


def table_eval(E, F, r_cut, G0, G1, r2):
    G0 = np.ascontiguousarray(G0, dtype=np.float32); G1 = np.ascontiguousarray(G1, dtype=np.float32)
    return lib().orc_table_eval(E, F, float(r_cut), _ptr(G0), _ptr(G1), float(r2))


def table_forces(xi, xj, mj, E, F, r_cut, G0, G1, box=0.0, skip=None, window=0.0,
                 nthreads_=None):
    """O-T2: Eq. (2) through the table's interpolant. Returns (acc, amb)."""
    xi = _f64(xi, (-1, 3)); xj = _f64(xj, (-1, 3)); mj = _f64(mj)
    G0 = np.ascontiguousarray(G0, dtype=np.float32); G1 = np.ascontiguousarray(G1, dtype=np.float32)
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.int64)
    ni = len(xi)
    acc = np.empty((ni, 3)); amb = np.empty(ni)
    _chk(lib().orc_table_forces(ni, _ptr(xi), _ptr(sk), len(xj), _ptr(xj), _ptr(mj), E, F,
                                float(r_cut), _ptr(G0), _ptr(G1), float(box), float(window),
                                _ptr(acc), _ptr(amb), nthreads_ or nthreads()))
    return acc, amb


def table_potential(xi, xj, mj, E, F, r_cut, P0, P1, box=0.0, skip=None, window=0.0,
                    nthreads_=None):
    """Table-mode potential: phi_i = sum_j m_j psi~(s_ij) through a second
    table (P0, P1) of the same layout. Returns (phi, amb)."""
    xi = _f64(xi, (-1, 3)); xj = _f64(xj, (-1, 3)); mj = _f64(mj)
    P0 = np.ascontiguousarray(P0, dtype=np.float32); P1 = np.ascontiguousarray(P1, dtype=np.float32)
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.int64)
    ni = len(xi)
    phi = np.empty(ni); amb = np.empty(ni)
    _chk(lib().orc_table_potential(ni, _ptr(xi), _ptr(sk), len(xj), _ptr(xj), _ptr(mj), E, F,
                                   float(r_cut), _ptr(P0), _ptr(P1), float(box), float(window),
                                   _ptr(phi), _ptr(amb), nthreads_ or nthreads()))
    return phi, amb


def shape_forces(xi, xj, mj, shape_id, par, r_cut, box=0.0, skip=None, window=0.0,
                 nthreads_=None, with_absum=False):
    """O-T1: Eq. (2) with the closed-form shape, pairs with r < r_cut.
    Returns (acc, amb) or, with_absum, (acc, amb, sum_j |pair term|)."""
    xi = _f64(xi, (-1, 3)); xj = _f64(xj, (-1, 3)); mj = _f64(mj); par = _f64(par)
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.int64)
    ni = len(xi)
    acc = np.empty((ni, 3)); amb = np.empty(ni); absum = np.empty(ni)
    _chk(lib().orc_shape_forces(ni, _ptr(xi), _ptr(sk), len(xj), _ptr(xj), _ptr(mj),
                                int(shape_id), _ptr(par), float(r_cut), float(box),
                                float(window), _ptr(acc), _ptr(amb), _ptr(absum),
                                nthreads_ or nthreads()))
    return (acc, amb, absum) if with_absum else (acc, amb)


# ---------------------------------------------------------------- gradients

def grad_newton(x, m, w, eps, nthreads_=None):
    """All-pairs analytic (dL/dx (n,3), dL/dm (n,), L) for L = sum_i w_i . a_i."""
    x = _f64(x, (-1, 3)); m = _f64(m); w = _f64(w, (-1, 3))
    n = len(x)
    dx = np.empty((n, 3)); dm = np.empty(n); L = C.c_double()
    _chk(lib().orc_grad_newton(n, _ptr(x), _ptr(m), _ptr(w), float(eps), _ptr(dx), _ptr(dm),
                               C.byref(L), nthreads_ or nthreads()))
    return dx, dm, L.value


def grad_newton_at(x, m, w, eps, idx, nthreads_=None):
    x = _f64(x, (-1, 3)); m = _f64(m); w = _f64(w, (-1, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    dx = np.empty((len(idx), 3)); dm = np.empty(len(idx))
    _chk(lib().orc_grad_newton_at(len(x), _ptr(x), _ptr(m), _ptr(w), float(eps), len(idx),
                                  _ptr(idx), _ptr(dx), _ptr(dm), nthreads_ or nthreads()))
    return dx, dm


def grad_table(x, m, w, E, F, r_cut, v, box=0.0, nthreads_=None):
    x = _f64(x, (-1, 3)); m = _f64(m); w = _f64(w, (-1, 3))
    v = np.ascontiguousarray(v, dtype=np.float32)
    n = len(x)
    dx = np.empty((n, 3)); dm = np.empty(n); L = C.c_double()
    _chk(lib().orc_grad_table(n, _ptr(x), _ptr(m), _ptr(w), float(box), E, F, float(r_cut),
                              _ptr(v), _ptr(dx), _ptr(dm), C.byref(L), nthreads_ or nthreads()))
    return dx, dm, L.value


def grad_table_at(x, m, w, E, F, r_cut, v, idx, box=0.0, nthreads_=None):
    x = _f64(x, (-1, 3)); m = _f64(m); w = _f64(w, (-1, 3))
    v = np.ascontiguousarray(v, dtype=np.float32)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    dx = np.empty((len(idx), 3)); dm = np.empty(len(idx))
    _chk(lib().orc_grad_table_at(len(x), _ptr(x), _ptr(m), _ptr(w), float(box), E, F,
                                 float(r_cut), _ptr(v), len(idx), _ptr(idx), _ptr(dx),
                                 _ptr(dm), nthreads_ or nthreads()))
    return dx, dm


def grad_table_v(x, m, w, E, F, r_cut, v, box=0.0, nthreads_=None):
    x = _f64(x, (-1, 3)); m = _f64(m); w = _f64(w, (-1, 3))
    v = np.ascontiguousarray(v, dtype=np.float32)
    dv = np.empty(table_size(E, F))
    _chk(lib().orc_grad_table_v(len(x), _ptr(x), _ptr(m), _ptr(w), float(box), E, F,
                                float(r_cut), _ptr(v), _ptr(dv), nthreads_ or nthreads()))
    return dv


def fd_newton(x, m, w, eps, k, what, h=1e-6):
    """Central difference of L in x_k[what] (what = 0, 1, 2) or m_k (what = 3)."""
    x = _f64(x, (-1, 3)); m = _f64(m); w = _f64(w, (-1, 3))
    out = C.c_double()
    _chk(lib().orc_fd_newton(len(x), _ptr(x), _ptr(m), _ptr(w), float(eps), int(k), int(what),
                             float(h), C.byref(out)))
    return out.value


def fd_table(x, m, w, E, F, r_cut, v, k, what, h=1e-6, box=0.0):
    """Central difference for the table model; returns (value, kinked)."""
    x = _f64(x, (-1, 3)); m = _f64(m); w = _f64(w, (-1, 3))
    v = np.ascontiguousarray(v, dtype=np.float32)
    out = C.c_double(); kink = C.c_int()
    _chk(lib().orc_fd_table(len(x), _ptr(x), _ptr(m), _ptr(w), float(box), E, F, float(r_cut),
                            _ptr(v), int(k), int(what), float(h), C.byref(out), C.byref(kink)))
    return out.value, bool(kink.value)


def fd_table_v(x, m, w, E, F, r_cut, v, bidx, h=1e-6, box=0.0, nthreads_=None):
    x = _f64(x, (-1, 3)); m = _f64(m); w = _f64(w, (-1, 3))
    v = np.ascontiguousarray(v, dtype=np.float32)
    bidx = np.ascontiguousarray(bidx, dtype=np.int64)
    out = np.empty(len(bidx))
    _chk(lib().orc_fd_table_v(len(x), _ptr(x), _ptr(m), _ptr(w), float(box), E, F,
                              float(r_cut), _ptr(v), len(bidx), _ptr(bidx), float(h),
                              _ptr(out), nthreads_ or nthreads()))
    return out


# ---------------------------------------------------------------- tree
def tree_build(x, m, theta, ncrit, nleaf, quadrupole=False):
    """The grouped Barnes-Hut tree of Section 5.1. Returns a dict with the
    key order ``perm``, the groups (``g_i0``, ``g_ni``, ``g_node``, in key
    order), the lists (``j_off``, ``jlist``: k < n is sorted particle k,
    n + P t + q is pseudo-particle q of node t), per node the moments
    (``nM``, ``nS``, the second moment ``nT`` as xx, xy, xz, yy, yz, zz),
    ``nlevel``, ``nfirst``, ``ncount``, and the pseudo-particles
    (``pseudo``: x, y, z, m; ``npseudo`` = P, 1 for monopoles, 3 with
    quadrupoles)."""
    x = _f64(x, (-1, 3)); m = _f64(m)
    n = len(x)
    h = lib().orc_tree_build(n, _ptr(x), _ptr(m), float(theta), int(ncrit), int(nleaf),
                             int(bool(quadrupole)))
    if not h:
        raise ValueError("tree build failed")
    try:
        sz = np.zeros(5, dtype=np.int64)
        lib().orc_tree_sizes(h, _ptr(sz))
        n, nnodes, ng, nlist, npseudo = (int(v) for v in sz)
        out = dict(perm=np.empty(n, np.int64), g_i0=np.empty(ng, np.int64),
                   g_ni=np.empty(ng, np.int64), g_node=np.empty(ng, np.int64),
                   j_off=np.empty(ng + 1, np.int64), jlist=np.empty(max(nlist, 1), np.int64),
                   nM=np.empty(nnodes), nS=np.empty((nnodes, 3)),
                   nlevel=np.empty(nnodes, np.int32))
        lib().orc_tree_get(h, *(_ptr(out[k]) for k in ("perm", "g_i0", "g_ni", "g_node", "j_off",
                                                      "jlist", "nM", "nS", "nlevel")))
        out["jlist"] = out["jlist"][:nlist]
        out.update(nfirst=np.empty(nnodes, np.int64), ncount=np.empty(nnodes, np.int64),
                   nT=np.empty((nnodes, 6)), pseudo=np.empty((nnodes * npseudo, 4)),
                   npseudo=npseudo)
        lib().orc_tree_get_nodes(h, *(_ptr(out[k]) for k in ("nfirst", "ncount", "nT", "pseudo")))
        return out
    finally:
        lib().orc_tree_free(h)


def tree_forces(x, m, eps, theta, ncrit, nleaf, quadrupole=False):
    """Forces and potentials of all particles (input order) from the grouped
    tree's lists, each particle's own entry left out."""
    x = _f64(x, (-1, 3)); m = _f64(m)
    n = len(x)
    h = lib().orc_tree_build(n, _ptr(x), _ptr(m), float(theta), int(ncrit), int(nleaf),
                             int(bool(quadrupole)))
    if not h:
        raise ValueError("tree build failed")
    try:
        acc = np.empty((n, 3)); pot = np.empty(n)
        _chk(lib().orc_tree_forces(h, float(eps), _ptr(acc), _ptr(pot)))
        return acc, pot
    finally:
        lib().orc_tree_free(h)
