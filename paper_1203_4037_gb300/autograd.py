"""torch.autograd binding of the all-pairs force and its hand-written
backward kernel (an extension of the paper's method: L = sum_i w_i . a_i
differentiated with respect to positions, masses and the table's knot
values, so that a cutoff force shape can be fitted).

Forward and backward both run in the CUDA library through the C ABI
(pg_run_dev, pg_backward_dev); this module only marshals tensors.
"""

from __future__ import annotations

import torch

from . import Context, PG_NEWTON, PG_TABLE


class _Shared:
    """One pg context per (device, stream) reused across calls."""

    ctxs = {}

    @classmethod
    def get(cls, device):
        st = torch.cuda.current_stream(device)
        key = (device.index, st.cuda_stream)
        c = cls.ctxs.get(key)
        if c is None:
            c = Context(device.index or 0)
            c.set_stream(st.cuda_stream)
            c.set_self(True)
            cls.ctxs[key] = c
        return c


class PairForceFn(torch.autograd.Function):
    """a = force(x, m[, v]) for the all-pairs self mode (every particle on
    every other one). x: (n, 3) float64 CUDA, m: (n,) float64 CUDA,
    v: (2^(E+F),) float32 CUDA knot values (table mode) or None."""

    @staticmethod
    def forward(ctx, x, m, v, eps, r_cut, E, F):
        dev = x.device
        c = _Shared.get(dev)
        table = v is not None
        c.set_mode(PG_TABLE if table else PG_NEWTON)
        if table:
            c.set_table_values_dev(v.contiguous(), r_cut, E, F)
        else:
            c.set_eps(eps)
        x = x.contiguous()
        m = m.contiguous()
        c.set_j_dev(x, m)
        c.set_n(x.shape[0])      # the whole set: a smaller one than the last ends here
        c.set_i_dev(x)
        a = torch.empty_like(x)
        c.run_dev(a)
        ctx.save_for_backward(x, m, v if table else None)
        ctx.cfg = (eps, r_cut, E, F, table)
        return a

    @staticmethod
    def backward(ctx, grad_a):
        x, m, v = ctx.saved_tensors
        eps, r_cut, E, F, table = ctx.cfg
        c = _Shared.get(x.device)
        c.set_mode(PG_TABLE if table else PG_NEWTON)
        if table:
            c.set_table_values_dev(v.contiguous(), r_cut, E, F)
        else:
            c.set_eps(eps)
        c.set_j_dev(x, m)
        c.set_n(x.shape[0])
        c.set_i_dev(x)
        w = grad_a.contiguous().to(torch.float64)
        dx = torch.empty_like(x)
        dm = torch.empty_like(m)
        dv = torch.empty_like(v) if table else None
        c.backward_dev(w, dx, dm, dv)
        return dx, dm, dv, None, None, None, None


def newton_force(x, m, eps):
    """Softened Newton acceleration of every particle (Eq. 1, G = 1)."""
    return PairForceFn.apply(x, m, None, float(eps), 0.0, 0, 0)


def table_force(x, m, v, r_cut, E, F):
    """Tabulated central force (Eq. 2) with trainable knot values v."""
    return PairForceFn.apply(x, m, v, 0.0, float(r_cut), int(E), int(F))
