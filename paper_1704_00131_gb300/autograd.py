"""torch.autograd.Function for log|det(1 + B(beta,0))| and the energy estimator on
fixed field configurations, as functions of the hopping matrix K and of U.

The forward and backward values come from the library's adjoint kernels
(dqmc_logdet_backward, dqmc_energy_backward); this module only moves tensors.
The library treats K as symmetric and returns derivatives with K_xy and K_yx
varied together; for a full-matrix gradient (entries independent) the
off-diagonal pair derivative is split evenly between (x, y) and (y, x).
"""
from __future__ import annotations

import numpy as np
import torch

from . import dqmc
from .workloads import ModelSpec


def _pair_to_full(g: np.ndarray) -> np.ndarray:
    out = 0.5 * g
    idx = np.arange(g.shape[-1])
    out[..., idx, idx] = g[..., idx, idx]
    return out


class LogDetEnergy(torch.autograd.Function):
    """(K [N,N] float64, U scalar float64) -> (sum_s log|det(1+B^s(beta,0))| [n_cfg], Ener [n_cfg])."""

    @staticmethod
    def forward(ctx, K: torch.Tensor, U: torch.Tensor, fields: np.ndarray, dtau: float, L: int, n_wrap: int,
                field_type: int = 1):
        Kh = K.detach().to("cpu", torch.float64).numpy()
        m = ModelSpec(Kh, U=float(U.detach().cpu()), dtau=dtau, L=L, n_wrap=n_wrap, field_type=field_type)
        ens = dqmc.Ensemble([m], [0], precision="fp64")
        try:
            ld, gK_ld, gU_ld = ens.logdet_backward(0, fields)
            e, gK_e, gU_e = ens.energy_backward(0, fields)
        finally:
            ens.close()
        # one K shared by both flavors: derivatives add over flavors
        ctx.gK = (_pair_to_full(gK_ld.sum(axis=1)), _pair_to_full(gK_e.sum(axis=1)))
        ctx.gU = (gU_ld.sum(axis=1), gU_e)
        ctx.dev, ctx.dtype = K.device, K.dtype
        return (torch.as_tensor(ld.sum(axis=1), device=K.device, dtype=K.dtype),
                torch.as_tensor(e[:, 3], device=K.device, dtype=K.dtype))

    @staticmethod
    def backward(ctx, g_ld: torch.Tensor, g_e: torch.Tensor):
        a = g_ld.detach().cpu().numpy()
        b = g_e.detach().cpu().numpy()
        gK = np.einsum("c,cxy->xy", a, ctx.gK[0]) + np.einsum("c,cxy->xy", b, ctx.gK[1])
        gU = float(a @ ctx.gU[0] + b @ ctx.gU[1])
        return (torch.as_tensor(gK, device=ctx.dev, dtype=ctx.dtype), torch.as_tensor(gU, device=ctx.dev,
                                                                                        dtype=ctx.dtype),
                None, None, None, None, None)


def logdet_energy(K: torch.Tensor, U: torch.Tensor, fields: np.ndarray, dtau: float, L: int, n_wrap: int,
                  field_type: int = 1):
    return LogDetEnergy.apply(K, U, fields, dtau, L, n_wrap, field_type)
