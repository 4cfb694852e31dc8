"""torch.autograd.Function over the C ABI's forward/adjoint sweep.

TransportReadouts.apply(mua, mus, spec) runs the explicit scheme on the GPU
from a zero state with the given optical maps (torch tensors of the grid
shape) and returns the gated detector readouts y. Its backward calls
rte_adjoint with grad_output as dL/dy and returns dL/dmu_a and dL/dmu_s.
Both directions run in librte's kernels; this module only moves arguments.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import Plan


@dataclass
class SweepSpec:
    """Everything except the two differentiated maps."""
    shape: tuple
    dx: float
    N: int
    c: float
    g: np.ndarray
    dt: float
    nsteps: int
    ckpt_every: int
    src_voxel: np.ndarray
    src_amp: np.ndarray
    src_t0: np.ndarray
    src_fwhm: np.ndarray
    det_voxel: np.ndarray
    gates: np.ndarray
    pml_cells: int = 0
    pml_mu0: float = 0.0
    pml_mu1: float = 0.0
    precision: str = "fp32"
    src_moment: np.ndarray = field(default=None)


def _torch():
    import torch
    return torch


class TransportReadouts(_torch().autograd.Function):
    @staticmethod
    def forward(ctx, mua, mus, spec: SweepSpec):
        torch = _torch()
        a = mua.detach().to("cpu", torch.float64).numpy()
        s = mus.detach().to("cpu", torch.float64).numpy()
        plan = Plan(spec.shape, spec.dx, spec.N, spec.c, a, s, spec.g, spec.pml_cells, spec.pml_mu0,
                    spec.pml_mu1, spec.precision, stream=torch.cuda.current_stream().cuda_stream)
        mom = spec.src_moment if spec.src_moment is not None else np.zeros(len(spec.src_voxel))
        plan.set_sources(spec.src_voxel, mom, spec.src_amp, spec.src_t0, spec.src_fwhm)
        plan.set_detectors(spec.det_voxel)
        y = plan.forward(spec.dt, spec.nsteps, spec.ckpt_every, spec.gates)
        ctx.plan = plan
        ctx.dev = mua.device
        return torch.from_numpy(y).to(mua.device)

    @staticmethod
    def backward(ctx, grad_y):
        torch = _torch()
        plan = ctx.plan
        ga, gs = plan.adjoint(grad_y.detach().to("cpu", torch.float64).numpy())
        plan.close()
        ctx.plan = None
        return ga.to(ctx.dev), gs.to(ctx.dev), None
