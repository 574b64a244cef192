"""GB300 library for guaranteed upper-lower bounds on homogenized conductivity.

The compute path is the sm_103a shared library ``_build/libhomb.so`` (C ABI in
``include/homb.h``); ``binding`` marshals arguments to it and ``Bounds`` owns a
context and a torch-allocated device workspace. Importing this package without the
built library raises ImportError: there is no CPU fallback.
"""
from __future__ import annotations

from . import binding
from .binding import (HOM_BALL, HOM_BOX, HOM_DUAL, HOM_FF, HOM_FP32, HOM_FP64, HOM_MIXED, HOM_PRIMAL,
                      HombError, hom_batched_workspace_size, hom_bounds, hom_bounds_batched, hom_coefficient, hom_create, hom_destroy, hom_energy,
                      hom_fft, hom_kernel_timing, hom_last_error, hom_matvec, hom_problem_info,
                      hom_profile_kernel, hom_rhs, hom_set_slab_pass, hom_step_workspace_size, hom_version,
                      hom_workspace_size, make_opts)

__all__ = ["binding", "Bounds", "HombError", "hom_bounds", "hom_bounds_batched", "hom_batched_workspace_size",
           "hom_coefficient", "hom_create",
           "hom_destroy", "hom_energy", "hom_fft", "hom_kernel_timing", "hom_last_error",
           "hom_matvec", "hom_problem_info", "hom_profile_kernel", "hom_rhs", "hom_set_slab_pass",
           "hom_step_workspace_size", "hom_version", "hom_workspace_size", "make_opts",
           "HOM_FP64", "HOM_MIXED", "HOM_FP32", "HOM_FF", "HOM_PRIMAL", "HOM_DUAL", "HOM_BOX", "HOM_BALL"]


class Bounds:
    """Guaranteed bounds through hom_bounds with a reusable device workspace.

    >>> solver = Bounds(device=0)
    >>> out = solver(problem, precision=HOM_FP64, tol=1e-8)   # dict(upper, lower, mean, D, report)
    """

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device
        self.ctx = hom_create(device)
        self.ws = None

    def workspace(self, nbytes: int):
        torch = self.torch
        if self.ws is None or self.ws.numel() < nbytes:
            self.ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=f"cuda:{self.device}")
        return self.ws

    def __call__(self, problem, precision=HOM_FP64, tol=1e-8, max_iter=10000, check_every=8, sides=3,
                 stream=None, graph=0, dual_start=0, discretization=0, x0=None, fields=None, net=None):
        """hom_bounds on one problem; graph=-1 launches every CG kernel directly instead of
        replaying blocks of check_every iterations from captured CUDA graphs; dual_start=1
        starts the dual CG from the primal minimisers; discretization=1 runs GaNi (the
        paper's algorithm: N-grid CG, double-grid bounds; adds gani_A, gani_B). x0 / fields:
        optional complex128 device tensors [2, d, d, Nz, Ny, (N1+1)//2] of starting / converged
        fields (a start is projected and scaled by Rayleigh-Ritz). net: a network handle
        (binding.hom_net_load): the library computes the learned start itself."""
        opts = make_opts(precision, tol, max_iter, check_every, sides, graph, dual_start=dual_start,
                         discretization=discretization, net=net)
        nbytes = hom_workspace_size(self.ctx, problem, opts)
        ws = self.workspace(nbytes)
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device).cuda_stream
        return hom_bounds(self.ctx, problem, opts, ws.data_ptr(), ws.numel(), s,
                          None if x0 is None else x0.data_ptr(), None if fields is None else fields.data_ptr())

    def batched(self, problems, precision=HOM_MIXED, tol=1e-4, max_iter=10000, graph=0, autotune=0,
                stream=None, x0=None, fields=None, net=None):
        """hom_bounds_batched on a list of 2D problems (one persistent launch). x0 / fields:
        optional device tensors [n, 2, 2, 2, N, (N+1)//2] complex (starting / final fields);
        net: a network handle (hom_net_load) for the learned start of every cell."""
        opts = make_opts(precision, tol, max_iter, 8, 3, graph, autotune, net=net)
        nbytes = hom_batched_workspace_size(self.ctx, problems, opts)
        ws = self.workspace(nbytes)
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device).cuda_stream
        return hom_bounds_batched(self.ctx, problems, opts, ws.data_ptr(), ws.numel(), s,
                                  None if x0 is None else x0.data_ptr(),
                                  None if fields is None else fields.data_ptr())

    def close(self):
        if self.ctx is not None:
            hom_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
