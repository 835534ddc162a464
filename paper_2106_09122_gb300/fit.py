"""Ring-parameter retrieval through the simulator: model, loss, gradient, fit.

The paper's flow chart (Fig. 3) closes with retrieving exozodi parameters
from images; here the retrieval is gradient based.  Every arithmetic step
runs in libpsfsim (include/psfsim_fit.h): ring scene, S = A Z, float64 loss,
A^T r, chain rule.  Python only sequences the calls and takes the line
search's accept / reject decision on the float64 loss it reads back.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _binding as B
from .plan import Plan, _stream_ptr


def _vp(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


class RingProblem:
    """Device buffers for fitting theta = (R, w, i, g, B) to a target image."""

    def __init__(self, plan: Plan, N: int, S: float, r_max: float, target: torch.Tensor, sigma: float):
        self.lib = B.load()
        self.plan, self.N, self.S, self.r_max, self.sigma = plan, int(N), float(S), float(r_max), float(sigma)
        if plan.K != self.N * self.N:
            raise ValueError("plan columns must match the N x N scene")
        dev = plan.lib.device
        self.target = target.contiguous()
        f32 = dict(dtype=torch.float32, device=dev)
        self.z = torch.empty(plan.K, **f32)
        self.y = torch.empty(plan.M, **f32)
        self.r = torch.empty(plan.M, **f32)
        self.gz = torch.empty(plan.K, **f32)
        self.jac = torch.empty((5, plan.K), **f32)
        self.jy = torch.empty((5, plan.M), **f32)
        # out6 = (loss, dL/dtheta); the separate operators write straight into its views.
        self.out6 = torch.empty(6, dtype=torch.float64, device=dev)
        self.loss_d, self.dtheta = self.out6[:1], self.out6[1:]
        u8 = dict(dtype=torch.uint8, device=dev)
        self.fscr = torch.empty(max(plan.forward_scratch_bytes(5), 1), **u8)
        self.ascr = torch.empty(max(plan.adjoint_scratch_bytes(1), 1), **u8)
        nb = ctypes.c_size_t()
        B.check(self.lib.psfsim_ring_chain_scratch_bytes(self.N, ctypes.byref(nb)), "chain scratch")
        self.cscr = torch.empty(nb.value, **u8)
        B.check(self.lib.psfsim_loss_scratch_bytes(plan.M, ctypes.byref(nb)), "loss scratch")
        self.lscr = torch.empty(nb.value, **u8)
        # FP32 grid plans take the fused path (two launches per gradient, three
        # for FP32_SYM); its scratch holds arrival counters that must start at zero.
        self.fused = self.lib.psfsim_ring_gradient_scratch_bytes(plan.handle, ctypes.byref(nb)) == B.OK
        self.gscr = torch.zeros(max(nb.value, 256), **u8) if self.fused else None
        self.launches = 0

    # -- operators ---------------------------------------------------------
    def scene(self, theta, out: torch.Tensor | None = None) -> torch.Tensor:
        z = self.z if out is None else out
        th = np.ascontiguousarray(theta, dtype=np.float64)
        B.check(self.lib.psfsim_ring_scene(self.N, self.S, self.r_max, th.ctypes.data_as(ctypes.c_void_p), _vp(z),
                                           _stream_ptr(None)), "psfsim_ring_scene")
        self.launches += 1
        return z

    def chain(self, theta, gz: torch.Tensor) -> torch.Tensor:
        th = np.ascontiguousarray(theta, dtype=np.float64)
        B.check(self.lib.psfsim_ring_chain(self.N, self.S, self.r_max, th.ctypes.data_as(ctypes.c_void_p), _vp(gz),
                                           _vp(self.dtheta), _vp(self.cscr), self.cscr.numel(), _stream_ptr(None)),
                "psfsim_ring_chain")
        self.launches += 2
        return self.dtheta

    def residual_loss(self, y: torch.Tensor, target: torch.Tensor, want_residual: bool) -> torch.Tensor:
        B.check(self.lib.psfsim_residual_loss(_vp(y), _vp(target), y.numel(), self.sigma,
                                              _vp(self.r) if want_residual else None, _vp(self.loss_d),
                                              _vp(self.lscr), self.lscr.numel(), _stream_ptr(None)),
                "psfsim_residual_loss")
        self.launches += 2
        return self.loss_d

    # -- composite steps ---------------------------------------------------
    def enqueue_loss(self, theta) -> None:
        self.plan.forward(self.scene(theta), out=self.y, scratch=self.fscr)
        self.launches += 2
        self.residual_loss(self.y, self.target, False)

    def enqueue_forward_loss(self, theta) -> None:
        """First half (one launch): ring scene and Jacobian, S = A Z with residual and loss partials."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        B.check(self.lib.psfsim_ring_forward_loss(self.plan.handle, self.r_max, th.ctypes.data_as(ctypes.c_void_p),
                                                  _vp(self.target), self.sigma, _vp(self.z), _vp(self.y), _vp(self.r),
                                                  _vp(self.gscr), self.gscr.numel(), _stream_ptr(None)),
                "psfsim_ring_forward_loss")
        self.launches += 2 if self.plan.storage == "fp32_sym" else 1

    def enqueue_adjoint_chain(self, theta) -> None:
        """Second half (one launch): A^T r, its dot with the stored Jacobian, the final sums into out6."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        B.check(self.lib.psfsim_ring_adjoint_chain(self.plan.handle, self.r_max, th.ctypes.data_as(ctypes.c_void_p),
                                                   _vp(self.r), _vp(self.gz), _vp(self.out6), _vp(self.gscr),
                                                   self.gscr.numel(), _stream_ptr(None)),
                "psfsim_ring_adjoint_chain")
        self.launches += 1

    def enqueue_gradient(self, theta) -> None:
        """Ring -> forward -> loss and residual -> adjoint -> chain, all enqueued; the result lands
        in out6 = (loss, dL/dtheta)."""
        if self.fused:  # one C-ABI call enqueues both halves
            th = np.ascontiguousarray(theta, dtype=np.float64)
            B.check(self.lib.psfsim_ring_gradient(self.plan.handle, self.r_max, th.ctypes.data_as(ctypes.c_void_p),
                                                  _vp(self.target), self.sigma, _vp(self.z), _vp(self.y),
                                                  _vp(self.r), _vp(self.gz), _vp(self.out6), _vp(self.gscr),
                                                  self.gscr.numel(), _stream_ptr(None)),
                    "psfsim_ring_gradient")
            self.launches += 3 if self.plan.storage == "fp32_sym" else 2
            return
        self.plan.forward(self.scene(theta), out=self.y, scratch=self.fscr)
        self.residual_loss(self.y, self.target, True)
        self.plan.adjoint(self.r, out=self.gz, scratch=self.ascr)
        self.launches += 3
        self.chain(theta, self.gz)

    def loss(self, theta) -> float:
        self.enqueue_loss(theta)
        return float(self.loss_d.item())

    def loss_and_grad(self, theta):
        self.enqueue_gradient(theta)
        out = self.out6.cpu().numpy()
        return float(out[0]), out[1:].copy()

    def gauss_newton_diagonal(self, theta) -> np.ndarray:
        """H_mm = ||A dZ/dtheta_m||^2 / sigma^2 (float64), the Gauss-Newton diagonal.

        Used only to scale the descent direction, so each column A dZ/dtheta_m is
        taken as a central difference of two forward images of the ring kernel.
        """
        th = np.ascontiguousarray(theta, dtype=np.float64)
        out = np.empty(5)
        for m in range(5):
            h = 1e-4 * max(abs(th[m]), 1e-3 if m != 4 else abs(th[4]))
            tp, tm = th.copy(), th.copy()
            tp[m] += h
            tm[m] -= h
            self.scene(tp, out=self.jac[m])
            self.scene(tm, out=self.gz)
            self.plan.forward(self.jac[m], out=self.jy[m], scratch=self.fscr)
            self.plan.forward(self.gz, out=self.y, scratch=self.fscr)
            self.residual_loss(self.jy[m], self.y, False)
            out[m] = 2.0 * float(self.loss_d.item()) / (2.0 * h) ** 2
        return out

    def fit(self, theta0, steps: int = 200, c1: float = 1e-4, max_halvings: int = 40):
        """Preconditioned gradient descent with Armijo backtracking on the float64 loss."""
        theta = np.asarray(theta0, dtype=np.float64).copy()
        P = 1.0 / np.maximum(self.gauss_newton_diagonal(theta), 1e-300)
        loss, g = self.loss_and_grad(theta)
        hist = [loss]
        alpha = 1.0
        for _ in range(steps):
            d = -P * g
            slope = float(g @ d)
            if not slope < 0.0:
                break
            accepted = False
            for _ in range(max_halvings):
                trial = theta + alpha * d
                if trial[1] > 0 and abs(trial[3]) < 1 and abs(np.cos(trial[2])) > 1e-3:
                    lt = self.loss(trial)
                    if lt <= loss + c1 * alpha * slope:
                        accepted = True
                        break
                alpha *= 0.5
            if not accepted:
                break
            theta = trial
            loss, g = self.loss_and_grad(theta)
            hist.append(loss)
            alpha = min(alpha * 2.0, 1.0)
        return theta, np.array(hist)


class RingImage(torch.autograd.Function):
    """theta (float64 CPU [5]) -> simulated image S = A Z(theta) (CUDA float32 [M]).

    backward: dL/dtheta = (dZ/dtheta)^T A^T dL/dS through psfsim_adjoint and
    psfsim_ring_chain.
    """

    @staticmethod
    def forward(ctx, theta: torch.Tensor, problem: RingProblem):
        th = theta.detach().cpu().double().numpy()
        z = problem.scene(th, out=torch.empty_like(problem.z))
        y = problem.plan.forward(z)
        ctx.problem = problem
        ctx.theta = th
        return y

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        problem = ctx.problem
        gz = problem.plan.adjoint(gy.contiguous().float())
        dtheta = problem.chain(ctx.theta, gz).cpu().clone()
        return dtheta, None
