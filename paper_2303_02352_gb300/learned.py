"""Learned l1-Jacobi damping: the network, its training through the V-cycle
adjoint, and the selection that keeps it only where it beats plain l1-Jacobi.

The damping omega_i in (0, 2) of row i on level k multiplies the l1-Jacobi
diagonal, D_i = omega_i / M_ii (M_ii = sum_j |a_ij|, Sec. 3.1).  A network
4 -> 32 -> 32 -> 1 (ReLU, omega = 2 sigmoid) maps the row features of
``amg_features`` to omega.  Weights are kept as float32 master copies and used
in bf16; the forward and backward passes of the network, the adjoint of the
V-cycle and the Adam update are the library's CUDA kernels (C ABI); PyTorch
only holds device memory and chains the autograd Functions.

Training objective: the mean log residual-reduction factor of m stationary
V-cycle steps, L = (1/m) ln(|r_m| / |r_0|), r_{t+1} = r_t - A B(omega) r_t,
on random-coefficient diffusion problems built by the method's own setup.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import amg as _amg

NPARAM = 1249
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "omega_mlp.npz")


def init_theta(seed: int = 0) -> np.ndarray:
    """He-style initial weights (seeded); the last layer is zero, so omega = 1
    everywhere before training (plain l1-Jacobi, bit for bit)."""
    rng = np.random.default_rng(seed)
    t = np.zeros(NPARAM, dtype=np.float32)
    t[:128] = rng.standard_normal(128) * np.sqrt(2.0 / 4)
    t[160:160 + 1024] = rng.standard_normal(1024) * np.sqrt(2.0 / 32)
    return t


def _lib():
    return _amg.load()


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Network:
    """bf16 network weights with float32 master copy and Adam state (device)."""

    def __init__(self, theta: np.ndarray | None = None, device="cuda"):
        import torch
        self.torch = torch
        th = init_theta() if theta is None else np.asarray(theta, dtype=np.float32)
        self.theta = torch.tensor(th, dtype=torch.float32, device=device)
        self.w = self.theta.to(torch.bfloat16)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.t = 0

    def omega(self, feats):
        """omega (float64, n) for features (float32, n x 4): amg_mlp_forward."""
        return MLPFn.apply(feats, self.theta, self.w)

    def adam_step(self, grad, lr=3e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        st = _lib().amg_adam_step(NPARAM, self.theta.data_ptr(), grad.data_ptr(), self.m.data_ptr(),
                                  self.v.data_ptr(), self.w.data_ptr(), lr, beta1, beta2, eps, self.t, _stream())
        if st != 0:
            raise RuntimeError(f"amg_adam_step failed ({st})")

    def save(self, path=DEFAULT_WEIGHTS):
        os.makedirs(os.path.dirname(path), exist_ok=True)
        np.savez(path, theta=self.theta.cpu().numpy(),
                 w_bf16=self.w.view(self.torch.int16).cpu().numpy())

    @classmethod
    def load(cls, path=DEFAULT_WEIGHTS, device="cuda"):
        d = np.load(path)
        net = cls(d["theta"], device=device)
        import torch
        net.w = torch.tensor(d["w_bf16"], dtype=torch.int16, device=device).view(torch.bfloat16)
        return net


def _autograd():
    import torch

    class MLPFn(torch.autograd.Function):
        """omega = network(feats); gradient with respect to the master weights."""

        @staticmethod
        def forward(ctx, feats, theta, w):
            n = feats.shape[0]
            om = torch.empty(n, dtype=torch.float64, device=feats.device)
            st = _lib().amg_mlp_forward(n, feats.data_ptr(), w.data_ptr(), om.data_ptr(), _stream())
            if st != 0:
                raise RuntimeError(f"amg_mlp_forward failed ({st})")
            ctx.save_for_backward(feats, w)
            return om

        @staticmethod
        def backward(ctx, dom):
            feats, w = ctx.saved_tensors
            n = feats.shape[0]
            dom = dom.contiguous().to(torch.float64)
            grad = torch.empty(NPARAM, dtype=torch.float32, device=feats.device)
            ws = torch.empty(int(_lib().amg_mlp_workspace_bytes(n)), dtype=torch.uint8, device=feats.device)
            st = _lib().amg_mlp_backward(n, feats.data_ptr(), w.data_ptr(), dom.data_ptr(), grad.data_ptr(),
                                         ws.data_ptr(), _stream())
            if st != 0:
                raise RuntimeError(f"amg_mlp_backward failed ({st})")
            return None, grad, None

    class VCycleFn(torch.autograd.Function):
        """z = B(omega) r through amg_vcycle; backward through amg_vcycle_backward."""

        @staticmethod
        def forward(ctx, h, r, *omegas):
            for k, om in enumerate(omegas):
                h.set_omega(k, om.detach())
            z = h.vcycle(r.detach())
            ctx.h = h
            ctx.save_for_backward(r, *omegas)
            return z

        @staticmethod
        def backward(ctx, dz):
            r, *omegas = ctx.saved_tensors
            h = ctx.h
            for k, om in enumerate(omegas):
                h.set_omega(k, om.detach())
            dr, dom = h.vcycle_backward(r.detach(), dz.contiguous())
            return (None, dr, *dom)

    class SpMVFn(torch.autograd.Function):
        """y = A x on level 0 (A symmetric: the adjoint is the same product)."""

        @staticmethod
        def forward(ctx, h, x):
            ctx.h = h
            return h.spmv(0, x.detach())

        @staticmethod
        def backward(ctx, dy):
            return None, ctx.h.spmv(0, dy.contiguous())

    class LossFn(torch.autograd.Function):
        """(1/m) ln(|r_m| / |r_0|), r_{t+1} = r_t - A B(omega) r_t, with its
        gradient in every level's damping: both computed by the library
        (amg_vcycle_loss); the function only hands them to autograd."""

        @staticmethod
        def forward(ctx, h, r0, m, *omegas):
            for k, om in enumerate(omegas):
                h.set_omega(k, om.detach())
            loss, dom = h.vcycle_loss(r0.detach(), m, grad=True)
            ctx.dom = dom
            return torch.tensor(loss, dtype=torch.float64, device=r0.device)

        @staticmethod
        def backward(ctx, g):
            return (None, None, None, *[d * g for d in ctx.dom])

    return MLPFn, VCycleFn, SpMVFn, LossFn


MLPFn, VCycleFn, SpMVFn, LossFn = _autograd()


def level_features(h):
    return [h.features(k) for k in range(h.num_levels)]


def stationary_loss(h, omegas, r0, m: int):
    """(1/m) ln(|r_m| / |r_0|) with r_{t+1} = r_t - A B(omega) r_t: the loss and
    its gradient in the dampings come from the library (amg_vcycle_loss)."""
    return LossFn.apply(h, r0, m, *omegas)


def train(problems, steps: int = 200, m: int = 3, lr: float = 3e-3, seed: int = 0, net: Network | None = None,
          log=None):
    """Trains the network on hierarchies built by the library.  problems: list
    of CSR matrices.  Returns (net, losses)."""
    import torch
    from . import workloads as W
    net = net or Network(init_theta(seed))
    hs = [_amg.Hierarchy(A) for A in problems]
    feats = [level_features(h) for h in hs]
    losses = []
    for step in range(steps):
        p = step % len(hs)
        h = hs[p]
        r0 = torch.as_tensor(W.random_vector(h.n, 7919 * seed + step), device="cuda")
        theta = net.theta.detach().requires_grad_(True)
        omegas = [MLPFn.apply(f, theta, net.w) for f in feats[p]]
        loss = stationary_loss(h, omegas, r0, m)
        loss.backward()
        net.adam_step(theta.grad.contiguous(), lr=lr)
        losses.append(float(loss.detach()))
        if log and step % 10 == 0:
            log(f"step {step} problem {p} loss {losses[-1]:.4f}")
    for h in hs:
        h.close()
    return net, losses


def choose_damping(A, b, net: Network, tol=1e-6, maxit=1000, **params):
    """Solves with plain l1-Jacobi and with the learned damping; keeps the
    learned one only if it needs no more iterations.  Returns a dict."""
    import torch
    h = _amg.Hierarchy(A, **params)
    bt = torch.as_tensor(b, device="cuda")
    plain = h.pcg_solve(bt, tol=tol, maxit=maxit)
    h.apply_mlp(net.w)
    learned = h.pcg_solve(bt, tol=tol, maxit=maxit)
    use = learned["iters"] <= plain["iters"] and learned["status"] == 0
    if not use:
        h.apply_mlp(None)
    return {"handle": h, "plain_iters": plain["iters"], "learned_iters": learned["iters"], "use_learned": use,
            "plain": plain, "learned": learned}
