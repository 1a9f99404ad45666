"""Host logic of the checkpoint-and-recompute gradient (adjoint.py), on the
CPU: trajectory_functional drives a small nonlinear stand-in for the
simulation that has the same interface (step, field, set_accel,
refresh_field, functional, adjoint_step, field_adjoint), with the exact
adjoint of its own step.  Its gradient must equal torch's reverse-mode
derivative of the same recursion for every checkpoint spacing and both
state policies: a state handed to the wrong adjoint step, a checkpoint
restored without its acceleration, a skipped or repeated step, or a missing
final field adjoint changes it.

The stand-in step mirrors the split step's structure: the state is (f, g);
f' = A f + C g + a f^2 + b (C g)^2 (elementwise squares: the adjoint depends
on the step-start state), then g' = B f'; g^0 = B f^0."""
from types import SimpleNamespace

import pytest
import torch

from paper_1206_6152_gb300.adjoint import trajectory_functional

N_F, M = 8, 2                # f has 8 entries, g has shape (3, 2)
A_SQ, B_SQ = 0.1, 0.05


def _mats(seed=3):
    g = torch.Generator().manual_seed(seed)
    A = 0.9 * torch.eye(N_F, dtype=torch.float64) + 0.05 * torch.randn(N_F, N_F, generator=g,
                                                                        dtype=torch.float64)
    B = 0.3 * torch.randn(3 * M, N_F, generator=g, dtype=torch.float64)
    C = 0.2 * torch.randn(N_F, 3 * M, generator=g, dtype=torch.float64)
    P = torch.randn(M, N_F, generator=g, dtype=torch.float64)
    return A, B, C, P


def _advance(A, B, C, f, g):
    cg = C @ g.reshape(-1)
    fn = A @ f + cg + A_SQ * f * f + B_SQ * cg * cg
    return fn, (B @ fn).reshape(3, M)


class StandIn:
    def __init__(self, A, B, C, P):
        self.A, self.B, self.C, self.P = A, B, C, P
        self.f = torch.zeros(N_F, dtype=torch.float64)
        self.g = torch.zeros(3, M, dtype=torch.float64)
        self.cfg = SimpleNamespace(n=(M,))
        self.steps_taken = 0
        self.adjoint_steps = 0

    def refresh_field(self):
        self.g = (self.B @ self.f).reshape(3, M)

    def field(self):
        return None, None, self.g.clone()

    def set_accel(self, g):
        self.g = g.clone()

    def step(self, n=1):
        for _ in range(n):
            fn, self.g = _advance(self.A, self.B, self.C, self.f, self.g)
            self.f.copy_(fn)
            self.steps_taken += 1

    def functional(self, kind, lam_f, target=None):
        if kind == 0:
            lam_f.copy_(self.f)
            return 0.5 * float(self.f @ self.f)
        r = self.P @ self.f - target
        lam_f.copy_(self.P.T @ r)
        return 0.5 * float(r @ r)

    def adjoint_step(self, fs, gs, lam_f, lam_g):
        mu = lam_f + self.B.T @ lam_g.reshape(-1)              # cotangent of f'
        cg = self.C @ gs.reshape(-1)
        lam_f.copy_(self.A.T @ mu + 2 * A_SQ * fs * mu)
        lam_g.copy_((self.C.T @ (mu + 2 * B_SQ * cg * mu)).reshape(3, M))
        self.adjoint_steps += 1

    def field_adjoint(self, lam_g, lam_f):
        lam_f += self.B.T @ lam_g.reshape(-1)


def _reference(A, B, C, P, f0, nsteps, kind, target):
    f = f0.clone().requires_grad_(True)
    x, g = f, (B @ f).reshape(3, M)
    for _ in range(nsteps):
        x, g = _advance(A, B, C, x, g)
    J = 0.5 * (x @ x) if kind == 0 else 0.5 * ((P @ x - target) @ (P @ x - target))
    (grad,) = torch.autograd.grad(J, f)
    return float(J.detach()), grad


@pytest.mark.parametrize("keep", [True, False, None])
@pytest.mark.parametrize("every", [1, 3, 7, 10])
@pytest.mark.parametrize("kind", [0, 1])
def test_gradient_matches_reverse_mode(keep, every, kind):
    A, B, C, P = _mats()
    gen = torch.Generator().manual_seed(7)
    f0 = 0.5 + 0.3 * torch.rand(N_F, generator=gen, dtype=torch.float64)
    target = torch.randn(M, generator=gen, dtype=torch.float64)
    nsteps = 7
    J_ref, grad_ref = _reference(A, B, C, P, f0, nsteps, kind, target)
    sim = StandIn(A, B, C, P)
    x = f0.clone().requires_grad_(True)
    J = trajectory_functional(x, sim, nsteps, every=every, kind=kind,
                              target=target if kind else None, keep_states=keep)
    assert float(J.detach()) == pytest.approx(J_ref, rel=1e-13)
    J.backward()
    torch.testing.assert_close(x.grad, grad_ref, rtol=1e-11, atol=1e-13)
    assert sim.adjoint_steps == nsteps
    # forward: nsteps; backward: each segment's states again, the last one
    # of a segment excluded (keep), or quadratic recompute (no keep)
    nseg = (nsteps + every - 1) // every
    lens = [min(every, nsteps - s * every) for s in range(nseg)]
    if keep is False:
        extra = sum(L * (L - 1) // 2 for L in lens)
    else:
        extra = sum(L - 1 for L in lens)
    assert sim.steps_taken == nsteps + extra


def test_gradient_scales_with_the_upstream_cotangent():
    A, B, C, P = _mats()
    f0 = 0.5 + 0.3 * torch.rand(N_F, generator=torch.Generator().manual_seed(9), dtype=torch.float64)
    _, grad_ref = _reference(A, B, C, P, f0, 4, 0, None)
    x = f0.clone().requires_grad_(True)
    (2.5 * trajectory_functional(x, StandIn(A, B, C, P), 4, every=2)).backward()
    torch.testing.assert_close(x.grad, 2.5 * grad_ref, rtol=1e-11, atol=1e-13)
