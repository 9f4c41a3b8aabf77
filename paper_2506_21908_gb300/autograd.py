"""torch.autograd wrapper: pulse-envelope samples -> final magnetisation, differentiated by the
library's discrete adjoint (tddft_backward).

The envelope env(t) = sum_j a_j phi_j(t) uses piecewise-linear hat functions phi_j on nodes
spread uniformly over the run.  Two drives are supported:
  * laser (velocity gauge): E(t) = env(t) cos(omega t) pol, A(t_n) = -int_0^{t_n} E dt
    (the pulse form of Sec. 4.4 with the envelope as the free function);
  * magnetic: B(t_n) = env(t_n) pol (spin Zeeman coupling, Sec. 3.4).
Both tables are linear in a, so dL/da = M^T dL/d(table) exactly, with the same matrices M
that build the tables.  The forward call runs the propagation and its adjoint together (one
library call) and keeps dL/da for the backward pass.
"""
import numpy as np
import torch

from . import _lib


def hat(t, nodes, j):
    """Piecewise-linear hat function of node j evaluated at times t."""
    y = np.zeros(len(nodes))
    y[j] = 1.0
    return np.interp(t, nodes, y)


class PulseBasis:
    def __init__(self, times, nparams, mode="laser", omega=0.057, pol=(1.0, 0.0, 0.0), nquad=16):
        self.times = np.asarray(times, np.float64)
        self.nodes = np.linspace(self.times[0], self.times[-1], nparams)
        self.pol = np.asarray(pol, np.float64)
        self.mode = mode
        nt = len(self.times)
        self.MA = np.zeros((nt, nparams))
        self.MB = np.zeros((nt, nparams))
        if mode == "laser":
            x, w = np.polynomial.legendre.leggauss(nquad)
            for i in range(1, nt):
                a, b = self.times[i - 1], self.times[i]
                tq = 0.5 * (b - a) * x + 0.5 * (b + a)
                for j in range(nparams):
                    inc = 0.5 * (b - a) * (w * hat(tq, self.nodes, j) * np.cos(omega * tq)).sum()
                    self.MA[i, j] = self.MA[i - 1, j] - inc
        elif mode == "magnetic":
            for j in range(nparams):
                self.MB[:, j] = hat(self.times, self.nodes, j)
        else:
            raise ValueError("mode must be 'laser' or 'magnetic'")

    def tables(self, a):
        a = np.asarray(a, np.float64)
        return np.outer(self.MA @ a, self.pol), np.outer(self.MB @ a, self.pol)

    def chain(self, dA, dB):
        return self.MA.T @ (dA @ self.pol) + self.MB.T @ (dB @ self.pol)


class MagnetizationFromPulse(torch.autograd.Function):
    """L = sum_r dL_drho . rho_v(T) (default use: M_z(T)) as a function of the envelope samples."""

    @staticmethod
    def forward(ctx, a, handle, psi0, basis, nsteps, dL_drho, ckpt_every=50, B_static=None, A_static=None):
        A_tab, B_tab = basis.tables(a.detach().cpu().numpy())
        if B_static is not None:
            B_tab = B_tab + np.asarray(B_static, np.float64)
        if A_static is not None:
            A_tab = A_tab + np.asarray(A_static, np.float64)
        handle.set_fields(basis.times, A_tab, B_tab)
        handle.set_states(psi0, float(basis.times[0]))
        L, dA, dB = handle.backward(nsteps, dL_drho, ckpt_every=ckpt_every, nt=len(basis.times))
        ctx.save_for_backward(torch.from_numpy(basis.chain(dA, dB)))
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        (ga,) = ctx.saved_tensors
        return (grad_out * ga,) + (None,) * 8


def mz_seed(n, L):
    """dL/drho_v for L = M_z = int m_z dV on an n^3 grid of the cell L."""
    dV = float(np.prod(L)) / n ** 3
    seed = np.zeros((4, n, n, n))
    seed[0], seed[1] = dV, -dV
    return seed


def pulse_loss(handle, psi0, basis, nsteps, a, ckpt_every=50):
    """Convenience: M_z(T) for envelope a (torch tensor with requires_grad)."""
    return MagnetizationFromPulse.apply(a, handle, psi0, basis, nsteps, mz_seed(handle.n, handle._L), ckpt_every)
