"""Discrete adjoint of the BDF integration (test infrastructure, oracle).

The paper has no sensitivity analysis; this is the method the library adds,
written out plainly.  It differentiates the frozen-step map of an adaptive run:
the accepted steps (end time t_m, size h_m, order q_m) are fixed, and each
step's implicit BDF equation

    R_m = alpha_0^m y_m + sum_{i=1..q_m} alpha_i^m y_{m-i} - h_m f(y_m; k) = 0

(alpha from the nodes t_m, t_{m-1}, ..., as in oracle.bdf) is solved exactly.
For Phi = c^T y_N the Lagrangian conditions give, backwards in m,

    (alpha_0^m I - h_m J(y_m))^T lambda_m = c [m = N] - sum_{m'} alpha_{m'-m}^{m'} lambda_{m'}

over the later steps m' that reach back to y_m (m' - m <= q_{m'}), and

    dPhi / d log k_j = sum_m h_m R_j(y_m) (S^T lambda_m)_j,

because f = S R and R_j is proportional to k_j.  `forward_sensitivity` is the
independent tangent-linear version of the same map (one column per reaction),
and `frozen_forward` with perturbed k gives finite differences; both pin the
adjoint.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .bdf import BDFOptions, bdf_alphas, integrate_cell, lagrange_weights
from .kinetics import jacobian, reaction_rates
from .network import stoichiometry


def record_steps(desc, k, y0, t_end, opts: BDFOptions = BDFOptions()):
    """Adaptive run; returns the accepted steps [(t_m, h_m, q_m)], m = 1..N."""
    res = integrate_cell(desc, k, y0, t_end, opts, record=True)
    steps = []
    for e in res.log:
        if e["outcome"] == "accept":
            t_new = min(e["t"] + e["h"], t_end) if e["t"] + e["h"] < t_end else t_end
            steps.append((t_new, e["h"], e["q"]))
    return steps, res


def frozen_forward(desc, k, y0, steps, S=None, tol=1e-14, max_iter=30):
    """States y_0..y_N of the frozen-step map (full Newton to `tol`)."""
    if S is None:
        S = stoichiometry(desc)
    k = np.asarray(k, dtype=float)
    n = desc.n_s

    def f(y):
        return S @ reaction_rates(desc, k, y)

    Y, T = [np.array(y0, dtype=float)], [0.0]
    out = [Y[0].copy()]
    for (t_new, h, q) in steps:
        tau = [t_new] + T[:q]
        alpha = bdf_alphas(tau, h)
        psi = sum(alpha[i] * Y[i - 1] for i in range(1, q + 1))
        if len(Y) > q:
            wts = lagrange_weights(T[: q + 1], t_new)
            y = sum(wts[i] * Y[i] for i in range(q + 1))
        else:
            y = Y[0] + h * f(Y[0])
        for _ in range(max_iter):
            G = alpha[0] * y + psi - h * f(y)
            M = alpha[0] * np.eye(n) - h * jacobian(desc, k, y, S)
            delta = np.linalg.solve(M, -G)
            y = y + delta
            if np.max(np.abs(delta) / (np.abs(y) + 1e-300)) <= tol:
                break
        Y.insert(0, y)
        T.insert(0, t_new)
        del Y[6:]
        del T[6:]
        out.append(y.copy())
    return out


def _alphas_all(steps):
    """alpha^m for every step m = 1..N, recomputed from the step times."""
    T = [0.0]
    res = []
    for (t_new, h, q) in steps:
        res.append(bdf_alphas([t_new] + T[:q], h))
        T.insert(0, t_new)
        del T[6:]
    return res


def adjoint(desc, k, ys, steps, cot, S=None, with_y0=False):
    """dPhi/d log k (one row per cotangent) for Phi = cot^T y_N; with
    `with_y0` also dPhi/dy_0, the same backward recursion taken one step
    further: y_0 enters the equations of the steps m' with m' <= q_{m'}
    through alpha_{m'}^{m'} y_0, so dPhi/dy_0 = -sum_{m'} alpha_{m'}^{m'} lambda_{m'}."""
    if S is None:
        S = stoichiometry(desc)
    k = np.asarray(k, dtype=float)
    cot = np.atleast_2d(np.asarray(cot, dtype=float))
    N = len(steps)
    n = desc.n_s
    alphas = _alphas_all(steps)
    lam = [None] * (N + 1)
    grad = np.zeros((cot.shape[0], desc.n_r))
    for m in range(N, 0, -1):
        t_new, h, q = steps[m - 1]
        b = cot.T.copy() if m == N else np.zeros((n, cot.shape[0]))
        for mp in range(m + 1, min(N, m + 5) + 1):
            qp = steps[mp - 1][2]
            if mp - m <= qp:
                b -= alphas[mp - 1][mp - m] * lam[mp]
        A = alphas[m - 1][0] * np.eye(n) - h * jacobian(desc, k, ys[m], S)
        lam[m] = sla.solve(A.T, b)
        R = reaction_rates(desc, k, ys[m])
        grad += h * (S.T @ lam[m]).T * R[None, :]
    if not with_y0:
        return grad
    g0 = np.zeros((n, cot.shape[0]))
    for mp in range(1, min(N, 5) + 1):
        if mp <= steps[mp - 1][2]:
            g0 -= alphas[mp - 1][mp] * lam[mp]
    return grad, g0.T


def forward_sensitivity_y0(desc, k, ys, steps, S=None):
    """dy_N / dy_0 (n_s x n_s) through the frozen map: the tangent recursion of
    `forward_sensitivity` with the identity as initial tangent and no source."""
    if S is None:
        S = stoichiometry(desc)
    k = np.asarray(k, dtype=float)
    n = desc.n_s
    alphas = _alphas_all(steps)
    sens = [np.eye(n)]
    for m, (t_new, h, q) in enumerate(steps, start=1):
        a = alphas[m - 1]
        rhs = np.zeros((n, n))
        for i in range(1, q + 1):
            rhs -= a[i] * sens[m - i]
        A = a[0] * np.eye(n) - h * jacobian(desc, k, ys[m], S)
        sens.append(np.linalg.solve(A, rhs))
    return sens[-1]


def forward_sensitivity(desc, k, ys, steps, S=None):
    """dy_N / d log k_j for every j (n_s x n_r) through the same frozen map."""
    if S is None:
        S = stoichiometry(desc)
    k = np.asarray(k, dtype=float)
    n = desc.n_s
    alphas = _alphas_all(steps)
    sens = [np.zeros((n, desc.n_r))]
    for m, (t_new, h, q) in enumerate(steps, start=1):
        a = alphas[m - 1]
        rhs = h * S * reaction_rates(desc, k, ys[m])[None, :]
        for i in range(1, q + 1):
            rhs -= a[i] * sens[m - i]
        A = a[0] * np.eye(n) - h * jacobian(desc, k, ys[m], S)
        sens.append(np.linalg.solve(A, rhs))
    return sens[-1]
