"""Variable-step, variable-order BDF integrator with simplified Newton iterations.

Test infrastructure (oracle): see the package docstring.

The paper solves the stiff system with DLSODES, a BDF code with a sparse
Jacobian, at rtol 1e-4 / atol 1e-20 (Section 3), and states nothing more about
the solver.  This file fixes one concrete BDF method, which the CUDA library
implements independently; the oracle solves each Newton system with a dense
LAPACK LU (partial pivoting), the library with its own factorisation.

Method (per cell, everything FP64):

* History: the last accepted solutions y_n, y_{n-1}, ... (at most q_max + 1)
  and their times.  Order q (1..q_max) starts at 1.
* BDF formula of order q on the nodes tau_0 = t_{n+1}, tau_i = t_{n+1-i}:
  sum_i alpha_i y(tau_i) = h f(y_{n+1}) with alpha_i = h l_i'(tau_0), l_i the
  Lagrange basis polynomials on the q + 1 nodes.
* Predictor: the degree-q interpolant of the q + 1 newest history points,
  evaluated at t_{n+1}; the very first step uses y0 + h f(y0).
* Newton: G(y) = alpha_0 y + psi - h f(y), psi = sum_{i>=1} alpha_i y_{n+1-i};
  delta = M^-1 (-G/alpha_0) with M = I - gamma_J J, gamma = h / alpha_0; when
  gamma != gamma_J delta is scaled by 2 / (1 + gamma/gamma_J).  The rate
  estimate crate = max(0.3 crate, d_m / d_{m-1}) (d = WRMS norm of delta)
  persists across steps and is reset to 1 with every new Jacobian.  Converged
  when d_m min(1, crate) <= newton_tol; failed after newton_max iterations or
  when d_m > 2 d_{m-1}.
* Jacobian refresh (J at the predicted y, then M and its factorisation): at the
  first attempt, after j_age_max accepted steps, when |gamma/gamma_J - 1| >
  gamma_tol, and after a Newton failure that used an older Jacobian.  A Newton
  failure with a fresh Jacobian cuts h by 4.
* WRMS norm: ||v|| = sqrt(mean((v_i w_i)^2)), w_i = 1/(rtol |y_n,i| + atol).
* Error test: err = C_q ||y_{n+1} - y_pred||, C_q = h / (t_{n+1} - t_{n-q})
  (1/(q+1) until the history holds q + 1 points).  err <= 1 accepts.
* Step size: eta = 0.9 err^(-1/(q+1)); on rejection eta = max(0.2, eta) and
  after three rejections in a row the order drops to 1.  After acceptance, once
  q + 1 steps were taken at order q, orders q - 1 and q + 1 are also rated:
  est_{q-1} = h/(t_{n+1} - t_{n+1-q}) ||y_{n+1} - P_{q-1}(t_{n+1})|| (P_{q-1}
  interpolating the q newest old points), eta_{q-1} = 0.8 est^(-1/q);
  est_{q+1} = ||e_n - e_{n-1}|| / (q + 2) with e = y_{n+1} - y_pred of two
  consecutive steps at order q, eta_{q+1} = 0.7 est^(-1/(q+2)).  The largest
  eta wins (ties keep q).  eta is then clipped to [0.2, eta_max] (to at most 1
  right after a rejection) and values in [1, eta_keep) are set to 1.
* The last step is shortened to land on t_end.  Abundances are never clipped
  (clipping would break the element conservation that E.S = 0 guarantees).
* Fixed-step mode (fixed_h > 0): every step has h = fixed_h and is accepted,
  and the order rises to q_max as history accumulates (used for convergence
  order tests).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .kinetics import jacobian, reaction_rates
from .network import stoichiometry

STATUS_OK, STATUS_MAXSTEPS, STATUS_HMIN, STATUS_CONV, STATUS_NAN = 0, 1, 2, 3, 4


@dataclass
class BDFOptions:
    rtol: float = 1e-6
    atol: float = 1e-20
    q_max: int = 5
    max_steps: int = 100000
    j_age_max: int = 20
    gamma_tol: float = 0.3
    newton_max: int = 4
    newton_tol: float = 0.1
    eta_max: float = 5.0
    eta_keep: float = 1.5
    max_conv_fails: int = 10
    fixed_h: float = 0.0


@dataclass
class CellResult:
    y: np.ndarray
    t: float
    status: int = STATUS_OK
    steps: int = 0
    rejects: int = 0
    conv_fails: int = 0
    newton_iters: int = 0
    jac_evals: int = 0
    h_last: float = 0.0
    q_last: int = 1
    log: list = field(default_factory=list)


def wrms(v, w) -> float:
    return float(np.sqrt(np.mean((v * w) ** 2)))


def lagrange_weights(nodes, t):
    """w_i with p(t) = sum_i w_i y_i for the polynomial through (nodes_i, y_i)."""
    n = len(nodes)
    out = []
    for i in range(n):
        num, den = 1.0, 1.0
        for m in range(n):
            if m != i:
                num *= t - nodes[m]
                den *= nodes[i] - nodes[m]
        out.append(num / den)
    return out


def bdf_alphas(tau, h):
    """alpha_i = h l_i'(tau_0) for the Lagrange basis on nodes tau_0..tau_q."""
    q = len(tau) - 1
    a = [h * sum(1.0 / (tau[0] - tau[i]) for i in range(1, q + 1))]
    for i in range(1, q + 1):
        num = 1.0
        for m in range(1, q + 1):
            if m != i:
                num *= tau[0] - tau[m]
        den = 1.0
        for m in range(q + 1):
            if m != i:
                den *= tau[i] - tau[m]
        a.append(h * num / den)
    return a


def integrate_cell(desc, k, y0, t_end, opts: BDFOptions = BDFOptions(), S=None,
                   record=False, history=None) -> CellResult:
    """Integrate one cell (k'[n_r], y0[n_s]) from t = 0 to t_end.

    `history` = (times, states), newest first with times < 0, seeds the step
    history with exact past values (fixed-step order tests only)."""
    if S is None:
        S = stoichiometry(desc)
    k = np.asarray(k, dtype=float)

    def f(y):
        return S @ reaction_rates(desc, k, y)

    def jac(y):
        return jacobian(desc, k, y, S)

    y0 = np.array(y0, dtype=float)
    if not np.all(np.isfinite(k)):
        return CellResult(y=y0.copy(), t=0.0, status=STATUS_NAN)
    return integrate_system(f, jac, y0, t_end, opts, record, history)


def integrate_system(f, jac, y0, t_end, opts: BDFOptions = BDFOptions(), record=False,
                     history=None) -> CellResult:
    """The method above for any system dy/dt = f(y) with Jacobian jac(y)
    (dense n x n), from t = 0 to t_end."""
    y0 = np.array(y0, dtype=float)
    I = np.eye(y0.shape[0])
    res = CellResult(y=y0.copy(), t=0.0)
    if not np.all(np.isfinite(y0)):
        res.status = STATUS_NAN
        return res
    Y, T = [y0.copy()], [0.0]
    if history is not None:
        for th, yh in zip(*history):
            T.append(float(th))
            Y.append(np.array(yh, dtype=float))
    f0 = f(y0)
    fixed = opts.fixed_h > 0.0
    if fixed:
        h = opts.fixed_h
    else:
        w0 = 1.0 / (opts.rtol * np.abs(y0) + opts.atol)
        h = min(0.01 / max(wrms(f0, w0), 1e-300), t_end)
    t, q, n_at_q, e_prev = 0.0, 1, 0, None
    need_J, lu, gamma_J, j_age, crate = True, None, 1.0, 0, 1.0
    rejected, consec_rej, consec_cf = False, 0, 0

    while t < t_end:
        if res.steps >= opts.max_steps:
            res.status = STATUS_MAXSTEPS
            break
        final = t + h >= t_end
        if final:
            h = t_end - t
        t_new = t_end if final else t + h
        if t_new == t or h <= 0.0:
            res.status = STATUS_HMIN
            break
        if fixed:
            q = max(1, min(opts.q_max, len(Y) - 1))
        if len(Y) == 1:
            y_pred = Y[0] + h * f0
        else:
            wts = lagrange_weights(T[: q + 1], t_new)
            y_pred = sum(wts[i] * Y[i] for i in range(q + 1))
        alpha = bdf_alphas([t_new] + T[:q], h)
        psi = sum(alpha[i] * Y[i - 1] for i in range(1, q + 1))
        gamma = h / alpha[0]
        w = 1.0 / (opts.rtol * np.abs(Y[0]) + opts.atol)
        refresh = need_J or j_age >= opts.j_age_max or abs(gamma / gamma_J - 1.0) > opts.gamma_tol
        if refresh:
            J = jac(y_pred)
            lu = sla.lu_factor(I - gamma * J)
            gamma_J, j_age, crate, need_J = gamma, 0, 1.0, False
            res.jac_evals += 1
        scale = 2.0 / (1.0 + gamma / gamma_J) if gamma != gamma_J else 1.0
        y = y_pred.copy()
        conv, d_prev, n_it = False, 0.0, 0
        for m in range(opts.newton_max):
            G = alpha[0] * y + psi - h * f(y)
            delta = sla.lu_solve(lu, -G / alpha[0]) * scale
            y = y + delta
            n_it += 1
            d = wrms(delta, w)
            if not np.isfinite(d):
                break
            if m > 0:
                crate = max(0.3 * crate, d / d_prev)
            if d * min(1.0, crate) <= opts.newton_tol:
                conv = True
                break
            if m > 0 and d > 2.0 * d_prev:
                break
            d_prev = d
        res.newton_iters += n_it
        if fixed:
            conv = True
        if not conv:
            res.conv_fails += 1
            consec_cf += 1
            if record:
                res.log.append(dict(t=t, h=h, q=q, refresh=refresh, iters=n_it, outcome="conv_fail"))
            if consec_cf >= opts.max_conv_fails:
                res.status = STATUS_CONV
                break
            if not refresh:
                need_J = True
            else:
                h *= 0.25
                need_J = True
            rejected = True
            continue
        e = y - y_pred
        Cq = h / (t_new - T[q]) if len(Y) >= q + 1 else 1.0 / (q + 1)
        err = Cq * wrms(e, w)
        if not np.isfinite(err):
            res.status = STATUS_NAN
            break
        if err > 1.0 and not fixed:
            res.rejects += 1
            consec_rej += 1
            if record:
                res.log.append(dict(t=t, h=h, q=q, refresh=refresh, iters=n_it, outcome="reject", err=err))
            eta = max(0.2, 0.9 * err ** (-1.0 / (q + 1)))
            if consec_rej >= 3 and q > 1:
                q, n_at_q, e_prev = 1, 0, None
            rejected = True
            h *= eta
            continue
        # accepted: rate the neighbouring orders against the old history
        n_at_q += 1
        best_eta = 0.9 * max(err, 1e-10) ** (-1.0 / (q + 1))
        best_q = q
        if not fixed and n_at_q >= q + 1:
            if q > 1:
                wl = lagrange_weights(T[:q], t_new)
                p_lo = sum(wl[i] * Y[i] for i in range(q))
                est = h / (t_new - T[q - 1]) * wrms(y - p_lo, w)
                eta_lo = 0.8 * max(est, 1e-10) ** (-1.0 / q)
                if eta_lo > best_eta:
                    best_eta, best_q = eta_lo, q - 1
            if q < opts.q_max and e_prev is not None and len(Y) + 1 >= q + 2:
                est = wrms(e - e_prev, w) / (q + 2)
                eta_hi = 0.7 * max(est, 1e-10) ** (-1.0 / (q + 2))
                if eta_hi > best_eta:
                    best_eta, best_q = eta_hi, q + 1
        if record:
            res.log.append(dict(t=t, h=h, q=q, refresh=refresh, iters=n_it, outcome="accept", err=err,
                                y=y.copy()))
        t = t_new
        Y.insert(0, y)
        T.insert(0, t_new)
        del Y[opts.q_max + 1:]
        del T[opts.q_max + 1:]
        res.steps += 1
        j_age += 1
        consec_rej = consec_cf = 0
        if best_q != q:
            q, n_at_q, e_prev = best_q, 0, None
        else:
            e_prev = e
        if not fixed:
            eta = min(best_eta, 1.0 if rejected else opts.eta_max)
            eta = max(eta, 0.2)
            if 1.0 <= eta < opts.eta_keep:
                eta = 1.0
            h *= eta
        rejected = False
    res.y, res.t, res.h_last, res.q_last = Y[0], t, h, q
    return res


def solve_step(desc, k, hist_y, hist_t, t_new, h, S=None, tol=1e-14, max_iter=30, y_start=None):
    """Exact solution of one step's implicit BDF equation given its history.

    hist_y / hist_t: the q past solutions and times, newest first (y_{n},
    y_{n-1}, ...; the order is q = len(hist_y)); the step ends at t_new with
    size h.  Solves alpha_0 y + sum_{i=1..q} alpha_i y_{n+1-i} - h f(y) = 0
    (alpha_i = h l_i'(t_new) on the nodes t_new, hist_t) by full Newton with
    a fresh Jacobian every iteration until max |delta_i| / |y_i| <= tol
    (components that are exactly zero compared absolutely).  Starts from
    y_start, else from hist_y[0]."""
    if S is None:
        S = stoichiometry(desc)
    k = np.asarray(k, dtype=float)
    return solve_step_system(lambda y: S @ reaction_rates(desc, k, y), lambda y: jacobian(desc, k, y, S),
                             hist_y, hist_t, t_new, h, tol, max_iter, y_start)


def solve_step_system(f, jac, hist_y, hist_t, t_new, h, tol=1e-14, max_iter=30, y_start=None):
    """solve_step for any system dy/dt = f(y) with Jacobian jac(y)."""
    q = len(hist_y)
    alpha = bdf_alphas([t_new] + list(hist_t[:q]), h)
    psi = sum(alpha[i] * np.asarray(hist_y[i - 1], dtype=float) for i in range(1, q + 1))
    y = np.array(hist_y[0] if y_start is None else y_start, dtype=float)
    I = np.eye(y.shape[0])
    for _ in range(max_iter):
        G = alpha[0] * y + psi - h * f(y)
        delta = np.linalg.solve(alpha[0] * I - h * jac(y), -G)
        y = y + delta
        if np.all(np.abs(delta) <= tol * np.abs(y)):
            break
    return y


def integrate(desc, k, y0, t_end, opts: BDFOptions = BDFOptions(), cells=None):
    """Integrate every cell (columns of k'[n_r, C] and y0[n_s, C]) in turn."""
    S = stoichiometry(desc)
    C = y0.shape[1]
    cells = range(C) if cells is None else cells
    out = []
    for c in cells:
        out.append(integrate_cell(desc, k[:, c], y0[:, c], t_end, opts, S))
    return out
