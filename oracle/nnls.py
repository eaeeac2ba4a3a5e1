"""Non-negative least squares for source commissioning -- TEST INFRASTRUCTURE ONLY.

The commissioning problem of Sec. 2.2.3 (Eq. 8): min_{x >= 0} F(x) = ||A x - b||_2^2,
with one column of A per photon PSR and per effective electron unit.

* ``gradient_projection`` follows Sec. 2.2.4: x^{k+1} = P(x^k - s_k grad F(x^k)),
  P(y) = max(0, y), s_k from Armijo's rule along the projection arc, stopped
  when the relative change of F between two iterations falls below delta.
* ``gradient_projection_bb`` is the spectral projected gradient of Birgin,
  Martinez & Raydan (2000): Barzilai & Borwein's (1988) step length and a
  nonmonotone line search along the projected step.
* ``lawson_hanson`` is the active-set method of Lawson & Hanson (1974), with the
  passive-set least-squares solved through the normal equations.
* ``brute_force`` enumerates every support (tiny problems only).

Plain numpy in FP64; a library solve serves as the unconstrained step.
"""
from __future__ import annotations

import itertools

import numpy as np


def objective(A, b, x) -> float:
    r = A @ x - b
    return float(r @ r)


def kkt_residual(A, b, x) -> float:
    """Largest violation of x >= 0, grad >= 0, x * grad = 0 (grad = 2 A^T(Ax - b))."""
    g = 2.0 * A.T @ (A @ x - b)
    return float(max(np.max(np.clip(-x, 0, None), initial=0.0),
                     np.max(np.clip(-g, 0, None), initial=0.0),
                     np.max(np.abs(x * g), initial=0.0)))


def gradient_projection(A, b, x0=None, *, delta=1e-12, max_iter=200000, sigma=1e-4,
                        beta=0.5):
    """Projected gradient with Armijo line search (Sec. 2.2.4).  Initial step
    s_bar = 1 / lambda_max(A^T A) (power iteration); stop when
    |F_k - F_{k+1}| <= delta * F_k.  Returns (x, iterations, converged)."""
    m, n = A.shape
    x = np.ones(n) if x0 is None else np.array(x0, dtype=np.float64)
    x = np.maximum(x, 0.0)
    G = A.T @ A
    c = A.T @ b
    v = np.ones(n) / np.sqrt(n)
    for _ in range(100):
        w = G @ v
        v = w / np.linalg.norm(w)
    lam = float(v @ G @ v)
    s_bar = 1.0 / lam
    F = objective(A, b, x)
    for it in range(1, max_iter + 1):
        grad = 2.0 * (G @ x - c)
        s = s_bar
        while True:
            xn = np.maximum(x - s * grad, 0.0)
            Fn = objective(A, b, xn)
            if Fn <= F + sigma * float(grad @ (xn - x)) or s < 1e-30:
                break
            s *= beta
        change = abs(F - Fn)
        x, Fprev, F = xn, F, Fn
        if change <= delta * max(Fprev, 1e-300):
            return x, it, True
    return x, max_iter, False


def gradient_projection_bb(A, b, x0=None, *, delta=1e-12, max_iter=200000, memory=10, gamma=1e-4):
    """Spectral projected gradient (Birgin, Martinez & Raydan 2000): the step
    length before projection is Barzilai and Borwein's s's / s'y (s = x_k -
    x_{k-1}, y = grad_k - grad_{k-1}; the first is s_bar = 1 / lambda_max(A^T A)).
    Along d = P(x - alpha grad) - x the full step t = 1 is taken when F(x + t d)
    <= max(last `memory` values of F) + gamma t grad'd (a nonmonotone test);
    otherwise t becomes the minimiser of the quadratic through F(x), its slope
    and F(x + t d), kept within [0.1 t, 0.9 t] (t / 2 outside). Stop when
    P(x - alpha grad) = x or |F_k - F_{k+1}| <= delta * F_k.
    Returns (x, iterations, converged)."""
    m, n = A.shape
    x = np.ones(n) if x0 is None else np.array(x0, dtype=np.float64)
    x = np.maximum(x, 0.0)
    G = A.T @ A
    c = A.T @ b
    v = np.ones(n) / np.sqrt(n)
    for _ in range(100):
        w = G @ v
        v = w / np.linalg.norm(w)
    s_bar = 1.0 / float(v @ G @ v)
    alpha = s_bar
    F = objective(A, b, x)
    recent = [F]
    grad = 2.0 * (G @ x - c)
    for it in range(1, max_iter + 1):
        d = np.maximum(x - alpha * grad, 0.0) - x
        slope = float(grad @ d)
        if not np.any(d) or slope >= 0.0:
            return x, it, True
        F_ref = max(recent)
        t = 1.0
        while True:
            F_new = objective(A, b, x + t * d)
            if F_new <= F_ref + gamma * t * slope or t < 1e-30:
                break
            t_q = -0.5 * t * t * slope / (F_new - F - t * slope)
            t = t_q if 0.1 * t <= t_q <= 0.9 * t else 0.5 * t
        x_new = x + t * d
        grad_new = 2.0 * (G @ x_new - c)
        s, y = x_new - x, grad_new - grad
        sy = float(s @ y)
        alpha = min(max(float(s @ s) / sy, 1e-12 * s_bar), 1e12 * s_bar) if sy > 0.0 else 1e12 * s_bar
        change = abs(F - F_new)
        x, grad, F_prev, F = x_new, grad_new, F, F_new
        recent = (recent + [F])[-memory:]
        if change <= delta * max(F_prev, 1e-300):
            return x, it, True
    return x, max_iter, False


def lawson_hanson(A, b, *, tol=None, max_iter=None):
    """Active-set NNLS (Lawson & Hanson 1974). Returns (x, iterations)."""
    m, n = A.shape
    G = A.T @ A
    c = A.T @ b
    if tol is None:
        tol = 10.0 * np.finfo(float).eps * np.linalg.norm(G, 1) * max(m, n)
    max_iter = 3 * n if max_iter is None else max_iter
    P = np.zeros(n, dtype=bool)
    x = np.zeros(n)
    w = c - G @ x
    it = 0
    while (~P).any() and np.max(w[~P]) > tol and it < max_iter:
        j = np.argmax(np.where(P, -np.inf, w))
        P[j] = True
        while True:
            it += 1
            idx = np.flatnonzero(P)
            z = np.zeros(n)
            z[idx] = np.linalg.solve(G[np.ix_(idx, idx)], c[idx])
            if np.all(z[idx] > 0):
                x = z
                break
            neg = idx[z[idx] <= 0]
            alpha = np.min(x[neg] / (x[neg] - z[neg]))
            x = x + alpha * (z - x)
            P &= x > tol
            x[~P] = 0.0
        w = c - G @ x
    return x, it


def brute_force(A, b):
    """Every support S: least squares on S; the best one with x_S > 0."""
    m, n = A.shape
    best, bx = objective(A, b, np.zeros(n)), np.zeros(n)
    for k in range(1, n + 1):
        for S in itertools.combinations(range(n), k):
            S = list(S)
            xs, *_ = np.linalg.lstsq(A[:, S], b, rcond=None)
            if np.all(xs > 0):
                x = np.zeros(n)
                x[S] = xs
                f = objective(A, b, x)
                if f < best:
                    best, bx = f, x
    return bx
