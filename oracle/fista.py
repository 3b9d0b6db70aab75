"""FP64 accelerated proximal-gradient reconstruction -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may import this module; it imports nothing from the product.

The paper names, as the intended use of the matched pair H, H^T, iterative
image reconstruction that minimises a penalised least-squares functional with
proximal methods (Sec. 3 and Sec. 8, citing Beck's and Combettes-Pesquet's
texts on first-order and proximal splitting methods).  This is the plainest
such method for a non-negativity prior: FISTA (Beck and Teboulle's fast
iterative shrinkage-thresholding algorithm) on

    f(p) = 1/2 ||A p - y||^2  subject to  p >= 0,

where the proximal step of the constraint is the projection onto p >= 0.
With L >= ||A||^2, x_0 = p_init, z_1 = x_0 and t_1 = 1, iteration k = 1, 2, ...
computes

    x_k     = max(0, z_k - A^T (A z_k - y) / L)
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
    z_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1})

A and A^T are callables (the oracle's forward and adjoint operators, or a
dense matrix in the pins), so that every step is checkable by eye.

Parity: pinned by ``tests/test_oracle_pins.py::test_fista_nn_reaches_nnls``
(on a dense problem the iterates converge to scipy.optimize.nnls's solution,
an active-set method that shares nothing with this code).
"""
from __future__ import annotations

import math
from typing import Callable, List

import numpy as np


def fista_nn(A: Callable[[np.ndarray], np.ndarray], AT: Callable[[np.ndarray], np.ndarray], y: np.ndarray,
             p_init: np.ndarray, L: float, iters: int) -> List[np.ndarray]:
    """Iterates x_1 .. x_iters of FISTA with the non-negativity projection."""
    y = np.asarray(y, dtype=np.float64)
    x_prev = np.asarray(p_init, dtype=np.float64).copy()
    z = x_prev.copy()
    t = 1.0
    out = []
    for _ in range(iters):
        grad = AT(A(z) - y)
        x = np.maximum(0.0, z - grad / L)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = x + ((t - 1.0) / t_next) * (x - x_prev)
        x_prev, t = x, t_next
        out.append(x.copy())
    return out


# ---------------------------------------------------------------------------
# total-variation penalty
# ---------------------------------------------------------------------------
def grad3(x: np.ndarray) -> np.ndarray:
    """Forward differences along each axis of an array, zero at the last index
    (Neumann boundary): shape (ndim,) + x.shape."""
    out = np.zeros((x.ndim,) + x.shape)
    for a in range(x.ndim):
        n = x.shape[a]
        lo = [slice(None)] * x.ndim
        hi = [slice(None)] * x.ndim
        lo[a] = slice(0, n - 1)
        hi[a] = slice(1, n)
        out[(a,) + tuple(lo)] = x[tuple(hi)] - x[tuple(lo)]
    return out


def div3(p: np.ndarray) -> np.ndarray:
    """Minus the adjoint of grad3: <grad3 x, p> = -<x, div3 p>."""
    out = np.zeros(p.shape[1:])
    nd = p.shape[0]
    for a in range(nd):
        n = p.shape[1 + a]
        for i in range(n):
            idx = [slice(None)] * nd
            idx[a] = i
            term = np.zeros(out[tuple(idx)].shape)
            if i < n - 1:
                term = term + p[(a,) + tuple(idx)]
            if i >= 1:
                prev = list(idx)
                prev[a] = i - 1
                term = term - p[(a,) + tuple(prev)]
            out[tuple(idx)] += term
    return out


def tv_prox_nn(b: np.ndarray, tau: float, iters: int) -> np.ndarray:
    """argmin_{x >= 0} 1/2 ||x - b||^2 + tau TV(x), TV(x) = sum_i |grad3(x)_i|
    (isotropic), by Beck and Teboulle's fast gradient projection on the dual:
    with x(r) = max(0, b + tau div3 r) and the pointwise projection P onto
    |p| <= 1,
        p_k     = P(r_k + grad3(x(r_k)) / (4 ndim tau))
        t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
        r_{k+1} = p_k + ((t_k - 1) / t_{k+1}) (p_k - p_{k-1})
    and the answer x(p_iters).  4 ndim bounds ||grad3||^2."""
    b = np.asarray(b, dtype=np.float64)
    if tau <= 0:
        return np.maximum(0.0, b)
    step = 1.0 / (4.0 * b.ndim * tau)
    p_prev = np.zeros((b.ndim,) + b.shape)
    r = p_prev.copy()
    t = 1.0
    for _ in range(iters):
        x = np.maximum(0.0, b + tau * div3(r))
        q = r + step * grad3(x)
        nrm = np.sqrt(np.sum(q * q, axis=0))
        p = q / np.maximum(1.0, nrm)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        r = p + ((t - 1.0) / t_next) * (p - p_prev)
        p_prev, t = p, t_next
    return np.maximum(0.0, b + tau * div3(p_prev))


def fista_tv_nn(A: Callable[[np.ndarray], np.ndarray], AT: Callable[[np.ndarray], np.ndarray], y: np.ndarray,
                p_init: np.ndarray, L: float, lam: float, iters: int, inner: int) -> List[np.ndarray]:
    """FISTA on 1/2 ||A p - y||^2 + lam TV(p) subject to p >= 0: as fista_nn with
    the projection replaced by tv_prox_nn with tau = lam / L (inner iterations)."""
    y = np.asarray(y, dtype=np.float64)
    x_prev = np.asarray(p_init, dtype=np.float64).copy()
    z = x_prev.copy()
    t = 1.0
    out = []
    for _ in range(iters):
        grad = AT(A(z) - y)
        x = tv_prox_nn(z - grad / L, lam / L, inner)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = x + ((t - 1.0) / t_next) * (x - x_prev)
        x_prev, t = x, t_next
        out.append(x.copy())
    return out
