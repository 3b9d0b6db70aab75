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
