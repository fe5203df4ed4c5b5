"""FP64 preconditioned conjugate gradients (textbook form) -- TEST INFRASTRUCTURE ONLY.

Solves A x = b from x = 0 with the preconditioner applied as z = Minv @ r; stops a
right-hand side when |r| / |b| < tol (r the recursively updated residual), exactly the
stopping rule of the device solver.  Dense numpy; pinned in tests/test_oracle_pins.py.
"""
import numpy as np


def pcg(A, b, Minv=None, tol=1e-8, max_iter=1000):
    """Returns (x, iterations, relative residual) for one right-hand side."""
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    if bn == 0:
        return x, 0, 0.0
    z = r if Minv is None else Minv @ r
    p = z.copy()
    rz = r @ z
    it = 0
    rel = 1.0
    while it < max_iter:
        it += 1
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        rel = np.linalg.norm(r) / bn
        if rel < tol:
            break
        z = r if Minv is None else Minv @ r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, rel
