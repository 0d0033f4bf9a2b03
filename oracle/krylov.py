"""Oracle of the Krylov comparators (test infrastructure only).

The paper compares F3R with preconditioned CG and BiCGStab in fp64 (Sec. 5).
Both here take the textbook steps in fp64 numpy, with the preconditioner the
F3R nest wraps, P = D^-1/2 M D^-1/2 (D = |diag A| under diagonal scaling, M
the stored Jacobi preconditioner of the scaled matrix, rounded to its storage
precision), applied on the left-preconditioned residual as in Saad,
Iterative Methods for Sparse Linear Systems:

    pcg       Alg. 9.1 (preconditioned conjugate gradient)
    bicgstab  van der Vorst's BiCGStab with the preconditioner applied to the
              search directions (Saad Alg. 7.7 in right-preconditioned form)

Both stop when the recurrence residual satisfies ||r|| <= tol ||b||, then the
true residual ||b - A x|| decides; if it is not below tol the recurrence
starts again from x (at most 3 times).  Returned: x, iterations, history of
||r|| / ||b|| (last start), true relative residual, breakdown flag.
"""
import numpy as np


def preconditioner(prob_oracle, m_prec_key="m16"):
    """(d, m): P y = d * (m * (d * y)) from an oracle.Problem."""
    return prob_oracle.get("d"), prob_oracle.get(m_prec_key)


def _pcg_run(A, b, x, d, m, tol, max_iters):
    P = lambda y: d * (m * (d * y))  # noqa: E731
    r = b - A @ x
    z = P(r)
    p = z.copy()
    rho = float(r @ z)
    bb = float(b @ b)
    hist = []
    it = 0
    brk = False
    if float(r @ r) <= tol * tol * bb:
        return x, it, hist, brk
    while it < max_iters:
        q = A @ p
        pq = float(p @ q)
        if pq == 0.0 or not np.isfinite(pq):
            brk = True
            break
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        z = P(r)
        rho_new = float(r @ z)
        rr = float(r @ r)
        it += 1
        hist.append(np.sqrt(rr / bb))
        if rr <= tol * tol * bb or not np.isfinite(rr):
            break
        beta = rho_new / rho
        rho = rho_new
        p = z + beta * p
    return x, it, hist, brk


def _bicgstab_run(A, b, x, d, m, tol, max_iters):
    P = lambda y: d * (m * (d * y))  # noqa: E731
    r = b - A @ x
    rh = r.copy()
    bb = float(b @ b)
    rho = float(rh @ r)
    alpha = omega = 1.0
    beta = 0.0
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    hist = []
    it = 0
    brk = False
    if float(r @ r) <= tol * tol * bb:
        return x, it, hist, brk
    while it < max_iters:
        p = r + beta * (p - omega * v)
        ph = P(p)
        v = A @ ph
        rv = float(rh @ v)
        if rv == 0.0 or not np.isfinite(rv):
            brk = True
            break
        alpha = rho / rv
        s = r - alpha * v
        sh = P(s)
        t = A @ sh
        tt = float(t @ t)
        omega = float(t @ s) / tt if tt > 0.0 else 0.0
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho_new = float(rh @ r)
        rr = float(r @ r)
        it += 1
        hist.append(np.sqrt(rr / bb))
        if rr <= tol * tol * bb or not np.isfinite(rr):
            break
        if rho_new == 0.0 or omega == 0.0:
            brk = True
            break
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
    return x, it, hist, brk


def solve(method, A, b, d, m, tol=1e-9, max_iters=100000, x0=None):
    """method: 'cg' or 'bicgstab'.  Returns dict(x, iters, hist, rel, breakdown, restarts)."""
    run = {"cg": _pcg_run, "bicgstab": _bicgstab_run}[method]
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    total = 0
    nb = np.linalg.norm(b)
    rel = np.linalg.norm(b - A @ x) / nb if nb > 0 else 0.0
    hist, brk, starts = [], False, 0
    for starts in range(4):
        x, it, hist, brk = run(A, b, x, d, m, tol, max_iters - total)
        total += it
        rel = np.linalg.norm(b - A @ x) / nb if nb > 0 else 0.0
        if not rel >= tol or brk or total >= max_iters:
            break
    return {"x": x, "iters": total, "hist": np.array(hist), "rel": rel, "breakdown": brk, "restarts": starts}
