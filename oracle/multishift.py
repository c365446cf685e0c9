"""ORACLE -- test infrastructure only.

Multi-shift BiCGstab in plain numpy FP64: one Krylov space, one matrix-vector
product pair per iteration, solves (A + sigma_k) x_k = b for every shift
sigma_k at once (the method of shifted-system Krylov solvers, Jegerlehner
1996 and Frommer 2003; it is not in arXiv:0911.3191).  Here it pins the
scalar recurrences that the CUDA multi-shift solver follows; the solutions
themselves are checked against their definition (a solve per shift).

Derivation, with t the seed variable and phi_n, theta_n the BiCG residual and
direction polynomials (phi_{n+1} = phi_n - alpha_n t theta_n,
theta_{n+1} = phi_{n+1} + beta_n theta_n) and psi_n = prod_j (1 - omega_j t):

* Krylov spaces are shift invariant, so the BiCG residual polynomial of the
  shifted system is phi_n(s - sigma) / f_n with f_n = phi_n(-sigma), which
  obeys f_{n+1} = f_n + alpha_n sigma g_n, g_{n+1} = f_{n+1} + beta_n g_n
  (g_n = theta_n(-sigma), f_0 = g_0 = 1).
* Matching the three-term recurrences gives the shifted BiCG scalars
  alpha^s_n = alpha_n f_n / f_{n+1}, beta^s_n = beta_n (f_n / f_{n+1})^2.
* The stabilising factor 1 - omega^s (t + sigma) is proportional to
  1 - omega t for omega^s = omega / (1 + omega sigma), with factor
  1 / (1 + omega sigma); pi_n = prod_{j<n} (1 + omega_j sigma).
* Hence r^s_n = r_n / (pi_n f_n) and s^s_n = s_n / (pi_n f_{n+1}) are
  multiples of the seed's vectors; x^s and p^s are kept per shift:
  x^s += alpha^s p^s + omega^s s^s,
  p^s = r^s_{n+1} + beta^s (p^s - omega^s A^s p^s) with
  A^s p^s = (r^s_n - s^s_n) / alpha^s (no extra matrix-vector product).
"""
from __future__ import annotations

import numpy as np


def multishift_bicgstab(apply_A, b, shifts, tol=1e-10, maxiter=10000):
    """Solve (A + shifts[k]) x_k = b for all k; shifts[0] must be the seed
    shift 0 relative to A (pass A itself as the seed).  Returns
    (xs, iterations, seed residual history).  A shift stops being updated once
    its residual |r^s| <= tol |b|; the loop ends when all have."""
    b = np.asarray(b, dtype=np.complex128)
    shifts = [float(s) for s in shifts]
    if not shifts or shifts[0] != 0.0:
        raise ValueError("shifts[0] must be 0: the seed system drives the iteration")
    n = len(shifts)
    bnorm = np.linalg.norm(b)
    xs = [np.zeros_like(b) for _ in range(n)]
    ps = [b.copy() for _ in range(n)]
    r = b.copy()
    r_tilde = b.copy()
    rho = np.vdot(r_tilde, r)
    f = np.ones(n, dtype=np.complex128)
    g = np.ones(n, dtype=np.complex128)
    pi = np.ones(n, dtype=np.complex128)
    active = [True] * n
    hist = []
    it = 0
    for it in range(1, maxiter + 1):
        v = apply_A(ps[0])
        alpha = rho / np.vdot(r_tilde, v)
        s = r - alpha * v
        t = apply_A(s)
        omega = np.vdot(t, s) / np.vdot(t, t)
        r_new = s - omega * t
        rho_new = np.vdot(r_tilde, r_new)
        beta = (alpha / omega) * (rho_new / rho)
        for k in range(n):
            if not active[k]:
                continue
            sig = shifts[k]
            f_next = f[k] + alpha * sig * g[k]
            alpha_s = alpha * f[k] / f_next
            omega_s = omega / (1.0 + omega * sig)
            pi_next = pi[k] * (1.0 + omega * sig)
            beta_s = beta * (f[k] / f_next) ** 2
            r_s = r / (pi[k] * f[k])           # r^s_n
            s_s = s / (pi[k] * f_next)         # s^s_n
            xs[k] = xs[k] + alpha_s * ps[k] + omega_s * s_s
            Ap = (r_s - s_s) / alpha_s         # A^s p^s_n
            rn_s = r_new / (pi_next * f_next)  # r^s_{n+1}
            ps[k] = rn_s + beta_s * (ps[k] - omega_s * Ap)
            g[k] = f_next + beta * g[k]
            f[k] = f_next
            pi[k] = pi_next
            if np.linalg.norm(rn_s) <= tol * bnorm:
                active[k] = False
        r, rho = r_new, rho_new
        hist.append(np.linalg.norm(r) / bnorm)
        if not any(active):
            break
    return xs, it, hist
