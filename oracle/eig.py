"""Oracle for the smallest Hessian eigenvalue (second-order test, paper §1 definition of
SP-II and the eigenvalue diagnostics of §4.1 / §4.3).

Test infrastructure, not product code (see oracle/__init__.py).  FP64 throughout.

The paper plots the smallest Hessian eigenvalues but does not say how it computed
them.  Two methods are kept here:
  * dense_eigs: assemble H column by column in an orthonormal basis of the zero-mean
    subspace and call numpy.linalg.eigh (small grids only);
  * lanczos_lambda_min: Lanczos on the congruent operator K = M^{-1/2} H M^{-1/2}
    with M = Lambda + sigma (diagonal in reciprocal space, sigma > 0), full
    re-orthogonalisation, then a Rayleigh-Ritz step for H itself on the subspace
    V = M^{-1/2} Q: the smallest eigenvalue theta of the pencil (Q^T K Q, Q^T M^{-1} Q).
    Because Q^T K Q is Lanczos's tridiagonal T_k, the pencil is (T_k, G_k) with
    G_k = Q^T M^{-1} Q.  theta is an upper bound on lambda_min(H) that converges to
    it; K has the same inertia as H (Sylvester), so the smallest Ritz value kappa of
    T_k has the sign of lambda_min(H).
The spectral spread of H (Lambda reaches ~(|Bk|_max)^4) makes plain Lanczos on H
impractically slow; the congruence bounds K's spectrum by O(1).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import fft, lb
from .subproblem import dense_hessian


def dense_eigs(p: lb.Problem, psi: np.ndarray, count: int | None = None):
    """All (or the `count` smallest) eigenvalues of H on zero-mean fields, ascending,
    with eigenvectors as physical fields normalised in <.,.>_N."""
    hc, u = dense_hessian(p, psi)
    s, q = np.linalg.eigh(hc)
    if count is not None:
        s, q = s[:count], q[:, :count]
    vecs = [(np.sqrt(p.n) * (u @ q[:, i])).reshape(p.shape) for i in range(q.shape[1])]
    return s, vecs


def default_sigma(p: lb.Problem, psi: np.ndarray) -> float:
    """Shift of the congruence M = Lambda + sigma: max(1e-2, max_x |F''(psi(x))|)."""
    return max(1e-2, float(np.max(np.abs(lb.f2(p, np.asarray(psi, np.float64))))))


def lanczos_lambda_min(p: lb.Problem, psi: np.ndarray, k_max: int = 300, tol: float = 1e-9,
                       check_every: int = 10, sigma: float | None = None,
                       v0: np.ndarray | None = None, seed: int = 0):
    """Preconditioned Lanczos + Rayleigh-Ritz estimate of lambda_min(H).

    Stops when the Ritz residual ||H u - theta u|| / ||u|| <= tol (checked every
    `check_every` steps) or after k_max steps.  Returns a dict with theta (the
    estimate), kappa (smallest Ritz value of K), the Ritz vector u (<u,u>_N = 1),
    the residual norm and the number of Lanczos steps.
    """
    psi = np.asarray(psi, np.float64)
    if sigma is None:
        sigma = default_sigma(p, psi)
    m = lb.lam(p) + sigma
    m_isqrt = 1.0 / np.sqrt(m)

    def minv_half(v):
        return fft.inverse(m_isqrt * fft.forward(v))

    def kop(v):
        return lb.project(minv_half(lb.hessvec(p, psi, minv_half(v))))

    if v0 is None:
        v0 = np.random.default_rng(seed).standard_normal(p.shape)
    q = lb.project(np.asarray(v0, np.float64))
    q = q / lb.norm(q)
    qs = [q]
    mq = [minv_half(q)]                       # M^{-1/2} q_j
    alpha, beta = [], []
    q_prev = np.zeros_like(q)
    b_prev = 0.0
    result = None
    for j in range(1, k_max + 1):
        w = kop(qs[-1])
        a = lb.inner(qs[-1], w)
        w = w - a * qs[-1] - b_prev * q_prev
        for _ in range(2):                    # full re-orthogonalisation (twice)
            for qi in qs:
                w = w - lb.inner(qi, w) * qi
        # K maps the constant field to 0, an eigenvalue below every other one;
        # rounding would let Lanczos amplify a mean component, so remove it each step
        w = lb.project(w)
        b = lb.norm(w)
        alpha.append(a)
        beta.append(b)
        done = (j % check_every == 0) or j == k_max or b <= 1e-14
        if done:
            k = len(alpha)
            t = np.diag(alpha) + np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)
            gram = np.array([[lb.inner(mq[i], mq[l]) for l in range(k)] for i in range(k)])
            th, y = scipy.linalg.eigh(t, gram)
            kap = float(np.linalg.eigvalsh(t)[0])
            u = sum(y[i, 0] * mq[i] for i in range(k))
            u = u / lb.norm(u)
            res = lb.norm(lb.hessvec(p, psi, u) - th[0] * u)
            result = {"theta": float(th[0]), "kappa": kap, "vector": u, "residual": res,
                      "steps": k, "sigma": sigma}
            if res <= tol or b <= 1e-14:
                break
        q_prev = qs[-1]
        b_prev = b
        qn = w / b
        qs.append(qn)
        mq.append(minv_half(qn))
    return result
