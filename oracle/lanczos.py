"""Plain Lanczos ground state in FP64 (oracle, test only).

Sec. 6.6: the sector ground state is found with the simple Lanczos procedure
without re-orthogonalisation.  Recurrence (Paige form):

    w = H v_j - beta_j v_{j-1};  alpha_j = <v_j, w>;  w -= alpha_j v_j;
    beta_{j+1} = ||w||;  v_{j+1} = w / beta_{j+1}.

Stopping (the paper leaves it open; reading used on both sides): after each
step the lowest eigenpair (theta_j, y) of the (j+1)x(j+1) tridiagonal matrix
is found and the Ritz residual estimate beta_{j+1} |y_j| (the norm of
H psi - theta psi for psi = V y in exact arithmetic) is formed; stop when it is
<= tol * max(1, |theta_j|), when beta_{j+1} <= breakdown * max_i(|alpha_i|,
beta_i) (invariant subspace found), or after ``maxit`` steps
(lanc_niter = 512).  The residual test converges the vector as well as the
energy, which the Green's function needs.
"""
from __future__ import annotations

import math

import numpy as np

from workloads import splitmix64_uniform_array


def start_vector(seed: int, dim: int) -> np.ndarray:
    """Lanczos start vector: element i is u_i - 1/2 with u_i the i-th uniform
    of a SplitMix64 stream started at ``seed`` (sector order), normalised."""
    v = splitmix64_uniform_array(seed, dim) - 0.5
    return v / np.linalg.norm(v)


def sturm_count(alpha, beta, x: float) -> int:
    """Number of eigenvalues of the symmetric tridiagonal matrix
    (diag alpha, off-diagonal beta[1:]) that are smaller than x (Sturm
    sequence of the LDL^T factorisation of T - x)."""
    k = len(alpha)
    cnt = 0
    q = 1.0
    for i in range(k):
        off = beta[i] * beta[i] if i > 0 else 0.0
        q = (alpha[i] - x) - (off / q if i > 0 else 0.0)
        if q == 0.0:
            q = -1e-300
        if q < 0.0:
            cnt += 1
    return cnt


def tridiag_bounds(alpha, beta):
    """Gershgorin interval of the tridiagonal matrix."""
    k = len(alpha)
    lo, hi = math.inf, -math.inf
    for i in range(k):
        r = (abs(beta[i]) if i > 0 else 0.0) + (abs(beta[i + 1]) if i + 1 < k else 0.0)
        lo = min(lo, alpha[i] - r)
        hi = max(hi, alpha[i] + r)
    return lo, hi


def tridiag_lowest(alpha, beta) -> float:
    """Lowest eigenvalue by bisection on the Sturm count (FP64).

    ``beta[i]`` couples rows i-1 and i (beta[0] unused)."""
    lo, hi = tridiag_bounds(alpha, beta)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if sturm_count(alpha, beta, mid) >= 1:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def tridiag_vector(alpha, beta, theta: float) -> np.ndarray:
    """Eigenvector of T for the eigenvalue theta by inverse iteration with
    the tridiagonal (Thomas) solver, normalised, largest-magnitude entry > 0."""
    k = len(alpha)
    y = np.ones(k) / math.sqrt(k)
    shift = theta - 1e-13 * max(1.0, abs(theta))
    for _ in range(4):
        # solve (T - shift) x = y
        d = np.array([alpha[i] - shift for i in range(k)], dtype=np.float64)
        c = np.array([beta[i + 1] if i + 1 < k else 0.0 for i in range(k)])
        b = y.copy()
        for i in range(1, k):
            if d[i - 1] == 0.0:
                d[i - 1] = 1e-300
            m = beta[i] / d[i - 1]
            d[i] -= m * c[i - 1]
            b[i] -= m * b[i - 1]
        x = np.zeros(k)
        if d[k - 1] == 0.0:
            d[k - 1] = 1e-300
        x[k - 1] = b[k - 1] / d[k - 1]
        for i in range(k - 2, -1, -1):
            x[i] = (b[i] - c[i] * x[i + 1]) / d[i]
        y = x / np.linalg.norm(x)
    if y[int(np.argmax(np.abs(y)))] < 0:
        y = -y
    return y


def lanczos_ground(matvec, v0, maxit=512, tol=1e-12, breakdown=1e-13, min_iter=2):
    """First Lanczos pass: returns dict with alpha[k], beta[k+1]
    (beta[0] = 0), theta and residual-estimate histories, e0, k and the stop
    reason."""
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    alpha, beta = [], [0.0]
    thetas, rests = [], []
    tnorm = 0.0
    reason = "maxit"
    for j in range(maxit):
        w = matvec(v) - beta[j] * v_prev
        a = float(np.dot(v, w))
        w = w - a * v
        b = float(np.linalg.norm(w))
        alpha.append(a)
        beta.append(b)
        tnorm = max(tnorm, abs(a), b)
        th = tridiag_lowest(alpha, beta[:len(alpha)])
        y = tridiag_vector(alpha, beta[:len(alpha)], th)
        thetas.append(th)
        rests.append(b * abs(y[-1]))
        if b <= breakdown * tnorm:
            reason = "breakdown"
            break
        if rests[-1] <= tol * max(1.0, abs(th)) and j + 1 >= min_iter:
            reason = "converged"
            break
        v_prev, v = v, w / b
    k = len(alpha)
    return dict(alpha=np.array(alpha), beta=np.array(beta), thetas=np.array(thetas),
                rests=np.array(rests), e0=thetas[-1], k=k, reason=reason)


def lanczos_ground_vector(matvec, v0, alpha, beta, y) -> np.ndarray:
    """Second pass: rebuild v_0..v_{k-1} with the stored coefficients and
    accumulate psi = sum_j y_j v_j (back-transform of the Ritz vector)."""
    k = len(alpha)
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    psi = y[0] * v
    for j in range(k - 1):
        w = matvec(v) - beta[j] * v_prev - alpha[j] * v
        v_prev, v = v, w / beta[j + 1]
        psi += y[j + 1] * v
    return psi


def ground_state(matvec, dim, seed=0x5EED, maxit=512, tol=1e-12):
    """E0 and normalised psi of a sector: first pass, Ritz vector of the
    tridiagonal matrix, second pass."""
    v0 = start_vector(seed, dim)
    r = lanczos_ground(matvec, v0, maxit=maxit, tol=tol)
    y = tridiag_vector(r["alpha"], r["beta"][:r["k"]], r["e0"])
    psi = lanczos_ground_vector(matvec, v0, r["alpha"], r["beta"], y)
    psi /= np.linalg.norm(psi)
    r["psi"] = psi
    r["y"] = y
    return r


def rayleigh_residual(matvec, psi):
    """FP64 Rayleigh quotient E = <psi,H psi>/<psi,psi> and the residual
    norm ||H psi - E psi|| / ||psi||."""
    hp = matvec(psi)
    nn = float(np.dot(psi, psi))
    e = float(np.dot(psi, hp)) / nn
    r = float(np.linalg.norm(hp - e * psi)) / math.sqrt(nn)
    return e, r


def lanczos_chain(matvec, phi, nsteps, breakdown=1e-13):
    """Lanczos tridiagonalisation started from phi/||phi|| (Sec. 6.8):
    returns (a[0..n-1], b[1..n-1]) with b[0] = 0, stopping early on
    breakdown (the chain then spans an invariant subspace)."""
    v = phi / np.linalg.norm(phi)
    v_prev = np.zeros_like(v)
    a, b = [], [0.0]
    tnorm = 0.0
    for j in range(nsteps):
        w = matvec(v) - b[j] * v_prev
        aj = float(np.dot(v, w))
        w = w - aj * v
        bj = float(np.linalg.norm(w))
        a.append(aj)
        tnorm = max(tnorm, abs(aj), bj)
        if j == nsteps - 1 or bj <= breakdown * tnorm:
            break
        b.append(bj)
        v_prev, v = v, w / bj
    return np.array(a), np.array(b)
