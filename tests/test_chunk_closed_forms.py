"""The per-chunk closed forms the kernels use instead of per-step recursions,
checked in plain numpy on small random models (no oracle, no CUDA).

A chunk's filter aggregate (Sec. 3's elements folded over its steps, started
from a given state z) gives log p(y_chunk | z) = c + eta^T z - z^T J z / 2,
the conditional mean A z + b and covariance C.  From it, with the filter
state or prediction (m, P) at the chunk's start:
  1. the chunk's log-likelihood (a Gaussian integral): the sequential
     prediction-error sum;
  2. the smoother chunk aggregate (product of the RTS elements): moments of
     the start state given the chunk, cross-covariance V A^T, closing step;
  3. the mean-adjoint chunk aggregate: Pi = N^{-1} A^T F^T,
     gamma = N^{-1}(eta - J m), N = I + J P;
  4. the covariance-adjoint chunk term:
     L = (u gamma^T + gamma u^T)/2 + gamma gamma^T/2 - N^{-1} J / 2, u = Pi mb.
Each is compared with the recursion it replaces, with missing steps and with
a series start (F = 0, Q = P_inf) inside the chunk.
"""
import numpy as np
import pytest
from scipy.linalg import expm, solve_continuous_lyapunov


def model(d, lam):
    """Companion drift with the repeated eigenvalue -lam (a Matern form) and
    noise on the last state."""
    c = np.poly(-lam * np.ones(d))[1:]           # monic (s + lam)^d
    G = np.zeros((d, d))
    G[:-1, 1:] = np.eye(d - 1)
    G[-1, :] = -c[::-1]
    W = np.zeros((d, d))
    W[-1, -1] = 2.0
    return G, W, solve_continuous_lyapunov(G, -W)


def disc(G, W, h):
    d = G.shape[0]
    M = np.zeros((2 * d, 2 * d))
    M[:d, :d], M[:d, d:], M[d:, d:] = G, W, -G.T
    E = expm(M * h)
    F = E[:d, :d]
    Q = E[:d, d:] @ F.T
    return F, (Q + Q.T) / 2


def problem(seed, d, n, reset_at=None):
    rng = np.random.default_rng(seed)
    G, W, Pinf = model(d, rng.uniform(0.8, 2.0))
    FQ = [disc(G, W, h) for h in rng.uniform(0.05, 0.5, n + 1)]
    if reset_at is not None:
        FQ[reset_at] = (np.zeros((d, d)), Pinf)
    y = rng.normal(size=n + 1)
    obs = rng.uniform(size=n + 1) > 0.25
    A0 = rng.normal(size=(d, d))
    P0 = A0 @ A0.T * 0.2 + 0.05 * np.eye(d)
    return FQ, y, obs, rng.normal(size=d), P0, 0.05, rng


def kf_step(x, P, F, Q, y, ob, R):
    """One Kalman step; returns the filtered state, the prediction, v, 1/S and
    the step's log-likelihood term."""
    xm, Pm = F @ x, F @ P @ F.T + Q
    S = Pm[0, 0] + R
    Si = 1.0 / S if ob else 0.0
    v = (y - xm[0]) if ob else 0.0
    K = Pm[:, 0] * Si
    ll = -0.5 * (np.log(2 * np.pi * S) + v * v / S) if ob else 0.0
    return xm + K * v, Pm - np.outer(K, Pm[0, :]), xm, Pm, v, Si, ll


def fold(FQ, y, obs, R, ks, first_without_transition=False):
    """Sec. 3's elements folded over the steps ks from the identity, in the
    fold's update form; also the zero-start log-likelihood c."""
    d = FQ[0][0].shape[0]
    A, b, C = np.eye(d), np.zeros(d), np.zeros((d, d))
    eta, J, c = np.zeros(d), np.zeros((d, d)), 0.0
    for i, k in enumerate(ks):
        F, Q = FQ[k]
        if i == 0 and first_without_transition:
            F, Q = np.eye(d), np.zeros((d, d))
        Pm, bm, w = F @ C @ F.T + Q, F @ b, (F @ A)[0]
        S = Pm[0, 0] + R
        Si = 1.0 / S if obs[k] else 0.0
        r = (y[k] - bm[0]) if obs[k] else 0.0
        K = Pm[:, 0] * Si
        J, eta = J + np.outer(w, w) * Si, eta + w * Si * r
        if obs[k]:
            c += -0.5 * (np.log(2 * np.pi * S) + r * r * Si)
        b, C, A = bm + K * r, Pm - np.outer(K, Pm[0, :]), F @ A - np.outer(K, w)
    return A, b, C, eta, J, c


CASES = [(2, 9, None), (3, 12, None), (3, 12, 5), (2, 7, 1)]


@pytest.mark.parametrize("d,n,reset", CASES)
def test_chunk_loglik_is_the_prediction_error_sum(d, n, reset):
    FQ, y, obs, m, P, R, _ = problem(10 + d + n, d, n, reset)
    x, Pk, ll = m, P, 0.0
    for k in range(n):
        x, Pk, _, _, _, _, l = kf_step(x, Pk, *FQ[k], y[k], obs[k], R)
        ll += l
    A, b, C, eta, J, c = fold(FQ, y, obs, R, range(n))
    M = np.eye(d) + P @ J
    r = eta - J @ m
    closed = (c + eta @ m - 0.5 * m @ J @ m + 0.5 * r @ np.linalg.solve(M, P @ r)
              - 0.5 * np.linalg.slogdet(M)[1])
    assert abs(closed - ll) <= 1e-11 * max(1.0, abs(ll))
    # and the aggregate's conditional moments are the filter's at the end
    mu = np.linalg.solve(M, m + P @ eta)
    assert np.allclose(A @ mu + b, x, atol=1e-11)
    assert np.allclose(A @ np.linalg.solve(M, P) @ A.T + C, Pk, atol=1e-11)


@pytest.mark.parametrize("d,n,reset", CASES)
def test_smoother_chunk_aggregate_closed_form(d, n, reset):
    """Elements a .. b-1 (E_k = P_k F_{k+1}^T (P^-_{k+1})^{-1}, g_k, L_k)
    composed, against the closed form from the filter state at a, the
    aggregate of steps a+1 .. b-1 and the prediction of step b."""
    FQ, y, obs, m, P, R, _ = problem(20 + d + n, d, n, reset)
    a, bb = 0, n                        # elements 0 .. n-1 need the prediction of step n
    xs, Ps = [m], [P]                   # filtered states at a, a+1, ...
    x, Pk = m, P
    preds = {}
    for k in range(a + 1, bb + 1):
        x, Pk, xm, Pm, _, _, _ = kf_step(x, Pk, *FQ[k], y[k], obs[k], R)
        xs.append(x)
        Ps.append(Pk)
        preds[k] = (xm, Pm)
    E, g, L = np.eye(d), np.zeros(d), np.zeros((d, d))
    for k in range(bb - 1, a - 1, -1):  # compose later elements first: e_k x agg
        xk, Pk_ = xs[k - a], Ps[k - a]
        xm, Pm = preds[k + 1]
        Ek = Pk_ @ FQ[k + 1][0].T @ np.linalg.inv(Pm)
        gk, Lk = xk - Ek @ xm, Pk_ - Ek @ Pm @ Ek.T
        E, g, L = Ek @ E, Ek @ g + gk, Ek @ L @ Ek.T + Lk
    A, _, _, eta, J, _ = fold(FQ, y, obs, R, range(a + 1, bb))
    M = np.eye(d) + P @ J
    mu, V = np.linalg.solve(M, m + P @ eta), np.linalg.solve(M, P)
    Sig = V @ A.T
    Fb = FQ[bb][0]
    xm, Pm = preds[bb]
    Ec = Sig @ Fb.T @ np.linalg.inv(Pm)
    gc, Lc = mu - Ec @ xm, V - Ec @ (Sig @ Fb.T).T
    for got, want in ((Ec, E), (gc, g), (Lc, L)):
        assert np.allclose(got, want, atol=1e-11 * max(1.0, np.abs(want).max()))


@pytest.mark.parametrize("d,n,reset", CASES)
def test_adjoint_chunk_aggregates_closed_form(d, n, reset):
    """The mean adjoint mb_k = (I - e0 K_k^T) F_{k+1}^T mb_{k+1} + e0 v_k/S_k
    and the covariance adjoint L <- A (F^T L F) A^T + B through the chunk
    k0 .. k1-1, against Pi, gamma and L in closed form."""
    FQ, y, obs, m, P, R, rng = problem(30 + d + n, d, n, reset)
    k0, k1 = 0, n - 1
    e0 = np.eye(d)[0]
    x, Pk, rec = m, P, []
    for k in range(k0, k1):
        x, Pk, xm, Pm, v, Si, _ = kf_step(x, Pk, *FQ[k], y[k], obs[k], R)
        rec.append((xm, Pm, v, Si))
    mb1 = rng.normal(size=d)
    F1 = FQ[k1][0]
    Lrec, mb = np.zeros((d, d)), mb1.copy()
    for k in range(k1 - 1, k0 - 1, -1):
        Fn = FQ[k + 1][0]
        xb = Fn.T @ mb
        xm, Pm, v, Si = rec[k - k0]
        K = Pm[:, 0] * Si
        kx, vSi = K @ xb, v * Si
        c = -0.5 * (Si - vSi * vSi)
        Amat = np.eye(d) - np.outer(e0, K)
        B = (vSi / 2) * (np.outer(xb, e0) + np.outer(e0, xb)) + (c - vSi * kx) * np.outer(e0, e0)
        Lrec = Amat @ (Fn.T @ Lrec @ Fn) @ Amat.T + B
        mb = xb.copy()
        mb[0] += vSi - kx
    A, _, _, eta, J, _ = fold(FQ, y, obs, R, range(k0, k1), first_without_transition=True)
    m0, P0 = rec[0][0], rec[0][1]
    N = np.eye(d) + J @ P0
    Pi = np.linalg.solve(N, A.T @ F1.T)
    gam = np.linalg.solve(N, eta - J @ m0)
    assert np.allclose(Pi @ mb1 + gam, mb, atol=1e-11 * max(1.0, np.abs(mb).max()))
    u = Pi @ mb1
    Lc = 0.5 * (np.outer(u, gam) + np.outer(gam, u)) + 0.5 * np.outer(gam, gam) - 0.5 * np.linalg.solve(N, J)
    assert np.allclose(Lc, Lrec, atol=1e-11 * max(1.0, np.abs(Lrec).max()))


def test_a_wrong_cross_term_is_detected():
    """The symmetrised cross term is the one that matches: the unhalved one
    does not (guards the test against a vacuous comparison)."""
    FQ, y, obs, m, P, R, rng = problem(41, 3, 12)
    k0, k1 = 0, 11
    e0 = np.eye(3)[0]
    x, Pk, rec = m, P, []
    for k in range(k0, k1):
        x, Pk, xm, Pm, v, Si, _ = kf_step(x, Pk, *FQ[k], y[k], obs[k], R)
        rec.append((xm, Pm, v, Si))
    mb1 = rng.normal(size=3)
    Lrec, mb = np.zeros((3, 3)), mb1.copy()
    for k in range(k1 - 1, k0 - 1, -1):
        Fn = FQ[k + 1][0]
        xb = Fn.T @ mb
        xm, Pm, v, Si = rec[k - k0]
        K = Pm[:, 0] * Si
        kx, vSi = K @ xb, v * Si
        Amat = np.eye(3) - np.outer(e0, K)
        B = (vSi / 2) * (np.outer(xb, e0) + np.outer(e0, xb)) + (-0.5 * (Si - vSi * vSi) - vSi * kx) * np.outer(e0, e0)
        Lrec = Amat @ (Fn.T @ Lrec @ Fn) @ Amat.T + B
        mb = xb.copy()
        mb[0] += vSi - kx
    A, _, _, eta, J, _ = fold(FQ, y, obs, R, range(k0, k1), first_without_transition=True)
    N = np.eye(3) + J @ rec[0][1]
    Pi = np.linalg.solve(N, A.T @ FQ[k1][0].T)
    gam = np.linalg.solve(N, eta - J @ rec[0][0])
    u = Pi @ mb1
    wrong = np.outer(u, gam) + np.outer(gam, u) + 0.5 * np.outer(gam, gam) - 0.5 * np.linalg.solve(N, J)
    assert not np.allclose(wrong, Lrec, atol=1e-6)
