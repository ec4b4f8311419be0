"""Oracle model formation: kernel -> continuous SDE (G, L, q, H) -> P_inf -> balancing.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and is never a fallback for it.

Paper: Corenflos, Zhao, Sarkka, "Temporal Gaussian Process Regression in
Logarithmic Time".

* SDE form of the GP, Sec. 2, Eq. (ssmodel): dx/dt = G x + L w, y = H x + e,
  with w white noise of spectral density q.  For Matern kernels the form is
  exact; the RBF kernel is approximated through a Taylor series of its spectral
  density (Sec. 2 and Sec. 5.1, order 6).
* Stationary covariance P_inf solves G P + P G^T + L q L^T = 0, by the
  vectorised closed form of Sec. 4.1.
* Balancing by a diagonal similarity D, Sec. 4.2, Eq. (scaled-ssmodel):
  z = D^{-1} x, so G' = D^{-1} G D, L' = D^{-1} L, H' = H D and the
  initial covariance becomes D^{-1} P_inf D^{-1}.  (The paper prints
  D^{-1} P_inf D, which is not symmetric; the state change z = D^{-1} x gives
  D^{-1} P_inf D^{-1}.)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import gamma


@dataclass
class SSModel:
    """A continuous-time state-space form of a stationary GP (Sec. 2)."""

    G: np.ndarray          # d x d drift
    L: np.ndarray          # d x 1 dispersion
    q: float               # white-noise spectral density
    H: np.ndarray          # 1 x d measurement row
    Pinf: np.ndarray = field(default=None)   # stationary covariance (Sec. 4.1)
    D: np.ndarray = field(default=None)      # balancing diagonal (Sec. 4.2), 1 if unbalanced

    @property
    def d(self) -> int:
        return self.G.shape[0]

    @property
    def W(self) -> np.ndarray:
        """L q L^T, the diffusion of Eq. (ss-gp-formation)."""
        return self.q * (self.L @ self.L.T)


def lyapunov(G: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Solve G P + P G^T + W = 0 by vectorisation (Sec. 4.1):

    (I (x) G + G (x) I) vec(P) = -vec(W).
    """
    d = G.shape[0]
    I = np.eye(d)
    K = np.kron(I, G) + np.kron(G, I)
    P = np.linalg.solve(K, -W.reshape(-1)).reshape(d, d)
    return 0.5 * (P + P.T)


def matern(nu: float, lengthscale: float, variance: float) -> SSModel:
    """Exact SDE of a Matern kernel with nu = p + 1/2 (Sec. 2, Matern case).

    The Matern spectral density is
        S(w) = variance * 2 sqrt(pi) Gamma(nu + 1/2) / Gamma(nu) * lam^(2 nu) / (lam^2 + w^2)^(nu + 1/2),
    lam = sqrt(2 nu) / lengthscale.  With (lam^2 + w^2)^(p+1) = |(lam + i w)^(p+1)|^2
    the monic Hurwitz factor is a(s) = (s + lam)^(p+1), so the SDE is the
    companion form of a(s) driven in its last coordinate with
    q = variance * 2 sqrt(pi) Gamma(nu + 1/2) / Gamma(nu) * lam^(2 nu).
    """
    p = int(round(nu - 0.5))
    assert abs(nu - (p + 0.5)) < 1e-12 and p >= 0
    d = p + 1
    lam = math.sqrt(2.0 * nu) / lengthscale
    # a(s) = sum_k binom(d, k) lam^(d-k) s^k ; companion last row = -a_k, k < d
    a = np.array([math.comb(d, k) * lam ** (d - k) for k in range(d)])
    G = np.zeros((d, d))
    for i in range(d - 1):
        G[i, i + 1] = 1.0
    G[d - 1, :] = -a
    L = np.zeros((d, 1)); L[d - 1, 0] = 1.0
    H = np.zeros((1, d)); H[0, 0] = 1.0
    q = variance * 2.0 * math.sqrt(math.pi) * gamma(nu + 0.5) / gamma(nu) * lam ** (2 * nu)
    m = SSModel(G=G, L=L, q=float(q), H=H)
    m.Pinf = lyapunov(m.G, m.W)
    m.D = np.ones(d)
    return m


def rbf_taylor(order: int, lengthscale: float, variance: float) -> SSModel:
    """Taylor approximation of the RBF kernel's spectral density (Sec. 2; order 6
    in Sec. 5.1), followed by spectral factorisation.

    S(w) = variance sqrt(2 pi) l exp(-l^2 w^2 / 2)
         ~ variance sqrt(2 pi) l / sum_{k<=n} (l^2 w^2 / 2)^k / k!.
    With s = i w the denominator is P(s) = sum_k (l^2/2)^k (-1)^k s^(2k) / k!,
    which factors as c a(s) a(-s) with a monic and Hurwitz (the n roots of P
    with negative real part) and c = (l^2/2)^n / n!.  Then S = q / |a(i w)|^2
    with q = variance sqrt(2 pi) l / c, i.e. the companion SDE of a(s).
    """
    n = int(order)
    ell2h = 0.5 * lengthscale * lengthscale
    # coefficients of P(s) in decreasing powers of s (degree 2n)
    coef = np.zeros(2 * n + 1)
    for k in range(n + 1):
        coef[2 * n - 2 * k] = ell2h ** k * (-1.0) ** k / math.factorial(k)
    roots = np.roots(coef)
    lhp = roots[roots.real < 0.0]
    assert lhp.size == n, "spectral factorisation: expected n stable roots"
    a_desc = np.real(np.poly(lhp))          # monic, decreasing powers
    a = a_desc[::-1][:n]                    # a_0 .. a_{n-1}
    G = np.zeros((n, n))
    for i in range(n - 1):
        G[i, i + 1] = 1.0
    G[n - 1, :] = -a
    L = np.zeros((n, 1)); L[n - 1, 0] = 1.0
    H = np.zeros((1, n)); H[0, 0] = 1.0
    c = ell2h ** n / math.factorial(n)
    q = variance * math.sqrt(2.0 * math.pi) * lengthscale / c
    m = SSModel(G=G, L=L, q=float(q), H=H)
    m.Pinf = lyapunov(m.G, m.W)
    m.D = np.ones(n)
    return m


def osborne_scaling(G: np.ndarray, max_sweeps: int = 100) -> np.ndarray:
    """Osborne's balancing (Sec. 4.2): a diagonal D making the off-diagonal
    2-norms of each row and column of D^{-1} G D equal, restricted to powers of
    two so that the scaling is exact.  Normalised to D_0 = 1."""
    d = G.shape[0]
    Dv = np.ones(d)
    for _ in range(max_sweeps):
        changed = False
        for i in range(d):
            B = (G * Dv[None, :]) / Dv[:, None]     # current D^{-1} G D
            c = math.sqrt(sum(B[j, i] ** 2 for j in range(d) if j != i))
            r = math.sqrt(sum(B[i, j] ** 2 for j in range(d) if j != i))
            if c == 0.0 or r == 0.0:
                continue
            f = 2.0 ** round(0.5 * math.log2(r / c))
            if f != 1.0:
                Dv[i] *= f
                changed = True
        if not changed:
            break
    return Dv / Dv[0]


def balance(m: SSModel) -> SSModel:
    """Return the balanced model of Eq. (scaled-ssmodel) with z = D^{-1} x."""
    Dv = osborne_scaling(m.G)
    Dinv = 1.0 / Dv
    G = (m.G * Dv[None, :]) * Dinv[:, None]
    L = m.L * Dinv[:, None]
    H = m.H * Dv[None, :]
    Pinf = m.Pinf * Dinv[:, None] * Dinv[None, :]
    return SSModel(G=G, L=L, q=m.q, H=H, Pinf=Pinf, D=Dv * m.D)


def make_model(kind: str, lengthscale: float, variance: float, order: int = 6,
               balanced: bool = False) -> SSModel:
    """kind in {'matern12', 'matern32', 'matern52', 'rbf'}."""
    if kind == "matern12":
        m = matern(0.5, lengthscale, variance)
    elif kind == "matern32":
        m = matern(1.5, lengthscale, variance)
    elif kind == "matern52":
        m = matern(2.5, lengthscale, variance)
    elif kind == "rbf":
        m = rbf_taylor(order, lengthscale, variance)
    else:
        raise ValueError(kind)
    return balance(m) if balanced else m


# ---------------------------------------------------------------------------
# Covariance functions used by the dense-GP check (Lemma of the supplement).
# ---------------------------------------------------------------------------

def matern_kernel(nu: float, lengthscale: float, variance: float):
    """Textbook Matern covariance for nu in {1/2, 3/2, 5/2}."""
    def k(tau):
        r = np.abs(tau) / lengthscale
        if nu == 0.5:
            return variance * np.exp(-r)
        if nu == 1.5:
            s = math.sqrt(3.0) * r
            return variance * (1.0 + s) * np.exp(-s)
        if nu == 2.5:
            s = math.sqrt(5.0) * r
            return variance * (1.0 + s + s * s / 3.0) * np.exp(-s)
        raise ValueError(nu)
    return k


def ssm_kernel(m: SSModel):
    """Covariance of the SDE's stationary output, k(tau) = H exp(G |tau|) P_inf H^T,
    evaluated through the eigendecomposition of G (a library routine).  Only
    for diagonalisable G (the RBF Taylor forms); the Matern drifts have one
    repeated eigenvalue and use the textbook covariance instead."""
    lam, V = np.linalg.eig(m.G)
    if np.linalg.cond(V) > 1e8:
        raise ValueError("ssm_kernel needs a diagonalisable drift")
    Vinv = np.linalg.inv(V)
    left = (m.H @ V).ravel()                     # H V
    right = (Vinv @ m.Pinf @ m.H.T).ravel()      # V^{-1} P_inf H^T
    coef = left * right

    def k(tau):
        a = np.abs(np.asarray(tau))
        out = np.zeros(a.shape, dtype=np.complex128)
        for c, l in zip(coef, lam):
            out += c * np.exp(l * a)
        return out.real
    return k


# ---------------------------------------------------------------------------
# Derivatives of the model with respect to the log hyperparameters, for the
# forward-mode gradient of the log marginal likelihood (Sec. 2, parameter
# estimation).  In the unbalanced companion form built above, both families
# have drift coefficients a_k proportional to lengthscale^(k - d) (Matern:
# a_k = binom(d, k) lam^(d - k) with lam = sqrt(2 nu) / lengthscale; RBF: the
# roots of P(s), a polynomial in lengthscale * s, scale as 1 / lengthscale)
# and a white-noise density q proportional to variance * lengthscale^(1 - 2d)
# (Matern: lam^(2 nu) = lam^(2d - 1); RBF: lengthscale / lengthscale^(2n)).
# Hence, with G[d-1, k] = -a_k and W = q L L^T,
#   d G[d-1, k] / d log l = -(d - k) G[d-1, k],  dW / d log l = (1 - 2d) W,
#   dG / d log s2 = 0,                           dW / d log s2 = W,
# and dP_inf follows from differentiating G P + P G^T + W = 0:
#   G dP + dP G^T + (dG P + P dG^T + dW) = 0.
# ---------------------------------------------------------------------------

def model_tangent(m: SSModel, param: str):
    """(dG, dW, dP_inf) of an unbalanced model for param in
    {'log_lengthscale', 'log_variance'}."""
    d = m.d
    if not np.all(m.D == 1.0):
        raise ValueError("model_tangent needs the unbalanced model")
    W = m.W
    if param == "log_lengthscale":
        dG = np.zeros((d, d))
        for k in range(d):
            dG[d - 1, k] = -(d - k) * m.G[d - 1, k]
        dW = (1.0 - 2.0 * d) * W
    elif param == "log_variance":
        dG = np.zeros((d, d))
        dW = W.copy()
    else:
        raise ValueError(param)
    dPinf = lyapunov(m.G, dG @ m.Pinf + m.Pinf @ dG.T + dW)
    return dG, dW, dPinf


def matern_kernel_dlogl(nu: float, lengthscale: float, variance: float):
    """d k / d log(lengthscale) of the textbook Matern covariance, written out
    from k(tau) = variance f(r), r = sqrt(2 nu) |tau| / lengthscale:
    d k / d log l = -r variance f'(r)."""
    def dk(tau):
        r = np.abs(tau) / lengthscale
        if nu == 0.5:
            return variance * r * np.exp(-r)
        if nu == 1.5:
            s = math.sqrt(3.0) * r
            return variance * s * s * np.exp(-s)
        if nu == 2.5:
            s = math.sqrt(5.0) * r
            return variance * s * s * (1.0 + s) / 3.0 * np.exp(-s)
        raise ValueError(nu)
    return dk
