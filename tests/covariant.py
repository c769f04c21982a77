"""Covariant (4-D) stress-energy forms of ideal GRMHD, written independently
of the oracle's 3+1 formulas so the tests can check the latter against them.

T^{mu nu} = (rho h + b^2) u^mu u^nu + (p + b^2/2) g^{mu nu} - b^mu b^nu, with
u^0 = W/alpha, u^i = W (v^i - beta^i/alpha), b^0 = W (B.v)/alpha,
b^i = (B^i + alpha b^0 u^i)/W.  Conserved D = rho W, S_j = alpha T^0_j,
tau = alpha^2 T^00 - D; fluxes along i: F(D) = alpha rho u^i,
F(S_j) = alpha T^i_j, F(tau) = alpha^2 T^{i0} - F(D),
F(B^j) = alpha (b^j u^i - b^i u^j).  Sources (stationary metric):
S(S_j) = alpha/2 T^{mu nu} d_j g_{mu nu},
S(tau) = alpha (T^{mu 0} d_mu alpha - alpha T^{mu nu} Gamma^0_{mu nu}).
"""
import numpy as np


def four_metric(alpha, beta, g):
    bl = g @ beta
    G = np.zeros((4, 4))
    G[0, 0] = -alpha * alpha + beta @ bl
    G[0, 1:] = G[1:, 0] = bl
    G[1:, 1:] = g
    return G


def inv_four_metric(alpha, beta, gi):
    Gi = np.zeros((4, 4))
    Gi[0, 0] = -1.0 / alpha ** 2
    Gi[0, 1:] = Gi[1:, 0] = beta / alpha ** 2
    Gi[1:, 1:] = gi - np.outer(beta, beta) / alpha ** 2
    return Gi


def stress_energy(P, alpha, beta, g, gamma_ad):
    gi = np.linalg.inv(g)
    rho, p = P[0], P[1]
    ut = np.asarray(P[2:5], float)
    B = np.asarray(P[5:8], float)
    W = np.sqrt(1.0 + ut @ g @ ut)
    v = ut / W
    u = np.zeros(4)
    u[0] = W / alpha
    u[1:] = W * (v - beta / alpha)
    b = np.zeros(4)
    b[0] = W * (B @ g @ v) / alpha
    b[1:] = (B + alpha * b[0] * u[1:]) / W
    G = four_metric(alpha, beta, g)
    Gi = inv_four_metric(alpha, beta, gi)
    b2 = b @ G @ b
    rhoh = rho + gamma_ad / (gamma_ad - 1.0) * p
    T = (rhoh + b2) * np.outer(u, u) + (p + 0.5 * b2) * Gi - np.outer(b, b)
    return T, u, b, G, Gi, W


def conserved(P, alpha, beta, g, gamma_ad):
    T, u, b, G, Gi, W = stress_energy(P, alpha, beta, g, gamma_ad)
    D = P[0] * W
    S = alpha * (T[0, :] @ G[:, 1:])
    tau = alpha * alpha * T[0, 0] - D
    return D, S, tau


def fluxes(P, alpha, beta, g, gamma_ad, i):
    """D, S_j, tau and B^j fluxes along direction i (no GLM term)."""
    T, u, b, G, Gi, W = stress_energy(P, alpha, beta, g, gamma_ad)
    FD = alpha * P[0] * u[1 + i]
    FS = alpha * (T[1 + i, :] @ G[:, 1:])
    Ftau = alpha * alpha * T[1 + i, 0] - FD
    FB = alpha * (b[1:] * u[1 + i] - b[1 + i] * u[1:])
    return FD, FS, Ftau, FB


def sources(P, metric_fn, x, gamma_ad, h=1e-5):
    """S(S_j) and S(tau) with metric derivatives by fourth-order central
    differences of the 4-metric built from metric_fn(x) -> (alpha, beta, g)."""
    alpha, beta, g = metric_fn(x)
    T, u, b, G, Gi, W = stress_energy(P, alpha, beta, g, gamma_ad)
    dG = np.zeros((4, 4, 4))   # dG[mu] = d_mu g_{..}; d_t = 0
    dal = np.zeros(4)
    for k in range(3):
        def at(s):
            y = np.array(x, float)
            y[k] += s
            a_, b_, g_ = metric_fn(y)
            return four_metric(a_, b_, g_), a_
        Gp1, ap1 = at(h)
        Gm1, am1 = at(-h)
        Gp2, ap2 = at(2 * h)
        Gm2, am2 = at(-2 * h)
        dG[1 + k] = (8 * (Gp1 - Gm1) - (Gp2 - Gm2)) / (12 * h)
        dal[1 + k] = (8 * (ap1 - am1) - (ap2 - am2)) / (12 * h)
    SS = np.array([0.5 * alpha * np.sum(T * dG[1 + j]) for j in range(3)])
    # Gamma^0_{mu nu} = 1/2 g^{0 s} (d_mu g_{s nu} + d_nu g_{s mu} - d_s g_{mu nu})
    Gam0 = np.zeros((4, 4))
    for m in range(4):
        for n in range(4):
            Gam0[m, n] = 0.5 * sum(Gi[0, s] * (dG[m][s, n] + dG[n][s, m] - dG[s][m, n]) for s in range(4))
    Stau = alpha * (T[:, 0] @ dal - alpha * np.sum(T * Gam0))
    return SS, Stau
