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


def glm_source(P, metric_fn, x, ch, kappa, h=1e-5):
    """Source of the cleaning scalar psi for the conservative form
        d_t(sqrt(gamma) psi) + d_i[sqrt(gamma) (alpha ch^2 B^i - beta^i psi)] = sqrt(gamma) S
    implied by the covariant damped cleaning equation
        (d_t - beta^i d_i) psi = -alpha ch^2 D_i B^i - alpha kappa psi
    (the time derivative along the normal observer; D_i B^i the covariant
    divergence) in a stationary metric:
        S_cov = -alpha kappa psi + ch^2 B^i d_i alpha - psi D_i beta^i,
        D_i beta^i = d_i(sqrt(gamma) beta^i) / sqrt(gamma).
    Returns (S_cov, psi beta^i d_i ln sqrt(gamma)).  alpha, beta^i and
    sqrt(gamma) are read off the inverse 4-metric of metric_fn(y) ->
    (alpha, beta, g): alpha = (-g^00)^(-1/2), beta^i = alpha^2 g^0i,
    sqrt(gamma) = sqrt(-det g_4) / alpha; derivatives by fourth-order central
    differences."""
    def lapse_shift_vol(y):
        a_, b_, g_ = metric_fn(y)
        G = four_metric(a_, b_, g_)
        Gi = np.linalg.inv(G)
        al = 1.0 / np.sqrt(-Gi[0, 0])
        be = al * al * Gi[0, 1:]
        sg = np.sqrt(-np.linalg.det(G)) / al
        return al, be, sg

    alpha, beta, sg = lapse_shift_vol(np.asarray(x, float))
    dal = np.zeros(3)
    dln = np.zeros(3)
    div = 0.0
    for k in range(3):
        vals = []
        for s in (h, -h, 2 * h, -2 * h):
            y = np.array(x, float)
            y[k] += s
            vals.append(lapse_shift_vol(y))
        (a1, b1, s1), (am1, bm1, sm1), (a2, b2, s2), (am2, bm2, sm2) = vals
        dal[k] = (8 * (a1 - am1) - (a2 - am2)) / (12 * h)
        dln[k] = (8 * (np.log(s1) - np.log(sm1)) - (np.log(s2) - np.log(sm2))) / (12 * h)
        div += (8 * (s1 * b1[k] - sm1 * bm1[k]) - (s2 * b2[k] - sm2 * bm2[k])) / (12 * h) / sg
    B = np.asarray(P[5:8], float)
    psi = P[8]
    s_cov = -alpha * kappa * psi + ch * ch * (B @ dal) - psi * div
    return s_cov, psi * (beta @ dln)
