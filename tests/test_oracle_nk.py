"""Pins of the oracle's Jacobian-free Newton-Krylov inversion (Grid.c2p = "nk")
against facts that do not come from the oracle's own solver.

The Newton-Krylov step solves the same momentum and energy equations in
(Z, v^2) as the Newton-Raphson one, with GMRES on difference quotients in
place of the analytic Jacobian, so:
- a primitive state sent to conserved variables and back is recovered (the
  exact answer is the input, by construction);
- the root agrees with a 50-digit bisection of the energy equation;
- it converges from the previous stage's state without the backup solver,
  and to the same root as the analytic Newton iteration (two different
  algorithms on one system);
- a step of the torus with either solver gives the same state up to the
  stopping tolerance, but not the same bits (the switch is effective).
CPU only."""
import math

import numpy as np
import pytest

import oracle
import problems as pb
from tests.test_oracle_pins import ks_grid, random_state


def _grid(coords):
    g = ks_grid("mks") if coords == "mks" else pb.periodic_box(gamma_ad=4.0 / 3.0)
    return g.with_(rho_floor=1e-30, p_floor=1e-30, rho_floor_pow=0.0, p_floor_pow=0.0)


@pytest.mark.parametrize("coords", ["cart", "mks"])
def test_nk_round_trip(coords):
    """prim -> con -> prim over rho in [1e-8, 1e2], p/rho in [1e-6, 1e2],
    W in [1, 20], sigma in [0, 100], from a guess 0.1% away: backward error
    <= 5e-14, forward error within the conditioning bound of the analytic
    Newton pin (1e-12 or 8 cond eps), and no cell needs the backup.  (The
    analytic pin's backward bound is 1e-14: the stopping test looks at dZ
    only, and the last accepted step of Newton-Krylov carries the difference
    quotients' error, about 1e-8 of the step times the Jacobian's condition,
    in v^2: 1.3e-14 for a sigma = 63, W = 14 state of this sample.)"""
    g = _grid(coords)
    nk = oracle.Point(g.with_(c2p="nk"))
    rng = np.random.default_rng(17)
    for _ in range(300):
        x = [math.log(rng.uniform(1.3, 100)), rng.uniform(0.05, 0.95), 1.0] if coords == "mks" else [0.5] * 3
        m = nk.metric(x, derivs=False)
        rho = 10 ** rng.uniform(-8, 2)
        p = rho * 10 ** rng.uniform(-6, 2)
        W = 1 + 19 * rng.random() ** 2
        d = rng.normal(size=3)
        u = d * math.sqrt((W * W - 1) / (d @ m.g @ d))
        e = rng.normal(size=3)
        sigma = 100 * rng.random() ** 2
        B = e * math.sqrt(sigma * rho * W * W / (e @ m.g @ e))
        P = np.array([rho, p, *u, *B, 0.01])
        U = nk.prim2con(m, P)
        Q, st = nk.con2prim(m, U, P * (1 + 1e-3 * rng.normal(size=9)))
        assert st == 0, (P, st)
        back = np.abs(nk.prim2con(m, Q)[:5] - U[:5]).max() / np.abs(U[:5]).max()
        assert back < 5e-14
        cond = (U[4] + U[0] + np.abs(U[1:4]).sum() + B @ m.g @ B) / p
        unorm = max(math.sqrt(u @ m.g @ u), 1e-300)
        err = np.abs(Q[:5] - P[:5]) / np.array([rho, p, unorm, unorm, unorm])
        assert err.max() < max(1e-12, 8 * cond * 2.2e-16), (P, Q, err, cond)


def test_nk_agrees_with_high_precision_root():
    """Z = rho h W^2 from a 50-digit bisection of the energy equation (v^2
    eliminated with the momentum equation) equals the Newton-Krylov result to
    1e-12."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    pt = oracle.Point(pb.periodic_box(gamma_ad=4.0 / 3.0, c2p="nk"))
    m = pt.metric([0.5] * 3)
    rng = np.random.default_rng(18)
    for _ in range(5):
        P = random_state(rng, m.g, sigma_max=20.0, wmax=6.0)
        U = pt.prim2con(m, P)
        Q, st = pt.con2prim(m, U, P * (1 + 1e-2 * rng.normal(size=9)))
        assert st == 0
        D, S, tau, B = (mp.mpf(U[0]), [mp.mpf(s) for s in U[1:4]], mp.mpf(U[4]), [mp.mpf(b) for b in U[5:8]])
        S2 = sum(s * s for s in S)
        B2 = sum(b * b for b in B)
        BS = sum(b * s for b, s in zip(B, S))
        gam = mp.mpf(4) / 3

        def v2(Z):
            return (S2 + BS * BS * (2 * Z + B2) / (Z * Z)) / (Z + B2) ** 2

        def f(Z):
            w2 = v2(Z)
            pr = (gam - 1) / gam * (Z * (1 - w2) - D * mp.sqrt(1 - w2))
            return Z - pr + B2 * (1 + w2) / 2 - BS * BS / (2 * Z * Z) - (tau + D)

        Zt = mp.mpf((P[0] + 4 * P[1]) * (1 + P[2:5] @ m.g @ P[2:5]))
        lo, hi = Zt * (1 - mp.mpf("1e-6")), Zt * (1 + mp.mpf("1e-6"))
        assert f(lo) < 0 < f(hi)
        for _ in range(300):
            mid = (lo + hi) / 2
            if f(mid) > 0:
                hi = mid
            else:
                lo = mid
        Z = (lo + hi) / 2
        W = 1 / mp.sqrt(1 - v2(Z))
        assert float(D / W) == pytest.approx(Q[0], rel=1e-12)
        Zq = (Q[0] + 4 * Q[1]) * (1 + Q[2:5] @ Q[2:5])
        assert Zq == pytest.approx(float(Z), rel=1e-12)


@pytest.mark.parametrize("sigma_max, wmax, spread", [(10.0, 5.0, 1e-3), (1e3, 10.0, 1e-3), (10.0, 5.0, 3e-2)])
def test_nk_and_newton_reach_the_same_root(sigma_max, wmax, spread):
    """Random states (strongly magnetized and fast ones too) from guesses 0.1%
    and 3% away: both solvers succeed without the backup and agree to 1e-11
    (or 8 cond eps where recovering p from the energy is ill-conditioned)."""
    g = pb.periodic_box(gamma_ad=4.0 / 3.0, rho_floor=1e-30, p_floor=1e-30)
    newton, nk = oracle.Point(g), oracle.Point(g.with_(c2p="nk"))
    m = newton.metric([0.5] * 3)
    rng = np.random.default_rng(19)
    for _ in range(200):
        P = random_state(rng, m.g, sigma_max=sigma_max, wmax=wmax)
        U = newton.prim2con(m, P)
        guess = P * (1 + spread * rng.normal(size=9))
        Qa, sa = newton.con2prim(m, U, guess)
        Qb, sb = nk.con2prim(m, U, guess)
        assert sa == 0 and sb == 0, (P, sa, sb)
        unorm = max(np.abs(Qa[2:5]).max(), 1e-300)
        err = np.abs(Qa[:5] - Qb[:5]) / np.array([Qa[0], Qa[1], unorm, unorm, unorm])
        cond = (U[4] + U[0] + np.abs(U[1:4]).sum() + P[5:8] @ m.g @ P[5:8]) / P[1]
        assert err.max() <= max(1e-11, 8 * cond * 2.2e-16), (P, err, cond)


def test_torus_step_with_nk_matches_newton():
    """One step of the 2-D torus (floors, atmosphere, magnetized torus) with
    each solver: the same state to 1e-11 (energy-scaled), the same inversion
    outcomes, and not the same bits."""
    from tests.test_gpu_parity import energy_scaled
    g = pb.torus_2d(nblock=16, nroot=(6, 4))
    P = pb.fm_torus_prims(g)
    outs = []
    for c2p in ("newton", "nk"):
        o = oracle.Oracle(g.with_(c2p=c2p))
        o.set_prims(P)
        dt = o.cfl_dt()
        o.step(dt)
        outs.append((o.cons(), o.c2p_status()))
    err = energy_scaled(outs[1][0], outs[0][0], g)
    assert np.all(err <= 1e-11), err
    assert (outs[0][1] != outs[1][1]).mean() <= 1e-3
    assert not np.array_equal(outs[0][0], outs[1][0])
