"""Pins of the oracle's IMEX treatment of the stiff cleaning damping
(IMEX-SSP2(2,2,2) of Pareschi & Russo 2005: the explicit SSP-RK2 stages plus
an L-stable implicit part for -alpha kappa psi) against facts that do not come
from the oracle: on a uniform state with no field the cleaning scalar obeys
d psi/dt = -kappa psi exactly, so the explicit path must follow the stability
polynomial 1 - z + z^2/2 of every two-stage second-order Runge-Kutta method
(unstable for z > 2), the IMEX path must stay bounded for any z and damp to
zero as z grows (L-stability), and both must converge to exp(-kappa t) at
second order.  With kappa = 0 the IMEX path is the explicit one bit for bit,
and the fluxes of D, S_i, tau never see psi, so one stage of each form gives
the same hydrodynamics.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import problems as pb


def _uniform(kappa, imex, psi0=0.3):
    g = pb.periodic_box(ndim=2, nblock=4, nroot=2, kappa=kappa, imex=imex, ch=1.0)
    P = pb.empty_prims(g)
    P[:, 0] = 1.0
    P[:, 1] = 0.5
    P[:, 8] = psi0
    o = oracle.Oracle(g)
    o.set_prims(P)
    return o


def _psi_after(kappa, imex, dt, n):
    o = _uniform(kappa, imex)
    for _ in range(n):
        o.step(dt)
    psi = o.prims()[:, 8]
    assert np.ptp(psi) <= 1e-15 * max(1.0, np.abs(psi).max())  # stays uniform
    return float(psi.flat[0])


def test_explicit_damping_follows_the_two_stage_stability_polynomial():
    for z in (0.5, 1.5, 3.0):
        got = _psi_after(1.0, False, z, 4) / 0.3
        assert got == pytest.approx((1 - z + z * z / 2) ** 4, rel=1e-13)
    assert abs(_psi_after(1.0, False, 3.0, 4)) > 0.3  # explicit: grows for z > 2


@pytest.mark.parametrize("z", [3.0, 10.0, 1e2, 1e4])
def test_imex_damping_is_bounded_and_l_stable(z):
    r1 = _psi_after(1.0, True, z, 1) / 0.3
    r4 = _psi_after(1.0, True, z, 4) / 0.3
    assert abs(r1) < 1.0
    assert r4 == pytest.approx(r1 ** 4, rel=1e-12, abs=1e-300)
    if z >= 1e4:
        assert abs(r1) < 1e-3  # the amplification vanishes as z -> infinity


@pytest.mark.parametrize("imex", [False, True])
def test_damping_converges_at_second_order(imex):
    errs = []
    for n in (8, 16, 32):
        psi = _psi_after(1.0, imex, 1.0 / n, n)
        errs.append(abs(psi - 0.3 * math.exp(-1.0)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.9, (errs, orders)


def test_imex_without_damping_is_the_explicit_step():
    g = pb.periodic_box(ndim=2, nblock=8, nroot=2, kappa=0.0)
    P = pb.random_periodic_prims(g)
    outs = []
    for imex in (False, True):
        o = oracle.Oracle(g.with_(imex=imex))
        o.set_prims(P)
        dt = o.cfl_dt()
        o.step(dt)
        o.step(dt)
        outs.append(o.cons())
    assert np.array_equal(outs[0], outs[1])


def test_one_imex_stage_leaves_the_hydrodynamics_of_the_explicit_stage():
    g = pb.periodic_box(ndim=2, nblock=8, nroot=2, kappa=5.0)
    P = pb.random_periodic_prims(g)
    outs = []
    for imex in (False, True):
        o = oracle.Oracle(g.with_(imex=imex))
        o.set_prims(P)
        dt = o.cfl_dt()
        o.stage(1, dt)
        outs.append(o.cons())
    assert np.array_equal(outs[0][:, :5], outs[1][:, :5])
    assert not np.array_equal(outs[0][:, 8], outs[1][:, 8])


def _telegraph_l1(n, imex, kappa=20.0, eps=1e-4, t_end=0.25):
    """Flat fluid at rest with B^x = eps sin(2 pi x) (so div B != 0), psi = 0:
    the cleaning pair obeys d_t B^x = -d_x psi, d_t psi = -ch^2 d_x B^x -
    kappa psi, so B^x = b(t) sin(kx), psi = p(t) cos(kx) with
    (b, p)(t) = expm([[0, k], [-ch^2 k, -kappa]] t) (eps, 0).  Returns the L1
    error of B^x at t_end (the field's back-reaction on the fluid is
    O(eps^2))."""
    sl = pytest.importorskip("scipy.linalg")
    g = pb.Grid(ndim=2, nx=(n, 4, 1), nroot=(1, 1, 1), xmin=(0, 0, 0), xmax=(1.0, 4.0 / n, 1.0),
                gamma_ad=5.0 / 3.0, kappa=kappa, ch=1.0, imex=imex, cfl=0.4)
    x = pb.cell_centres(g)[0]
    k = 2 * math.pi
    P = pb.empty_prims(g)
    P[:, 0] = 1.0
    P[:, 1] = 1.0
    P[:, 5] = eps * np.sin(k * x)
    o = oracle.Oracle(g)
    o.set_prims(P)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(o.cfl_dt(), t_end - t)
        o.step(dt)
        t += dt
    b, _ = sl.expm(np.array([[0.0, k], [-k, -kappa]]) * t_end) @ np.array([eps, 0.0])
    return float(np.mean(np.abs(o.prims()[:, 5] - b * np.sin(k * x))))


@pytest.mark.parametrize("imex", [False, True])
def test_coupled_cleaning_system_converges_at_second_order(imex):
    """Order >= 1.75 from 64 to 128 to 256 cells (PPM clips the smooth
    extrema, so the L1 order settles near 1.9).  The stage-1 fluxes of the IMEX scheme must see the implicit first stage
    Y1 (psi scaled by 1/(1 + gamma alpha kappa dt)); evaluated at psi_n the
    scheme drops to first order on this coupled problem."""
    e = [_telegraph_l1(n, imex) for n in (64, 128, 256)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(orders) > 1.75, (e, orders)
