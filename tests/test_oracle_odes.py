"""Closed forms of the source terms on uniform states (CPU only).

On a uniform state over flat bathymetry every flux difference vanishes in
cells more than 4 n cells from the walls after n steps (radius-2 stencil,
two stages), so those cells follow the scheme's time integrator applied to
the source ODE alone:

* Coriolis (eq:swe): d(hu, hv)/dt = f (hv, -hu). SSP-RK2 (eq:rk2) applied
  to it is the linear map R = I + dt A + (dt A)^2 / 2; the oracle must match
  R^n exactly and the continuous rotation at second order in dt.
* Bottom drag: d(hu)/dt = -C_d u |u| has hu(t) = hu0 / (1 + C_d |u0| t / h);
  the semi-implicit update eq:rk2_semiimp converges to it at first order
  (for a constant rate s it reduces to the implicit Euler factor
  1/(1 + dt s) per step).
"""
import numpy as np

from tests import helpers


def _uniform(nx, depth, hu0, hv0, f=0.0, cd=0.0, dx=10e3, dt=50.0):
    wl = helpers.flat(nx, nx, depth=depth, dx=dx, dy=dx, f=f, theta=0.37, cd=cd,
                      dt_fixed=dt)
    wl.hu = np.full((nx, nx), hu0)
    wl.hv = np.full((nx, nx), hv0)
    return wl


def test_inertial_oscillation_discrete_propagator(oracle_mod):
    f, dt, n = 1e-3, 50.0, 20
    wl = _uniform(200, 10.0, 1.0, 0.5, f=f, dt=dt)
    e, u, v, *_ = oracle_mod.Oracle(wl).run(n)
    A = f * np.array([[0.0, 1.0], [-1.0, 0.0]])
    R = np.eye(2) + dt * A + 0.5 * (dt * A) @ (dt * A)
    y = np.linalg.matrix_power(R, n) @ np.array([1.0, 0.5])
    c = 100
    assert abs(u[c, c] - y[0]) < 1e-13
    assert abs(v[c, c] - y[1]) < 1e-13
    assert e[c, c] == 0.0


def test_inertial_oscillation_second_order(oracle_mod):
    f, T = 1e-3, 1000.0
    errs = []
    for n in (10, 20, 40):
        dt = T / n
        wl = _uniform(4 * 4 * n + 20, 10.0, 1.0, 0.5, f=f, dt=dt)
        e, u, v, *_ = oracle_mod.Oracle(wl).run(n)
        c = wl.nx // 2
        exact = (np.cos(f * T) + 0.5 * np.sin(f * T), 0.5 * np.cos(f * T) - np.sin(f * T))
        errs.append(np.hypot(u[c, c] - exact[0], v[c, c] - exact[1]))
    o1 = np.log2(errs[0] / errs[1])
    o2 = np.log2(errs[1] / errs[2])
    assert 1.8 < o1 < 2.2 and 1.8 < o2 < 2.2, (errs, o1, o2)


def test_friction_closed_form_first_order(oracle_mod):
    cd, h, hu0, T = 0.01, 1.0, 1.0, 200.0
    exact = hu0 / (1.0 + cd * abs(hu0 / h) * T / h)
    errs = []
    for n in (10, 20, 40):
        dt = T / n
        wl = _uniform(4 * 4 * n + 20, h, hu0, 0.0, cd=cd, dx=1e3, dt=dt)
        e, u, v, *_ = oracle_mod.Oracle(wl).run(n)
        c = wl.nx // 2
        assert v[c, c] == 0.0
        errs.append(abs(u[c, c] - exact))
    o1 = np.log2(errs[0] / errs[1])
    o2 = np.log2(errs[1] / errs[2])
    assert 0.8 < o1 < 1.2 and 0.8 < o2 < 1.2, (errs, o1, o2)
    assert errs[-1] < 0.02 * exact


def test_friction_constant_rate_is_implicit_euler(oracle_mod):
    """With a uniform flow the drag rate is the same in both stages only to
    first order; with hu tiny against h the rate is near-constant and the
    per-step factor approaches 1/(1 + dt s)."""
    cd, h, hu0, dt, n = 1e-2, 100.0, 1e-3, 10.0, 4
    wl = _uniform(60, h, hu0, 0.0, cd=cd, dx=1e3, dt=dt)
    e, u, v, *_ = oracle_mod.Oracle(wl).run(n)
    s = cd * abs(hu0 / h) / h
    c = 30
    assert abs(u[c, c] - hu0 / (1 + dt * s) ** n) < 1e-12 * hu0
