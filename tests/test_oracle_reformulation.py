"""The local reformulation of Section 3.1 against the recursive form it
replaces (CPU only).

The test builds the face values of h the way the original scheme defines
them: the Coriolis primitive V by the prefix sum of eq:recursiveV, the cell
averages K of eq:discK, limited differences of K, and h^E, h^W from
eq:hOnFaces_E / eq:hOnFaces_W. The oracle computes them with the local
expressions eq:Kbackwards and eq:hE only; both must agree to round-off."""
import numpy as np

from tests import helpers


def _recursive_faces(eta, v, f, HE, HW, dx, g, theta_mm):
    nx = eta.shape[0]
    V = np.zeros(nx + 1)                      # V_{i-1/2}, V_{-1/2} = 0
    for i in range(nx):
        V[i + 1] = V[i] + dx / g * f[i] * v[i]
    K = g * (eta - 0.5 * (V[1:] + V[:-1]))
    out_E = np.full(nx, np.nan)
    out_W = np.full(nx, np.nan)
    for i in range(1, nx - 1):
        bw = (K[i] - K[i - 1]) / dx
        fw = (K[i + 1] - K[i]) / dx
        ce = 0.5 * (bw + fw)
        a, b, c = theta_mm * bw, ce, theta_mm * fw
        if a > 0 and b > 0 and c > 0:
            Kx = min(a, b, c)
        elif a < 0 and b < 0 and c < 0:
            Kx = max(a, b, c)
        else:
            Kx = 0.0
        out_E[i] = (K[i] + 0.5 * dx * Kx) / g + V[i + 1] + HE[i]
        out_W[i] = (K[i] - 0.5 * dx * Kx) / g + V[i] + HW[i]
    return out_E, out_W


def test_local_equals_recursive(oracle_mod):
    nx, ny = 48, 6
    rng = np.random.default_rng(7)
    wl = helpers.flat(nx, ny, depth=80.0, dx=1500.0, dy=1500.0)
    Hc = 80.0 + 10 * rng.standard_normal((ny + 1, nx + 1))
    wl.H = Hc
    wl.f = 1e-4 + 3e-5 * rng.standard_normal((ny, nx))
    wl.theta = np.zeros((ny, nx))
    wl.eta = 0.3 * np.sin(np.arange(nx) / 5.0)[None, :] + 0.05 * rng.standard_normal((ny, nx))
    wl.hu = 2.0 * rng.standard_normal((ny, nx))
    wl.hv = 5.0 + 3.0 * rng.standard_normal((ny, nx))
    o = oracle_mod.Oracle(wl)
    etaE, etaW, hE, hW = o.recon_x(wl.eta, wl.hu, wl.hv)
    for j in range(ny):
        Hbar = 0.25 * (Hc[j, :-1] + Hc[j, 1:] + Hc[j + 1, :-1] + Hc[j + 1, 1:])
        HE = 0.5 * (Hc[j, 1:] + Hc[j + 1, 1:])
        HW = 0.5 * (Hc[j, :-1] + Hc[j + 1, :-1])
        v = wl.hv[j] / (wl.eta[j] + Hbar)
        rE, rW = _recursive_faces(wl.eta[j], v, wl.f[j], HE, HW, wl.dx, 9.81, 1.3)
        sl = slice(1, nx - 1)
        assert np.abs(hE[j, sl] - rE[sl]).max() < 1e-10
        assert np.abs(hW[j, sl] - rW[sl]).max() < 1e-10
        # and the slopes really are non-trivial
        assert np.abs(hE[j, sl] - hW[j, sl]).max() > 1e-3


def _h_form_flux(L, R, Hf, d, g=9.81, kappa=1e-2):
    """eqn:numerical_flux on Q = [h, hu, hv] with the physical flux of eq:swe
    (pressure g h^2 / 2) and desingularised velocities (eq:desing_ours); zero
    when a+ = a-."""
    def desing(h):
        r = max(abs(h), min(h * h / (2 * kappa) + kappa / 2, kappa))
        return -r if h < 0 else r

    def side(s):
        h, eta, hu, hv = s
        u, v = hu / desing(h), hv / desing(h)
        hu, hv = h * u, h * v
        if d == 0:
            F = np.array([hu, hu * u + 0.5 * g * h * h, hu * v])
            un = u
        else:
            F = np.array([hv, hv * u, hv * v + 0.5 * g * h * h])
            un = v
        return F, np.array([h, hu, hv]), un, np.sqrt(g * h)

    FL, QL, uL, cL = side(L)
    FR, QR, uR, cR = side(R)
    ap = max(uL + cL, uR + cR, 0.0)
    am = min(uL - cL, uR - cR, 0.0)
    if ap - am == 0.0:
        return np.zeros(3)
    return (ap * FL - am * FR) / (ap - am) + ap * am / (ap - am) * (QR - QL)


def test_eta_form_equals_h_form(oracle_mod):
    """The eta-variable flux (pressure g eta (eta + 2 H_f)/2) differs from the
    h-form flux of eqn:numerical_flux by exactly the constant g H_f^2/2 in the
    normal momentum, for wet, partly dry and fully dry faces alike (Section
    3.2 replaces h by eta for accuracy without changing the scheme)."""
    rng = np.random.default_rng(17)
    g = 9.81
    n_checked = 0
    for trial in range(4000):
        Hf = float(rng.choice([rng.uniform(-3, 5), rng.uniform(5, 3000)]))
        sides = []
        for _ in range(2):
            kind = rng.integers(0, 4)
            h = 0.0 if kind == 0 else float(rng.uniform(0, 0.02) if kind == 1 else rng.uniform(0, 50))
            hu = 0.0 if kind == 0 and rng.random() < 0.7 else float(rng.normal(0, 2))
            hv = 0.0 if kind == 0 and rng.random() < 0.7 else float(rng.normal(0, 2))
            sides.append((h, h - Hf, hu, hv))
        for d in (0, 1):
            eta_flux = oracle_mod.face_flux(sides[0], sides[1], Hf, d)
            shift = np.zeros(3)
            shift[1 + d] = 0.5 * g * Hf * Hf
            href = _h_form_flux(sides[0], sides[1], Hf, d)
            scale = max(np.abs(href).max(), 0.5 * g * Hf * Hf, 1.0)
            assert np.abs(eta_flux + shift - href).max() <= 1e-11 * scale, (sides, Hf, d)
            n_checked += 1
    assert n_checked == 8000
