"""Pins for the FP64 oracle against things other than itself: closed forms,
paper-stated special cases, brute-force dense algebra, finite differences,
published known-answer vectors.  CPU only."""
import math
import os

import numpy as np
import pytest
from scipy.optimize import brentq, minimize_scalar

from oracle import pta_oracle as O
from paper_2607_06834_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pos(theta_deg):
    t = math.radians(theta_deg)
    return np.array([[0.0, 0.0, 1.0], [math.sin(t), 0.0, math.cos(t)]])


def _hd(theta_deg):
    return O.hellings_downs(_pos(theta_deg))[0, 1]


# --------------------------------------------------------------- Eq. (HD)
def test_hd_golden_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "hellings_downs.txt"))
            if l.strip() and not l.startswith("#")]
    for kind, th, val, tol, *_ in rows:
        th, val, tol = float(th), float(val), float(tol)
        if kind == "value":
            got = O.hellings_downs(_pos(th))[0, 0] if th == 0.0 else _hd(th)
            assert abs(got - val) <= tol, (kind, th, got)
        elif kind == "limit":
            assert abs(_hd(th) - val) <= tol
        elif kind == "zero":
            root = math.degrees(brentq(lambda d: _hd(math.degrees(d)), math.radians(th - 5),
                                       math.radians(th + 5)))
            assert abs(root - th) <= tol * 100, root
        elif kind == "min":
            r = minimize_scalar(_hd, bounds=(60, 100), method="bounded", options={"xatol": 1e-8})
            assert abs(r.x - th) <= tol * 100 and abs(r.fun - val) <= tol


def test_hd_matrix_pd_and_diag():
    rng = np.random.default_rng(0)
    v = rng.normal(size=(40, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    G = O.hellings_downs(v)
    assert np.allclose(np.diag(G), 1.0)
    assert np.allclose(G, G.T)
    assert np.linalg.eigvalsh(G).min() > 0.0


# --------------------------------------------------------------- Eq. (power_law)
def test_power_law_hand_value():
    T = 10 * O.YEAR_S
    rho = O.power_law(-14.7, 13.0 / 3.0, np.array([1, 10]), T)
    # computed by hand from the equation: sqrt(rho_1) = 268.5 ns, sqrt(rho_10) = 1.83 ns
    assert abs(math.sqrt(rho[0]) - 268.5) < 0.2
    assert abs(math.sqrt(rho[1]) - 1.83) < 0.01


def test_power_law_matches_characteristic_strain_route():
    """rho_k = S(f_k)/T with the one-sided PSD S = h_c^2/(12 pi^2 f^3) and the
    characteristic strain h_c = A (f/f_yr)^((3 - gamma)/2)."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        la, g = rng.uniform(-18, -12), rng.uniform(0.5, 6.5)
        T = rng.uniform(3, 30) * O.YEAR_S
        k = np.arange(1, 31)
        f = k / T
        hc = 10 ** la * (f / O.F_YR) ** ((3 - g) / 2)
        S = hc ** 2 / (12 * math.pi ** 2 * f ** 3)
        np.testing.assert_allclose(O.power_law(la, g, k, T), S / T * 1e18, rtol=1e-12)


def test_power_law_invariants():
    T = 12 * O.YEAR_S
    k = np.arange(1, 20)
    for g in (1.0, 13 / 3, 6.0):
        r = O.power_law(-15, g, k, T)
        np.testing.assert_allclose(r[1] / r[0], 2.0 ** -g, rtol=1e-13)
        np.testing.assert_allclose(O.power_law(-14, g, k, T) / r, 100.0, rtol=1e-12)
    # at f = f_yr the spectrum is independent of gamma
    Tyr = 7 * O.YEAR_S
    vals = [O.power_law(-15, g, np.array([7]), Tyr)[0] for g in (0.5, 3.0, 6.5)]
    np.testing.assert_allclose(vals, vals[0], rtol=1e-12)


# --------------------------------------------------------------- Eq. (WN_cov)
def _golden_rows(name):
    return [[float(v) for v in l.split()] for l in open(os.path.join(GOLDEN, name))
            if l.strip() and not l.startswith("#")]


def test_white_noise_golden_values():
    """N_ii against values worked by hand from Eq. (WN_cov) (tests/golden/white_noise.txt);
    each TOA has its own backend so EFAC/EQUAD are picked per row."""
    from types import SimpleNamespace
    rows = _golden_rows("white_noise.txt")
    psr = SimpleNamespace(sigma_s=np.array([r[0] * 1e-6 for r in rows]),
                          backend=np.arange(len(rows), dtype=np.int32),
                          efac=np.array([r[1] for r in rows]),
                          equad_s=np.array([r[2] * 1e-6 for r in rows]))
    np.testing.assert_allclose(O.white_noise_var(psr), [r[3] for r in rows], rtol=1e-12)
    # backend selection: the same sigma under two backends takes each backend's EFAC/EQUAD
    psr2 = SimpleNamespace(sigma_s=np.array([1e-6, 1e-6]), backend=np.array([1, 0], dtype=np.int32),
                           efac=np.array([1.2, 0.8]), equad_s=np.array([0.5e-6, 0.1e-6]))
    np.testing.assert_allclose(O.white_noise_var(psr2), [0.64e6 + 1e4, 1.69e6], rtol=1e-12)


def test_chromatic_weight_golden_values():
    """DM basis weight (nu_ref/nu)^2, nu_ref = 1400 MHz, against hand values
    (tests/golden/chromatic_weight.txt): 4 at 700 MHz, 1/4 at 2800 MHz."""
    rows = _golden_rows("chromatic_weight.txt")
    nu = np.array([r[0] for r in rows])
    np.testing.assert_allclose(O.chromatic_weight(nu), [r[1] for r in rows], rtol=1e-14)
    # and the oracle's DM columns are the achromatic ones times that weight, row by row
    arr = synth.small_array(npsr=1, ntoa=40, n_gwb=2, n_rn=3, n_dm=2, seed=8)
    orc = O.Oracle(arr)
    F = orc.get_F(0)
    w = (1400.0 / arr.pulsars[0].freqs_mhz) ** 2
    np.testing.assert_allclose(F[:, 2 * orc.na:], F[:, :4] * w[:, None], rtol=1e-13)


# --------------------------------------------------------------- Eq. (Fourier_series)
def test_fourier_basis_orthogonal_on_dense_grid():
    T = 1.0
    n = 4000
    t = (np.arange(n) + 0.5) / n * T
    F = O.fourier_basis(t, T, 6)
    G = F.T @ F / (n / 2)
    np.testing.assert_allclose(G, np.eye(12), atol=1e-10)
    # column order [sin k, cos k]: a = e_{2k} picks sin(2 pi k t/T)
    np.testing.assert_allclose(F[:, 4], np.sin(2 * math.pi * 3 * t / T), atol=1e-15)
    np.testing.assert_allclose(F[:, 5], np.cos(2 * math.pi * 3 * t / T), atol=1e-15)


# --------------------------------------------------------------- Eq. (Gmatrix_proj)
@pytest.mark.parametrize("m,nb", [(3, 1), (11, 3)])
def test_ntilde_three_routes_agree(m, nb):
    arr = synth.small_array(npsr=1, ntoa=70, m=m, nbackend=nb, seed=5)
    p = arr.pulsars[0]
    N = O.white_noise_var(p)
    A = O.ntilde_inv_G(N, p.M)
    B = O.ntilde_inv_svd(N, p.M)
    C = O.ntilde_inv_woodbury(N, p.M, np.eye(p.n))
    scale = np.abs(A).max()
    assert np.abs(A - B).max() < 1e-11 * scale
    assert np.abs(A - C).max() < 1e-11 * scale
    # projector properties: N~^-1 M = 0, N~^-1 N N~^-1 = N~^-1
    assert np.abs(A @ p.M).max() < 1e-10 * scale * np.abs(p.M).max()
    np.testing.assert_allclose(A @ (N[:, None] * A), A, atol=1e-11 * scale)
    # invariance to a change of timing-model parameterisation M -> M R
    R = np.random.default_rng(0).normal(size=(p.m, p.m)) + 3 * np.eye(p.m)
    D = O.ntilde_inv_woodbury(N, p.M @ R, np.eye(p.n))
    assert np.abs(D - C).max() < 1e-10 * scale


# --------------------------------------------------------------- whole posterior vs brute force
def _closed_form_logZ(orc, x):
    """logp_full is exactly quadratic in z at fixed theta (no CW): integrate it."""
    Dz = orc.Dz

    def f(z):
        xx = x.copy()
        xx[:Dz] = z
        return orc.logp_full(xx)
    c0 = f(np.zeros(Dz))
    H = np.zeros((Dz, Dz))
    g = np.zeros(Dz)
    for i in range(Dz):
        e = np.zeros(Dz)
        e[i] = 1.0
        g[i] = (f(e) - f(-e)) / 2
        for j in range(i, Dz):
            e2 = np.zeros(Dz)
            e2[j] = 1.0
            H[i, j] = H[j, i] = -(f(e + e2) - f(e - e2) - f(-e + e2) + f(-e - e2)) / 4
    _, ld = np.linalg.slogdet(H)
    return c0 + 0.5 * g @ np.linalg.solve(H, g) + 0.5 * Dz * math.log(2 * math.pi) - 0.5 * ld


@pytest.mark.parametrize("kw", [
    dict(npsr=2, ntoa=40, m=3, n_gwb=2, n_rn=3, n_dm=2, seed=1),
    dict(npsr=3, ntoa=30, m=3, n_gwb=3, n_rn=2, n_dm=0, seed=2),
    dict(npsr=2, ntoa=45, m=9, n_gwb=2, n_rn=2, n_dm=1, seed=4, nbackend=2),
    # free spectral models (Sec. "Priors"): one variance parameter per bin
    dict(npsr=2, ntoa=40, m=3, n_gwb=3, n_rn=2, n_dm=1, seed=5, gwb_free=True),
    dict(npsr=3, ntoa=35, m=3, n_gwb=2, n_rn=3, n_dm=0, seed=6, gwb_free=True, rn_free=True),
])
def test_marginal_likelihood_matches_dense_gaussian(kw):
    arr = synth.small_array(**kw)
    orc = O.Oracle(arr)
    for s in range(2):
        x = synth.make_points(arr, 1, seed=10 + s)[0].astype(np.float64)
        a = _closed_form_logZ(orc, x)
        b = orc.dense_marginal(x)
        assert abs(a - b) <= 1e-9 * abs(b), (a, b)


def test_logdet_cancellation_prior_whitened():
    arr = synth.small_array(npsr=3, ntoa=30, m=3, n_gwb=3, n_rn=4, n_dm=2, seed=7)
    orc = O.Oracle(arr)
    X = synth.make_points(arr, 20, seed=8).astype(np.float64)
    c = orc.data_constant()
    for x in X:
        d = orc.logp_full(x) - (orc.logp(x) + c)
        assert abs(d - (-0.5 * orc.Dz * math.log(2 * math.pi))) < 1e-8


def test_gram_form_equivalence():
    """Eq. (raw_posterior) and Eq. (stochastic_posterior) differ by an a-independent
    constant, -1/2 dt^T N~^-1 dt."""
    arr = synth.small_array(npsr=2, ntoa=50, m=3, n_gwb=3, n_rn=3, n_dm=1, seed=9)
    orc = O.Oracle(arr)
    x = synth.make_points(arr, 1, seed=1)[0].astype(np.float64)
    rng = np.random.default_rng(0)
    diffs = []
    for _ in range(10):
        a = rng.normal(scale=200.0, size=(orc.npsr, orc.P))
        diffs.append(orc.raw_posterior_exponent(a, x) - orc.gram_posterior_exponent(a, x))
    const = sum(-0.5 * orc.dt_ns[I] @ O.ntilde_inv_woodbury(orc.Nvar[I], arr.pulsars[I].M, orc.dt_ns[I])
                for I in range(orc.npsr))
    np.testing.assert_allclose(diffs, const, rtol=1e-9, atol=1e-7 * abs(const))


# --------------------------------------------------------------- gradient
def _fd_grad(orc, x, idx, rel=1e-6):
    out = []
    for j in idx:
        h = rel * max(1.0, abs(x[j]))
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        out.append((orc.logp(xp) - orc.logp(xm)) / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("kw", [
    dict(npsr=3, ntoa=40, m=3, n_gwb=3, n_rn=4, n_dm=2, seed=11),
    dict(npsr=3, ntoa=40, m=5, n_gwb=4, n_rn=2, n_dm=0, seed=12, nbackend=2),
    dict(npsr=2, ntoa=40, m=3, n_gwb=2, n_rn=2, n_dm=1, seed=13, cw=True),
    dict(npsr=3, ntoa=40, m=3, n_gwb=3, n_rn=4, n_dm=2, seed=14, gwb_free=True, rn_free=True),
    dict(npsr=2, ntoa=40, m=4, n_gwb=4, n_rn=2, n_dm=0, seed=15, gwb_free=True),
])
def test_gradient_central_differences(kw):
    arr = synth.small_array(**kw)
    orc = O.Oracle(arr)
    x = synth.make_points(arr, 1, seed=21)[0].astype(np.float64)
    if arr.cw:
        c = orc.lay["th_cw"]
        x[c: c + 8] = [9.5, -7.8, -13.5, 0.3, 1.0, 0.2, 2.0, 1.0]
    g = orc.grad(x)
    idx = np.arange(orc.D)
    fd = _fd_grad(orc, x, idx)
    scale = np.abs(g).max()
    err = np.abs(fd - g)
    assert np.all(err <= 1e-6 * np.abs(g) + 1e-7 * scale), (np.argmax(err / (np.abs(g) + 1e-7 * scale)), err.max())


# --------------------------------------------------------------- CW invariants
def _cw_case():
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0, 15 * O.YEAR_S, 300))
    pos = np.array([0.3, -0.5, 0.81])
    pos /= np.linalg.norm(pos)
    th = np.array([9.4, -7.9, -14.0, 0.4, 0.9, -0.3, 4.0, 1.2])
    return t, pos, th


def test_cw_zero_amplitude_and_zero_distance():
    t, pos, th = _cw_case()
    th0 = th.copy()
    th0[2] = -40.0
    assert np.abs(O.cw_signal(t, pos, th0, 1.0, 0.3)).max() < 1e-20
    # pulsar at zero distance with its phase equal to Phi0: pulsar term = Earth term
    assert np.abs(O.cw_signal(t, pos, th, 0.0, th[7])).max() < 1e-9
    assert np.abs(O.cw_signal(t, pos, th, 1.0, 0.3)).max() > 1.0


def test_cw_polarisation_flip():
    t, pos, th = _cw_case()
    th2 = th.copy()
    th2[4] += math.pi / 2
    np.testing.assert_allclose(O.cw_signal(t, pos, th2, 1.3, 0.7), -O.cw_signal(t, pos, th, 1.3, 0.7),
                               rtol=1e-9, atol=1e-12)


def test_cw_phase_derivative_is_frequency():
    """d Phi/dt from Eq. (phase_evolve) equals omega(t) of Eq. (CW_evolve)."""
    mc = 10 ** 9.7 * O.TSUN_S
    w0 = math.pi * 10 ** -7.6
    for t in (0.0, 3e8, 9e8):
        h = 1e3
        d = (O.cw_phase(t + h, mc, w0)[0] - O.cw_phase(t - h, mc, w0)[0]) / (2 * h)
        assert d == pytest.approx(O.cw_phase(t, mc, w0)[1], rel=1e-6, abs=0)


def test_cw_taylor_form_small_x():
    mc = 10 ** 8.5 * O.TSUN_S
    w0 = math.pi * 10 ** -8.4
    t = np.linspace(0, 1e8, 11)
    np.testing.assert_allclose(O.cw_phase_taylor(t, mc, w0), O.cw_phase(t, mc, w0)[0], rtol=1e-4, atol=1e-9)


def test_cw_antenna_pattern_identity():
    """F+^2 + Fx^2 = (1 - Omega.p)^2 / 4 for any source and pulsar direction."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        p = rng.normal(size=3)
        p /= np.linalg.norm(p)
        fp, fx, op = O.cw_geometry(rng.uniform(-1, 1), rng.uniform(0, 2 * math.pi), p)
        assert fp * fp + fx * fx == pytest.approx(0.25 * (1 - op) ** 2, rel=1e-12)


def test_cw_special_geometry_golden_values():
    """Earth-term delay at t = 0 for geometries where the antenna pattern and the
    polarisation factors reduce to closed form (tests/golden/cw_special_geometry.txt,
    derived by hand from the circular-binary model of Sec. "Deterministic signals and
    continuous waves"): pins the amplitude h/(2 w0^(2/3) w^(1/3)), the inclination
    factors (1 + cos^2 i) and 2 cos i, the polarisation rotation and both patterns."""
    for line in open(os.path.join(GOLDEN, "cw_special_geometry.txt")):
        if line.startswith("#") or not line.strip():
            continue
        case, *v = line.split()
        px, py, pz, cosi, psi, phi0, phiI, s_ns = map(float, v)
        th = np.array([9.0, -8.0, -14.0, cosi, psi, 1.0, 0.0, phi0])
        s = O.cw_signal(np.array([0.0]), np.array([px, py, pz]), th, 1.3, phiI)
        assert abs(s[0] - s_ns) <= 1e-9 * abs(s_ns), (case, s[0], s_ns)


def test_cw_chirp_rate_is_quadrupole_formula():
    """Eq. (CW_evolve) at t = 0 must reproduce the quadrupole-formula chirp of a circular
    binary, d omega/dt = (96/5) Mc^(5/3) omega^(11/3) (Peters & Mathews 1963, with
    omega = pi f_gw and Mc in seconds), for several masses and frequencies."""
    for lmc, lf in ((8.5, -8.3), (9.4, -7.9), (10.0, -7.6)):
        mc = 10 ** lmc * O.TSUN_S
        w0 = math.pi * 10 ** lf
        h = 1e4
        dw = (O.cw_phase(h, mc, w0)[1] - O.cw_phase(-h, mc, w0)[1]) / (2 * h)
        assert dw == pytest.approx(96.0 / 5.0 * mc ** (5.0 / 3.0) * w0 ** (11.0 / 3.0), rel=1e-6, abs=0)


# --------------------------------------------------------------- Philox + HMC
def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(s, 16) for s in line.split()]
        assert O.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_hmc_normals_moments():
    z = np.concatenate([O.hmc_normals(7, it, 3, 101) for it in range(200)])
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1) < 0.02


def test_hmc_reversibility_and_gaussian_target():
    rng = np.random.default_rng(0)
    D = 6
    prec = np.diag(np.linspace(0.5, 3.0, D))

    def lg(x):
        return -0.5 * x @ prec @ x, -prec @ x
    x0 = rng.normal(size=D)
    lp0, g0 = lg(x0)
    p0 = rng.normal(size=D)
    # integrate forward, flip momentum, integrate back: returns to the start
    x, p, g = x0.copy(), p0.copy(), g0.copy()
    eps = 0.1
    for _ in range(15):
        p = p + 0.5 * eps * g
        x = x + eps * p
        g = lg(x)[1]
        p = p + 0.5 * eps * g
    p = -p
    for _ in range(15):
        p = p + 0.5 * eps * g
        x = x + eps * p
        g = lg(x)[1]
        p = p + 0.5 * eps * g
    np.testing.assert_allclose(x, x0, atol=1e-10)
    # sampling: moments of N(0, prec^-1)
    xs = []
    x, lp, g = x0, lp0, g0
    for it in range(4000):
        p0 = O.hmc_normals(11, it, 0, D)
        u = O.hmc_uniform(11, it, 0)
        x, lp, g, _ = O.hmc_trajectory(lg, x, lp, g, 0.3, 8, p0, u)
        xs.append(x)
    xs = np.array(xs[500:])
    np.testing.assert_allclose(xs.var(0), 1 / np.diag(prec), rtol=0.15)
    assert np.abs(xs.mean(0)).max() < 0.1


def test_hmc_bounded_coordinates_sample_the_box():
    """Box-bounded coordinates moved in logit space: a flat target on [lo, hi] (logp = 0
    inside) must be sampled uniformly (mean (lo + hi)/2, variance (hi - lo)^2 / 12), next
    to an unbounded Gaussian coordinate (N(1, 0.5^2)); no proposal leaves the box."""
    lo = np.array([-20.0, 0.0, -np.inf])
    hi = np.array([-10.0, 7.0, np.inf])

    def lg(x):
        if not (lo[0] < x[0] < hi[0] and lo[1] < x[1] < hi[1]):
            return -math.inf, np.zeros(3)
        return -0.5 * ((x[2] - 1.0) / 0.5) ** 2, np.array([0.0, 0.0, -(x[2] - 1.0) / 0.25])
    x = np.array([-12.0, 6.5, 0.0])
    lp, g = lg(x)
    xs = []
    for it in range(6000):
        p0 = O.hmc_normals(13, it, 0, 3)
        u = O.hmc_uniform(13, it, 0)
        x, lp, g, _ = O.hmc_trajectory(lg, x, lp, g, 0.4, 6, p0, u, bounds=(lo, hi))
        assert math.isfinite(lp)
        xs.append(x)
    xs = np.array(xs[500:])
    assert abs(xs[:, 0].mean() - (-15.0)) < 0.3 and abs(xs[:, 1].mean() - 3.5) < 0.25
    np.testing.assert_allclose(xs[:, :2].var(0), [100.0 / 12, 49.0 / 12], rtol=0.12)
    assert abs(xs[:, 2].mean() - 1.0) < 0.05 and abs(xs[:, 2].std() - 0.5) < 0.05



def test_tempered_posterior_limits_and_linearity():
    """Eq. (tempered_post): beta = 0 leaves the prior alone (closed form: logp = -|z|^2/2
    + log p(theta), gradient -z on the whitened coefficients, 0 on the box-prior
    hyper-parameters); logp and its gradient are affine in beta."""
    arr = synth.small_array(npsr=2, ntoa=[40, 55], m=[3, 4], n_gwb=2, n_rn=3, n_dm=2, seed=21)
    orc = O.Oracle(arr)
    x = synth.make_points(arr, 1, seed=4)[0].astype(np.float64)
    dz = orc.Dz
    lp0 = orc.logp(x, beta=0.0)
    assert lp0 == pytest.approx(-0.5 * float(x[:dz] @ x[:dz]) + orc.log_prior_theta(x), rel=1e-14, abs=1e-12)
    g0 = orc.grad(x, beta=0.0)
    np.testing.assert_allclose(g0[:dz], -x[:dz], rtol=0, atol=1e-12)
    assert np.all(g0[dz:] == 0.0)
    lp1, g1 = orc.logp(x), orc.grad(x)
    for beta in (0.25, 0.6):
        assert orc.logp(x, beta=beta) == pytest.approx((1 - beta) * lp0 + beta * lp1, rel=1e-12)
        np.testing.assert_allclose(orc.grad(x, beta=beta), (1 - beta) * g0 + beta * g1, rtol=1e-10, atol=1e-10)


def test_tempered_gradient_central_differences():
    arr = synth.small_array(npsr=2, ntoa=[40, 55], m=[3, 4], n_gwb=2, n_rn=3, n_dm=2, seed=22)
    orc = O.Oracle(arr)
    x = synth.make_points(arr, 1, seed=5)[0].astype(np.float64)
    beta = 0.37
    g = orc.grad(x, beta=beta)
    rng = np.random.default_rng(1)
    for j in rng.choice(orc.D, size=12, replace=False):
        h = 1e-6 * max(1.0, abs(x[j]))
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        fd = (orc.logp(xp, beta=beta) - orc.logp(xm, beta=beta)) / (2 * h)
        assert fd == pytest.approx(g[j], rel=1e-5, abs=1e-6 * max(1.0, abs(g).max()))



def test_free_spectrum_reduces_to_power_law():
    """A free spectrum whose per-bin variances are set to the power law's values gives
    the power-law posterior exactly (Sec. "Priors": both are choices of rho_k / kappa_Ik),
    and the free-spectrum gradient summed with the power law's chain rule
    (d rho_k / d log10 A = 2 ln10 rho_k) reproduces the power-law gradient."""
    kw = dict(npsr=2, ntoa=40, m=3, n_gwb=3, n_rn=3, n_dm=1, seed=8)
    arr_pl = synth.small_array(**kw)
    arr_fr = synth.small_array(**kw, gwb_free=True, rn_free=True)
    pl, fr = O.Oracle(arr_pl), O.Oracle(arr_fr)
    x = synth.make_points(arr_pl, 1, seed=3)[0].astype(np.float64)
    z_ach, z_dm, th_rn, th_dm, th_gwb, _ = pl.unpack(x)
    rho, kappa, _ = pl.spectra(th_rn, th_dm, th_gwb)
    lp, lf = pl.lay, fr.lay
    xf = np.zeros(fr.D)
    xf[: pl.Dz] = x[: pl.Dz]
    xf[lf["th_dm"]: lf["th_dm"] + 2 * arr_pl.npsr] = x[lp["th_dm"]: lp["th_dm"] + 2 * arr_pl.npsr]
    xf[lf["th_gwb"]: lf["th_gwb"] + 3] = np.log10(rho[:3] / 1e18)
    for I in range(2):
        xf[lf["th_rn"] + 3 * I: lf["th_rn"] + 3 * I + 3] = np.log10(kappa[I, :3] / 1e18)
    assert fr.logp(xf) == pytest.approx(pl.logp(x), rel=1e-12)
    gp, gf = pl.grad(x), fr.grad(xf)
    np.testing.assert_allclose(gf[: pl.Dz], gp[: pl.Dz], rtol=1e-10, atol=1e-12)
    # d/d log10 A_GWB = sum_k (d/d log10 rho_k)(d log10 rho_k / d log10 A) = 2 sum_k g_k
    assert 2.0 * gf[lf["th_gwb"]: lf["th_gwb"] + 3].sum() == pytest.approx(gp[lp["th_gwb"]], rel=1e-10)
    for I in range(2):
        assert 2.0 * gf[lf["th_rn"] + 3 * I: lf["th_rn"] + 3 * I + 3].sum() == \
            pytest.approx(gp[lp["th_rn"] + 2 * I], rel=1e-10)
