"""Pins for the oracle's CURN-posterior transform (Eqs. PTA_standard_transform_curn,
standardized_stochastic_posterior; the tempered T_beta of App. "tempered likelihoods")
against things other than itself.  CPU only.

* One pulsar: the HD prior has no off-diagonal part, so the CURN moments are the exact
  conditional posterior moments of a and the transform whitens it exactly:
  logp(z) + |z|^2 / 2 does not depend on z and equals the dense time-domain marginal
  likelihood (Fourier coefficients and timing model integrated out) minus the dropped
  data constant.  Tempered: still z-independent (the tempered posterior in a is
  Gaussian with the moments of T_beta).
* Several pulsars with HD correlations: logp_full is exactly quadratic in z (a is
  affine in z), and its integral over z equals the dense marginal likelihood: the
  Jacobian det L_CURN and the prior normalisation are both checked by this.
* beta = 0: the transform is a = sqrt(phi_CURN) z; for one pulsar this is the
  prior-whitened transform, so the two oracles agree.
* With a circular binary (Eq. decenter_det_PTA) the same exactness and integral hold with
  the mean abar = Sigma F^T N~^-1 (dt - h).
* The gradient against central differences, power-law and free spectra, tempered."""
import math

import numpy as np
import pytest

from oracle import pta_oracle as O
from paper_2607_06834_b300 import synth


def _z_variants(orc, x, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        y = x.copy()
        y[: orc.Dz] = rng.normal(size=orc.Dz)
        out.append(y)
    return out


@pytest.mark.parametrize("kw", [
    dict(npsr=1, ntoa=50, m=3, n_gwb=3, n_rn=4, n_dm=2, seed=3),
    dict(npsr=1, ntoa=60, m=5, n_gwb=4, n_rn=2, n_dm=0, seed=4, nbackend=2),
    dict(npsr=1, ntoa=45, m=3, n_gwb=3, n_rn=3, n_dm=1, seed=5, gwb_free=True, rn_free=True),
])
def test_single_pulsar_exact_whitening(kw):
    arr = synth.small_array(**kw)
    orc = O.Oracle(arr, transform="curn")
    for x in synth.make_points(arr, 2, seed=7).astype(np.float64):
        ref = orc.dense_marginal(x) - orc.data_constant()
        for y in _z_variants(orc, x, 4, seed=11):
            v = orc.logp(y) + 0.5 * y[: orc.Dz] @ y[: orc.Dz]
            assert abs(v - ref) <= 1e-9 * abs(ref), (v, ref)
        tempered = [orc.logp(y, beta=0.35) + 0.5 * y[: orc.Dz] @ y[: orc.Dz] for y in _z_variants(orc, x, 4, 12)]
        assert np.ptp(tempered) <= 1e-9 * abs(tempered[0])


def test_beta_zero_single_pulsar_equals_prior_whitened():
    arr = synth.small_array(npsr=1, ntoa=40, m=3, n_gwb=3, n_rn=4, n_dm=2, seed=6)
    oc, op = O.Oracle(arr, transform="curn"), O.Oracle(arr)
    for x in synth.make_points(arr, 3, seed=8).astype(np.float64):
        assert abs(oc.logp(x, beta=0.0) - op.logp(x, beta=0.0)) < 1e-10 * max(1.0, abs(op.logp(x, beta=0.0)))
        np.testing.assert_allclose(oc.grad(x, beta=0.0), op.grad(x, beta=0.0), rtol=1e-9, atol=1e-9)


def _closed_form_logZ(orc, x):
    """Integral over z of exp(logp_full), exactly quadratic in z at fixed theta."""
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
    dict(npsr=3, ntoa=30, m=3, n_gwb=3, n_rn=2, n_dm=1, seed=2),
    dict(npsr=2, ntoa=45, m=5, n_gwb=2, n_rn=3, n_dm=0, seed=9, nbackend=2),
    dict(npsr=3, ntoa=35, m=3, n_gwb=2, n_rn=2, n_dm=1, seed=10, gwb_free=True, rn_free=True),
])
def test_integral_over_z_is_the_marginal_likelihood(kw):
    arr = synth.small_array(**kw)
    orc = O.Oracle(arr, transform="curn")
    for s in range(2):
        x = synth.make_points(arr, 1, seed=20 + s)[0].astype(np.float64)
        a = _closed_form_logZ(orc, x)
        b = orc.dense_marginal(x)
        assert abs(a - b) <= 1e-9 * abs(b), (a, b)


def _fd_grad(orc, x, beta, rel=1e-6):
    out = np.zeros(orc.D)
    for j in range(orc.D):
        h = rel * max(1.0, abs(x[j]))
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        out[j] = (orc.logp(xp, beta=beta) - orc.logp(xm, beta=beta)) / (2 * h)
    return out


@pytest.mark.parametrize("kw,beta", [
    (dict(npsr=3, ntoa=40, m=3, n_gwb=3, n_rn=4, n_dm=2, seed=11), 1.0),
    (dict(npsr=3, ntoa=40, m=5, n_gwb=4, n_rn=2, n_dm=0, seed=12, nbackend=2), 0.4),
    (dict(npsr=3, ntoa=40, m=3, n_gwb=3, n_rn=4, n_dm=2, seed=14, gwb_free=True, rn_free=True), 1.0),
    (dict(npsr=2, ntoa=40, m=4, n_gwb=4, n_rn=2, n_dm=1, seed=15, gwb_free=True), 0.7),
])
def test_gradient_central_differences(kw, beta):
    arr = synth.small_array(**kw)
    orc = O.Oracle(arr, transform="curn")
    x = synth.make_points(arr, 1, seed=21)[0].astype(np.float64)
    g = orc.grad(x, beta=beta)
    fd = _fd_grad(orc, x, beta)
    scale = np.abs(g).max()
    err = np.abs(fd - g)
    assert np.all(err <= 1e-6 * np.abs(g) + 1e-7 * scale), (np.argmax(err / (np.abs(g) + 1e-7 * scale)), err.max())


def _cw_point(orc, arr, seed):
    x = synth.make_points(arr, 1, seed=seed)[0].astype(np.float64)
    c = orc.lay["th_cw"]
    x[c: c + 8] = [9.5, -7.8, -13.5, 0.3, 1.0, 0.2, 2.0, 1.0]
    return x


def test_deterministic_signal_single_pulsar_exact_whitening():
    """Eq. decenter_det_PTA: with a circular binary the conditional posterior of a is still
    Gaussian with the CURN covariance and mean abar = Sigma F^T N~^-1 (dt - h); for one pulsar
    logp(z) + |z|^2/2 is independent of z and equals the dense marginal likelihood of dt - h
    (minus the dropped constant) plus the CW prior."""
    arr = synth.small_array(npsr=1, ntoa=60, m=3, n_gwb=3, n_rn=3, n_dm=1, seed=8, cw=True)
    orc = O.Oracle(arr, transform="curn")
    x = _cw_point(orc, arr, 3)
    ref = orc.dense_marginal(x) - orc.data_constant() + orc.log_prior_theta(x)
    for y in _z_variants(orc, x, 4, seed=5):
        v = orc.logp(y) + 0.5 * y[: orc.Dz] @ y[: orc.Dz]
        assert abs(v - ref) <= 1e-9 * abs(ref), (v, ref)


def test_deterministic_signal_integral_and_gradient():
    arr = synth.small_array(npsr=2, ntoa=40, m=3, n_gwb=2, n_rn=2, n_dm=1, seed=13, cw=True)
    orc = O.Oracle(arr, transform="curn")
    x = _cw_point(orc, arr, 21)
    a = _closed_form_logZ(orc, x)
    b = orc.dense_marginal(x) + orc.log_prior_theta(x)
    assert abs(a - b) <= 1e-9 * abs(b), (a, b)
    for beta in (1.0, 0.6):
        g = orc.grad(x, beta=beta)
        fd = _fd_grad(orc, x, beta)
        scale = np.abs(g).max()
        err = np.abs(fd - g)
        assert np.all(err <= 1e-6 * np.abs(g) + 1e-7 * scale), (np.argmax(err / (np.abs(g) + 1e-7 * scale)), err.max())
