"""GPU parity of the CURN-posterior transform (Eq. PTA_standard_transform_curn; tempered
T_beta of App. "tempered likelihoods") through the C ABI against the oracle's CURN mode.

Under this transform every z ~ N(0, I) maps to coefficients near the conditional
posterior, so the FP32 target (|dlogp| <= 1e-3 nats, relative gradient-norm error <= 1e-4)
applies at every point.  FP64 and Gram contractions: relative 1e-9 on logp, 1e-6 on the
gradient (the transform itself is FP64 in every mode)."""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import pta_oracle as O
from paper_2607_06834_b300 import abi, synth

pytestmark = pytest.mark.gpu

LOGP_ABS = 1e-3
GRAD_REL = 1e-4
FP64_REL = 1e-9

CASES = [
    # several 128-TOA tiles, a 2048-TOA chunk boundary, RN-only bins, DM
    dict(npsr=4, ntoa=[150, 700, 2300, 4500], m=[3, 9, 12, 7], n_gwb=5, n_rn=8, n_dm=6, seed=31, nbackend=2),
    # GWB-only bins (n_gwb > n_rn), no DM
    dict(npsr=3, ntoa=[90, 1300, 2049], m=[4, 3, 10], n_gwb=8, n_rn=3, n_dm=0, seed=32, nbackend=3),
    # free spectral models
    dict(npsr=3, ntoa=[400, 900, 1500], m=[3, 6, 8], n_gwb=4, n_rn=5, n_dm=3, seed=47, nbackend=2,
         gwb_free=True, rn_free=True),
]


def _engine(arr, prec):
    from paper_2607_06834_b300.engine import Engine
    eng = Engine(arr, precision=prec)
    eng.set_transform("curn")
    return eng


def _eval(eng, X):
    x = torch.tensor(np.asarray(X, dtype=np.float32), device="cuda")
    lp, g, st = eng.logp_and_grad(x)
    torch.cuda.synchronize()
    return lp.cpu().numpy(), g.cpu().numpy(), st.cpu().numpy()


def _grad_rel(g, go):
    return np.linalg.norm(g - go, axis=-1) / np.maximum(np.linalg.norm(go, axis=-1), 1e-30)


def _check(prec, lp, g, lo, go, tag):
    err, rel = np.abs(lp - lo), _grad_rel(g, go)
    print(f"{tag} {prec}: max |dlogp| {err.max():.2e} (|logp| ~ {np.abs(lo).max():.3g}) max grad rel {rel.max():.2e}")
    if prec in ("fp64", "gram"):
        assert np.max(err / np.maximum(1.0, np.abs(lo))) < FP64_REL
        assert rel.max() < 1e-6
    else:
        assert err.max() < LOGP_ABS and rel.max() < GRAD_REL


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "gram"])
def test_curn_small_arrays_match_oracle(kw, prec):
    arr = synth.small_array(**kw)
    orc = O.Oracle(arr, transform="curn")
    X = synth.make_points(arr, 12, seed=61)
    Xd = X.astype(np.float64)
    lo = np.array([orc.logp(x) for x in Xd])
    go = np.array([orc.grad(x) for x in Xd])
    eng = _engine(arr, prec)
    lp, g, st = _eval(eng, X)
    assert np.all(st == 0)
    _check(prec, lp, g, lo, go, "curn small")


@pytest.mark.parametrize("prec", ["fp32", "gram"])
def test_curn_tempered_matches_oracle(prec):
    arr = synth.small_array(**CASES[0])
    orc = O.Oracle(arr, transform="curn")
    B = 8
    X = synth.make_points(arr, B, seed=62)
    beta = np.array([1.0, 0.5, 0.1, 0.0, 0.3, 0.9, 0.05, 0.7])
    eng = _engine(arr, prec)
    eng.set_beta(torch.tensor(beta, device="cuda"))
    lp, g, st = _eval(eng, X)
    assert np.all(st == 0)
    Xd = X.astype(np.float64)
    lo = np.array([orc.logp(x, beta=b) for x, b in zip(Xd, beta)])
    go = np.array([orc.grad(x, beta=b) for x, b in zip(Xd, beta)])
    _check(prec, lp, g, lo, go, "curn tempered")
    eng.set_beta(None)


def test_curn_paper_config_nodm():
    """The paper's NANOGrav-15-yr model (67 pulsars, RN 30 / HD-GWB 14 bins, no DM:
    P = 60, the factor in shared memory), 64 chains, sampled against the oracle."""
    arr = synth.make_array("ng15_nodm")
    orc = O.Oracle(arr, transform="curn")
    B = 64
    X = synth.make_points(arr, B, seed=63)
    eng = _engine(arr, "fp32")
    lp, g, st = _eval(eng, X)
    assert np.all(st == 0)
    idx = [0, 17, B - 1]
    Xd = X[idx].astype(np.float64)
    lo = np.array([orc.logp(x) for x in Xd])
    go = np.array([orc.grad(x) for x in Xd])
    _check("fp32", lp[idx], g[idx], lo, go, "curn ng15_nodm")


def test_curn_ng15_global_factor():
    """67 pulsars with 100 DM bins (P = 260: the double-word factor over a cluster of two
    CTAs; FP64 mode keeps it in the global inverse buffer), 16 chains, two sampled
    against the oracle."""
    arr = synth.make_array("ng15")
    orc = O.Oracle(arr, transform="curn")
    X = synth.make_points(arr, 16, seed=64)
    eng = _engine(arr, "fp32")
    lp, g, st = _eval(eng, X)
    assert np.all(st == 0)
    idx = [3, 11]
    Xd = X[idx].astype(np.float64)
    lo = np.array([orc.logp(x) for x in Xd])
    go = np.array([orc.grad(x) for x in Xd])
    _check("fp32", lp[idx], g[idx], lo, go, "curn ng15")


@pytest.mark.parametrize("n_dm", [110, 160, 235])
@pytest.mark.parametrize("prec", ["fp32", "gram"])
def test_curn_cluster_factor_matches_oracle(n_dm, prec):
    """P = 240, 340, 490: above one CTA's shared memory the double-word factorisation runs over
    a thread-block cluster of 2, 4 and 8 CTAs (interleaved row pairs); 4 chains against the
    oracle, the 340 case also tempered."""
    kw = dict(npsr=3, ntoa=[600, 900, 1300], m=[3, 6, 8], n_gwb=6, n_rn=10, n_dm=n_dm, seed=71, nbackend=2)
    arr = synth.small_array(**kw)
    orc = O.Oracle(arr, transform="curn")
    X = synth.make_points(arr, 4, seed=72)
    beta = np.array([1.0, 0.6, 0.2, 0.0]) if n_dm == 160 else np.ones(4)
    eng = _engine(arr, prec)
    if n_dm == 160:
        eng.set_beta(torch.tensor(beta, device="cuda"))
    lp, g, st = _eval(eng, X)
    assert np.all(st == 0)
    Xd = X.astype(np.float64)
    lo = np.array([orc.logp(x, beta=b) for x, b in zip(Xd, beta)])
    go = np.array([orc.grad(x, beta=b) for x, b in zip(Xd, beta)])
    _check(prec, lp, g, lo, go, f"curn cluster P={20 + 2 * n_dm}")


def test_curn_hmc_trajectory_and_rejections():
    from paper_2607_06834_b300 import sampler
    arr = synth.small_array(**CASES[1])
    eng = _engine(arr, "fp32")
    X = torch.tensor(synth.make_points(arr, 8, seed=65), device="cuda")
    res = sampler.run_hmc(eng, X, n_warmup=40, n_samples=20, n_leapfrog=8, seed=3)
    lp_end, _, st = eng.logp_and_grad(res.state.x.contiguous())
    assert np.all(st.cpu().numpy() == 0) and np.all(np.isfinite(lp_end.cpu().numpy()))
    assert 0.2 < res.accept_rate <= 1.0
    # the allocation-free entry point keeps no per-chain factors
    B = 4
    x = torch.tensor(synth.make_points(arr, B, seed=66), device="cuda")
    lp = torch.empty(B, dtype=torch.float64, device="cuda")
    rc = abi.lib.pta_logp_and_grad_noalloc(eng._h, B, C.c_void_p(x.data_ptr()), C.c_void_p(lp.data_ptr()),
                                           None, None, None)
    assert rc == abi.PTA_EINVAL
    # back to the prior-whitened transform: the default path's result
    eng.set_transform("prior")
    ref = _engine(arr, "fp32")
    ref.set_transform("prior")
    a, _, _ = _eval(eng, x.cpu().numpy())
    b, _, _ = _eval(ref, x.cpu().numpy())
    np.testing.assert_array_equal(a, b)


CW_CASE = dict(npsr=3, ntoa=[150, 700, 2300], m=[3, 9, 12], n_gwb=4, n_rn=5, n_dm=3, seed=41, nbackend=2, cw=True)


def _cw_points(orc, arr, B, seed):
    X = synth.make_points(arr, B, seed=seed)
    c = orc.lay["th_cw"]
    X[0, c: c + 8] = [9.5, -7.8, -13.5, 0.3, 1.0, 0.2, 2.0, 1.0]  # a loud binary in one chain
    return X


@pytest.mark.parametrize("tempered", [False, True])
def test_curn_deterministic_signal_matches_oracle(tempered):
    """Eq. decenter_det_PTA on the FP32 path: the mean abar = Sigma F^T N~^-1 (dt - h) from an
    extra TOA pass, and the CW gradient through it from another; every block of the gradient
    (z, noise, GWB, CW) against the oracle, with and without per-chain temperatures."""
    arr = synth.small_array(**CW_CASE)
    orc = O.Oracle(arr, transform="curn")
    B = 8
    X = _cw_points(orc, arr, B, 67)
    beta = np.array([1.0, 0.5, 0.1, 0.0, 0.3, 0.9, 0.05, 0.7]) if tempered else np.ones(B)
    eng = _engine(arr, "fp32")
    if tempered:
        eng.set_beta(torch.tensor(beta, device="cuda"))
    lp, g, st = _eval(eng, X)
    assert np.all(st == 0)
    Xd = X.astype(np.float64)
    lo = np.array([orc.logp(x, beta=b) for x, b in zip(Xd, beta)])
    go = np.array([orc.grad(x, beta=b) for x, b in zip(Xd, beta)])
    _check("fp32", lp, g, lo, go, "curn cw" + (" tempered" if tempered else ""))
    c = orc.lay["th_cw"]
    relcw = _grad_rel(g[:, c:], go[:, c:])
    print(f"cw block grad rel {relcw.max():.2e}")
    assert relcw.max() < GRAD_REL


def test_curn_deterministic_signal_hmc():
    from paper_2607_06834_b300 import sampler
    arr = synth.small_array(**CW_CASE)
    orc = O.Oracle(arr, transform="curn")
    eng = _engine(arr, "fp32")
    X = torch.tensor(_cw_points(orc, arr, 8, 68), device="cuda")
    res = sampler.run_hmc(eng, X, n_warmup=30, n_samples=10, n_leapfrog=6, seed=4, unit_mass=eng.layout["d_z"])
    lp_end, _, st = eng.logp_and_grad(res.state.x.contiguous())
    assert np.all(st.cpu().numpy() == 0) and np.all(np.isfinite(lp_end.cpu().numpy()))
    assert 0.2 < res.accept_rate <= 1.0
