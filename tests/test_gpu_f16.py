"""GPU parity of the exact-split fp16 tensor-core path (PTA_PREC_F16SPLIT) against the FP64
oracle, held to the FP32 bar: |dlogp| <= 1e-3 nats at near-posterior points (the
CURN-conditional draw of the coefficients, Eq. PTA_standard_transform_curn) and
relative gradient-norm error <= 1e-4; at prior-random points, where chi2 is orders of
magnitude above the noise level, |dlogp| <= 1e-3 + 8 u |logp| with u = 2^-24 (the
leading products are exact and the rest carry FP32-level rounding)."""
import numpy as np
import pytest
import torch

from oracle import pta_oracle as O
from paper_2607_06834_b300 import synth

pytestmark = pytest.mark.gpu

LOGP_ABS = 1e-3
GRAD_REL = 1e-4
REL_RANDOM = 8 * 2.0 ** -24

RAGGED = [
    dict(npsr=4, ntoa=[150, 700, 2300, 4500], m=[3, 9, 12, 7], n_gwb=5, n_rn=8, n_dm=6, seed=31, nbackend=2),
    dict(npsr=3, ntoa=[90, 1300, 2049], m=[4, 3, 10], n_gwb=8, n_rn=3, n_dm=0, seed=32, nbackend=3),
]


def _engine(arr, prec):
    from paper_2607_06834_b300.engine import Engine
    return Engine(arr, precision=prec)


def _eval(eng, X):
    x = torch.tensor(np.asarray(X, dtype=np.float32), device="cuda")
    lp, g, st = eng.logp_and_grad(x)
    torch.cuda.synchronize()
    return lp.cpu().numpy(), g.cpu().numpy(), st.cpu().numpy()


def _oracle(orc, X):
    X = np.asarray(X, dtype=np.float32).astype(np.float64)
    return np.array([orc.logp(x) for x in X]), np.array([orc.grad(x) for x in X])


def _grad_rel(g, go):
    return np.linalg.norm(g - go, axis=-1) / np.maximum(np.linalg.norm(go, axis=-1), 1e-30)


def test_tiny_1000_points():
    arr = synth.make_array("tiny3")
    orc = O.Oracle(arr)
    X = synth.make_points(arr, 1000, seed=6834)
    X[:16] = np.array([O.curn_point(orc, x.astype(np.float64), 1.0, seed=i) for i, x in enumerate(X[:16])])
    lo, go = _oracle(orc, X)
    lp, g, st = _eval(_engine(arr, "f16split"), X)
    assert np.all(st == 0)
    err = np.abs(lp - lo)
    print(f"tiny f16split: max |dlogp| near {err[:16].max():.2e}, random {err[16:].max():.2e}; "
          f"max grad rel {_grad_rel(g, go).max():.2e}")
    assert err[:16].max() < LOGP_ABS
    assert np.all(err <= LOGP_ABS + REL_RANDOM * np.abs(lo))
    assert np.max(_grad_rel(g, go)) < GRAD_REL


@pytest.mark.parametrize("kw", RAGGED)
@pytest.mark.parametrize("B", [70, 130])
def test_ragged_arrays(kw, B):
    """Partial tiles, a 2048-TOA unit boundary, RN-only and GWB-only bins, a partial
    block of chains and two column chunks of the F^T w kernel."""
    arr = synth.small_array(**kw)
    orc = O.Oracle(arr)
    X = synth.make_points(arr, B, seed=5)
    X[:6] = np.array([O.curn_point(orc, x.astype(np.float64), 1.0, seed=i) for i, x in enumerate(X[:6])])
    sample = list(range(6)) + [B // 2, 64, B - 1]
    lo, go = _oracle(orc, X[sample])
    eng = _engine(arr, "f16split")
    lp, g, st = _eval(eng, X)
    assert np.all(st == 0)
    err = np.abs(lp[sample] - lo)
    rel = _grad_rel(g[sample], go)
    print(f"f16split ragged B={B}: max |dlogp| near {err[:6].max():.2e} random {err[6:].max():.2e}; "
          f"max grad rel {rel.max():.2e}")
    assert err[:6].max() < LOGP_ABS
    assert np.all(err <= LOGP_ABS + REL_RANDOM * np.abs(lo))
    assert rel.max() < GRAD_REL
    # a chain's result does not depend on the rest of the batch
    lp1, g1, _ = _eval(eng, X[B - 1:B])
    assert lp1[0] == lp[B - 1] and np.array_equal(g1[0], g[B - 1])


def test_ng15_batch256_sampled():
    """The bench's launch configuration (256 chains in one call), 16 near-posterior
    chains spread over the batch held to the absolute bar, 3 prior-random ones."""
    arr = synth.make_array("ng15")
    orc = O.Oracle(arr)
    X = synth.make_points(arr, 256, seed=6836)
    near = [5 + 16 * j for j in range(16)]
    for j, i in enumerate(near):
        X[i] = O.curn_point(orc, X[i].astype(np.float64), 1.0, seed=j)
    eng = _engine(arr, "f16split")
    lp, g, st = _eval(eng, X)
    assert np.all(st == 0)
    sample = [0, 77, 255] + near
    lo, go = _oracle(orc, X[sample])
    err = np.abs(lp[sample] - lo)
    rel = _grad_rel(g[sample], go)
    print(f"f16split ng15: 16 near-posterior chains: max |dlogp| {err[3:].max():.2e}, max grad rel "
          f"{rel[3:].max():.2e}; random: {err[:3].max():.2e} at |logp| {np.abs(lo[:3]).max():.3g}")
    assert err[3:].max() < LOGP_ABS
    assert np.all(err[:3] <= LOGP_ABS + REL_RANDOM * np.abs(lo[:3]))
    assert rel.max() < GRAD_REL
