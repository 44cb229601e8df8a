"""GPU parity at the scale-up size: 150 pulsars, 1.0e6 TOAs (1k-30k per pulsar over up
to 30 yr), 100 GWB / 30 red-noise / 150 DM bins (P = 500 coefficients per pulsar,
dense FP64 150 x 150 Cholesky in 30 bins, GWB-only bins above), 1024 chains in one
launch, the configuration the scale-up measurement times.  The FP64 oracle takes
minutes per gradient here, so outputs are sampled: logp of three chains (one at a
near-posterior point) and the full gradient of the near-posterior chain.  Tolerances
as in test_gpu_parity."""
import numpy as np
import pytest
import torch

from oracle import pta_oracle as O
from paper_2607_06834_b300 import synth

pytestmark = pytest.mark.gpu

LOGP_ABS = 1e-3
GRAD_REL = 1e-4
REL_RANDOM_FP32 = 8 * 2.0 ** -24
FP64_REL = 1e-9


def test_scale150_b1024_sampled():
    from paper_2607_06834_b300.engine import Engine
    arr = synth.make_array("scale150")
    orc = O.Oracle(arr)
    B = synth.WORKLOADS["scale150"]["chains"]
    X = synth.make_points(arr, B, seed=6834 + 4)
    near = 100
    X[near] = O.curn_point(orc, X[near].astype(np.float64), 1.0, seed=5)
    eng = Engine(arr, precision="fp32")
    x = torch.tensor(X, device="cuda")
    lp, g, st = eng.logp_and_grad(x)
    torch.cuda.synchronize()
    lp, g, st = lp.cpu().numpy(), g.cpu().numpy(), st.cpu().numpy()
    assert np.all(st == 0) and np.all(np.isfinite(lp))
    Xd = X.astype(np.float64)
    for i in (0, near, B - 1):
        lo = orc.logp(Xd[i])
        err = abs(lp[i] - lo)
        print(f"scale150 chain {i}: logp {lo:.3f} |d| {err:.2e}")
        assert err < (LOGP_ABS if i == near else LOGP_ABS + REL_RANDOM_FP32 * abs(lo))
    go = orc.grad(Xd[near])
    rel = np.linalg.norm(g[near] - go) / np.linalg.norm(go)
    print(f"scale150 chain {near}: grad rel {rel:.2e}")
    assert rel < GRAD_REL
    # the Gram form on the whole batch (compensated FP32, FP64-level agreement)
    eng.set_precision("gram")
    lpg, gg, stg = eng.logp_and_grad(x)
    torch.cuda.synchronize()
    lpg, gg = lpg.cpu().numpy(), gg.cpu().numpy()
    assert np.all(stg.cpu().numpy() == 0)
    for i in (0, near, B - 1):
        lo = orc.logp(Xd[i])
        assert abs(lpg[i] - lo) / max(1.0, abs(lo)) < FP64_REL
    assert np.linalg.norm(gg[near] - go) / np.linalg.norm(go) < 1e-6
    # the plain FP64 path on the same chain
    eng.set_precision("fp64")
    lp64, g64, st64 = eng.logp_and_grad(x[near:near + 1].contiguous())
    torch.cuda.synchronize()
    lo = orc.logp(Xd[near])
    assert int(st64.item()) == 0
    assert abs(float(lp64.item()) - lo) / max(1.0, abs(lo)) < FP64_REL
    assert np.linalg.norm(g64.cpu().numpy()[0] - go) / np.linalg.norm(go) < 1e-6
