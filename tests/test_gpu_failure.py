"""Failure detection of the bounded device waits, made on purpose without a GPU
fault: a test hook makes the BF16 tensor-core kernel withhold one MMA completion
signal, so its epilogue's bounded mbarrier wait runs out.  The kernel must finish,
report status bit 4 for its chains, and leave the context usable: the next
evaluation, with the hook off, repeats the clean result bit for bit."""
import numpy as np
import pytest
import torch

from paper_2607_06834_b300 import abi, synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_timeout_reports_status_and_context_survives():
    from paper_2607_06834_b300.engine import Engine
    arr = synth.make_array("tiny3")
    eng = Engine(arr, precision="bf16x3")
    x = torch.tensor(synth.make_points(arr, 6, seed=3), device="cuda")
    lp0, g0, st0 = eng.logp_and_grad(x)
    torch.cuda.synchronize()
    assert int(st0.abs().sum()) == 0
    lp0, g0 = lp0.cpu().numpy().copy(), g0.cpu().numpy().copy()
    eng._check(abi.lib.pta_debug_inject(eng._h, 1), "pta_debug_inject")
    lp1, g1, st1 = eng.logp_and_grad(x)
    torch.cuda.synchronize()
    st1 = st1.cpu().numpy()
    assert np.all((st1 & 4) == 4), st1
    eng._check(abi.lib.pta_debug_inject(eng._h, 0), "pta_debug_inject")
    lp2, g2, st2 = eng.logp_and_grad(x)
    torch.cuda.synchronize()
    assert int(st2.abs().sum()) == 0
    assert np.array_equal(lp2.cpu().numpy(), lp0) and np.array_equal(g2.cpu().numpy(), g0)
