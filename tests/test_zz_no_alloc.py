"""The allocation-free entry point (pta_logp_and_grad_noalloc), for callers that cannot
call cudaMalloc at evaluation time: its results must equal the allocating entry
point's on the same inputs, on two calls in a row (the shared workspace keeps the
previous call's contents).  Collected last so a stop-at-first-failure run has run
every other test before it."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2607_06834_b300 import abi, synth

pytestmark = pytest.mark.gpu

LOGP_ABS = 1e-3
GRAD_REL = 1e-4


def _call(fn, eng, x):
    B = x.shape[0]
    lp = torch.empty(B, dtype=torch.float64, device=x.device)
    g = torch.empty_like(x)
    st = torch.empty(B, dtype=torch.int32, device=x.device)
    rc = fn(eng._h, B, C.c_void_p(x.data_ptr()), C.c_void_p(lp.data_ptr()), C.c_void_p(g.data_ptr()),
            C.c_void_p(st.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, abi.lib.pta_last_error(eng._h)
    torch.cuda.synchronize()
    return lp.cpu().numpy(), g.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("kw", [
    None,  # the 3-pulsar array
    dict(npsr=4, ntoa=[150, 700, 2300, 4500], m=[3, 9, 12, 7], n_gwb=5, n_rn=8, n_dm=6, seed=31, nbackend=2),
])
def test_noalloc_matches_allocating_entry(kw):
    from paper_2607_06834_b300.engine import Engine
    arr = synth.make_array("tiny3") if kw is None else synth.small_array(**kw)
    eng = Engine(arr, precision="fp32")
    for call in range(2):
        X = torch.tensor(synth.make_points(arr, 9, seed=100 + call), device="cuda")
        lp_ref, g_ref, st_ref = _call(abi.lib.pta_logp_and_grad, eng, X)
        lp, g, st = _call(abi.lib.pta_logp_and_grad_noalloc, eng, X)
        assert np.array_equal(st, st_ref)
        assert np.all(np.abs(lp - lp_ref) <= LOGP_ABS)
        assert np.all(np.linalg.norm(g - g_ref, axis=1) <= GRAD_REL * np.linalg.norm(g_ref, axis=1))


@pytest.mark.parametrize("precision", ["fp32", "gram"])
def test_noalloc_tempered_free_spectra(precision):
    """Feature combination on the allocation-free entry point: free spectral models for
    the GWB and the red noise, a per-chain inverse temperature, and the Gram form."""
    from paper_2607_06834_b300.engine import Engine
    arr = synth.small_array(npsr=3, ntoa=[400, 900, 1500], m=[3, 6, 8], n_gwb=4, n_rn=5, n_dm=3, seed=47,
                            nbackend=2, gwb_free=True, rn_free=True)
    eng = Engine(arr, precision=precision)
    B = 7
    X = torch.tensor(synth.make_points(arr, B, seed=404), device="cuda")
    eng.set_beta(torch.linspace(0.1, 1.0, B, dtype=torch.float64))
    lp_ref, g_ref, st_ref = _call(abi.lib.pta_logp_and_grad, eng, X)
    lp, g, st = _call(abi.lib.pta_logp_and_grad_noalloc, eng, X)
    assert np.all(st_ref == 0) and np.array_equal(st, st_ref)
    assert np.all(np.abs(lp - lp_ref) <= LOGP_ABS)
    assert np.all(np.linalg.norm(g - g_ref, axis=1) <= GRAD_REL * np.linalg.norm(g_ref, axis=1))
    # more chains than the temperatures given: refused, nothing computed
    X2 = torch.tensor(synth.make_points(arr, B + 1, seed=405), device="cuda")
    lp2 = torch.empty(B + 1, dtype=torch.float64, device="cuda")
    rc = abi.lib.pta_logp_and_grad_noalloc(eng._h, B + 1, C.c_void_p(X2.data_ptr()), C.c_void_p(lp2.data_ptr()),
                                           None, None, None)
    assert rc == abi.PTA_EINVAL
    eng.set_beta(None)


def test_noalloc_rejects_oversized_batch():
    from paper_2607_06834_b300.engine import Engine
    eng = Engine(synth.make_array("ng15"), precision="fp32")
    B = 200  # about 1.2 MB of workspace per chain at this size: above the fixed array
    x = torch.zeros((B, eng.D), dtype=torch.float32, device="cuda")
    lp = torch.empty(B, dtype=torch.float64, device="cuda")
    rc = abi.lib.pta_logp_and_grad_noalloc(eng._h, B, C.c_void_p(x.data_ptr()), C.c_void_p(lp.data_ptr()),
                                           None, None, None)
    assert rc == abi.PTA_EINVAL
    assert b"use fewer chains" in abi.lib.pta_last_error(eng._h)
