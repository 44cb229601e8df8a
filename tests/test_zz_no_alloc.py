"""The allocation-free entry point (pta_logp_and_grad_noalloc), for callers that cannot
call cudaMalloc at evaluation time.  It runs the same kernels as the allocating entry
point on the same inputs, only with its workspace in the library's fixed device array,
so its results must equal the allocating call's bit for bit, on two calls in a row (the
shared workspace keeps the previous call's contents).  Collected last so a
stop-at-first-failure run has run every other test before it."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2607_06834_b300 import abi, synth

pytestmark = pytest.mark.gpu

ARRAYS = {
    "tiny3": None,
    # ragged tiles, a 2048-TOA chunk boundary, red-noise-only bins and DM
    "ragged_dm": dict(npsr=4, ntoa=[150, 700, 2300, 4500], m=[3, 9, 12, 7], n_gwb=5, n_rn=8, n_dm=6, seed=31,
                      nbackend=2),
    # GWB-only bins (n_gwb > n_rn): the chol(Gamma) kernels
    "gwb_only_bins": dict(npsr=3, ntoa=[90, 1300, 2049], m=[4, 3, 10], n_gwb=8, n_rn=3, n_dm=0, seed=32,
                          nbackend=3),
}


def _array(name):
    kw = ARRAYS[name]
    return synth.make_array("tiny3") if kw is None else synth.small_array(**kw)


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


def _same(a, b):
    lp, g, st = a
    lp_ref, g_ref, st_ref = b
    assert np.array_equal(st, st_ref)
    assert np.array_equal(lp, lp_ref), np.max(np.abs(lp - lp_ref))
    assert np.array_equal(g, g_ref), np.max(np.abs(g - g_ref))


@pytest.mark.parametrize("precision", ["fp32", "fp64", "tf32x3", "tf32", "gram"])
@pytest.mark.parametrize("name", list(ARRAYS))
def test_noalloc_matches_allocating_entry(name, precision):
    from paper_2607_06834_b300.engine import Engine
    arr = _array(name)
    eng = Engine(arr, precision=precision)
    for call in range(2):
        X = torch.tensor(synth.make_points(arr, 9, seed=100 + call), device="cuda")
        ref = _call(abi.lib.pta_logp_and_grad, eng, X)  # first: the FP64 path builds its stored basis here
        _same(_call(abi.lib.pta_logp_and_grad_noalloc, eng, X), ref)
        assert np.all(ref[2] == 0) and np.all(np.isfinite(ref[0]))
    eng.close()


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
    ref = _call(abi.lib.pta_logp_and_grad, eng, X)
    assert np.all(ref[2] == 0)
    _same(_call(abi.lib.pta_logp_and_grad_noalloc, eng, X), ref)
    # more chains than the temperatures given: refused, nothing computed
    X2 = torch.tensor(synth.make_points(arr, B + 1, seed=405), device="cuda")
    lp2 = torch.empty(B + 1, dtype=torch.float64, device="cuda")
    rc = abi.lib.pta_logp_and_grad_noalloc(eng._h, B + 1, C.c_void_p(X2.data_ptr()), C.c_void_p(lp2.data_ptr()),
                                           None, None, None)
    assert rc == abi.PTA_EINVAL
    eng.set_beta(None)
    eng.close()


def _refused(eng, B=3):
    x = torch.zeros((B, eng.D), dtype=torch.float32, device="cuda")
    lp = torch.empty(B, dtype=torch.float64, device="cuda")
    rc = abi.lib.pta_logp_and_grad_noalloc(eng._h, B, C.c_void_p(x.data_ptr()), C.c_void_p(lp.data_ptr()),
                                           None, None, None)
    return rc, abi.lib.pta_last_error(eng._h)


def test_noalloc_documented_refusals():
    """Each refusal the header documents returns its code and computes nothing."""
    from paper_2607_06834_b300.engine import Engine
    arr = _array("ragged_dm")
    eng = Engine(arr, precision="fp64")          # stored FP64 basis not built yet
    rc, msg = _refused(eng)
    assert rc == abi.PTA_ESTATE and b"FP64 basis" in msg
    eng.set_precision("bf16x3")
    rc, msg = _refused(eng)
    assert rc == abi.PTA_EINVAL and b"BF16" in msg
    eng.set_precision("fp32")
    eng.set_transform("curn")
    rc, msg = _refused(eng)
    assert rc == abi.PTA_EINVAL and b"CURN" in msg
    eng.close()
    cw = synth.small_array(npsr=2, ntoa=[150, 300], m=[3, 4], n_gwb=2, n_rn=2, seed=3, cw=True)
    eng = Engine(cw, precision="fp32")
    rc, msg = _refused(eng)
    assert rc == abi.PTA_EINVAL and b"continuous-wave" in msg
    eng.close()


def test_noalloc_rejects_oversized_batch():
    from paper_2607_06834_b300.engine import Engine
    eng = Engine(synth.make_array("ng15"), precision="fp32")
    rc, msg = _refused(eng, B=200)  # about 1.3 MB of workspace per chain at this size: above the fixed array
    assert rc == abi.PTA_EINVAL and b"use fewer chains" in msg
    eng.close()
