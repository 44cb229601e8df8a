"""CPU checks of the C ABI: the in-tree library loads, exports every entry point the
header declares, and rejects bad host input with error codes (no device work)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2607_06834_b300 import abi, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ptahmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pta_[a-z_0-9]+)\s*\(", src)))


def test_header_symbols_exported():
    names = declared_symbols()
    assert len(names) >= 11
    for n in names:
        assert hasattr(abi.lib, n), n
    assert set(names) == set(abi.EXPORTED)


def test_check_build_exports_and_error_codes():
    """the check build (libptahmc_check.so) exports the same entry points; the error codes of
    the binding are the header's"""
    from paper_2607_06834_b300 import build
    if not os.path.exists(build.LIB_CHECK):
        pytest.skip("check build not built")
    lib = C.CDLL(build.LIB_CHECK)
    for n in declared_symbols():
        assert hasattr(lib, n), n
    hdr = open(os.path.join(ROOT, "include", "ptahmc.h")).read()
    codes = {k: int(v) for k, v in re.findall(r"#define (PTA_E[A-Z]+|PTA_OK) \(?(-?\d+)\)?", hdr)}
    for k, v in codes.items():
        assert getattr(abi, k) == v, k
    assert codes["PTA_ECHECK"] == -6


def _ctx(**kw):
    d = abi.ModelDesc(kw.get("n_gwb", 2), kw.get("n_rn", 2), kw.get("n_dm", 0), 0, 1, 0.0)
    h = C.c_void_p()
    rc = abi.lib.pta_create(C.byref(h), C.byref(d))
    return rc, h


def _desc(p, keep):
    pd = abi.PulsarDesc()
    arrs = {k: np.ascontiguousarray(getattr(p, k), dtype=np.float64)
            for k in ("toas_s", "freqs_mhz", "resid_s", "sigma_s", "efac", "equad_s", "M")}
    arrs["backend"] = np.ascontiguousarray(p.backend, dtype=np.int32)
    keep.append(arrs)
    pd.n, pd.m, pd.n_backend = p.M.shape[0], p.M.shape[1], len(p.efac)
    for k in ("toas_s", "freqs_mhz", "resid_s", "sigma_s", "efac", "equad_s", "M"):
        setattr(pd, k, arrs[k].ctypes.data_as(C.POINTER(C.c_double)))
    pd.backend = arrs["backend"].ctypes.data_as(C.POINTER(C.c_int32))
    pd.pos = (C.c_double * 3)(*p.pos)
    pd.dist_kpc = p.dist_kpc
    return pd, arrs


def test_create_rejects_bad_model():
    d = abi.ModelDesc(0, 0, 0, 0, 1, 0.0)
    h = C.c_void_p()
    assert abi.lib.pta_create(C.byref(h), C.byref(d)) == abi.PTA_EINVAL
    d = abi.ModelDesc(2, 2, 0, 0, 9, 0.0)
    assert abi.lib.pta_create(C.byref(h), C.byref(d)) == abi.PTA_EINVAL


def test_add_pulsar_validation():
    rc, h = _ctx()
    assert rc == 0
    arr = synth.small_array(npsr=1, ntoa=30, m=3, seed=0)
    keep = []
    pd, arrs = _desc(arr.pulsars[0], keep)
    arrs["sigma_s"][3] = -1.0
    assert abi.lib.pta_add_pulsar(h, C.byref(pd)) == abi.PTA_EINVAL
    assert b"sigma" in abi.lib.pta_last_error(h)
    arrs["sigma_s"][3] = 1e-7
    arrs["backend"][0] = 5
    assert abi.lib.pta_add_pulsar(h, C.byref(pd)) == abi.PTA_EINVAL
    arrs["backend"][0] = 0
    pd.m = pd.n
    assert abi.lib.pta_add_pulsar(h, C.byref(pd)) == abi.PTA_EINVAL
    pd.m = 3
    arrs["resid_s"][0] = np.nan
    assert abi.lib.pta_add_pulsar(h, C.byref(pd)) == abi.PTA_EINVAL
    arrs["resid_s"][0] = 0.0
    assert abi.lib.pta_add_pulsar(h, C.byref(pd)) == abi.PTA_OK
    # calls that need a finalized context report a state error
    lay = abi.Layout()
    assert abi.lib.pta_layout(h, C.byref(lay)) == abi.PTA_ESTATE
    x = C.c_void_p(1)
    assert abi.lib.pta_logp_and_grad(h, 1, x, x, None, None, None) == abi.PTA_ESTATE
    assert abi.lib.pta_set_hyperprior(h, 1.0, 0.0, 0.0, 7.0) == abi.PTA_EINVAL
    abi.lib.pta_destroy(h)


def test_null_arguments():
    assert abi.lib.pta_create(None, None) == abi.PTA_EINVAL
    assert abi.lib.pta_add_pulsar(None, None) == abi.PTA_EINVAL
    assert abi.lib.pta_logp_and_grad(None, 1, None, None, None, None, None) == abi.PTA_EINVAL
    assert abi.lib.pta_last_error(None) == b"null context"


def test_toa_config_table_is_queryable_without_a_gpu():
    from paper_2607_06834_b300 import engine
    n = engine.toa_config_count()
    assert n >= 8
    shapes = [engine.toa_config_info(i) for i in range(n)]
    for s in shapes:
        assert s["chains_per_cta"] in (32, 64) and s["toas_per_tile"] in (32, 64)
        assert s["rows_per_thread"] >= 1 and 0 <= s["order"] < 8
    assert len({tuple(s.values()) for s in shapes}) == n   # no duplicate entries
    with pytest.raises(IndexError):
        engine.toa_config_info(n)
