"""The check build (libptahmc_check.so, nvcc -DPTA_CHECK) on the GPU.

Every instrumented index is tested before use: the LDL sweeps' triangle elements, staging entries
and L D^1/2 outputs, the cluster sweep's per-CTA parts, the work units' TOA ranges, the
exact-split kernels' bulk copies and TMA coordinates, the CURN slot writes.  A child process
loads the check build and evaluates cases that reach every one of them: the NANOGrav-15-yr-like
batch on the exact-split path, the CURN transform with the factor in one CTA (P = 60) and over
clusters of 2, 4 and 8 CTAs (P = 260, 340, 490), a ragged array, and an HMC trajectory.  Every
call must return PTA_OK, so no check failed, with the release build's results."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RAGGED = dict(npsr=4, ntoa=[150, 700, 2300, 4500], m=[3, 9, 12, 7], n_gwb=5, n_rn=8, n_dm=6, seed=31, nbackend=2)


def _cases():
    from paper_2607_06834_b300 import synth
    wide = lambda nd: synth.small_array(npsr=3, ntoa=[600, 900, 1300], m=[3, 6, 8], n_gwb=6, n_rn=10, n_dm=nd,
                                        seed=71, nbackend=2)
    return [
        ("ng15_f16split", lambda: synth.make_array("ng15_b256"), "f16split", "prior", 32),
        ("ng15_gram", lambda: synth.make_array("ng15_b256"), "gram", "prior", 16),
        ("ng15nodm_curn", lambda: synth.make_array("ng15_nodm"), "f16split", "curn", 8),
        ("ng15_curn_c2", lambda: synth.make_array("ng15"), "f16split", "curn", 4),
        ("wide340_curn_c4", lambda: wide(160), "gram", "curn", 4),
        ("wide490_curn_c8", lambda: wide(235), "fp32", "curn", 4),
        ("ragged_f16split", lambda: synth.small_array(**RAGGED), "f16split", "prior", 8),
    ]


def _run_all(out):
    """evaluate every case with the library this process loaded; save the results to out"""
    import torch

    from paper_2607_06834_b300 import abi, sampler, synth
    from paper_2607_06834_b300.engine import Engine
    res = {}
    for name, make, prec, tr, B in _cases():
        arr = make()
        eng = Engine(arr, precision=prec)
        eng.set_transform(tr)
        x = torch.tensor(synth.make_points(arr, B, seed=808), device="cuda")
        lp, g, st = eng.logp_and_grad(x)
        torch.cuda.synchronize()
        res[name + "_logp"] = lp.cpu().numpy()
        res[name + "_grad"] = g.cpu().numpy()
        res[name + "_stat"] = st.cpu().numpy()
        eng.close()
    arr = synth.small_array(**RAGGED)
    eng = Engine(arr, precision="f16split")
    x = torch.tensor(synth.make_points(arr, 8, seed=809), device="cuda")
    r = sampler.run_hmc(eng, x, n_warmup=4, n_samples=4, n_leapfrog=4, seed=5)
    res["hmc_x"] = r.state.x.cpu().numpy()
    eng.close()
    np.savez(out, **res)
    print(json.dumps({"lib": os.path.basename(abi.LIB_PATH)}))


@pytest.fixture(scope="module")
def check_lib():
    from paper_2607_06834_b300 import build
    if build.needs_build(build.LIB_CHECK):
        build.build(check=True)
    return build.LIB_CHECK


def test_check_build_matches_release(check_lib, tmp_path):
    out_c, out_r = str(tmp_path / "check.npz"), str(tmp_path / "release.npz")
    code = f"import sys; sys.path.insert(0, {ROOT!r}); import tests.test_gpu_check_build as t; t._run_all(sys.argv[1])"
    env = dict(os.environ, PTA_CHECK_BUILD="1")
    p = subprocess.run([sys.executable, "-c", code, out_c], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    assert json.loads(p.stdout.strip().splitlines()[-1])["lib"] == "libptahmc_check.so"
    _run_all(out_r)
    c, r = np.load(out_c), np.load(out_r)
    nbit = 0
    for k in r.files:
        a, b = c[k], r[k]
        nbit += int(np.array_equal(a, b))
        if k == "hmc_x":  # an accept decision may flip on a last-bit difference: the run itself must pass
            assert np.all(np.isfinite(a)), k
        elif k.endswith("_stat"):
            assert np.all(a == 0) and np.array_equal(a, b), k
        elif k.endswith("_logp"):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-9, err_msg=k)
        else:
            np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max(), err_msg=k)
    print(f"check build: {len(r.files)} arrays, {nbit} bit-identical to the release build")
