#!/usr/bin/env python
"""Throughput of the batched log posterior + gradient (the HMC hot path).

One step = one pta_logp_and_grad call over all chains of the workload: prior
spectra + FP64 per-frequency Cholesky + transform, TOA-domain contractions, FP64
timing-model solve, adjoint and final sum.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): chains are independent, so every rank runs its own batch of
chains on its own GPU (weak scaling, no data-path collective); a barrier and a
max-over-ranks of the timed duration use the process group.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ng15_b256"
WORKLOAD_DESC = "NANOGrav-15-yr-like: 67 pulsars, 3.0e5 TOAs, RN 30 / DM 100 / HD-GWB 14 bins, 256 chains"
METRIC = "logp+grad evals/s (all chains) at 67-psr size vs FP64 plain path; % roofline"
DTYPE = {"fp32": "f32", "fp64": "f64", "tf32x3": "tf32x3", "tf32": "tf32", "bf16x3": "bf16x3",
         "gram": "f32 (compensated)", "f16split": "f16 (exact split, f32 accumulate)"}
DTYPE_DETAIL = {"fp32": "FP32 TOA contractions (SIMT)", "fp64": "FP64 TOA contractions (stored basis)",
                "tf32x3": "3-term split TF32 tensor-core TOA contractions, FP32 accumulation",
                "tf32": "single TF32 tensor-core TOA contractions, FP32 accumulation",
                "bf16x3": "3-term split BF16 tensor-core TOA contractions, FP32 accumulation",
                "gram": "Gram form: per-pulsar F^T N~^-1 F products in compensated FP32 (hi/lo, Dot2)",
                "f16split": "exact-split fp16 tensor-core TOA contractions (tcgen05 kind::f16): stored projected "
                            "basis and FP64 coefficients cut into 4 fp16 pieces, exact leading levels, "
                            "10 MMAs per K step for F a and 6 for F^T w"}
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # SMs x FP32 lanes x 2 flop x max SM clock
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12     # SMs x 2 FP64 FMA/clk x 2 flop x max SM clock
# The dense-bin Cholesky outside FP64 mode runs in double-word (float pair) arithmetic on
# the FP32 pipes: one multiply-add of the algorithm issues 14 FP32 operations (an exact
# product with three fused multiply-adds, TwoSum and a renormalisation), so its peak in
# flop of the algorithm is the FP32 operation rate x 2 / 14.
# the HMC legs sample with the headline evaluation path
HMC_PRECISION = "f16split"
HMC_PATH = "exact-split tensor-core path"
DW_OPS_PER_FMA = 14
DW_PEAK_TFLOPS = 148 * 128 * 2.032e9 * 2 / DW_OPS_PER_FMA / 1e12


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel from one ncu capture, valid only while the kernel's sources are the ones
# profiled (sha256 of each file); see profiles/.
CAPTURED_TRAFFIC = {
    "k_chol_forward_dw": {"bytes": (7.477248 + 78.906112) * 1e6, "profile": "profiles/k_chol_forward_dw_ng15_b256.md",
                          "sources": {"k_prior.cu": "577a257f2b1635253165b9e54b638f14c8155b1975415154e5661089bec34220",
                                      "dw_ldl.cuh": "f0f4f50e696915f9891833b063ccc90b6bd9e024447d1020ad7d16f07c3dd3af",
                                      "dwarith.cuh": "487efa32b981977af53e8f51e037f947a3a1373050868a1543ad1ac2869bdae0",
                                      "pta_check.cuh": "8922e66311c1eaef8cef83b01d22f538ca1c01ce3714480bf04d301dd04618a6",
                                      "pta_internal.cuh":
                                          "77ac6b320ff664cb6fc0ede00f32a73d8b1e294df681d41d324ca9dc63c03f45"}},
    "k_f16_res": {"bytes": (743.047168 + 286.591488) * 1e6, "profile": "profiles/k_f16_res_ng15_b256.md",
                  "sources": {"k_toa_f16.cu": "0ee63d4252e783834f58afda7beab9780ef47efe3837d7b726ec5fa22d7eb71c",
                              "dwarith.cuh": "487efa32b981977af53e8f51e037f947a3a1373050868a1543ad1ac2869bdae0",
                              "pta_check.cuh": "8922e66311c1eaef8cef83b01d22f538ca1c01ce3714480bf04d301dd04618a6",
                              "pta_internal.cuh": "77ac6b320ff664cb6fc0ede00f32a73d8b1e294df681d41d324ca9dc63c03f45",
                              "tc_ptx.cuh": "3c9784327356c5b1fdfbf233ac793b19bb50883f641ee44cceddaaed2465521c"}},
    "k_f16_ftw": {"bytes": (835.902208 + 39.038464) * 1e6, "profile": "profiles/k_f16_ftw_ng15_b256.md",
                  "sources": {"k_toa_f16.cu": "0ee63d4252e783834f58afda7beab9780ef47efe3837d7b726ec5fa22d7eb71c",
                              "dwarith.cuh": "487efa32b981977af53e8f51e037f947a3a1373050868a1543ad1ac2869bdae0",
                              "pta_check.cuh": "8922e66311c1eaef8cef83b01d22f538ca1c01ce3714480bf04d301dd04618a6",
                              "pta_internal.cuh": "77ac6b320ff664cb6fc0ede00f32a73d8b1e294df681d41d324ca9dc63c03f45",
                              "tc_ptx.cuh": "3c9784327356c5b1fdfbf233ac793b19bb50883f641ee44cceddaaed2465521c"}},
}


def captured_traffic(kernel):
    """DRAM bytes per launch of `kernel` (dram__bytes_read.sum + dram__bytes_write.sum)
    from one ncu capture, valid only while the kernel's source files are the ones
    profiled (sha256 of each file); None otherwise."""
    import hashlib
    rec = CAPTURED_TRAFFIC.get(kernel)
    if rec is None:
        return None
    csrc = os.path.join(ROOT, "paper_2607_06834_b300", "csrc")
    for f, h in rec["sources"].items():
        try:
            if hashlib.sha256(open(os.path.join(csrc, f), "rb").read()).hexdigest() != h:
                return None
        except OSError:
            return None
    return {"bytes_per_launch": rec["bytes"], "profile": rec["profile"]}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except Exception:
            return None
    return None


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.strip().split(", ") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


def toa_flops_per_launch(arr, B):
    """Algorithmic flops of the TOA contractions per launch: F a (2 n P), F^T w (2 n P)
    and M^T w (2 n m) per chain and pulsar, unpadded TOA counts."""
    na = max(arr.n_gwb, arr.n_rn)
    P = 2 * na + 2 * arr.n_dm
    return float(B * sum(2 * p.n * (2 * P + p.m) for p in arr.pulsars))


def toa_flops_f16(arr, B):
    """Algorithmic flops of the exact-split path's contractions per launch: F~ a and
    F~^T w (2 n P each) per chain and pulsar, plus M c_s (2 n m) with a signal."""
    na = max(arr.n_gwb, arr.n_rn)
    P = 2 * na + 2 * arr.n_dm
    return float(B * sum(2 * p.n * (2 * P + (p.m if arr.cw else 0)) for p in arr.pulsars))


def toa_issued_f16(arr, B):
    """Tensor flops the exact-split kernels issue per launch (launch shapes of
    k_f16_res and k_f16_ftw): per 128-TOA tile, 16-column step and chain block of NC,
    MMAs of N = 4, 3, 2, 1 x NC; per 32-TOA stage, 144-column chunk and 128 chains, six
    MMAs of N = 144 (the last chunk rounded up to 16)."""
    na = max(arr.n_gwb, arr.n_rn)
    P = 2 * na + 2 * arr.n_dm
    kxm = -(-(P + (max(p.m for p in arr.pulsars) if arr.cw else 0)) // 32) * 32
    nc = 64 if 4 * 16384 + 4 * kxm * 64 * 2 + 64 * 16 <= 227 * 1024 else 32
    res = ftw = 0.0
    for p in arr.pulsars:
        npad = -(-p.n // 128) * 128
        kx = -(-(P + (p.m if arr.cw else 0)) // 32) * 32
        res += (npad // 128) * (kx // 16) * 2.0 * 128 * 10 * nc * 16 * (-(-B // nc))
        for q0 in range(0, P, 144):
            nq = -(-min(144, P - q0) // 16) * 16
            ftw += (npad // 32) * 2 * 6 * 2.0 * 128 * nq * 16 * (-(-B // 128))
    return res + ftw


def chol_roofline(arr, B, kms, fp64, size=""):
    """Roofline record of the dense-bin factorisation kernel: algorithmic flop (2n^3/3 + 2n^2
    per bin and chain, the factor and its inverse) over its own CUDA-event time, against the
    FP64 pipe's peak (FP64 mode) or the double-word peak on the FP32 pipes."""
    flops = chol_flops_per_launch(arr, B)
    ach = flops / (kms * 1e-3) / 1e12
    if fp64:
        return {"kernel": f"k_chol_forward (FP64 {size}Cholesky + inverse + transform, dense bins)", "bound": "alu",
                "unit": "TFLOP/s", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "peak_source": "derived: 148 SM x 2 FP64 FMA/clk x 2 flop x 2.032 GHz", "kernel_ms": kms,
                "algorithmic_flop": flops}
    return {"kernel": f"k_chol_forward_dw (double-word {size}Cholesky + inverse + transform, dense bins)",
            "bound": "alu", "unit": "TFLOP/s", "achieved": ach, "peak": DW_PEAK_TFLOPS,
            "peak_source": f"derived: 148 SM x 128 FP32 lanes x 2.032 GHz x 2 flop / {DW_OPS_PER_FMA} FP32 "
                           "operations per double-word multiply-add",
            "kernel_ms": kms, "algorithmic_flop": flops,
            "fp64_peak_frac": ach / FP64_PEAK_TFLOPS,
            "note": "achieved counts the algorithm's flop (FP64-equivalent work at ~48-bit precision); "
                    "fp64_peak_frac compares it with what the FP64 pipe could do at most"}


def chol_flops_per_launch(arr, B):
    """FP64 flops of the dense-bin prior forward per launch: Cholesky (np^3/3),
    triangular inverse (np^3/3) and the transform (2 x np^2) per (chain, bin)."""
    npsr = arr.npsr
    nb = min(arr.n_gwb, arr.n_rn)
    return float(B * nb * (2 * npsr ** 3 / 3 + 2 * npsr ** 2))


def curn_flops_per_launch(arr, B):
    """FP64 flops of the CURN factorisation per launch: the LDL^T sweep with the inverse
    (P^3/3 multiply-adds) and the transform's triangular products (3 P^2 flop) per
    (pulsar, chain)."""
    P = 2 * max(arr.n_gwb, arr.n_rn) + 2 * arr.n_dm
    return float(B * arr.npsr * (2.0 * P ** 3 / 3.0 + 3.0 * P ** 2))


def curn_factor_mode(P):
    """Which CURN forward kernel the library runs outside FP64 mode (the rule of
    launch_curn_forward): 1 = k_curn_forward_dw, the triangle in one CTA's shared memory;
    C > 1 = k_curn_forward_dwc over a cluster of C CTAs (row pairs interleaved); 0 = FP64."""
    lim = 226 * 1024
    stage = 6 * (P // 2 + 1) * 16
    prow = P * (P + 2) // 2 if P % 2 == 0 else (P + 1) ** 2 // 2
    if stage + prow * 8 <= lim:
        return 1
    npairs, cstage = (P + 1) // 2, (10 * (P // 2 + 1) + 8) * 16
    for C in (2, 4, 8):
        part = max(4 * M * (k + 1) + 2 * C * M * (M - 1)
                   for k in range(C) for M in [(npairs - k + C - 1) // C if npairs > k else 0])
        if cstage + 2 * P * 8 + part * 8 <= lim:
            return C
    return 0


def curn_variant(dev, steps):
    """The CURN-posterior transform (Eq. PTA_standard_transform_curn) against the default
    prior-whitened one on the same batch: the paper's NANOGrav-15-yr model (RN 30 /
    HD-GWB 14 bins, no DM: P = 60, the factor in one CTA's shared memory) with 64 and 256
    chains, and the 100-DM-bin workload (P = 260, the factor over a cluster of two CTAs)
    with 256 chains, on the headline path.  CUDA events per step with L2 flushed; the
    factorisation stage is the CURN forward stage minus the prior-whitened one, in double
    words (curn_factor_mode)."""
    import ctypes as C
    import torch
    from paper_2607_06834_b300 import abi, synth
    from paper_2607_06834_b300.engine import Engine
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peak = FP64_PEAK_TFLOPS
    out = []
    for name, B in (("ng15_nodm", 64), ("ng15_nodm", 256), ("ng15_b256", 256)):
        arr = synth.make_array(name)
        eng = Engine(arr, precision=HMC_PRECISION)
        x = torch.tensor(synth.make_points(arr, B, seed=6834 + 7), device=dev)
        rec = {"workload": name, "chains": B, "P": 2 * max(arr.n_gwb, arr.n_rn) + 2 * arr.n_dm}
        for tr in ("prior", "curn"):
            eng.set_transform(tr)
            for _ in range(3):
                eng.logp_and_grad(x)
            torch.cuda.synchronize()
            abi.lib.pta_profile_enable(eng._h, 1)
            abi.lib.pta_profile_read(eng._h, None, None, 1)
            n = max(3, min(steps, 10 if name != "ng15_b256" else 3))
            ev = []
            for _ in range(n):
                flush.zero_()
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record()
                eng.logp_and_grad(x)
                a1.record()
                ev.append((a0, a1))
            torch.cuda.synchronize()
            sm = (C.c_double * abi.NSTAGES)()
            abi.lib.pta_profile_read(eng._h, sm, None, 1)
            abi.lib.pta_profile_enable(eng._h, 0)
            ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
            rec[tr] = {"value": B / (ms * 1e-3), "unit": "evals/s", "ms_per_step": ms,
                       "stage_ms": dict(zip(abi.STAGES, [round(v / n, 4) for v in sm]))}
        fac_ms = rec["curn"]["stage_ms"]["prior_forward"] - rec["prior"]["stage_ms"]["prior_forward"]
        ach = curn_flops_per_launch(arr, B) / (fac_ms * 1e-3) / 1e12
        P = rec["P"]
        mode = curn_factor_mode(P)
        if mode:
            kern = "k_curn_forward_dw" if mode == 1 else f"k_curn_forward_dwc<{mode}>"
            rec["roofline"] = {"kernel": f"{kern} + k_curn_whiten (double-word LDL^T sweep with inverse)",
                               "bound": "alu", "unit": "TFLOP/s", "achieved": ach, "peak": DW_PEAK_TFLOPS,
                               "peak_source": f"derived: 148 SM x 128 FP32 lanes x 2.032 GHz x 2 flop / "
                                              f"{DW_OPS_PER_FMA} FP32 operations per double-word multiply-add",
                               "frac": ach / DW_PEAK_TFLOPS, "fp64_peak_frac": ach / peak, "stage_ms": fac_ms,
                               "factor_in": "shared memory" if mode == 1 else
                               f"distributed shared memory of a {mode}-CTA cluster"}
        else:
            rec["roofline"] = {"kernel": "k_curn_forward + k_curn_whiten (FP64 LDL^T sweep with inverse)",
                               "bound": "alu", "unit": "TFLOP/s", "achieved": ach, "peak": peak,
                               "peak_source": "derived: 148 SM x 2 FP64 FMA/clk x 2 flop x 2.032 GHz",
                               "frac": ach / peak, "stage_ms": fac_ms,
                               "factor_in": "shared memory" if (P * (P + 1) // 2 + 8 * P) * 8 <= 200 * 1024
                               else "global inverse buffer"}
        eng.close()
        out.append(rec)
    return out


def scale150_leg(dev, steps: int, peaks):
    """The scale-up configuration: 150 pulsars, 1.0e6 TOAs (1k-30k per pulsar over up to
    30 yr), 100 GWB / 30 red-noise / 150 DM bins (P = 500), 1024 chains in one call.
    Evals/s of the exact-split path (headline mode) and the FP32 SIMT path, the plain
    FP64 path on the same batch, stage and kernel times, the dominant kernel's roofline
    and the end-to-end rate through host buffers.  L2 flushed between timed steps."""
    import ctypes as C
    import torch
    from paper_2607_06834_b300 import abi, synth
    from paper_2607_06834_b300.engine import Engine
    arr = synth.make_array("scale150")
    B = synth.WORKLOADS["scale150"]["chains"]
    t0 = time.perf_counter()
    eng = Engine(arr, precision="f16split")
    setup_s = time.perf_counter() - t0
    X = synth.make_points(arr, B, seed=6834 + 4)
    x = torch.tensor(X, device=dev)
    out = (torch.empty(B, dtype=torch.float64, device=dev), torch.empty_like(x),
           torch.empty(B, dtype=torch.int32, device=dev))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    rec = {"workload": "150 pulsars, 1.0e6 TOAs, GWB 100 / RN 30 / DM 150 bins (P = 500), 1024 chains",
           "ntoa": arr.ntoa, "chains": B, "host_setup_s": setup_s}

    def timed(prec, n):
        eng.set_precision(prec)
        for _ in range(2):
            eng.logp_and_grad(x, out=out)
        torch.cuda.synchronize()
        assert int((out[2] != 0).sum()) == 0, "non-finite or out-of-prior chains in the scale-up batch"
        abi.lib.pta_profile_enable(eng._h, 1)
        abi.lib.pta_profile_read(eng._h, None, None, 1)
        ev = []
        for _ in range(n):
            flush.zero_()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            eng.logp_and_grad(x, out=out)
            a1.record()
            ev.append((a0, a1))
        torch.cuda.synchronize()
        sm = (C.c_double * abi.NSTAGES)()
        abi.lib.pta_profile_read(eng._h, sm, None, 1)
        abi.lib.pta_profile_enable(eng._h, 0)
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        st = [v / n for v in sm]
        return {"value": B / (ms * 1e-3), "unit": "evals/s", "ms_per_step": ms, "steps": n,
                "stage_ms": dict(zip(abi.STAGES, [round(v, 3) for v in st])),
                "kernel_ms": dict(zip(abi.KERNEL_TIMERS, [round(v, 3) for v in st[len(abi.STAGES):]]))}

    n = max(3, min(steps, 5))
    rec["f16split"] = timed("f16split", n)
    eng.set_cholesky("fp64")  # the same path with the FP64 dense-bin Cholesky (150 x 150)
    rec["f16split_chol_fp64"] = timed("f16split", n)
    eng.set_cholesky("dw")
    rec["fp32"] = timed("fp32", n)
    rec["fp64_plain_path"] = timed("fp64", 1)
    rec["f16split_vs_fp64_plain_path"] = rec["f16split"]["value"] / rec["fp64_plain_path"]["value"]
    # roofline of the dominant kernel in the headline mode
    f = rec["f16split"]
    kms = f["kernel_ms"]
    dom = max(kms, key=kms.get)
    if dom == "chol_forward":
        rec["roofline"] = chol_roofline(arr, B, kms[dom], False, "150 x 150 ")
    else:
        bf16 = (peaks or {}).get("bf16_tflops", 1800.0)
        flops = toa_flops_f16(arr, B) / 2  # one of the two contractions per kernel
        rec["roofline"] = {"kernel": {"toa_res": "k_f16_res", "toa_ftw": "k_f16_ftw"}[dom], "bound": "tensor",
                           "unit": "TFLOP/s", "achieved": flops / (kms[dom] * 1e-3) / 1e12, "peak": bf16,
                           "peak_source": "measured bf16 burst (fp16 has the same dense rate)"}
    rec["roofline"]["frac"] = rec["roofline"]["achieved"] / rec["roofline"]["peak"]
    rec["roofline"]["kernel_ms"] = kms[dom]
    # end to end through host buffers: x in, logp and gradient out, every step
    eng.set_precision("f16split")
    xh = torch.tensor(X).pin_memory()
    lh = torch.empty(B, dtype=torch.float64).pin_memory()
    gh = torch.empty(tuple(x.shape), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n):
        x.copy_(xh, non_blocking=True)
        eng.logp_and_grad(x, out=out)
        lh.copy_(out[0], non_blocking=True)
        gh.copy_(out[1], non_blocking=True)
    e1.record()
    e1.synchronize()
    rec["e2e"] = {"value": B / (e0.elapsed_time(e1) / n * 1e-3), "unit": "evals/s",
                  "h2d_bytes_per_step": int(x.numel() * 4), "d2h_bytes_per_step": int(B * 8 + x.numel() * 4)}
    eng.close()
    return rec


_ORC = None


def _oracle_worker_init(workload: str):
    """Process-pool worker: its own FP64 oracle (stored basis) of the workload."""
    global _ORC
    from oracle import pta_oracle as O
    from paper_2607_06834_b300 import synth
    _ORC = O.Oracle(synth.make_array(workload))


def _oracle_eval(x):
    _ORC.logp(x)
    _ORC.grad(x)
    return 1


def oracle_pool(workload: str):
    """A spawn-started pool (safe after CUDA use) of one single-threaded oracle per host
    core, bounded by memory (about 1 GB per worker at the 67-pulsar size)."""
    import multiprocessing as mp
    ncpu = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    try:
        avail_gb = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE") / 2 ** 30
    except (ValueError, OSError):
        avail_gb = 16.0
    nproc = max(1, min(ncpu, 64, int(avail_gb // 1.5)))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"   # one BLAS thread per worker: the pool is the parallelism
    try:
        pool = mp.get_context("spawn").Pool(nproc, initializer=_oracle_worker_init, initargs=(workload,))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool, nproc


def oracle_rate(workload: str, steps: int, warmup: int):
    """The FP64 oracle, as it stands, on the host cores: each step evaluates logp + grad
    of one chain per worker process (B = #workers chains in parallel).  Returns
    (evals/s, workers, timed seconds, steps timed)."""
    from paper_2607_06834_b300 import synth
    pool, nproc = oracle_pool(workload)
    try:
        arr = synth.make_array(workload)
        X = synth.make_points(arr, nproc * (steps + warmup), seed=6834 + 2).astype(np.float64)
        for i in range(warmup):
            pool.map(_oracle_eval, list(X[i * nproc:(i + 1) * nproc]), chunksize=1)
        t0 = time.perf_counter()
        for i in range(warmup, warmup + steps):
            pool.map(_oracle_eval, list(X[i * nproc:(i + 1) * nproc]), chunksize=1)
        dt = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    return nproc * steps / dt, nproc, dt, steps


def cpu_baseline(workload: str, steps: int):
    value, nproc, dt, steps = oracle_rate(workload, steps, 1)
    return {"value": value, "unit": "evals/s", "cores": int(nproc), "kind": "oracle",
            "sample": f"{steps} steps of {nproc} chains of the {workload} workload, one chain per process "
                      f"({nproc} spawned processes, one BLAS thread each; {dt:.1f} s timed; numpy FP64)"}


RHAT_CONVERGED = 1.05


def ess_rate(ess: float, rhat: float, seconds: float):
    """ESS per second of a parameter group, published only when its split R-hat is at most
    RHAT_CONVERGED: an ESS of chains that have not mixed is not an effective sample size."""
    if not np.isfinite(rhat) or rhat > RHAT_CONVERGED:
        return {"ess_per_s": "unconverged", "rhat": float(rhat)}
    return {"ess_per_s": float(ess) / seconds, "rhat": float(rhat)}


def hmc_ess_tiny(dev):
    """Control run of the same driver on the 3-pulsar, 10-bin array (64 chains,
    20 leapfrog steps), where the posterior is benign enough to mix in seconds."""
    import torch
    from paper_2607_06834_b300 import sampler, synth
    from paper_2607_06834_b300.engine import Engine
    arr = synth.make_array("tiny3")
    eng = Engine(arr, precision="fp32")
    lay = eng.layout
    x0 = torch.tensor(synth.make_points(arr, 64, seed=6834 + 30), device=dev)
    th0 = lay["d_z"]
    res = sampler.run_hmc(eng, x0, n_warmup=400, n_samples=400, n_leapfrog=20, record=slice(0, eng.D),
                          seed=6834 + 30, eps0=0.05, init_dz=th0, consensus=100)
    e = sampler.ess_columns(res.draws)
    rh = np.array([sampler.split_rhat(res.draws[:, :, k]) for k in range(res.draws.shape[2])])
    g0 = lay["th_gwb"]
    t = res.sampling_s
    eng.close()
    return {"workload": "3 pulsars x 200 TOAs, RN/GWB 10 bins, 64 chains, 20 leapfrog steps, FP32 path",
            "warmup_trajectories": 400, "sampling_trajectories": 400,
            "gwb": ess_rate(np.nanmin(e[g0:g0 + 2]), np.nanmax(rh[g0:g0 + 2]), t),
            "all_parameters": ess_rate(np.nanmedian(e), np.nanmax(rh), t),
            "ess_gwb_min": float(np.nanmin(e[g0:g0 + 2])), "ess_median": float(np.nanmedian(e)),
            "rhat_max": float(np.nanmax(rh)), "rhat_median": float(np.nanmedian(rh)), "sampling_s": t,
            "accept_rate": res.accept_rate, "stuck_chains": res.stats["stuck_chains"]}


def hmc_ess(args, dev):
    """HMC effective samples per second on the NG15-like array plus a circular binary:
    64 chains, trajectories of 20 leapfrog steps (one CUDA graph each), warm-up with
    step-size and diagonal-mass adaptation, then the sampling iterations timed; ESS by
    the multi-chain Geyer estimator over the hyper-parameters and CW parameters."""
    import torch
    from paper_2607_06834_b300 import sampler, synth
    from paper_2607_06834_b300.engine import Engine
    name = "ng15_cw"
    arr = synth.make_array(name)
    B, L = synth.WORKLOADS[name]["chains"], 20
    eng = Engine(arr, precision=HMC_PRECISION)
    lay = eng.layout
    x0 = torch.tensor(synth.make_points(arr, B, seed=6834 + 3), device=dev)
    th0 = lay["d_z"]
    # record the hyper-parameters and CW parameters plus every 50th whitened coefficient
    zpick = np.arange(0, th0, 50)
    rec = np.concatenate([zpick, np.arange(th0, eng.D)])
    res = sampler.run_hmc(eng, x0, n_warmup=args.hmc_warmup, n_samples=args.hmc_samples, n_leapfrog=L,
                          record=torch.tensor(rec, device=dev), seed=6834 + 3, eps0=0.01, init_dz=th0,
                          consensus=args.hmc_warmup // 4)
    e_all = sampler.ess_columns(res.draws)
    rh_all = np.array([sampler.split_rhat(res.draws[:, :, k]) for k in range(res.draws.shape[2])])
    nz = len(zpick)
    e, rh = e_all[nz:], rh_all[nz:]
    e_z = float(np.nanmedian(e_all[:nz]))
    g0 = lay["th_gwb"] - th0
    cw0 = lay["th_cw"] - th0
    e_gwb = float(np.nanmin(e[g0:g0 + 2]))
    e_med = float(np.nanmedian(e))
    e_cw = float(np.nanmedian(e[cw0:cw0 + 8]))
    t = res.sampling_s
    eng.close()
    return {"workload": "NANOGrav-15-yr-like array + circular SMBHB (Earth and pulsar terms), "
                        f"{B} chains, {L} leapfrog steps per trajectory, {HMC_PATH}",
            "warmup_trajectories": args.hmc_warmup, "sampling_trajectories": args.hmc_samples,
            "gwb": ess_rate(e_gwb, np.nanmax(rh[g0:g0 + 2]), t),
            "theta_median": ess_rate(e_med, np.nanmax(rh), t),
            "cw": ess_rate(e_cw, np.nanmax(rh[cw0:cw0 + 8]), t),
            "ess_gwb_min": e_gwb, "ess_theta_median": e_med, "ess_cw_median": e_cw, "ess_z_median": e_z,
            "start": "conditional mode in z, then all chains restart from the best chain after a quarter "
                     "of the warm-up (consensus start)",
            "sampling_s": t, "warmup_s": res.warmup_s,
            "ms_per_trajectory": 1e3 * t / max(args.hmc_samples, 1),
            "evals_per_s": B * L * args.hmc_samples / t, "accept_rate": res.accept_rate, "step": res.step,
            "rhat_gwb_max": float(np.nanmax(rh[g0:g0 + 2])), "rhat_theta_median": float(np.nanmedian(rh)),
            "init": "z at the conditional mode given the starting hyper-parameters (batched CG)",
            "stuck_chains": res.stats["stuck_chains"], "chain_accept_min": res.stats["chain_accept_min"],
            "step_range": [res.stats["step_min"], res.stats["step_max"]],
            "ess_estimator": "multi-chain, Geyer initial monotone sequence"}


def hmc_ess_transforms(args, dev):
    """HMC effective samples per second on the model of the paper's NANOGrav-15-yr
    analysis (67 pulsars, RN 30 / HD-GWB 14 bins, no DM), 64 chains, 20 leapfrog steps,
    under the CURN-posterior transform (Eq. PTA_standard_transform_curn; z keeps unit
    mass, z ~ N(0, 1) starts near the posterior) and, as the control, under the
    prior-whitened transform (z started at its conditional mode).  Same warm-up (step
    size, diagonal mass of the hyper-parameters, consensus start), same draws."""
    import torch
    from paper_2607_06834_b300 import sampler, synth
    from paper_2607_06834_b300.engine import Engine
    name = "ng15_nodm"
    arr = synth.make_array(name)
    B, L = synth.WORKLOADS[name]["chains"], 20
    out = {"workload": "paper's NANOGrav-15-yr model (RN 30 / HD-GWB 14 bins, no DM) on the 67-pulsar "
                       f"array, {B} chains, {L} leapfrog steps per trajectory, {HMC_PATH}",
           "warmup_trajectories": {"curn": args.hmc_warmup_curn, "prior": args.hmc_warmup},
           "sampling_trajectories": {"curn": args.hmc_samples_curn, "prior": args.hmc_samples}}
    for tr in ("curn", "prior"):
        ns = args.hmc_samples_curn if tr == "curn" else args.hmc_samples
        nw = args.hmc_warmup_curn if tr == "curn" else args.hmc_warmup
        eng = Engine(arr, precision=HMC_PRECISION)
        eng.set_transform(tr)
        lay = eng.layout
        th0 = lay["d_z"]
        x0 = torch.tensor(synth.make_points(arr, B, seed=6834 + 3), device=dev)
        kw = dict(unit_mass=th0, init_dz=0) if tr == "curn" else dict(init_dz=th0)
        res = sampler.run_hmc(eng, x0, n_warmup=nw, n_samples=ns, n_leapfrog=L,
                              record=slice(th0, eng.D), seed=6834 + 3, eps0=0.01,
                              consensus=nw // 4, **kw)
        e = sampler.ess_columns(res.draws)
        rh = np.array([sampler.split_rhat(res.draws[:, :, k]) for k in range(res.draws.shape[2])])
        g0 = lay["th_gwb"] - th0
        t = res.sampling_s
        out[tr] = {"gwb": ess_rate(np.nanmin(e[g0:g0 + 2]), np.nanmax(rh[g0:g0 + 2]), t),
                   "theta": ess_rate(np.nanmedian(e), np.nanmax(rh), t),
                   "ess_gwb_min": float(np.nanmin(e[g0:g0 + 2])), "ess_theta_median": float(np.nanmedian(e)),
                   "rhat_gwb_max": float(np.nanmax(rh[g0:g0 + 2])), "rhat_theta_median": float(np.nanmedian(rh)),
                   "rhat_theta_max": float(np.nanmax(rh)), "sampling_s": t, "warmup_s": res.warmup_s,
                   "ms_per_trajectory": 1e3 * t / max(ns, 1),
                   "evals_per_s": B * L * ns / t, "accept_rate": res.accept_rate, "step": res.step,
                   "gwb_posterior_mean": [float(v) for v in res.draws[:, :, g0:g0 + 2].reshape(-1, 2).mean(0)],
                   "gwb_posterior_std": [float(v) for v in res.draws[:, :, g0:g0 + 2].reshape(-1, 2).std(0)],
                   "stuck_chains": res.stats["stuck_chains"]}
        eng.close()
    # the same model with a circular binary, CURN transform with the signal-dependent mean
    # (Eq. decenter_det_PTA)
    arr = synth.make_array("ng15_nodm_cw")
    eng = Engine(arr, precision=HMC_PRECISION)
    eng.set_transform("curn")
    lay = eng.layout
    th0 = lay["d_z"]
    x0 = torch.tensor(synth.make_points(arr, B, seed=6834 + 5), device=dev)
    res = sampler.run_hmc(eng, x0, n_warmup=args.hmc_warmup, n_samples=args.hmc_samples, n_leapfrog=L,
                          record=slice(th0, eng.D), seed=6834 + 5, eps0=0.01, consensus=args.hmc_warmup // 4,
                          unit_mass=th0, init_dz=0)
    e = sampler.ess_columns(res.draws)
    rh = np.array([sampler.split_rhat(res.draws[:, :, k]) for k in range(res.draws.shape[2])])
    g0, c0 = lay["th_gwb"] - th0, lay["th_cw"] - th0
    t = res.sampling_s
    out["curn_with_cw"] = {"workload": "same model + circular SMBHB (Earth and pulsar terms), CURN transform with "
                                       "the signal-dependent mean",
                           "gwb": ess_rate(np.nanmin(e[g0:g0 + 2]), np.nanmax(rh[g0:g0 + 2]), t),
                           "theta": ess_rate(np.nanmedian(e), np.nanmax(rh), t),
                           "cw": ess_rate(np.nanmedian(e[c0:c0 + 8]), np.nanmax(rh[c0:c0 + 8]), t),
                           "ess_gwb_min": float(np.nanmin(e[g0:g0 + 2])), "ess_theta_median": float(np.nanmedian(e)),
                           "ess_cw_median": float(np.nanmedian(e[c0:c0 + 8])),
                           "rhat_gwb_max": float(np.nanmax(rh[g0:g0 + 2])),
                           "rhat_theta_median": float(np.nanmedian(rh)), "rhat_cw_max": float(np.nanmax(rh[c0:c0 + 8])),
                           "sampling_s": t, "warmup_s": res.warmup_s,
                           "ms_per_trajectory": 1e3 * t / max(args.hmc_samples, 1), "accept_rate": res.accept_rate,
                           "step": res.step, "stuck_chains": res.stats["stuck_chains"]}
    eng.close()
    out["ess_estimator"] = "multi-chain, Geyer initial monotone sequence"
    out["bounded_coordinates"] = "hyper-parameters move in logit space inside each trajectory"
    out["paper_context"] = {"ess_per_s": 1.53, "note": "the paper's figure for this model on the real "
                            "NANOGrav 15-yr data, one RTX 3090, JAX/NumPyro NUTS: context, not the same run "
                            "(synthetic data here, fixed-length HMC, another GPU)"}
    return out


def reduce_timing(ms: float, chains: int, world: int, pg=None, device=None):
    """Max over ranks of the per-step time (ms) and the whole-job throughput: every
    rank evaluates its own ``chains`` chains, so value = world x chains / max time."""
    import torch
    if pg is not None and world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * chains / (ms * 1e-3)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    value, nproc, dt, steps = oracle_rate(WORKLOAD, args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_DESC, "chains_per_step": nproc},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": int(nproc), "kind": "oracle",
                             "sample": f"each step: {nproc} chains, one per spawned process (one BLAS thread each)"},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_2607_06834_b300 import abi, synth
    from paper_2607_06834_b300.engine import Engine
    arr = synth.make_array(args.workload)
    B = args.chains if args.chains > 0 else synth.WORKLOADS[args.workload]["chains"]
    X = synth.make_points(arr, B, seed=6834 + 2 + 1000 * rank)
    eng = Engine(arr, precision=args.precision)
    if args.transform != "prior":
        eng.set_transform(args.transform)
    D = eng.D
    tuned = None
    if args.precision == "fp32":  # the autotuner picks the SIMT tile shape (setup, not timed)
        from paper_2607_06834_b300.engine import toa_config_info
        if args.toa_config >= 0:      # fixed shape (profiling runs: no tuning launches)
            eng.set_toa_config(args.toa_config)
            tuned = {"entry": args.toa_config, **toa_config_info(args.toa_config), "fixed": True}
        else:
            chosen, table = eng.autotune(B)
            tuned = {"entry": chosen, **toa_config_info(chosen),
                     "candidates_ms": {str(k): round(v, 4) for k, v in sorted(table.items())}}
    dev = torch.device("cuda", local)
    x = torch.tensor(X, device=dev)
    logp = torch.empty(B, dtype=torch.float64, device=dev)
    grad = torch.empty_like(x)
    status = torch.empty(B, dtype=torch.int32, device=dev)
    out = (logp, grad, status)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 126 MB L2
    for _ in range(args.warmup):
        eng.logp_and_grad(x, out=out)
    torch.cuda.synchronize()
    assert int((status != 0).sum()) == 0, "non-finite or out-of-prior chains in the bench batch"

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    abi.lib.pta_profile_enable(eng._h, 1)
    abi.lib.pta_profile_read(eng._h, None, None, 1)
    clocks = Clocks(local) if rank == 0 or True else None
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record()
        eng.logp_and_grad(x, out=out)
        ends[i].record()
    barrier()
    t_wall = time.perf_counter() - t_wall
    ck = clocks.stop() if clocks else None
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = float(np.sum(step_ms)) / args.steps
    stage_ms = (C.c_double * abi.NSTAGES)()
    stage_n = (C.c_longlong * abi.NSTAGES)()
    abi.lib.pta_profile_read(eng._h, stage_ms, stage_n, 1)
    abi.lib.pta_profile_enable(eng._h, 0)
    stage_ms = [v / args.steps for v in stage_ms]
    kernel_ms = dict(zip(abi.KERNEL_TIMERS, stage_ms[len(abi.STAGES):]))  # single kernels inside the stages
    stage_ms = stage_ms[:len(abi.STAGES)]
    launches = int(sum(stage_n))
    ms, value = reduce_timing(ms, B, world, pg, dev)
    if rank != 0:
        pg.destroy_process_group()
        return
    # roofline of the dominant stage's kernel
    dom = int(np.argmax(stage_ms))  # main stages only
    peaks = measured_peaks()
    bf16_peak = (peaks or {}).get("bf16_tflops", 1800.0)
    toa_roof = None
    if args.precision == "f16split":
        flops = toa_flops_f16(arr, B)
        issued = toa_issued_f16(arr, B)
        ms_toa = stage_ms[abi.STAGES.index("toa")]
        kms = {k: kernel_ms[k] for k in ("toa_res", "toa_ftw")}
        toa_roof = {"kernel": "k_f16_pack + k_f16_res + k_f16_ftw (TOA contractions, tcgen05 kind::f16, exact split)",
                    "bound": "tensor", "unit": "TFLOP/s", "achieved": flops / (ms_toa * 1e-3) / 1e12,
                    "peak": bf16_peak, "peak_source": "measured bf16 burst (fp16 has the same dense rate)",
                    "stage_ms": ms_toa, "kernel_ms": kms, "algorithmic_flop": flops, "issued_flop": issued,
                    "issued_tflops": issued / (ms_toa * 1e-3) / 1e12,
                    "issued_frac": issued / (ms_toa * 1e-3) / 1e12 / bf16_peak,
                    "note": "the exact split issues about 10 products per algorithmic one in F~ a and 6 in "
                            "F~^T w: frac is algorithmic flops over the dense peak, issued_frac the tensor "
                            "pipe's share of it"}
        toa_roof["frac"] = toa_roof["achieved"] / toa_roof["peak"]
    chol_dominant = args.transform != "curn" and kernel_ms["chol_forward"] > 0 and (
        abi.STAGES[dom] == "prior_forward" or
        (args.precision == "f16split" and kernel_ms["chol_forward"] >= max(kernel_ms["toa_res"], kernel_ms["toa_ftw"])))
    if chol_dominant:  # the longest single kernel (the exact-split TOA stage runs three)
        roof = chol_roofline(arr, B, kernel_ms["chol_forward"], args.precision == "fp64")
    elif abi.STAGES[dom] == "toa" and toa_roof is not None:
        roof = dict(toa_roof)
    elif abi.STAGES[dom] == "toa" and args.precision in ("tf32x3", "tf32"):
        flops = toa_flops_per_launch(arr, B)
        terms = 3 if args.precision == "tf32x3" else 1
        tf32_peak = bf16_peak * (1.1 / 2.25)
        roof = {"kernel": f"k_toa_tc<{terms}> (TOA contractions, tcgen05 kind::tf32)", "bound": "tensor",
                "unit": "TFLOP/s", "achieved": flops / (stage_ms[dom] * 1e-3) / 1e12, "peak": tf32_peak,
                "peak_source": "measured bf16 burst x nominal TF32/BF16 ratio 1.1/2.25",
                "pipe_terms": terms}
    elif abi.STAGES[dom] == "toa" and args.precision == "gram":
        P = 2 * max(arr.n_gwb, arr.n_rn) + 2 * arr.n_dm
        flops = 2.0 * P * P * arr.npsr * B
        roof = {"kernel": "k_gram (Gram form, compensated FP32 P x P products)", "bound": "alu",
                "unit": "TFLOP/s", "achieved": flops / (stage_ms[dom] * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 flop x 2.032 GHz",
                "note": "algorithmic 2 P^2 flop per (pulsar, chain); the error-free products and sums issue "
                        "about 11 FP32 operations per multiply-add"}
    elif abi.STAGES[dom] == "toa" and args.precision == "bf16x3":
        flops = toa_flops_per_launch(arr, B)
        roof = {"kernel": "k_toa_bf16 (TOA contractions, tcgen05 kind::f16, 3-term BF16 split)",
                "bound": "tensor", "unit": "TFLOP/s", "achieved": flops / (stage_ms[dom] * 1e-3) / 1e12,
                "peak": bf16_peak, "peak_source": "measured bf16 burst (cuBLAS)", "pipe_terms": 3}
    elif abi.STAGES[dom] == "toa":
        flops = toa_flops_per_launch(arr, B)
        shape = f"<{tuned['chains_per_cta']},{tuned['toas_per_tile']},{tuned['rows_per_thread']},{tuned['order']}>" \
            if tuned else ""
        roof = {"kernel": f"k_toa_simt{shape} (TOA contractions)", "bound": "alu", "unit": "TFLOP/s",
                "achieved": flops / (stage_ms[dom] * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 flop x 2.032 GHz"}
    elif args.transform == "curn":
        flops = curn_flops_per_launch(arr, B) + chol_flops_per_launch(arr, B)
        P = 2 * max(arr.n_gwb, arr.n_rn) + 2 * arr.n_dm
        mode = 0 if args.precision == "fp64" else curn_factor_mode(P)
        if mode:
            kern = "k_curn_forward_dw" if mode == 1 else f"k_curn_forward_dwc<{mode}>"
            roof = {"kernel": f"prior stage with {kern} (double-word LDL^T sweep with inverse)", "bound": "alu",
                    "unit": "TFLOP/s", "achieved": flops / (stage_ms[dom] * 1e-3) / 1e12, "peak": DW_PEAK_TFLOPS,
                    "peak_source": f"derived: 148 SM x 128 FP32 lanes x 2.032 GHz x 2 flop / "
                                   f"{DW_OPS_PER_FMA} FP32 operations per double-word multiply-add"}
        else:
            roof = {"kernel": "prior stage with k_curn_forward (FP64 LDL^T sweep with inverse)", "bound": "alu",
                    "unit": "TFLOP/s", "achieved": flops / (stage_ms[dom] * 1e-3) / 1e12,
                    "peak": FP64_PEAK_TFLOPS, "peak_source": "derived: 148 SM x 2 FP64 FMA/clk x 2 flop x 2.032 GHz"}
    else:
        roof = chol_roofline(arr, B, kernel_ms["chol_forward"], args.precision == "fp64")
    roof["frac"] = roof["achieved"] / roof["peak"]
    tr = captured_traffic(roof["kernel"].split(" ")[0])
    roof["traffic"] = tr["bytes_per_launch"] if tr else None  # DRAM bytes per launch (ncu), None if stale
    roof["traffic_source"] = tr["profile"] if tr else None
    if toa_roof is not None:
        toa_roof["traffic"] = {k: (captured_traffic(k) or {}).get("bytes_per_launch") for k in ("k_f16_res", "k_f16_ftw")}
    roof["stage_ms"] = dict(zip(abi.STAGES, [round(v, 4) for v in stage_ms]))
    # end to end through the public call with host buffers (pinned), copies inside the timed
    # region: every step copies its input x host->device and its logp and gradient
    # device->host.  Steps are pipelined the way a sampler loop runs them: copies in,
    # compute (L2 flush, then the evaluation) and copies out on three streams, two buffer
    # sets, ordered by events; the timed region runs from the first copy in to the last
    # copy out.
    xh = torch.tensor(X).pin_memory()
    lh = [torch.empty(B, dtype=torch.float64).pin_memory() for _ in range(2)]
    gh = [torch.empty((B, D), dtype=torch.float32).pin_memory() for _ in range(2)]
    xd = [torch.empty_like(x) for _ in range(2)]
    od = [(torch.empty(B, dtype=torch.float64, device=dev), torch.empty_like(x),
           torch.empty(B, dtype=torch.int32, device=dev)) for _ in range(2)]
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_cmp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    n_e2e = max(4, args.steps)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for i in range(n_e2e):
        k = i % 2
        with torch.cuda.stream(s_in):
            if i >= 2:
                s_in.wait_event(ev_cmp[k])      # step i-2 finished reading xd[k]
            xd[k].copy_(xh, non_blocking=True)
            ev_in[k].record(s_in)
        with torch.cuda.stream(s_cmp):
            s_cmp.wait_event(ev_in[k])
            if i >= 2:
                s_cmp.wait_event(ev_out[k])     # step i-2's results copied out of od[k]
            flush.zero_()
            eng.logp_and_grad(xd[k], out=od[k])
            ev_cmp[k].record(s_cmp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_cmp[k])
            lh[k].copy_(od[k][0], non_blocking=True)
            gh[k].copy_(od[k][1], non_blocking=True)
            ev_out[k].record(s_out)
    e1.record(s_out)
    e1.synchronize()
    e2e_ms = e0.elapsed_time(e1) / n_e2e
    # the plain FP64 GPU path on the same workload (the metric's comparison)
    fp64 = None
    if not args.skip_fp64:
        eng.set_precision("fp64")
        eng.logp_and_grad(x, out=out)
        torch.cuda.synchronize()
        n64 = 2
        e0.record()
        for _ in range(n64):
            eng.logp_and_grad(x, out=out)
        e1.record()
        e1.synchronize()
        ms64 = e0.elapsed_time(e1) / n64
        x1 = x[:1].contiguous()
        eng.logp_and_grad(x1)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            eng.logp_and_grad(x1)
        e1.record()
        e1.synchronize()
        ms64_1 = e0.elapsed_time(e1) / 5
        fp64 = {"value": B / (ms64 * 1e-3), "unit": "evals/s", "ms_per_step": ms64, "chains": B,
                "single_chain_ms": ms64_1, "speedup_of_value": (B / (ms * 1e-3)) / (B / (ms64 * 1e-3))}
        eng.set_precision(args.precision)
    # the other evaluation modes on the same workload and batch (same protocol: L2
    # flushed, CUDA events per step); the headline stays the FP32 TOA form
    variants = {}
    if not args.skip_variants:
        accuracy = {"gram": "FP64-level (parity at FP64 tolerances)",
                    "fp32": "FP32 bar at the 67-pulsar size (max 5.0e-4 nats over 16 near-posterior points); "
                            "1.6e-3 nats at one of 8 near-posterior points at the 150-pulsar size",
                    "f16split": "max 1.8e-4 nats over 16 near-posterior points, gradient 1.1e-5",
                    "bf16x3": "reported: 8e-3 nats at a near-posterior point",
                    "tf32x3": "reported: 2.5e-3 nats at a near-posterior point"}
        accuracy["f16split_chol_fp64"] = accuracy["f16split"]
        for key in ("fp32", "f16split", "f16split_chol_fp64", "gram", "bf16x3", "tf32x3"):
            prec = key.split("_")[0]
            if key == args.precision:
                continue
            try:
                eng.set_precision(prec)
                eng.set_cholesky("fp64" if key.endswith("chol_fp64") else "dw")
                vt = None
                if prec == "fp32":  # the autotuner picks the SIMT tile shape (setup, not timed)
                    from paper_2607_06834_b300.engine import toa_config_info
                    chosen, _ = eng.autotune(B)
                    vt = {"entry": chosen, **toa_config_info(chosen)}
                for _ in range(3):
                    eng.logp_and_grad(x, out=out)
                torch.cuda.synchronize()
                vs, ve = [], []
                for i in range(max(5, args.steps // 2)):
                    flush.zero_()
                    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a0.record()
                    eng.logp_and_grad(x, out=out)
                    a1.record()
                    vs.append(a0)
                    ve.append(a1)
                torch.cuda.synchronize()
                vms = float(np.mean([a.elapsed_time(b) for a, b in zip(vs, ve)]))
                variants[key] = {"value": B / (vms * 1e-3), "unit": "evals/s", "ms_per_step": vms,
                                 "detail": DTYPE_DETAIL[prec] + ("; FP64 dense-bin Cholesky (pta_set_cholesky)"
                                                                 if key.endswith("chol_fp64") else ""),
                                 "accuracy": accuracy[key]}
                if vt:
                    variants[key]["toa_kernel_autotuned"] = vt
            except Exception as exc:  # a mode this model cannot run
                variants[key] = {"unavailable": str(exc)}
        eng.set_cholesky("dw")
        eng.set_precision(args.precision)
        if tuned and tuned.get("entry") is not None:
            eng.set_toa_config(tuned["entry"])
        variants["curn_transform"] = curn_variant(dev, args.steps)
    scale = None if (args.skip_scale150 or args.workload != WORKLOAD) else scale150_leg(dev, args.steps, peaks)
    cpu = None if args.skip_cpu else cpu_baseline(args.workload, args.cpu_steps)
    hmc = None if args.skip_hmc else hmc_ess(args, dev)
    if hmc is not None:
        hmc["control_small_array"] = hmc_ess_tiny(dev)
        hmc["transforms_paper_model"] = hmc_ess_transforms(args, dev)
    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision],
            "dtype_detail": DTYPE_DETAIL[args.precision] + (
                "; FP64 Cholesky, log-det, timing-model solve and sums" if args.precision == "fp64" else
                "; dense-bin Cholesky sweep and its adjoint in double-word (float pair, ~48-bit) arithmetic on the "
                "FP32 pipes; FP64 pivots' square roots, log-det, timing-model solve and sums"),
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC if (args.workload, args.chains) == (WORKLOAD, 0)
                       else f"{args.workload}, {B} chains", "transform": args.transform,
                       "chains_per_gpu": B, "ntoa": arr.ntoa, "npsr": arr.npsr,
                       "precision": args.precision, "l2": "flushed between timed steps (512 MB write)",
                       "toa_kernel_autotuned": tuned,
                       # the metric is quoted against the plain FP64 GPU path on the same batch
                       "vs_fp64_plain_path": None if fp64 is None else
                       {"fp64_evals_per_s": fp64["value"], "ratio": value / fp64["value"]}},
            "roofline": roof, "roofline_toa": toa_roof, "cpu_baseline": cpu,
            "e2e": {"value": world * B / (e2e_ms * 1e-3), "unit": "evals/s",
                    "h2d_bytes_per_step": int(B * D * 4), "d2h_bytes_per_step": int(B * 8 + B * D * 4)},
            "gpu_launches": launches, "fp64_plain_path": fp64, "variants": variants or None, "hmc": hmc,
            "scale150": scale,
            "clocks": ck,
            "wall_s_timed": t_wall, "measured_peaks": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")} if peaks else None}
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="f16split")
    ap.add_argument("--cpu-steps", type=int, default=2, help="oracle steps (one chain per host core each)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-hmc", action="store_true")
    ap.add_argument("--skip-variants", action="store_true")
    ap.add_argument("--skip-scale150", action="store_true")
    ap.add_argument("--toa-config", type=int, default=-1, help="fixed FP32 TOA kernel entry (default: autotune)")
    # profiling runs of a single kernel on another shape (the headline keeps the defaults)
    ap.add_argument("--workload", default=WORKLOAD, help="synthetic workload (synth.WORKLOADS key)")
    ap.add_argument("--chains", type=int, default=0, help="chains (default: the workload's)")
    ap.add_argument("--transform", default="prior", choices=["prior", "curn"])
    ap.add_argument("--hmc-warmup", type=int, default=400)
    ap.add_argument("--hmc-samples", type=int, default=200)
    ap.add_argument("--hmc-samples-curn", type=int, default=2000,
                    help="sampling trajectories of the CURN leg on the paper's model")
    ap.add_argument("--hmc-warmup-curn", type=int, default=1000,
                    help="warm-up trajectories of the CURN leg on the paper's model")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
