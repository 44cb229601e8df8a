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
         "gram": "f32 (compensated)"}
DTYPE_DETAIL = {"fp32": "FP32 TOA contractions (SIMT)", "fp64": "FP64 TOA contractions (stored basis)",
                "tf32x3": "3-term split TF32 tensor-core TOA contractions, FP32 accumulation",
                "tf32": "single TF32 tensor-core TOA contractions, FP32 accumulation",
                "bf16x3": "3-term split BF16 tensor-core TOA contractions, FP32 accumulation",
                "gram": "Gram form: per-pulsar F^T N~^-1 F products in compensated FP32 (hi/lo, Dot2)"}
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # SMs x FP32 lanes x 2 flop x max SM clock
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12     # SMs x 2 FP64 FMA/clk x 2 flop x max SM clock


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel from one ncu capture, valid only while the kernel's sources are the ones
# profiled (sha256 of each file); see profiles/.
CAPTURED_TRAFFIC = {
    ("fp32", 90): {"bytes": 99.4e6, "profile": "profiles/k_toa_simt_ng15_b256.md",
                   "sources": {"k_toa.cu": "c8d87cf044a8314097a12141a102f2f6f1655504562fa633692ac1885ff3e7ed",
                               "pta_internal.cuh": "6980f278b2d07f527a51f8b84b6aecf336252fc4f05fe8ed5ba6b76aa628bb97"}},
}


def captured_traffic(precision, entry):
    import hashlib
    rec = CAPTURED_TRAFFIC.get((precision, entry))
    if rec is None:
        return None
    csrc = os.path.join(ROOT, "paper_2607_06834_b300", "csrc")
    for f, h in rec["sources"].items():
        try:
            if hashlib.sha256(open(os.path.join(csrc, f), "rb").read()).hexdigest() != h:
                return None
        except OSError:
            return None
    return rec["bytes"]


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


def curn_variant(dev, steps):
    """The CURN-posterior transform (Eq. PTA_standard_transform_curn) against the default
    prior-whitened one on the same batch: the paper's NANOGrav-15-yr model (RN 30 /
    HD-GWB 14 bins, no DM: P = 60, the factor in shared memory) with 64 and 256 chains,
    and the 100-DM-bin workload (P = 260, the factor in the global inverse buffer) with
    256 chains.  CUDA events per step with L2 flushed; the FP64 factorisation stage is
    the CURN forward stage minus the prior-whitened one."""
    import ctypes as C
    import torch
    from paper_2607_06834_b300 import abi, synth
    from paper_2607_06834_b300.engine import Engine
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peak = FP64_PEAK_TFLOPS
    out = []
    for name, B in (("ng15_nodm", 64), ("ng15_nodm", 256), ("ng15_b256", 256)):
        arr = synth.make_array(name)
        eng = Engine(arr, precision="fp32")
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
        rec["roofline"] = {"kernel": "k_curn_forward + k_curn_whiten (FP64 LDL^T sweep with inverse)",
                           "bound": "alu", "unit": "TFLOP/s", "achieved": ach, "peak": peak,
                           "peak_source": "derived: 148 SM x 2 FP64 FMA/clk x 2 flop x 2.032 GHz",
                           "frac": ach / peak, "stage_ms": fac_ms,
                           "factor_in": "shared memory" if (rec["P"] * (rec["P"] + 1) // 2 + 8 * rec["P"]) * 8
                           <= 200 * 1024 else "global inverse buffer"}
        eng.close()
        out.append(rec)
    return out


def cpu_baseline(arr, n_eval: int):
    """The FP64 oracle, as it stands, on the host cores: logp + grad of n_eval chains."""
    from oracle import pta_oracle as O
    from paper_2607_06834_b300 import synth
    try:
        from threadpoolctl import threadpool_info
        cores = max([t.get("num_threads", 1) for t in threadpool_info()] or [1])
    except Exception:
        cores = os.cpu_count()
    orc = O.Oracle(arr)
    X = synth.make_points(arr, n_eval, seed=6834 + 2).astype(np.float64)
    orc.logp(X[0])
    t0 = time.perf_counter()
    for x in X:
        orc.logp(x)
        orc.grad(x)
    dt = time.perf_counter() - t0
    return {"value": n_eval / dt, "unit": "evals/s", "cores": int(cores), "kind": "oracle",
            "sample": f"{n_eval} single-chain logp+grad evaluations of the {WORKLOAD} workload "
                      f"({dt:.1f} s, numpy FP64)"}


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
            "ess_per_s_gwb_min": float(np.nanmin(e[g0:g0 + 2])) / t, "ess_per_s_median": float(np.nanmedian(e)) / t,
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
    eng = Engine(arr, precision="fp32")
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
                        f"{B} chains, {L} leapfrog steps per trajectory, FP32 path",
            "warmup_trajectories": args.hmc_warmup, "sampling_trajectories": args.hmc_samples,
            "ess_per_s_gwb_min": e_gwb / t, "ess_per_s_theta_median": e_med / t,
            "ess_per_s_cw_median": e_cw / t,
            "ess_gwb_min": e_gwb, "ess_theta_median": e_med, "ess_cw_median": e_cw,
            "ess_z_median": e_z, "ess_per_s_z_median": e_z / t,
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
                       f"array, {B} chains, {L} leapfrog steps per trajectory, FP32 path",
           "warmup_trajectories": args.hmc_warmup, "sampling_trajectories": args.hmc_samples}
    for tr in ("curn", "prior"):
        eng = Engine(arr, precision="fp32")
        eng.set_transform(tr)
        lay = eng.layout
        th0 = lay["d_z"]
        x0 = torch.tensor(synth.make_points(arr, B, seed=6834 + 3), device=dev)
        kw = dict(unit_mass=th0, init_dz=0) if tr == "curn" else dict(init_dz=th0)
        res = sampler.run_hmc(eng, x0, n_warmup=args.hmc_warmup, n_samples=args.hmc_samples, n_leapfrog=L,
                              record=slice(th0, eng.D), seed=6834 + 3, eps0=0.01,
                              consensus=args.hmc_warmup // 4, **kw)
        e = sampler.ess_columns(res.draws)
        rh = np.array([sampler.split_rhat(res.draws[:, :, k]) for k in range(res.draws.shape[2])])
        g0 = lay["th_gwb"] - th0
        t = res.sampling_s
        out[tr] = {"ess_per_s_gwb_min": float(np.nanmin(e[g0:g0 + 2])) / t,
                   "ess_per_s_theta_median": float(np.nanmedian(e)) / t,
                   "ess_gwb_min": float(np.nanmin(e[g0:g0 + 2])), "ess_theta_median": float(np.nanmedian(e)),
                   "rhat_gwb_max": float(np.nanmax(rh[g0:g0 + 2])), "rhat_theta_median": float(np.nanmedian(rh)),
                   "rhat_theta_max": float(np.nanmax(rh)), "sampling_s": t, "warmup_s": res.warmup_s,
                   "ms_per_trajectory": 1e3 * t / max(args.hmc_samples, 1),
                   "evals_per_s": B * L * args.hmc_samples / t, "accept_rate": res.accept_rate, "step": res.step,
                   "gwb_posterior_mean": [float(v) for v in res.draws[:, :, g0:g0 + 2].reshape(-1, 2).mean(0)],
                   "gwb_posterior_std": [float(v) for v in res.draws[:, :, g0:g0 + 2].reshape(-1, 2).std(0)],
                   "stuck_chains": res.stats["stuck_chains"]}
        eng.close()
    # the same model with a circular binary, CURN transform with the signal-dependent mean
    # (Eq. decenter_det_PTA)
    arr = synth.make_array("ng15_nodm_cw")
    eng = Engine(arr, precision="fp32")
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
                           "ess_per_s_gwb_min": float(np.nanmin(e[g0:g0 + 2])) / t,
                           "ess_per_s_theta_median": float(np.nanmedian(e)) / t,
                           "ess_per_s_cw_median": float(np.nanmedian(e[c0:c0 + 8])) / t,
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
    from paper_2607_06834_b300 import synth
    from oracle import pta_oracle as O
    arr = synth.make_array(WORKLOAD)
    orc = O.Oracle(arr)
    X = synth.make_points(arr, args.steps + args.warmup, seed=6834 + 2).astype(np.float64)
    for i in range(args.warmup):
        orc.logp(X[i])
        orc.grad(X[i])
    t0 = time.perf_counter()
    for i in range(args.warmup, args.warmup + args.steps):
        orc.logp(X[i])
        orc.grad(X[i])
    dt = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([t.get("num_threads", 1) for t in threadpool_info()] or [1])
    except Exception:
        cores = os.cpu_count()
    value = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_DESC, "chains_per_step": 1},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": int(cores), "kind": "oracle",
                             "sample": "one single-chain logp+grad evaluation per step"},
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
    launches = int(sum(stage_n))
    ms, value = reduce_timing(ms, B, world, pg, dev)
    if rank != 0:
        pg.destroy_process_group()
        return
    # roofline of the dominant stage's kernel
    dom = int(np.argmax(stage_ms))
    peaks = measured_peaks()
    if abi.STAGES[dom] == "toa" and args.precision in ("tf32x3", "tf32"):
        flops = toa_flops_per_launch(arr, B)
        terms = 3 if args.precision == "tf32x3" else 1
        tf32_peak = (peaks or {}).get("bf16_tflops", 1800.0) * (1.1 / 2.25)
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
                "peak": (peaks or {}).get("bf16_tflops", 1800.0),
                "peak_source": "measured bf16 burst (cuBLAS)", "pipe_terms": 3}
    elif abi.STAGES[dom] == "toa":
        flops = toa_flops_per_launch(arr, B)
        shape = f"<{tuned['chains_per_cta']},{tuned['toas_per_tile']},{tuned['rows_per_thread']},{tuned['order']}>" \
            if tuned else ""
        roof = {"kernel": f"k_toa_simt{shape} (TOA contractions)", "bound": "alu", "unit": "TFLOP/s",
                "achieved": flops / (stage_ms[dom] * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 flop x 2.032 GHz"}
    elif args.transform == "curn":
        flops = curn_flops_per_launch(arr, B) + chol_flops_per_launch(arr, B)
        roof = {"kernel": "prior stage with k_curn_forward (FP64 LDL^T sweep with inverse)", "bound": "alu",
                "unit": "TFLOP/s", "achieved": flops / (stage_ms[dom] * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "peak_source": "derived: 148 SM x 2 FP64 FMA/clk x 2 flop x 2.032 GHz"}
    else:
        flops = chol_flops_per_launch(arr, B)
        roof = {"kernel": "k_chol_forward (FP64 Cholesky + inverse + transform)", "bound": "alu",
                "unit": "TFLOP/s", "achieved": flops / (stage_ms[dom] * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "peak_source": "derived: 148 SM x 2 FP64 FMA/clk x 2 flop x 2.032 GHz"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = captured_traffic(args.precision, tuned["entry"]) \
        if (tuned and abi.STAGES[dom] == "toa") else None
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
        for prec in ("gram", "bf16x3", "tf32x3"):
            if prec == args.precision:
                continue
            try:
                eng.set_precision(prec)
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
                variants[prec] = {"value": B / (vms * 1e-3), "unit": "evals/s", "ms_per_step": vms,
                                  "detail": DTYPE_DETAIL[prec],
                                  "accuracy": {"gram": "FP64-level (parity at FP64 tolerances)",
                                               "bf16x3": "reported: 8e-3 nats at a near-posterior point",
                                               "tf32x3": "reported: 2.5e-3 nats at a near-posterior point"}[prec]}
            except Exception as exc:  # a mode this model cannot run
                variants[prec] = {"unavailable": str(exc)}
        eng.set_precision(args.precision)
        if tuned and tuned.get("entry") is not None:
            eng.set_toa_config(tuned["entry"])
        variants["curn_transform"] = curn_variant(dev, args.steps)
    cpu = None if args.skip_cpu else cpu_baseline(arr, args.cpu_evals)
    hmc = None if args.skip_hmc else hmc_ess(args, dev)
    if hmc is not None:
        hmc["control_small_array"] = hmc_ess_tiny(dev)
        hmc["transforms_paper_model"] = hmc_ess_transforms(args, dev)
    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision],
            "dtype_detail": DTYPE_DETAIL[args.precision] + "; FP64 Cholesky, log-det, timing-model solve and sums",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC if (args.workload, args.chains) == (WORKLOAD, 0)
                       else f"{args.workload}, {B} chains", "transform": args.transform,
                       "chains_per_gpu": B, "ntoa": arr.ntoa, "npsr": arr.npsr,
                       "precision": args.precision, "l2": "flushed between timed steps (512 MB write)",
                       "toa_kernel_autotuned": tuned},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": world * B / (e2e_ms * 1e-3), "unit": "evals/s",
                    "h2d_bytes_per_step": int(B * D * 4), "d2h_bytes_per_step": int(B * 8 + B * D * 4)},
            "gpu_launches": launches, "fp64_plain_path": fp64, "variants": variants or None, "hmc": hmc,
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
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--cpu-evals", type=int, default=16)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-hmc", action="store_true")
    ap.add_argument("--skip-variants", action="store_true")
    ap.add_argument("--toa-config", type=int, default=-1, help="fixed FP32 TOA kernel entry (default: autotune)")
    # profiling runs of a single kernel on another shape (the headline keeps the defaults)
    ap.add_argument("--workload", default=WORKLOAD, help="synthetic workload (synth.WORKLOADS key)")
    ap.add_argument("--chains", type=int, default=0, help="chains (default: the workload's)")
    ap.add_argument("--transform", default="prior", choices=["prior", "curn"])
    ap.add_argument("--hmc-warmup", type=int, default=400)
    ap.add_argument("--hmc-samples", type=int, default=200)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
