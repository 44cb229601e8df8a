"""Seeded synthetic pulsar-timing-array inputs.

This module only draws numbers: TOA epochs, radio frequencies, uncertainties,
backends, timing-model design matrices, sky positions and synthetic residuals.
It holds none of the posterior's arithmetic (no Fourier basis, no Hellings-Downs
matrix, no power-law spectrum, no noise covariance, no marginalisation), so
both the CPU oracle and the CUDA path can be fed from it without sharing code.

Residuals are built from a sum of off-grid sinusoids with power-law-like
amplitudes (a common process, per-pulsar red noise, radio-frequency-dependent
dispersion-like noise), a small timing-model offset and white noise drawn as
two independent terms (scaled uncertainty plus a quadrature term).  They have
the magnitudes of real post-fit residuals (tens of ns to a few us) but are not
drawn from the model the posterior assumes.

Workload shapes follow the paper's analyses (Sec. "Analyses of real and
simulated datasets"): a NANOGrav-15-yr-like array of 67 pulsars with ~3e5 TOAs,
30 red-noise bins, 14 GWB bins, and a 150-pulsar 1e6-TOA scale-up.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DAY = 86400.0
YEAR = 365.25 * DAY
MJD0_S = 53000.0 * DAY  # absolute time origin of the synthetic TOAs (s)

# Parameter-space sizes of the synthetic workloads.  Keys:
#   npsr, ntoa_total, ntoa_range, span_yr (lo, hi), m_range, n_gwb, n_rn, n_dm,
#   cw, chains, mode ('uniform' epochs for the tiny case, 'epochs' otherwise)
WORKLOADS = {
    "tiny3": dict(npsr=3, ntoa_total=600, ntoa_range=(200, 200), span_yr=(10.0, 10.0),
                  m_range=(3, 3), n_gwb=10, n_rn=10, n_dm=0, cw=False, chains=1,
                  mode="uniform", nbackend=(1, 1)),
    "ng15": dict(npsr=67, ntoa_total=300_000, ntoa_range=(2000, 20000), span_yr=(3.0, 16.0),
                 m_range=(8, 80), n_gwb=14, n_rn=30, n_dm=100, cw=False, chains=1,
                 mode="epochs", nbackend=(1, 4)),
    "ng15_b256": dict(npsr=67, ntoa_total=300_000, ntoa_range=(2000, 20000), span_yr=(3.0, 16.0),
                      m_range=(8, 80), n_gwb=14, n_rn=30, n_dm=100, cw=False, chains=256,
                      mode="epochs", nbackend=(1, 4)),
    "ng15_cw": dict(npsr=67, ntoa_total=300_000, ntoa_range=(2000, 20000), span_yr=(3.0, 16.0),
                    m_range=(8, 80), n_gwb=14, n_rn=30, n_dm=100, cw=True, chains=64,
                    mode="epochs", nbackend=(1, 4)),
    # the model of the paper's NANOGrav-15-yr analysis (Sec. "Analyses of real and simulated
    # datasets"): intrinsic red noise with 30 bins and an HD-correlated GWB with 14, no DM
    # (P = 60 coefficients per pulsar), on the same 67-pulsar array
    "ng15_nodm": dict(npsr=67, ntoa_total=300_000, ntoa_range=(2000, 20000), span_yr=(3.0, 16.0),
                      m_range=(8, 80), n_gwb=14, n_rn=30, n_dm=0, cw=False, chains=64,
                      mode="epochs", nbackend=(1, 4)),
    # the same model with a circular binary (the paper's joint GWB + RN + CW analysis shape)
    "ng15_nodm_cw": dict(npsr=67, ntoa_total=300_000, ntoa_range=(2000, 20000), span_yr=(3.0, 16.0),
                         m_range=(8, 80), n_gwb=14, n_rn=30, n_dm=0, cw=True, chains=64,
                         mode="epochs", nbackend=(1, 4)),
    "scale150": dict(npsr=150, ntoa_total=1_000_000, ntoa_range=(1000, 30000), span_yr=(5.0, 30.0),
                     m_range=(8, 80), n_gwb=100, n_rn=30, n_dm=150, cw=False, chains=1024,
                     mode="epochs", nbackend=(1, 4)),
}
# The five workloads in order of the build's configuration list.
WORKLOAD_ORDER = ["tiny3", "ng15", "ng15_b256", "ng15_cw", "scale150"]


@dataclass
class Pulsar:
    toas_s: np.ndarray        # (n,) f64, absolute seconds
    freqs_mhz: np.ndarray     # (n,) f64
    resid_s: np.ndarray       # (n,) f64
    sigma_s: np.ndarray       # (n,) f64
    backend: np.ndarray       # (n,) int32 in [0, n_backend)
    efac: np.ndarray          # (n_backend,) f64
    equad_s: np.ndarray       # (n_backend,) f64
    M: np.ndarray             # (n, m) f64 row-major
    pos: np.ndarray           # (3,) unit vector
    dist_kpc: float

    @property
    def n(self) -> int:
        return int(self.toas_s.shape[0])

    @property
    def m(self) -> int:
        return int(self.M.shape[1])


@dataclass
class Array:
    pulsars: list
    n_gwb: int
    n_rn: int
    n_dm: int
    cw: bool
    name: str = ""
    meta: dict = field(default_factory=dict)
    gwb_free: bool = False    # free spectral model for the GWB: one log10 rho per bin
    rn_free: bool = False     # free spectral model for every pulsar's red noise

    @property
    def npsr(self) -> int:
        return len(self.pulsars)

    @property
    def ntoa(self) -> int:
        return sum(p.n for p in self.pulsars)


def _toa_counts(rng, npsr, total, lo, hi):
    if lo == hi:
        return [lo] * npsr
    raw = np.exp(rng.uniform(math.log(lo), math.log(hi), npsr))
    raw *= total / raw.sum()
    counts = np.clip(np.round(raw), lo, hi).astype(int)
    # nudge so the total matches as closely as the bounds allow
    for _ in range(10 * npsr):
        d = total - counts.sum()
        if d == 0:
            break
        i = rng.integers(npsr)
        step = int(np.sign(d)) * min(abs(d), 50)
        counts[i] = int(np.clip(counts[i] + step, lo, hi))
    return counts.tolist()


def _sky(rng):
    ct = rng.uniform(-1.0, 1.0)
    ph = rng.uniform(0.0, 2.0 * math.pi)
    st = math.sqrt(max(0.0, 1.0 - ct * ct))
    return np.array([st * math.cos(ph), st * math.sin(ph), ct])


def _times(rng, n, t_end, span_s, mode):
    t_start = t_end - span_s
    if mode == "uniform":
        return np.sort(rng.uniform(t_start, t_end, n))
    cadence = rng.uniform(14.0, 30.0) * DAY
    n_ep = max(4, int(span_s / cadence))
    epochs = np.sort(t_start + (np.arange(n_ep) + rng.uniform(0.0, 1.0, n_ep) * 0.5) * (span_s / n_ep))
    which = np.sort(rng.integers(0, n_ep, n))
    return np.sort(epochs[which] + rng.uniform(0.0, 3600.0, n)), which


def _design_matrix(rng, t, nu, backend, nb, m_target, span_s):
    tc = 0.5 * (t.min() + t.max())
    tau = (t - tc) / (0.5 * max(span_s, DAY))
    cols = [np.ones_like(t), tau, tau * tau]
    if m_target > 3:
        ya = 2.0 * math.pi * t / YEAR
        cols += [np.sin(ya), np.cos(ya), tau * np.sin(ya), tau * np.cos(ya),
                 np.sin(2 * ya), np.cos(2 * ya)]
        for b in range(1, nb):
            cols.append((backend == b).astype(float))
        wnu = (1400.0 / nu) ** 2
        edges = np.arange(t.min(), t.max() + 182.625 * DAY, 182.625 * DAY)
        for lo in edges:
            if len(cols) >= m_target:
                break
            sel = (t >= lo) & (t < lo + 182.625 * DAY)
            if sel.sum() >= 4:
                cols.append(np.where(sel, wnu, 0.0))
    cols = cols[:m_target]
    return np.stack(cols, axis=1)


def _red_process(rng, t, span_s, rms_ns, gamma, ncomp=32):
    f = np.exp(rng.uniform(math.log(0.4 / span_s), math.log(40.0 / span_s), ncomp))
    amp = f ** (-0.5 * gamma)
    ph = rng.uniform(0.0, 2.0 * math.pi, ncomp)
    sig = (amp[None, :] * np.sin(2.0 * math.pi * f[None, :] * t[:, None] + ph[None, :])).sum(1)
    s = sig.std()
    return sig * (rms_ns / s if s > 0 else 0.0)


def make_array(name: str, seed: int | None = None) -> Array:
    """Draw the synthetic array named ``name`` (a key of WORKLOADS)."""
    w = WORKLOADS[name]
    if seed is None:
        # the 67-pulsar workloads share one array (same seed; the draws do not depend on n_dm)
        seed = {"tiny3": 2607, "ng15": 2608, "ng15_b256": 2608, "ng15_cw": 2608, "ng15_nodm": 2608,
                "ng15_nodm_cw": 2608, "scale150": 2611}[name]
    rng = np.random.default_rng(seed)
    npsr = w["npsr"]
    counts = _toa_counts(rng, npsr, w["ntoa_total"], *w["ntoa_range"])
    span_hi = w["span_yr"][1] * YEAR
    t_end = MJD0_S + span_hi
    # a common red process shared by all pulsars (defined on absolute time)
    common_f = np.exp(rng.uniform(math.log(0.4 / span_hi), math.log(30.0 / span_hi), 24))
    common_a = common_f ** (-13.0 / 6.0)
    common_p = rng.uniform(0.0, 2.0 * math.pi, 24)
    cw_f = 10.0 ** rng.uniform(-8.5, -7.5)
    pulsars = []
    for I in range(npsr):
        n = counts[I]
        span = span_hi if I == 0 else rng.uniform(*w["span_yr"]) * YEAR
        tt = _times(rng, n, t_end, span, w["mode"])
        t = tt[0] if isinstance(tt, tuple) else tt
        nb = int(rng.integers(w["nbackend"][0], w["nbackend"][1] + 1))
        if isinstance(tt, tuple):
            ep_backend = rng.integers(0, nb, tt[1].max() + 1)
            backend = ep_backend[tt[1]].astype(np.int32)
        else:
            backend = rng.integers(0, nb, n).astype(np.int32)
        nu = rng.uniform(400.0, 3000.0, n)
        sigma_ns = np.exp(rng.uniform(math.log(100.0), math.log(1000.0), n))
        efac = rng.uniform(0.8, 1.5, nb)
        equad_ns = np.exp(rng.uniform(math.log(10.0), math.log(300.0), nb))
        m_target = int(rng.integers(w["m_range"][0], w["m_range"][1] + 1))
        M = _design_matrix(rng, t, nu, backend, nb, m_target, span)
        # synthetic residual in ns
        tr = t - MJD0_S
        common = (common_a[None, :] * np.sin(2 * math.pi * common_f[None, :] * tr[:, None]
                                              + common_p[None, :])).sum(1)
        common *= 100.0 / max(common.std(), 1e-30)
        rn = _red_process(rng, tr, span, 10.0 ** rng.uniform(0.5, 3.0), rng.uniform(2.0, 5.0))
        dm = _red_process(rng, tr, span, 10.0 ** rng.uniform(1.0, 2.7), rng.uniform(1.0, 4.0))
        dm *= (1400.0 / nu) ** 2 if w["n_dm"] else 0.0  # no chromatic noise where the model has none
        tm = M @ rng.normal(0.0, 100.0, M.shape[1])
        white = (sigma_ns * efac[backend] * rng.normal(size=n)
                 + equad_ns[backend] * rng.normal(size=n))
        resid_ns = common + rn + dm + tm + white
        if w["cw"]:
            resid_ns += rng.uniform(10.0, 50.0) * np.sin(2 * math.pi * cw_f * tr + rng.uniform(0, 2 * math.pi))
        pulsars.append(Pulsar(
            toas_s=t, freqs_mhz=nu, resid_s=resid_ns * 1e-9, sigma_s=sigma_ns * 1e-9,
            backend=backend, efac=efac, equad_s=equad_ns * 1e-9, M=np.ascontiguousarray(M),
            pos=_sky(rng), dist_kpc=float(rng.uniform(0.5, 5.0))))
    return Array(pulsars=pulsars, n_gwb=w["n_gwb"], n_rn=w["n_rn"], n_dm=w["n_dm"],
                 cw=w["cw"], name=name, meta=dict(seed=seed, chains=w["chains"]))


def small_array(npsr=2, ntoa=60, m=3, n_gwb=2, n_rn=2, n_dm=0, cw=False, seed=0,
                span_yr=5.0, nbackend=1, gwb_free=False, rn_free=False) -> Array:
    """A hand-sized array for brute-force checks (dense N x N algebra).  ``ntoa`` and
    ``m`` may be per-pulsar lists (ragged arrays)."""
    rng = np.random.default_rng(seed)
    span = span_yr * YEAR
    t_end = MJD0_S + span
    ntoas = list(ntoa) if np.ndim(ntoa) else [ntoa] * npsr
    ms = list(m) if np.ndim(m) else [m] * npsr
    pulsars = []
    for I in range(npsr):
        ntoa, m = ntoas[I], ms[I]
        t = np.sort(rng.uniform(t_end - span * rng.uniform(0.6, 1.0), t_end, ntoa))
        if I == 0:
            t[0] = t_end - span
        nu = rng.uniform(400.0, 3000.0, ntoa)
        backend = rng.integers(0, nbackend, ntoa).astype(np.int32)
        sigma_ns = np.exp(rng.uniform(math.log(100.0), math.log(1000.0), ntoa))
        efac = rng.uniform(0.8, 1.5, nbackend)
        equad_ns = np.exp(rng.uniform(math.log(10.0), math.log(300.0), nbackend))
        M = _design_matrix(rng, t, nu, backend, nbackend, m, span)
        tr = t - MJD0_S
        resid_ns = (_red_process(rng, tr, span, 300.0, 3.0, ncomp=8)
                    + (1400.0 / nu) ** 2 * _red_process(rng, tr, span, 50.0, 2.0, ncomp=8)
                    + sigma_ns * efac[backend] * rng.normal(size=ntoa)
                    + equad_ns[backend] * rng.normal(size=ntoa))
        pulsars.append(Pulsar(
            toas_s=t, freqs_mhz=nu, resid_s=resid_ns * 1e-9, sigma_s=sigma_ns * 1e-9,
            backend=backend, efac=efac, equad_s=equad_ns * 1e-9, M=np.ascontiguousarray(M),
            pos=_sky(rng), dist_kpc=float(rng.uniform(0.5, 5.0))))
    return Array(pulsars=pulsars, n_gwb=n_gwb, n_rn=n_rn, n_dm=n_dm, cw=cw, name="small",
                 meta=dict(seed=seed), gwb_free=gwb_free, rn_free=rn_free)


# ---------------------------------------------------------------------------
# Parameter-vector layout.  Plain index bookkeeping, shared by convention with
# the C ABI (pta_layout) and the oracle, each of which states it independently:
#   z_ach[k][c][I]  k < N_a = max(n_gwb, n_rn), c in {0: sin, 1: cos}
#   z_dm [I][k][c]  k < n_dm
#   theta_rn [I][2] (log10 A, gamma) or, free spectrum, [I][n_rn] (log10 kappa_Ik, s^2),
#   theta_dm [I][2], theta_gwb [2] or, free spectrum, [n_gwb] (log10 rho_k, s^2),
#   theta_cw [8] (log10 Mc, log10 f, log10 h, cos iota, psi, cos theta, phi, Phi0)
#   followed by per-pulsar (L_I [kpc], Phi_I [rad]) when cw is on.
# ---------------------------------------------------------------------------
def layout(arr: Array) -> dict:
    npsr = arr.npsr
    na = max(arr.n_gwb, arr.n_rn)
    nd = arr.n_dm
    o = {}
    o["z_ach"] = 0
    o["z_dm"] = na * 2 * npsr
    o["dz"] = o["z_dm"] + npsr * nd * 2
    o["n_th_rn"] = arr.n_rn if arr.rn_free else 2
    o["n_th_gwb"] = arr.n_gwb if arr.gwb_free else 2
    o["th_rn"] = o["dz"]
    o["th_dm"] = o["th_rn"] + o["n_th_rn"] * npsr
    o["th_gwb"] = o["th_dm"] + (2 * npsr if nd > 0 else 0)
    o["th_cw"] = o["th_gwb"] + o["n_th_gwb"]
    o["d"] = o["th_cw"] + ((8 + 2 * npsr) if arr.cw else 0)
    o["na"] = na
    return o


def make_points(arr: Array, B: int, seed: int = 6834, spread: float = 1.0,
                z_scale: float = 1.0) -> np.ndarray:
    """Evaluation points x[B, D] (float32): z ~ N(0, z_scale^2), hyper-parameters
    drawn around the injection values, CW parameters from their prior ranges.  Free
    spectral parameters (log10 of the per-bin variance in s^2) are drawn from
    U(-19, -13), the band the injected processes span."""
    rng = np.random.default_rng(seed)
    L = layout(arr)
    x = np.zeros((B, L["d"]), dtype=np.float64)
    x[:, : L["dz"]] = z_scale * rng.normal(size=(B, L["dz"]))
    npsr = arr.npsr
    nr = L["n_th_rn"]
    for I in range(npsr):
        if arr.rn_free:
            x[:, L["th_rn"] + nr * I: L["th_rn"] + nr * (I + 1)] = rng.uniform(-19.0, -13.0, (B, nr))
        else:
            x[:, L["th_rn"] + 2 * I] = rng.uniform(-16.0, -13.5, B)
            x[:, L["th_rn"] + 2 * I + 1] = rng.uniform(2.0, 5.0, B)
        if arr.n_dm:
            x[:, L["th_dm"] + 2 * I] = rng.uniform(-14.5, -13.0, B)
            x[:, L["th_dm"] + 2 * I + 1] = rng.uniform(1.0, 4.0, B)
    if arr.gwb_free:
        x[:, L["th_gwb"]: L["th_gwb"] + L["n_th_gwb"]] = rng.uniform(-19.0, -13.0, (B, L["n_th_gwb"]))
    else:
        x[:, L["th_gwb"]] = -14.7 + spread * rng.uniform(-0.5, 0.5, B)
        x[:, L["th_gwb"] + 1] = 13.0 / 3.0 + spread * rng.uniform(-1.0, 1.0, B)
    if arr.cw:
        c = L["th_cw"]
        x[:, c + 0] = rng.uniform(8.5, 10.0, B)
        x[:, c + 1] = rng.uniform(-8.5, -7.5, B)
        x[:, c + 2] = -14.5 + rng.uniform(-0.3, 0.3, B)
        x[:, c + 3] = rng.uniform(-1.0, 1.0, B)
        x[:, c + 4] = rng.uniform(0.0, math.pi, B)
        x[:, c + 5] = rng.uniform(-1.0, 1.0, B)
        x[:, c + 6] = rng.uniform(0.0, 2 * math.pi, B)
        x[:, c + 7] = rng.uniform(0.0, 2 * math.pi, B)
        for I in range(npsr):
            x[:, c + 8 + 2 * I] = np.maximum(0.05, arr.pulsars[I].dist_kpc + rng.normal(0.0, 0.2, B))
            x[:, c + 9 + 2 * I] = rng.uniform(0.0, 2 * math.pi, B)
    return x.astype(np.float32)
