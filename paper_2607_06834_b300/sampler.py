"""Host-side driver of the batched HMC sampler (Sec. "Hamiltonian Monte Carlo";
the paper samples the prior-whitened posterior with NumPyro's HMC).

Every transition is one ``Engine.hmc_trajectory`` call: momentum draw, L leapfrog
steps with the fused log posterior + adjoint, and the Metropolis test all run in
the CUDA library (one CUDA graph per batch size and trajectory length).  This
module only chooses the step size and the diagonal inverse mass during warm-up
and computes effective sample sizes from the stored draws:

* step size: dual averaging of Hoffman & Gelman (2014, Sec. 3.2), one per chain
  on that chain's accept indicators, jittered by +-10 % per trajectory;
* inverse mass: windowed estimates of the per-coordinate posterior variance
  (the median over chains of the within-chain variances, so that chains which
  have not met, or one that is stuck, do not set it), in windows that double in
  length (the scheme Stan and NumPyro use), regularised towards 1e-3 as n/(n + 5);
* effective sample size: the multi-chain estimator with Geyer's initial
  monotone sequence (Geyer 1992; Vehtari et al. 2021, Sec. 3.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


# ---------------------------------------------------------------------------
# effective sample size
# ---------------------------------------------------------------------------
def _autocov(x: np.ndarray) -> np.ndarray:
    """Biased autocovariance of each row of x [M, N] at lags 0..N-1 (FFT)."""
    M, N = x.shape
    xc = x - x.mean(axis=1, keepdims=True)
    n2 = 1 << (2 * N - 1).bit_length()
    f = np.fft.rfft(xc, n=n2, axis=1)
    ac = np.fft.irfft(f * np.conj(f), n=n2, axis=1)[:, :N]
    return ac / N


def ess(draws: np.ndarray) -> float:
    """Effective sample size of one scalar from draws [M chains, N iterations]."""
    x = np.asarray(draws, dtype=np.float64)
    if x.ndim == 1:
        x = x[None, :]
    M, N = x.shape
    if N < 4:
        return float("nan")
    acov = _autocov(x)
    chain_var = acov[:, 0] * N / (N - 1.0)
    W = chain_var.mean()
    var_plus = W * (N - 1.0) / N
    if M > 1:
        var_plus += x.mean(axis=1).var(ddof=1)
    if not var_plus > 0:
        return float("nan")
    rho = 1.0 - (W - acov.mean(axis=0)) / var_plus
    rho[0] = 1.0
    # Geyer: sums of adjacent pairs, truncated at the first non-positive pair and
    # forced to be non-increasing
    tau = -1.0
    prev = math.inf
    for t in range(0, N - 1, 2):
        pair = rho[t] + rho[t + 1]
        if pair <= 0.0:
            break
        pair = min(pair, prev)
        prev = pair
        tau += 2.0 * pair
    tau = max(tau, 1.0 / math.log10(M * N))
    return float(M * N / tau)


def ess_columns(draws: np.ndarray) -> np.ndarray:
    """ESS of every column of draws [M, N, K] -> [K]."""
    return np.array([ess(draws[:, :, k]) for k in range(draws.shape[2])])


def split_rhat(draws: np.ndarray) -> float:
    """Split potential scale reduction of one scalar, draws [M, N] (Gelman et al.,
    Bayesian Data Analysis 3rd ed., Sec. 11.4): each chain is cut in halves and
    R = sqrt(var+ / W)."""
    x = np.asarray(draws, dtype=np.float64)
    M, N = x.shape
    h = N // 2
    if h < 2:
        return float("nan")
    x = np.concatenate([x[:, :h], x[:, N - h:]], axis=0)
    W = x.var(axis=1, ddof=1).mean()
    var_plus = W * (h - 1.0) / h + x.mean(axis=1).var(ddof=1)
    return float(np.sqrt(var_plus / W)) if W > 0 else float("inf")


# ---------------------------------------------------------------------------
# initialisation
# ---------------------------------------------------------------------------
def conditional_mode(engine, x: torch.Tensor, dz: int, iters: int = 100) -> torch.Tensor:
    """Move the whitened coefficients z = x[:, :dz] of every chain towards the mode of
    the posterior at fixed hyper-parameters.  log p is exactly quadratic in z there
    (a = L(theta) z enters the residual linearly and the prior is N(0, I)), so
    g(z) = b - H z with H symmetric positive definite, and conjugate gradients
    solve H z = b chain by chain.  Each iteration takes a fresh gradient at z (the
    exact residual) and one at z + s p, s = 1 / rms(p), for H p = (g(z) - g(z + s p)) / s
    (exact for a quadratic up to rounding); beta is Fletcher-Reeves.  A chain whose
    step does not raise log p (rounding in the FP32 gradients) keeps its last point
    and stops."""
    x = x.clone().contiguous()
    lp, g, st = engine.logp_and_grad(x)
    r = g[:, :dz].double()
    active = (st == 0)
    p = r.clone()
    rr = (r * r).sum(1)
    lp = lp.double()
    for it in range(iters):
        if not bool(active.any()):
            break
        sc = 1.0 / (p * p).mean(1).sqrt().clamp_min(1e-30)
        xp = x.clone()
        xp[:, :dz] += (sc[:, None] * p).float()
        _, gp, _ = engine.logp_and_grad(xp)
        Hp = (r - gp[:, :dz].double()) / sc[:, None]
        pHp = (p * Hp).sum(1)
        ok = active & (pHp > 0)
        alpha = torch.where(ok, rr / pHp.clamp_min(1e-300), torch.zeros_like(rr))
        xn = x.clone()
        xn[:, :dz] += (alpha[:, None] * p).float()
        lpn, gn, stn = engine.logp_and_grad(xn)
        better = ok & (stn == 0) & (lpn.double() > lp)
        x = torch.where(better[:, None], xn, x)
        lp = torch.where(better, lpn.double(), lp)
        rn = gn[:, :dz].double()
        rr_new = (rn * rn).sum(1)
        beta = rr_new / rr.clamp_min(1e-300)
        pn = rn + beta[:, None] * p
        r = torch.where(better[:, None], rn, r)
        p = torch.where(better[:, None], pn, p)
        rr = torch.where(better, rr_new, rr)
        active = better
    return x


# ---------------------------------------------------------------------------
# warm-up adaptation
# ---------------------------------------------------------------------------
class DualAveraging:
    """Step-size adaptation of Hoffman & Gelman (2014), Sec. 3.2, on log(eps); one
    independent adaptation per chain (arrays of length B)."""

    def __init__(self, eps0, target: float = 0.8, gamma: float = 0.05, t0: float = 10.0,
                 kappa: float = 0.75):
        self.target, self.gamma, self.t0, self.kappa = target, gamma, t0, kappa
        self.restart(eps0)

    def restart(self, eps0):
        eps0 = np.asarray(eps0, dtype=np.float64)
        self.mu = np.log(10.0 * eps0)
        self.hbar = np.zeros_like(eps0)
        self.log_eps = np.log(eps0)
        self.log_eps_bar = np.zeros_like(eps0)
        self.m = 0

    def update(self, accept):
        self.m += 1
        m = self.m
        w = 1.0 / (m + self.t0)
        self.hbar = (1.0 - w) * self.hbar + w * (self.target - np.asarray(accept, dtype=np.float64))
        self.log_eps = self.mu - math.sqrt(m) / self.gamma * self.hbar
        eta = m ** (-self.kappa)
        self.log_eps_bar = eta * self.log_eps + (1.0 - eta) * self.log_eps_bar
        return np.exp(self.log_eps)

    @property
    def final(self):
        return np.exp(self.log_eps_bar)


def warmup_schedule(n: int, init: int = 15, term: int = 10, base: int = 25) -> list[tuple[int, int]]:
    """Mass-matrix windows [start, end) inside n warm-up iterations: a step-size-only
    start of ``init`` iterations, windows doubling from ``base``, and a step-size-only
    end of ``term``; the last window absorbs what is left."""
    if n < init + term + base:
        return [(init, max(init, n - term))] if n > init + term else []
    wins, s, w = [], init, base
    end = n - term
    while s < end:
        e = s + w
        if e + 2 * w > end:
            e = end
        wins.append((s, e))
        s, w = e, 2 * w
    return wins


@dataclass
class ChainState:
    """Everything a sampling run needs to continue: the chains' state (x, logp, grad
    on the device), the adapted step sizes and inverse mass, and the random-stream
    position.  The library's momenta and accept draws are Philox streams keyed by
    (seed, iteration), and the step jitter comes from a numpy generator whose state
    is kept here, so a resumed run repeats an uninterrupted one bit for bit."""
    x: torch.Tensor
    logp: torch.Tensor
    grad: torch.Tensor
    step: np.ndarray
    inv_mass: torch.Tensor
    seed: int
    iteration: int
    n_leapfrog: int
    jitter: float
    rng_state: dict


def save_state(path: str, st: ChainState) -> None:
    """Checkpoint a ChainState to an .npz file."""
    import json
    meta = dict(seed=st.seed, iteration=st.iteration, n_leapfrog=st.n_leapfrog, jitter=st.jitter,
                rng_state=st.rng_state)
    np.savez(path, x=st.x.cpu().numpy(), logp=st.logp.cpu().numpy(), grad=st.grad.cpu().numpy(),
             step=np.asarray(st.step), inv_mass=st.inv_mass.cpu().numpy(), meta=np.array(json.dumps(meta)))


def load_state(path: str, device=None) -> ChainState:
    """Read a checkpoint written by save_state onto ``device``."""
    import json
    z = np.load(path, allow_pickle=False)
    meta = json.loads(str(z["meta"]))
    dev = torch.device(device) if device is not None else torch.device("cpu")
    return ChainState(x=torch.tensor(z["x"], device=dev), logp=torch.tensor(z["logp"], device=dev),
                      grad=torch.tensor(z["grad"], device=dev), step=np.array(z["step"]),
                      inv_mass=torch.tensor(z["inv_mass"], device=dev), seed=int(meta["seed"]),
                      iteration=int(meta["iteration"]), n_leapfrog=int(meta["n_leapfrog"]),
                      jitter=float(meta["jitter"]), rng_state=meta["rng_state"])


def sample(engine, st: ChainState, n: int, record: slice | None = None):
    """Advance the chains by n trajectories with fixed step sizes and mass (updates
    ``st`` in place).  Returns (draws [n, B, K] on the device, accept counts [B])."""
    B, D = st.x.shape
    dev = st.x.device
    rng = np.random.default_rng()
    rng.bit_generator.state = st.rng_state
    rec = record if record is not None else slice(0, D)
    K = len(range(D)[rec]) if isinstance(rec, slice) else int(len(rec))
    draws = torch.empty((n, B, K), dtype=torch.float32, device=dev)
    accs = torch.zeros(B, dtype=torch.float64, device=dev)
    step = torch.empty(B, dtype=torch.float32, device=dev)
    for j in range(n):
        step.copy_(torch.tensor(st.step * (1.0 + st.jitter * (2.0 * rng.random(B) - 1.0)), dtype=torch.float32))
        acc = engine.hmc_trajectory(st.x, st.logp, st.grad, step, st.n_leapfrog, st.seed, st.iteration,
                                    inv_mass=st.inv_mass)
        st.iteration += 1
        accs += acc.double()
        draws[j].copy_(st.x[:, rec])
    st.rng_state = rng.bit_generator.state
    return draws, accs


@dataclass
class HMCResult:
    draws: np.ndarray                 # [chains, n_samples, K] of the recorded coordinates
    accept_rate: float                # mean over chains and sampling iterations
    step: float
    inv_mass: np.ndarray
    warmup_s: float
    sampling_s: float
    trajectories: int
    leapfrog: int
    stats: dict = field(default_factory=dict)
    state: ChainState | None = None   # where sampling stopped (checkpoint with save_state)


def run_hmc(engine, x0: torch.Tensor, n_warmup: int, n_samples: int, n_leapfrog: int,
            record=None, seed: int = 1, eps0: float = 0.05, target_accept: float = 0.651,
            jitter: float = 0.1, timer=None, init_dz: int = 0, init_iters: int = 100,
            consensus: int = 0, unit_mass: int = 0) -> HMCResult:
    """Warm up and sample ``x0.shape[0]`` chains.  ``engine`` provides ``D``,
    ``logp_and_grad(x)`` and ``hmc_trajectory(x, logp, grad, step, L, seed, it, inv_mass)``
    working on tensors of x0's device.  ``record`` (a slice or an index tensor) selects
    the coordinates stored for the ESS (default: all).  ``timer()`` returns seconds
    after synchronising the device (default: torch.cuda.synchronize + perf_counter).
    With ``init_dz`` > 0 the first init_dz coordinates start at their conditional mode
    (``conditional_mode``, counted in the warm-up time).  With ``consensus`` > 0 the
    chains first run that many warm-up trajectories from their own starts, then all
    restart from the state of the chain with the highest log posterior (the rest of
    the warm-up and the Philox momenta then separate them): chains that start in
    regions far apart would otherwise need far longer to meet than the run allows.
    The step size targets acceptance 0.651, the asymptotically optimal rate of HMC with a
    fixed number of leapfrog steps (Beskos, Pillai, Roberts, Sanz-Serna & Stuart 2013); the
    0.8 that NUTS implementations use left the accepted fraction near 0.93 here and halved
    the ESS of a 40-dimensional Gaussian test.
    With ``unit_mass`` > 0 the first unit_mass coordinates keep inverse mass 1 through
    the adaptation (coordinates that the transform standardizes by construction).
    Box-bounded coordinates (``engine.param_bounds()``) get their mass from the variance
    of u = logit((x - lo)/(hi - lo)), the coordinate the trajectory moves them in."""
    import time

    if timer is None:
        def timer():
            if x0.is_cuda:
                torch.cuda.synchronize(x0.device)
            return time.perf_counter()

    B, D = x0.shape
    dev = x0.device
    t_start = timer()
    x = x0.clone().contiguous()
    if init_dz > 0:
        x = conditional_mode(engine, x, init_dz, iters=init_iters)
    logp, grad, status = engine.logp_and_grad(x)
    if bool((status != 0).any()):
        raise ValueError("initial points outside the prior support")
    init_lp = float(logp.mean())
    inv_mass = torch.ones(D, dtype=torch.float32, device=dev)
    da = DualAveraging(np.full(B, eps0), target=target_accept)
    eps = np.full(B, eps0)
    rng = np.random.default_rng(seed)
    step = torch.empty(B, dtype=torch.float32, device=dev)
    windows = warmup_schedule(n_warmup)
    wi = 0
    # the trajectory moves box-bounded coordinates in u = logit((x - lo)/(hi - lo)): their
    # mass is adapted from the variance of u
    bnd = None
    if hasattr(engine, "param_bounds"):
        lo, hi = engine.param_bounds()
        m = np.isfinite(lo) & np.isfinite(hi)
        if m.any():
            idx = torch.tensor(np.nonzero(m)[0], device=dev)
            bnd = (idx, torch.tensor(lo[m], device=dev), torch.tensor(hi[m], device=dev))
    s1 = torch.zeros((B, D), dtype=torch.float64, device=dev)
    s2 = torch.zeros((B, D), dtype=torch.float64, device=dev)
    cnt = 0
    it = 0
    for i in range(n_warmup):
        step.copy_(torch.tensor(eps * (1.0 + jitter * (2.0 * rng.random(B) - 1.0)), dtype=torch.float32))
        acc = engine.hmc_trajectory(x, logp, grad, step, n_leapfrog, seed, it, inv_mass=inv_mass)
        it += 1
        eps = da.update(acc.cpu().numpy())
        if consensus > 0 and i == consensus - 1:
            lpf = torch.where(torch.isfinite(logp), logp, torch.full_like(logp, -math.inf))
            best = int(torch.argmax(lpf))
            x.copy_(x[best:best + 1].expand_as(x))
            grad.copy_(grad[best:best + 1].expand_as(grad))
            logp.fill_(float(logp[best]))
            eps = np.full(B, float(eps[best]))
            da.restart(eps)
        if wi < len(windows) and windows[wi][0] <= i < windows[wi][1]:
            xd = x.double()
            if bnd is not None:
                t = ((xd[:, bnd[0]] - bnd[1]) / (bnd[2] - bnd[1])).clamp(1e-12, 1.0 - 1e-12)
                xd[:, bnd[0]] = torch.log(t) - torch.log1p(-t)
            s1 += xd
            s2 += xd * xd
            cnt += 1
            if i == windows[wi][1] - 1:
                # within-chain variance, averaged over chains (chains that have not
                # met yet must not inflate it with their spread)
                mean = s1 / cnt
                var = ((s2 / cnt - mean * mean).clamp_min(0.0) * cnt / max(cnt - 1, 1)).median(0).values
                n = cnt * B  # draws behind the estimate
                var = (n / (n + 5.0)) * var + 1e-3 * (5.0 / (n + 5.0))
                if unit_mass > 0:  # coordinates standardized by construction keep unit mass
                    var[:unit_mass] = 1.0
                inv_mass = var.float().contiguous()
                s1.zero_()
                s2.zero_()
                cnt = 0
                wi += 1
                da.restart(eps)
    if n_warmup > 0:
        eps = da.final
    t_warm = timer()
    st = ChainState(x=x, logp=logp, grad=grad, step=np.asarray(eps, dtype=np.float64), inv_mass=inv_mass,
                    seed=seed, iteration=it, n_leapfrog=n_leapfrog, jitter=jitter,
                    rng_state=rng.bit_generator.state)
    draws, accs = sample(engine, st, n_samples, record)
    t_end = timer()
    d = draws.permute(1, 0, 2).cpu().numpy()
    chain_rate = (accs / max(n_samples, 1)).cpu().numpy()
    return HMCResult(draws=d, accept_rate=float(chain_rate.mean()), step=float(np.median(eps)),
                     inv_mass=inv_mass.cpu().numpy(), warmup_s=t_warm - t_start, sampling_s=t_end - t_warm,
                     trajectories=n_warmup + n_samples, leapfrog=n_leapfrog,
                     stats={"final_logp_mean": float(logp.mean()), "init_logp_mean": init_lp,
                            "chain_accept_min": float(chain_rate.min()),
                            "stuck_chains": int((chain_rate < 0.05).sum()),
                            "step_min": float(eps.min()), "step_max": float(eps.max())},
                     state=st)
