"""Host logic of the HMC driver (step-size and mass adaptation, effective sample
size), checked on the CPU against closed forms with a stand-in engine whose
trajectories are plain leapfrog + Metropolis on a Gaussian target."""
import math

import numpy as np
import pytest
import torch

from paper_2607_06834_b300 import sampler


def _ar1(rng, M, N, phi):
    x = np.empty((M, N))
    e = rng.normal(size=(M, N))
    x[:, 0] = e[:, 0] / math.sqrt(1 - phi * phi)
    for n in range(1, N):
        x[:, n] = phi * x[:, n - 1] + e[:, n]
    return x


@pytest.mark.parametrize("phi", [0.0, 0.5, 0.9, -0.5])
def test_ess_ar1_closed_form(phi):
    # an AR(1) chain has integrated autocorrelation time (1 + phi) / (1 - phi)
    rng = np.random.default_rng(11)
    M, N = 4, 20000
    x = _ar1(rng, M, N, phi)
    want = M * N * (1 - phi) / (1 + phi)
    got = sampler.ess(x)
    assert abs(got / want - 1) < 0.15, (got, want)


def test_ess_detects_unmixed_chains():
    # two chains stuck at different means: the between-chain variance must cut the ESS
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 5000))
    x[1] += 5.0
    assert sampler.ess(x) < 50


def test_warmup_schedule_windows():
    for n in (60, 150, 400, 1000):
        w = sampler.warmup_schedule(n)
        assert w[0][0] == 15 and w[-1][1] == n - 10
        for (a, b), (c, d) in zip(w, w[1:]):
            assert b == c and d - c >= b - a
    assert sampler.warmup_schedule(20) == []


class GaussEngine:
    """Stand-in for the CUDA engine: logp = -1/2 sum ((x - mu) / sigma)^2, with the same
    hmc_trajectory contract (in-place state update, accept flags returned)."""

    def __init__(self, mu, sigma, seed=0):
        self.mu = torch.tensor(mu, dtype=torch.float64)
        self.sig = torch.tensor(sigma, dtype=torch.float64)
        self.D = len(mu)
        self.g = torch.Generator().manual_seed(seed)

    def _lg(self, x):
        r = (x.double() - self.mu) / self.sig
        return -0.5 * (r * r).sum(1), (-r / self.sig).float()

    def logp_and_grad(self, x):
        lp, g = self._lg(x)
        return lp, g, torch.zeros(x.shape[0], dtype=torch.int32)

    def hmc_trajectory(self, x, logp, grad, step, L, seed, it, inv_mass=None):
        # random numbers keyed by (seed, iteration), like the library's Philox streams
        self.g.manual_seed(int(seed) * 1000003 + int(it))
        im = inv_mass.double() if inv_mass is not None else torch.ones(self.D, dtype=torch.float64)
        p = torch.randn(x.shape, generator=self.g, dtype=torch.float64) / im.sqrt()
        k0 = 0.5 * (p * p * im).sum(1)
        xs, gs = x.double().clone(), grad.double().clone()
        e = step.double()[:, None]
        for _ in range(L):
            p += 0.5 * e * gs
            xs += e * im * p
            lp1, g1 = self._lg(xs)
            gs = g1.double()
            p += 0.5 * e * gs
        k1 = 0.5 * (p * p * im).sum(1)
        u = torch.rand(x.shape[0], generator=self.g, dtype=torch.float64)
        acc = torch.log(u) < (-logp + k0) - (-lp1 + k1)
        x[acc] = xs[acc].float()
        grad[acc] = gs[acc].float()
        logp[acc] = lp1[acc]
        return acc.int()


def test_run_hmc_adapts_mass_and_samples_gaussian():
    sig = np.array([0.01, 0.05, 0.3, 1.0, 2.0, 0.1])
    mu = np.array([1.0, -2.0, 0.5, 0.0, 3.0, -0.7])
    eng = GaussEngine(mu, sig, seed=5)
    B = 32
    x0 = torch.tensor(np.random.default_rng(1).normal(size=(B, 6)) * 0.5 + mu * 0.9, dtype=torch.float32)
    res = sampler.run_hmc(eng, x0, n_warmup=300, n_samples=300, n_leapfrog=8, seed=2, eps0=0.01,
                          timer=lambda: 0.0)
    # the adapted inverse mass is the posterior variance
    np.testing.assert_allclose(res.inv_mass, sig ** 2, rtol=0.35)
    d = res.draws.reshape(-1, 6)
    assert np.all(np.abs(d.mean(0) - mu) < 4 * sig / math.sqrt(B * 30)), (d.mean(0) - mu) / sig
    np.testing.assert_allclose(d.std(0), sig, rtol=0.15)
    assert 0.6 < res.accept_rate < 0.97
    e = sampler.ess_columns(res.draws)
    assert np.all(e > 0.2 * B * 300 / 10)


def test_conditional_mode_solves_the_quadratic():
    # logp quadratic in the first dz coordinates with a badly conditioned precision
    rng = np.random.default_rng(4)
    dz, D = 12, 14
    Q, _ = np.linalg.qr(rng.normal(size=(dz, dz)))
    H = Q @ np.diag(np.logspace(0, 4, dz)) @ Q.T
    b = rng.normal(size=dz) * 10

    class QuadEngine:
        def logp_and_grad(self, x):
            z = x[:, :dz].double()
            g = torch.zeros(x.shape, dtype=torch.float32)
            gz_ = torch.tensor(b)[None, :] - z @ torch.tensor(H)
            g[:, :dz] = gz_.float()
            lp = (z @ torch.tensor(b)) - 0.5 * ((z @ torch.tensor(H)) * z).sum(1)
            return lp, g, torch.zeros(x.shape[0], dtype=torch.int32)

    x0 = torch.tensor(rng.normal(size=(3, D)), dtype=torch.float32)
    x = sampler.conditional_mode(QuadEngine(), x0, dz, iters=40)
    zstar = np.linalg.solve(H, b)
    np.testing.assert_allclose(x[:, :dz].numpy(), np.broadcast_to(zstar, (3, dz)), atol=2e-3 * np.abs(zstar).max())
    assert torch.equal(x[:, dz:], x0[:, dz:])


def test_split_rhat_flags_unmixed_chains():
    rng = np.random.default_rng(8)
    good = rng.normal(size=(4, 1000))
    assert abs(sampler.split_rhat(good) - 1.0) < 0.01
    bad = good.copy()
    bad[0] += 3.0
    assert sampler.split_rhat(bad) > 1.2


def test_checkpoint_resume_is_bit_exact(tmp_path):
    sig = np.array([0.1, 1.0, 0.5])
    mu = np.zeros(3)
    eng = GaussEngine(mu, sig)
    x0 = torch.tensor(np.random.default_rng(2).normal(size=(8, 3)), dtype=torch.float32)
    res = sampler.run_hmc(eng, x0, n_warmup=60, n_samples=5, n_leapfrog=5, seed=9, eps0=0.1, timer=lambda: 0.0)
    st = res.state
    path = str(tmp_path / "chains.npz")
    sampler.save_state(path, st)
    straight, _ = sampler.sample(eng, st, 12)
    st2 = sampler.load_state(path)
    first, _ = sampler.sample(eng, st2, 7)
    sampler.save_state(path, st2)
    st3 = sampler.load_state(path)
    second, _ = sampler.sample(eng, st3, 5)
    assert torch.equal(torch.cat([first, second]), straight)
    assert st3.iteration == st.iteration


def test_consensus_start_mixes_dispersed_chains():
    sig = np.array([0.05, 1.0, 0.3])
    mu = np.array([2.0, -1.0, 0.5])
    eng = GaussEngine(mu, sig, seed=4)
    B = 16
    x0 = torch.tensor(np.random.default_rng(5).normal(size=(B, 3)) * 20.0, dtype=torch.float32)
    res = sampler.run_hmc(eng, x0, n_warmup=200, n_samples=200, n_leapfrog=8, seed=6, eps0=0.01,
                          consensus=40, timer=lambda: 0.0, record=torch.tensor([0, 1, 2]))
    rh = [sampler.split_rhat(res.draws[:, :, k]) for k in range(3)]
    assert max(rh) < 1.05, rh
    assert np.all(np.abs(res.draws.reshape(-1, 3).mean(0) - mu) < 5 * sig / math.sqrt(B * 20))
