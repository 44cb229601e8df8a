"""FP64 CPU oracle for the standardized Fourier-coefficient PTA posterior.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package's smoke check and
the benchmark's CPU-baseline leg may import this module.  It shares no code
with the CUDA path and imports nothing from it.

Every function is the plain definition of the quantity it returns, written in
FP64 with numpy, following the paper (Gundersen, van Haasteren, Cornish,
Vallisneri, Meyers, "A new framework for lightning-fast gravitational wave
analysis of pulsar timing data"):

  * white-noise covariance N            Eq. (WN_cov), Sec. "White noise"
  * Fourier basis F, DM basis F_DM      Eq. (Fourier_series) and the text after
                                        it, Sec. "Red and chromatic noise"
  * prior covariance phi, HD ORF        Eqs. (prior_cov), (HD), Sec. "Priors"
  * power-law spectrum                  Eq. (power_law)
  * timing-model marginalisation N~^-1  Eq. (Gmatrix_proj) and its QR form
  * standardizing transform a = L z     Eqs. (standardizing_transform),
                                        (standardized_density) with mu = 0 and
                                        Sigma = phi (prior-whitened reading)
  * CURN-posterior transform            Eqs. (PTA_standard_transform_curn),
    a = ahat_CURN + L_CURN z            (standardized_stochastic_posterior); the
                                        tempered T_beta of App. "tempered likelihoods"
  * posterior with deterministic signal Eq. (raw_det_posterior)
  * CW phase / frequency evolution      Eqs. (phase_evolve), (CW_evolve),
                                        (phase_evolve_Taylor)
  * HMC leapfrog + Metropolis accept    Eqs. (Hamiltonian), (Hamilton's_eq),
                                        (Gaussian_momentum), (HMC_acceptance)

Units: residuals, uncertainties and covariances in ns / ns^2 (Sec. "Single
precision"), times in s.  The canonical log-posterior ``logp`` drops the
data-only constants that the paper drops (det 2 pi N, det M^T N^-1 M); the
function ``logp_full`` adds them back (and the (2 pi)^(-D_z/2) of the z
prior) so that it is a normalised density in z.

Pins (tests/test_oracle_*.py): HD closed-form values; power-law spectral ratios
and a hand value; three routes to N~^-1 agree; logp_full integrated over z in
closed form equals the dense time-domain Gaussian marginal likelihood with
C = N + F phi F^T; the log-det cancellation of the prior-whitened transform;
the Gram-form (Eq. stochastic_posterior) equivalence; central finite
differences of every gradient block; CW invariants (h -> 0, L -> 0 with equal
phases, psi -> psi + pi/2, dPhi/dt = omega(t), antenna-pattern identity);
Philox4x32-10 known-answer vectors; HMC reversibility and Gaussian moments;
hand-worked golden values (tests/golden/) for the white-noise variance, the DM
weight and the circular-binary delay at special geometries, and the quadrupole-
formula chirp rate for Eq. (CW_evolve).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

YEAR_S = 365.25 * 86400.0
F_YR = 1.0 / YEAR_S
NU_REF_MHZ = 1400.0
TSUN_S = 4.925490947641267e-06       # G Msun / c^3 in s
KPC_S = 1.0292712503e11              # 1 kpc / c in s
LN10 = math.log(10.0)

# uniform hyper-prior boxes (Sec. "Priors": log10 A ~ U(-20, -10), gamma ~ U(0, 7),
# identical for intrinsic red noise; the same box is used for DM)
PRIOR_LOG10A = (-20.0, -10.0)
PRIOR_GAMMA = (0.0, 7.0)
PRIOR_LOG10RHO = (-20.0, -5.0)   # free spectral model: log10 of the per-bin variance (s^2), Sec. "Priors"
# CW prior boxes (order: log10 Mc, log10 f, log10 h, cos iota, psi, cos theta, phi, Phi0)
PRIOR_CW = [(7.0, 10.5), (-9.0, -7.0), (-18.0, -11.0), (-1.0, 1.0), (0.0, math.pi),
            (-1.0, 1.0), (0.0, 2.0 * math.pi), (0.0, 2.0 * math.pi)]
PRIOR_PPHASE = (0.0, 2.0 * math.pi)
DIST_SIGMA_KPC = 0.2                 # pulsar-distance prior width (Sec. "Analyses")


# --------------------------------------------------------------------------- #
# Building blocks, each the definition printed in the paper.
# --------------------------------------------------------------------------- #
def hellings_downs(pos: np.ndarray) -> np.ndarray:
    """Eq. (HD): alpha_IJ = 3/2 b ln b - b/4 + 1/2 + delta_IJ/2, b = (1 - cos Theta_IJ)/2."""
    npsr = pos.shape[0]
    G = np.empty((npsr, npsr))
    for I in range(npsr):
        for J in range(npsr):
            cos_t = float(np.clip(np.dot(pos[I], pos[J]), -1.0, 1.0))
            b = 0.5 * (1.0 - cos_t)
            blnb = b * math.log(b) if b > 0.0 else 0.0
            G[I, J] = 1.5 * blnb - 0.25 * b + 0.5 + (0.5 if I == J else 0.0)
    return G


def power_law(log10A: float, gamma: float, k: np.ndarray, T: float) -> np.ndarray:
    """Eq. (power_law) in ns^2: rho_k = A^2/(12 pi^2) (1/T) (f_k / f_yr)^(-gamma) yr^3 / yr,
    i.e. A^2/(12 pi^2) f_yr^(gamma-3) f_k^(-gamma) / T with f_k = k/T, T in s."""
    A = 10.0 ** log10A
    f = np.asarray(k, dtype=float) / T
    rho_s2 = A * A / (12.0 * math.pi ** 2) * F_YR ** (gamma - 3.0) * f ** (-gamma) / T
    return rho_s2 * 1e18


def white_noise_var(psr) -> np.ndarray:
    """Eq. (WN_cov): N_ii = EFAC_mu^2 sigma_i^2 + EQUAD_mu^2, in ns^2."""
    s = psr.sigma_s * 1e9
    b = psr.backend
    return psr.efac[b] ** 2 * s * s + (psr.equad_s[b] * 1e9) ** 2


def fourier_basis(t_rel: np.ndarray, T: float, nf: int) -> np.ndarray:
    """Eq. (Fourier_series): columns [sin(2 pi k t/T), cos(2 pi k t/T)] for k = 1..nf,
    ordered so that F a = sum_k a_k sin + b_k cos with a = [a1, b1, a2, b2, ...]."""
    F = np.zeros((t_rel.shape[0], 2 * nf))
    for k in range(1, nf + 1):
        arg = 2.0 * math.pi * k * t_rel / T
        F[:, 2 * (k - 1)] = np.sin(arg)
        F[:, 2 * (k - 1) + 1] = np.cos(arg)
    return F


def chromatic_weight(freqs_mhz: np.ndarray) -> np.ndarray:
    """DM basis weight: F_DM = F / (K nu^2), with the constant absorbed into the DM
    amplitude and referenced to 1400 MHz: (nu_ref / nu)^2."""
    return (NU_REF_MHZ / freqs_mhz) ** 2


def ntilde_inv_woodbury(Nvar: np.ndarray, M: np.ndarray, v: np.ndarray) -> np.ndarray:
    """N~^-1 v with N~^-1 = N^-1 - N^-1 M (M^T N^-1 M)^-1 M^T N^-1 (the flat-prior
    timing-model marginalisation; equal to Eq. (Gmatrix_proj), see ntilde_inv_G)."""
    w = v / Nvar[:, None] if v.ndim == 2 else v / Nvar
    K = M.T @ (M / Nvar[:, None])
    b = M.T @ w
    c = np.linalg.solve(K, b)
    corr = M @ c
    return w - (corr / Nvar[:, None] if v.ndim == 2 else corr / Nvar)


def ntilde_inv_G(Nvar: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Eq. (Gmatrix_proj) with G = Q_2 from the (column-pivoted) QR decomposition of
    M (the text after Eq. (Gmatrix_proj)): N~^-1 = G (G^T N G)^-1 G^T.  Dense n x n."""
    n, m = M.shape
    Q, _R, _P = sla.qr(M, pivoting=True)
    G = Q[:, m:]
    GNG = G.T @ (Nvar[:, None] * G)
    return G @ np.linalg.solve(GNG, G.T)


def ntilde_inv_svd(Nvar: np.ndarray, M: np.ndarray) -> np.ndarray:
    """The same projector with G from the SVD of M (G = left singular vectors
    orthogonal to the column space of M)."""
    n, m = M.shape
    U, _s, _vt = np.linalg.svd(M, full_matrices=True)
    G = U[:, m:]
    return G @ np.linalg.solve(G.T @ (Nvar[:, None] * G), G.T)


def chol_tangent(L: np.ndarray, dPhi: np.ndarray) -> np.ndarray:
    """Forward-mode derivative of the Cholesky factor: for Phi = L L^T,
    dL = L tril_half(L^-1 dPhi L^-T), where tril_half keeps the strict lower
    triangle and half the diagonal (follows from dPhi = dL L^T + L dL^T with
    L^-1 dL lower triangular)."""
    X = sla.solve_triangular(L, dPhi, lower=True)
    Y = sla.solve_triangular(L, X.T, lower=True).T
    P = np.tril(Y, -1) + 0.5 * np.diag(np.diag(Y))
    return L @ P


# --------------------------------------------------------------------------- #
# CW: circular super-massive black-hole binary (Sec. "Deterministic signals and
# continuous waves", Eqs. (phase_evolve), (CW_evolve)).  The antenna pattern,
# polarisation amplitudes and pulsar term follow the published circular-binary
# model of Ellis, Siemens & Creighton (2012), restated from the physics.
# --------------------------------------------------------------------------- #
def cw_geometry(cos_gwtheta, gwphi, pos):
    """Propagation direction Omega, polarisation basis (m, n) and antenna patterns
    F+ = ((m.p)^2 - (n.p)^2) / (2 (1 + Omega.p)), Fx = (m.p)(n.p) / (1 + Omega.p)."""
    ct = cos_gwtheta
    st = np.sqrt(1.0 - ct * ct)
    sp, cp = np.sin(gwphi), np.cos(gwphi)
    omhat = -np.array([st * cp, st * sp, ct])
    mhat = np.array([sp, -cp, 0.0 * sp])
    nhat = np.array([-ct * cp, -ct * sp, st])
    mp = mhat @ pos
    np_ = nhat @ pos
    op = omhat @ pos
    fplus = 0.5 * (mp * mp - np_ * np_) / (1.0 + op)
    fcross = mp * np_ / (1.0 + op)
    return fplus, fcross, op


def cw_phase(t, mc_s, omega0):
    """Phase advance and frequency of the Earth term from Eqs. (phase_evolve) and
    (CW_evolve): omega = omega0 (1 - x)^(-3/8), x = (256/5) Mc^(5/3) omega0^(8/3) t,
    Phi - Phi0 = [omega0^(-5/3) - omega^(-5/3)] / (32 Mc^(5/3))."""
    x = 256.0 / 5.0 * mc_s ** (5.0 / 3.0) * omega0 ** (8.0 / 3.0) * t
    omega = omega0 * (1.0 - x) ** (-3.0 / 8.0)
    dphi = (omega0 ** (-5.0 / 3.0) - omega ** (-5.0 / 3.0)) / (32.0 * mc_s ** (5.0 / 3.0))
    return dphi, omega


def cw_phase_taylor(t, mc_s, omega0):
    """First-order form of Eq. (phase_evolve_Taylor): Phi - Phi0 ~ omega0 t."""
    xp = mc_s ** (5.0 / 3.0) * omega0 ** (8.0 / 3.0) * t
    return xp / (mc_s * omega0) ** (5.0 / 3.0)


def cw_signal(t_rel, pos, th, dist_kpc, pphase):
    """Deterministic CW delay h(theta) in ns at times t_rel (s from the array's first
    TOA) for one pulsar.  th = (log10 Mc[Msun], log10 f_gw[Hz], log10 h, cos iota, psi,
    cos theta, phi, Phi0).  Earth term r(t) and pulsar term r(t_p) with
    t_p = t - L (1 + Omega.p); the pulsar-term phase at t = 0 is the free parameter
    Phi_I (the paper treats pulsar phases as independent parameters).  Residual
    s = F+ (r+(t_p) - r+(t)) + Fx (rx(t_p) - rx(t))."""
    log10mc, log10f, log10h, cosi, psi, cos_gt, gwphi, phi0 = th
    mc = 10.0 ** log10mc * TSUN_S
    omega0 = np.pi * 10.0 ** log10f
    h = 10.0 ** log10h
    L = dist_kpc * KPC_S
    fplus, fcross, op = cw_geometry(cos_gt, gwphi, pos)
    tp = t_rel - L * (1.0 + op)
    # Earth term
    dphi_e, om_e = cw_phase(t_rel, mc, omega0)
    ph_e = phi0 + dphi_e
    # pulsar term: same evolution law, referenced so its phase at t = 0 is Phi_I
    dphi_p0, _ = cw_phase(-L * (1.0 + op), mc, omega0)
    dphi_p, om_p = cw_phase(tp, mc, omega0)
    ph_p = pphase + (dphi_p - dphi_p0)
    c2psi, s2psi = np.cos(2 * psi), np.sin(2 * psi)
    inc_p = 1.0 + cosi * cosi
    inc_x = 2.0 * cosi

    def pols(phase, om):
        alpha = h / (2.0 * omega0 ** (2.0 / 3.0) * om ** (1.0 / 3.0))
        s2, c2 = np.sin(2 * phase), np.cos(2 * phase)
        rp = alpha * (-s2 * inc_p * c2psi - c2 * inc_x * s2psi)
        rx = alpha * (-s2 * inc_p * s2psi + c2 * inc_x * c2psi)
        return rp, rx

    rp_e, rx_e = pols(ph_e, om_e)
    rp_p, rx_p = pols(ph_p, om_p)
    return (fplus * (rp_p - rp_e) + fcross * (rx_p - rx_e)) * 1e9


# --------------------------------------------------------------------------- #
# The posterior.
# --------------------------------------------------------------------------- #
class Oracle:
    """Plain FP64 posterior and gradient for one synthetic array.

    ``arr`` exposes ``pulsars`` (each with toas_s, freqs_mhz, resid_s, sigma_s,
    backend, efac, equad_s, M, pos, dist_kpc), ``n_gwb``, ``n_rn``, ``n_dm``, ``cw``.
    """

    def __init__(self, arr, store_basis: bool = True, transform: str = "prior"):
        if transform not in ("prior", "curn"):
            raise ValueError("transform must be 'prior' or 'curn'")
        self.transform_kind = transform
        self._curn_fixed = None
        self.arr = arr
        self.psrs = arr.pulsars
        self.npsr = len(self.psrs)
        self.n_gwb, self.n_rn, self.n_dm = arr.n_gwb, arr.n_rn, arr.n_dm
        self.cw = bool(arr.cw)
        # free spectral models (Sec. "Priors"): each rho_k / kappa_Ik its own parameter
        self.gwb_free = bool(getattr(arr, "gwb_free", False))
        self.rn_free = bool(getattr(arr, "rn_free", False))
        self.na = max(self.n_gwb, self.n_rn)
        self.P = 2 * self.na + 2 * self.n_dm
        tmin = min(p.toas_s.min() for p in self.psrs)
        tmax = max(p.toas_s.max() for p in self.psrs)
        self.t0, self.T = tmin, tmax - tmin               # Sec. "Red and chromatic noise"
        self.Gamma = hellings_downs(np.array([p.pos for p in self.psrs]))
        self.Nvar = [white_noise_var(p) for p in self.psrs]
        self.dt_ns = [p.resid_s * 1e9 for p in self.psrs]
        self.t_rel = [p.toas_s - self.t0 for p in self.psrs]
        self.F = [self.basis(I) for I in range(self.npsr)] if store_basis else None
        # parameter layout (same convention as the C ABI)
        o = {}
        o["z_dm"] = self.na * 2 * self.npsr
        o["dz"] = o["z_dm"] + self.npsr * self.n_dm * 2
        self.nthr = self.n_rn if self.rn_free else 2
        self.nthg = self.n_gwb if self.gwb_free else 2
        o["th_rn"] = o["dz"]
        o["th_dm"] = o["th_rn"] + self.nthr * self.npsr
        o["th_gwb"] = o["th_dm"] + (2 * self.npsr if self.n_dm else 0)
        o["th_cw"] = o["th_gwb"] + self.nthg
        o["d"] = o["th_cw"] + ((8 + 2 * self.npsr) if self.cw else 0)
        self.lay = o
        self.D = o["d"]
        self.Dz = o["dz"]

    # -- basis ------------------------------------------------------------------
    def basis(self, I: int) -> np.ndarray:
        p = self.psrs[I]
        t = p.toas_s - self.t0
        F = fourier_basis(t, self.T, self.na)
        if self.n_dm:
            Fd = fourier_basis(t, self.T, self.n_dm) * chromatic_weight(p.freqs_mhz)[:, None]
            F = np.concatenate([F, Fd], axis=1)
        return F

    def get_F(self, I):
        return self.F[I] if self.F is not None else self.basis(I)

    # -- parameter unpacking ----------------------------------------------------
    def unpack(self, x):
        x = np.asarray(x, dtype=np.float64)
        o, npsr, na, nd = self.lay, self.npsr, self.na, self.n_dm
        z_ach = x[: o["z_dm"]].reshape(na, 2, npsr)            # [k][c][I]
        z_dm = x[o["z_dm"]: o["dz"]].reshape(npsr, nd, 2)        # [I][k][c]
        th_rn = x[o["th_rn"]: o["th_rn"] + self.nthr * npsr].reshape(npsr, self.nthr)
        th_dm = x[o["th_dm"]: o["th_dm"] + 2 * npsr].reshape(npsr, 2) if nd else np.zeros((npsr, 2))
        th_gwb = x[o["th_gwb"]: o["th_gwb"] + self.nthg]
        th_cw = x[o["th_cw"]: o["d"]] if self.cw else None
        return z_ach, z_dm, th_rn, th_dm, th_gwb, th_cw

    def in_prior(self, x) -> bool:
        _, _, th_rn, th_dm, th_gwb, th_cw = self.unpack(x)
        def box(v, lo_hi):
            return bool(np.all((v > lo_hi[0]) & (v < lo_hi[1])))
        if self.rn_free:
            ok = box(th_rn, PRIOR_LOG10RHO)
        else:
            ok = box(th_rn[:, 0], PRIOR_LOG10A) and box(th_rn[:, 1], PRIOR_GAMMA)
        if self.gwb_free:
            ok = ok and box(th_gwb, PRIOR_LOG10RHO)
        else:
            ok = ok and box(th_gwb[0:1], PRIOR_LOG10A) and box(th_gwb[1:2], PRIOR_GAMMA)
        if self.n_dm:
            ok = ok and box(th_dm[:, 0], PRIOR_LOG10A) and box(th_dm[:, 1], PRIOR_GAMMA)
        if self.cw:
            for j in range(8):
                ok = ok and box(th_cw[j:j + 1], PRIOR_CW[j])
            dist = th_cw[8::2]
            ok = ok and bool(np.all(dist > 0.0)) and box(th_cw[9::2], PRIOR_PPHASE)
        return ok

    def param_bounds(self):
        """Per-coordinate prior support (lo, hi): the uniform boxes of Sec. "Priors" (and
        the CW box, pulsar phases in (0, 2 pi)); -inf/inf for z and pulsar distances."""
        lo = np.full(self.D, -np.inf)
        hi = np.full(self.D, np.inf)
        o = self.lay
        for I in range(self.npsr):
            if self.rn_free:
                sl = slice(o["th_rn"] + self.n_rn * I, o["th_rn"] + self.n_rn * (I + 1))
                lo[sl], hi[sl] = PRIOR_LOG10RHO
            else:
                lo[o["th_rn"] + 2 * I], hi[o["th_rn"] + 2 * I] = PRIOR_LOG10A
                lo[o["th_rn"] + 2 * I + 1], hi[o["th_rn"] + 2 * I + 1] = PRIOR_GAMMA
            if self.n_dm:
                lo[o["th_dm"] + 2 * I], hi[o["th_dm"] + 2 * I] = PRIOR_LOG10A
                lo[o["th_dm"] + 2 * I + 1], hi[o["th_dm"] + 2 * I + 1] = PRIOR_GAMMA
        if self.gwb_free:
            lo[o["th_gwb"]: o["th_gwb"] + self.n_gwb], hi[o["th_gwb"]: o["th_gwb"] + self.n_gwb] = PRIOR_LOG10RHO
        else:
            lo[o["th_gwb"]], hi[o["th_gwb"]] = PRIOR_LOG10A
            lo[o["th_gwb"] + 1], hi[o["th_gwb"] + 1] = PRIOR_GAMMA
        if self.cw:
            for j in range(8):
                lo[o["th_cw"] + j], hi[o["th_cw"] + j] = PRIOR_CW[j]
            for I in range(self.npsr):
                lo[o["th_cw"] + 9 + 2 * I], hi[o["th_cw"] + 9 + 2 * I] = PRIOR_PPHASE
        return lo, hi

    # -- spectra and prior covariance (Eqs. prior_cov, power_law) -----------------
    def spectra(self, th_rn, th_dm, th_gwb):
        ks = np.arange(1, self.na + 1)
        rho = np.zeros(self.na)
        if self.gwb_free:   # free spectral model: rho_k = 10^theta_k s^2, in ns^2
            rho[: self.n_gwb] = 10.0 ** np.asarray(th_gwb, dtype=float) * 1e18
        else:
            rho[: self.n_gwb] = power_law(th_gwb[0], th_gwb[1], ks[: self.n_gwb], self.T)
        kappa = np.zeros((self.npsr, self.na))
        for I in range(self.npsr):
            if self.rn_free:
                kappa[I, : self.n_rn] = 10.0 ** np.asarray(th_rn[I], dtype=float) * 1e18
            else:
                kappa[I, : self.n_rn] = power_law(th_rn[I, 0], th_rn[I, 1], ks[: self.n_rn], self.T)
        kdm = np.zeros((self.npsr, self.n_dm))
        if self.n_dm:
            kd = np.arange(1, self.n_dm + 1)
            for I in range(self.npsr):
                kdm[I] = power_law(th_dm[I, 0], th_dm[I, 1], kd, self.T)
        return rho, kappa, kdm

    def phi_bin(self, rho_k, kappa_k):
        """Eq. (prior_cov) restricted to one frequency bin: Phi_k = rho_k Gamma + diag(kappa_.k)."""
        return rho_k * self.Gamma + np.diag(kappa_k)

    # -- standardizing transform a = L z (prior-whitened) -------------------------
    def transform(self, z_ach, z_dm, rho, kappa, kdm):
        """a_{.,k,c} = L_k z_{.,k,c} with Phi_k = L_k L_k^T (Eq. standardizing_transform
        with mu = 0, Sigma = phi, batched over frequency bins); DM: a = sqrt(kappa) z.
        Returns per-pulsar coefficient vectors a_I[P] and the factors L_k."""
        a = np.zeros((self.npsr, self.P))
        Ls = []
        for k in range(self.na):
            Lk = np.linalg.cholesky(self.phi_bin(rho[k], kappa[:, k]))
            Ls.append(Lk)
            for c in range(2):
                a[:, 2 * k + c] = Lk @ z_ach[k, c]
        if self.n_dm:
            off = 2 * self.na
            for I in range(self.npsr):
                for k in range(self.n_dm):
                    for c in range(2):
                        a[I, off + 2 * k + c] = math.sqrt(kdm[I, k]) * z_dm[I, k, c]
        return a, Ls

    # -- CURN-posterior standardizing transform ------------------------------------
    # Eq. (PTA_standard_transform_curn): per pulsar, a_I = ahat_I + L_I z_I with
    # Sigma_I = (beta F_I^T N~_I^-1 F_I + phi_CURN,I^-1)^-1 = L_I L_I^T (Cholesky, lower)
    # and ahat_I = beta Sigma_I F_I^T N~_I^-1 dt_I.  phi_CURN is the prior covariance of
    # Eq. (prior_cov) with the inter-pulsar correlations dropped (alpha_IJ = delta_IJ,
    # Gamma_II = 1), diagonal per pulsar.  beta = 1 is the transform of the paper's main
    # result; beta < 1 the tempered transform T_beta of App. "tempered likelihoods".
    # The density sampled is Eq. (standardized_stochastic_posterior): the posterior of
    # Eq. (stochastic_posterior) at a(z) times det L_CURN, which (completing the square
    # back) is the likelihood times the HD prior N(a; 0, phi) times det L_CURN.
    def curn_fixed(self, I):
        """(F^T N~^-1 F, F^T N~^-1 dt) of pulsar I: parameter-independent."""
        if self._curn_fixed is None:
            self._curn_fixed = [None] * self.npsr
        if self._curn_fixed[I] is None:
            F = self.get_F(I)
            NF = ntilde_inv_woodbury(self.Nvar[I], self.psrs[I].M, F)
            self._curn_fixed[I] = (F.T @ NF, NF.T @ self.dt_ns[I])
        return self._curn_fixed[I]

    def curn_prior_var(self, I, rho, kappa, kdm):
        """Diagonal of phi_CURN for pulsar I: rho_k + kappa_Ik on both achromatic columns
        of bin k, kappa^DM_Ik on the DM columns."""
        phi = np.zeros(self.P)
        for k in range(self.na):
            phi[2 * k: 2 * k + 2] = rho[k] + kappa[I, k]
        for k in range(self.n_dm):
            phi[2 * self.na + 2 * k: 2 * self.na + 2 * k + 2] = kdm[I, k]
        return phi

    def curn_moments(self, I, phiC, beta, h=None):
        """ahat_I, L_I (lower Cholesky factor of Sigma_I) and Sigma_I.  With a deterministic
        signal h_I (Eq. decenter_det_PTA) the mean is abar_I = beta Sigma_I F^T N~^-1 (dt - h)."""
        FNF, FNd = self.curn_fixed(I)
        if h is not None:
            FNd = FNd - self.get_F(I).T @ ntilde_inv_woodbury(self.Nvar[I], self.psrs[I].M, h)
        Sigma = np.linalg.inv(beta * FNF + np.diag(1.0 / phiC))
        Sigma = 0.5 * (Sigma + Sigma.T)
        return beta * Sigma @ FNd, np.linalg.cholesky(Sigma), Sigma

    def z_per_pulsar(self, z_ach, z_dm):
        """z regrouped per pulsar in the coefficient order of a_I: z_I[2k + c] is
        z_ach[k][c][I], z_I[2 N_a + 2k + c] is z_dm[I][k][c] (the parameter layout of the
        prior-whitened transform, reused)."""
        Z = np.zeros((self.npsr, self.P))
        for k in range(self.na):
            for c in range(2):
                Z[:, 2 * k + c] = z_ach[k, c]
        for I in range(self.npsr):
            for k in range(self.n_dm):
                for c in range(2):
                    Z[I, 2 * self.na + 2 * k + c] = z_dm[I, k, c]
        return Z

    def curn_transform(self, z_ach, z_dm, rho, kappa, kdm, beta: float = 1.0, th_cw=None):
        """a_I = ahat_I + L_I z_I for every pulsar (abar_I with the deterministic signal,
        Eq. decenter_det_PTA); returns (a, [L_I])."""
        Z = self.z_per_pulsar(z_ach, z_dm)
        a = np.zeros((self.npsr, self.P))
        Ls = []
        for I in range(self.npsr):
            h = self.signal(th_cw, I) if self.cw else None
            ahat, L, _ = self.curn_moments(I, self.curn_prior_var(I, rho, kappa, kdm), beta, h)
            a[I] = ahat + L @ Z[I]
            Ls.append(L)
        return a, Ls

    def log_det_phi(self, rho, kappa, kdm) -> float:
        """log det phi over all coefficient columns (two per bin)."""
        ld = 0.0
        for k in range(self.na):
            ld += 2.0 * np.linalg.slogdet(self.phi_bin(rho[k], kappa[:, k]))[1]
        for I in range(self.npsr):
            for k in range(self.n_dm):
                ld += 2.0 * math.log(kdm[I, k])
        return ld

    def _logp_curn(self, x, beta, lpt):
        z_ach, z_dm, th_rn, th_dm, th_gwb, th_cw = self.unpack(x)
        rho, kappa, kdm = self.spectra(th_rn, th_dm, th_gwb)
        a, Ls = self.curn_transform(z_ach, z_dm, rho, kappa, kdm, beta, th_cw)
        chi2 = 0.0
        for I in range(self.npsr):
            r = self.dt_ns[I] - self.get_F(I) @ a[I] - self.signal(th_cw, I)
            chi2 += r @ ntilde_inv_woodbury(self.Nvar[I], self.psrs[I].M, r)
        logdetL = sum(float(np.sum(np.log(np.diag(L)))) for L in Ls)
        return (-0.5 * beta * chi2 - 0.5 * self._a_phi_a(a, rho, kappa, kdm)
                - 0.5 * self.log_det_phi(rho, kappa, kdm) + logdetL + lpt)

    def spectra_tangent(self, j, rho, kappa, kdm):
        """d(rho, kappa, kappa^DM) / d x_j for a hyper-parameter index j (closed forms of
        the power law and the free spectrum); None if x_j is not a spectral parameter."""
        o, npsr = self.lay, self.npsr
        drho, dkap, dkdm = np.zeros(self.na), np.zeros((npsr, self.na)), np.zeros((npsr, self.n_dm))
        ks = np.arange(1, self.na + 1)
        lnf = np.log(ks / self.T / F_YR)
        if o["th_rn"] <= j < o["th_rn"] + self.nthr * npsr:
            I, q = divmod(j - o["th_rn"], self.nthr)
            if self.rn_free:
                dkap[I, q] = LN10 * kappa[I, q]
            else:
                dkap[I] = (2 * LN10 if q == 0 else -lnf) * kappa[I]
        elif self.n_dm and o["th_dm"] <= j < o["th_dm"] + 2 * npsr:
            I, q = divmod(j - o["th_dm"], 2)
            lnfd = np.log(np.arange(1, self.n_dm + 1) / self.T / F_YR)
            dkdm[I] = (2 * LN10 if q == 0 else -lnfd) * kdm[I]
        elif o["th_gwb"] <= j < o["th_gwb"] + self.nthg:
            q = j - o["th_gwb"]
            if self.gwb_free:
                drho[q] = LN10 * rho[q]
            else:
                drho = (2 * LN10 if q == 0 else -lnf) * rho
        else:
            return None
        return drho, dkap, dkdm

    def _grad_curn(self, x, beta):
        """Gradient under the CURN transform.  z-block: d logp / d z_I = L_I^T gbar_I
        with gbar = beta F^T N~^-1 r - phi^-1 a (likelihood and HD prior in a).
        Hyper-parameters: the forward-mode derivative along each spectral parameter:
        at fixed a, 1/2 v^T dphi v - 1/2 tr(phi^-1 dphi) (v = phi^-1 a); through
        a(eta) = ahat + L z, gbar . da with dSigma = -Sigma dSigma^-1 Sigma,
        dL = chol_tangent(L, dSigma), dahat = beta dSigma F^T N~^-1 dt; and
        d log det L = tr(L^-1 dL).
        With the deterministic signal (Eq. decenter_det_PTA) the mean abar_I depends on the
        CW parameters too: d logp = beta w~ . dh + gbar_I . dabar_I with
        dabar_I = -beta Sigma_I F_I^T N~_I^-1 dh_I, dh by complex-step differentiation of
        ``cw_signal``; the mean's spectral tangent uses F^T N~^-1 (dt - h)."""
        g = np.zeros(self.D)
        if not math.isfinite(self.log_prior_theta(x)):
            return g
        z_ach, z_dm, th_rn, th_dm, th_gwb, th_cw = self.unpack(x)
        rho, kappa, kdm = self.spectra(th_rn, th_dm, th_gwb)
        npsr, na, nd, P = self.npsr, self.na, self.n_dm, self.P
        Z = self.z_per_pulsar(z_ach, z_dm)
        mom = []
        a = np.zeros((npsr, P))
        for I in range(npsr):
            phiC = self.curn_prior_var(I, rho, kappa, kdm)
            h = self.signal(th_cw, I) if self.cw else None
            ahat, L, Sigma = self.curn_moments(I, phiC, beta, h)
            a[I] = ahat + L @ Z[I]
            FNd = self.curn_fixed(I)[1]
            if h is not None:
                FNd = FNd - self.get_F(I).T @ ntilde_inv_woodbury(self.Nvar[I], self.psrs[I].M, h)
            mom.append((phiC, L, Sigma, FNd))
        gbar = np.zeros((npsr, P))
        wts = []
        for I in range(npsr):
            r = self.dt_ns[I] - self.get_F(I) @ a[I] - self.signal(th_cw, I)
            wts.append(ntilde_inv_woodbury(self.Nvar[I], self.psrs[I].M, r))
            gbar[I] = beta * (self.get_F(I).T @ wts[I])
        Phis = [self.phi_bin(rho[k], kappa[:, k]) for k in range(na)]
        v = np.zeros((npsr, P))
        for k in range(na):
            for c in range(2):
                v[:, 2 * k + c] = np.linalg.solve(Phis[k], a[:, 2 * k + c])
        for I in range(npsr):
            for k in range(nd):
                v[I, 2 * na + 2 * k: 2 * na + 2 * k + 2] = a[I, 2 * na + 2 * k: 2 * na + 2 * k + 2] / kdm[I, k]
        gbar -= v
        # z block, scattered back to the parameter layout
        GZ = np.array([mom[I][1].T @ gbar[I] for I in range(npsr)])
        o = self.lay
        gz = np.zeros((na, 2, npsr))
        for k in range(na):
            for c in range(2):
                gz[k, c] = GZ[:, 2 * k + c]
        g[: o["z_dm"]] = gz.reshape(-1)
        if nd:
            g[o["z_dm"]: o["dz"]] = GZ[:, 2 * na:].reshape(npsr, nd, 2).reshape(-1)
        for j in range(o["dz"], self.D):
            tan = self.spectra_tangent(j, rho, kappa, kdm)
            if tan is None:
                continue
            drho, dkap, dkdm = tan
            d = 0.0
            for k in range(na):  # HD prior at fixed a
                dPhi = drho[k] * self.Gamma + np.diag(dkap[:, k])
                if not np.any(dPhi):
                    continue
                for c in range(2):
                    d += 0.5 * v[:, 2 * k + c] @ dPhi @ v[:, 2 * k + c]
                d -= np.trace(np.linalg.solve(Phis[k], dPhi))
            for I in range(npsr):
                for k in range(nd):
                    if dkdm[I, k]:
                        vv = v[I, 2 * na + 2 * k: 2 * na + 2 * k + 2]
                        d += 0.5 * dkdm[I, k] * (vv @ vv) - dkdm[I, k] / kdm[I, k]
            for I in range(npsr):  # the transform a(eta) and log det L
                dphiC = self.curn_prior_var(I, drho, dkap, dkdm)
                if not np.any(dphiC):
                    continue
                phiC, L, Sigma, FNd = mom[I]
                dSinv = -dphiC / phiC ** 2                 # d(phi_CURN^-1), diagonal
                dSigma = -(Sigma * dSinv[None, :]) @ Sigma
                dL = chol_tangent(L, dSigma)
                da = beta * dSigma @ FNd + dL @ Z[I]
                d += gbar[I] @ da + np.trace(sla.solve_triangular(L, dL, lower=True))
            g[j] = d
        if self.cw:
            hstep = 1e-30
            for j in range(8 + 2 * npsr):
                pulsars = range(npsr) if j < 8 else [(j - 8) // 2]
                acc = 0.0
                for I in pulsars:
                    th8, dist, pph = self.cw_th(th_cw, I)
                    th8c = np.array(th8, dtype=complex)
                    dist_c, pph_c = complex(dist), complex(pph)
                    if j < 8:
                        th8c[j] += 1j * hstep
                    elif (j - 8) % 2 == 0:
                        dist_c += 1j * hstep
                    else:
                        pph_c += 1j * hstep
                    ds = np.imag(cw_signal(self.t_rel[I], self.psrs[I].pos, th8c, dist_c, pph_c)) / hstep
                    Fds = self.get_F(I).T @ ntilde_inv_woodbury(self.Nvar[I], self.psrs[I].M, ds)
                    acc += beta * (wts[I] @ ds) - beta * (gbar[I] @ (mom[I][2] @ Fds))
                g[o["th_cw"] + j] = acc
            for I in range(npsr):
                g[o["th_cw"] + 8 + 2 * I] += -(th_cw[8 + 2 * I] - self.psrs[I].dist_kpc) / DIST_SIGMA_KPC ** 2
        return g

    # -- deterministic signal ---------------------------------------------------
    def cw_th(self, th_cw, I):
        return th_cw[:8], th_cw[8 + 2 * I], th_cw[9 + 2 * I]

    def signal(self, th_cw, I):
        if not self.cw:
            return 0.0
        th8, dist, pph = self.cw_th(th_cw, I)
        return cw_signal(self.t_rel[I], self.psrs[I].pos, th8, dist, pph)

    # -- log posterior ----------------------------------------------------------
    def residuals(self, x, beta: float = 1.0):
        """Residuals r_I = dt_I - F_I a_I - h_I(theta) with a from the chosen
        standardizing transform (the CURN transform depends on beta when tempered)."""
        z_ach, z_dm, th_rn, th_dm, th_gwb, th_cw = self.unpack(x)
        rho, kappa, kdm = self.spectra(th_rn, th_dm, th_gwb)
        if self.transform_kind == "curn":
            a, Ls = self.curn_transform(z_ach, z_dm, rho, kappa, kdm, beta, th_cw)
        else:
            a, Ls = self.transform(z_ach, z_dm, rho, kappa, kdm)
        rs = [self.dt_ns[I] - self.get_F(I) @ a[I] - self.signal(th_cw, I) for I in range(self.npsr)]
        return rs, a, Ls, (rho, kappa, kdm)

    def chi2_terms(self, x, beta: float = 1.0):
        """Per-pulsar r_I^T N~_I^-1 r_I with r_I = dt_I - F_I a_I - h_I(theta)."""
        rs, *_ = self.residuals(x, beta)
        out = np.zeros(self.npsr)
        for I in range(self.npsr):
            wt = ntilde_inv_woodbury(self.Nvar[I], self.psrs[I].M, rs[I])
            out[I] = rs[I] @ wt
        return out

    def log_prior_theta(self, x) -> float:
        if not self.in_prior(x):
            return -math.inf
        lp = 0.0
        if self.cw:
            th_cw = self.unpack(x)[5]
            for I in range(self.npsr):
                d = (th_cw[8 + 2 * I] - self.psrs[I].dist_kpc) / DIST_SIGMA_KPC
                lp += -0.5 * d * d
        return lp

    def logp(self, x, beta: float = 1.0) -> float:
        """Canonical log posterior (the quantity the GPU path computes):
        -1/2 sum_I chi2_I - 1/2 |z|^2 + log p(theta), data-only constants dropped.
        Under the prior-whitened transform the Gaussian prior on a and the Jacobian
        det L combine to -1/2 |z|^2 - (D_z/2) log 2 pi (constant dropped here).
        beta < 1: the tempered posterior of Eq. (tempered_post), the likelihood raised
        to the power beta (its chi2 term scaled by beta), prior unchanged."""
        lpt = self.log_prior_theta(x)
        if not math.isfinite(lpt):
            return -math.inf
        x = np.asarray(x, dtype=np.float64)
        if self.transform_kind == "curn":
            return self._logp_curn(x, beta, lpt)
        z = x[: self.Dz]
        return -0.5 * beta * float(self.chi2_terms(x).sum()) - 0.5 * float(z @ z) + lpt

    def data_constant(self) -> float:
        """-1/2 sum_I [log det(2 pi N_I) + log det(M_I^T N_I^-1 M_I) - m_I log 2 pi]
        (the flat-prior integral over the timing-model offsets of Eq. likelihood)."""
        c = 0.0
        for I, p in enumerate(self.psrs):
            Nv = self.Nvar[I]
            M = p.M
            K = M.T @ (M / Nv[:, None])
            sign, ld = np.linalg.slogdet(K)
            c += -0.5 * (np.sum(np.log(2 * math.pi * Nv)) + ld - M.shape[1] * math.log(2 * math.pi))
        return c

    def logp_full(self, x) -> float:
        """Normalised log density in (z, theta) at fixed theta: logp + data_constant
        - (D_z/2) log 2 pi, with the prior on a and the Jacobian written out literally:
        log N(a; 0, phi) + log det L (Eqs. a_prior, standardized_density).  Under the CURN
        transform ``logp`` already carries the prior on a and det L_CURN literally."""
        x = np.asarray(x, dtype=np.float64)
        if self.transform_kind == "curn":
            return self.logp(x) + self.data_constant() - 0.5 * self.Dz * math.log(2 * math.pi)
        z_ach, z_dm, th_rn, th_dm, th_gwb, th_cw = self.unpack(x)
        rho, kappa, kdm = self.spectra(th_rn, th_dm, th_gwb)
        a, Ls = self.transform(z_ach, z_dm, rho, kappa, kdm)
        lp_a = 0.0
        logdetL = 0.0
        for k in range(self.na):
            Phi = self.phi_bin(rho[k], kappa[:, k])
            sign, ld = np.linalg.slogdet(2 * math.pi * Phi)
            for c in range(2):
                ak = a[:, 2 * k + c]
                lp_a += -0.5 * ak @ np.linalg.solve(Phi, ak) - 0.5 * ld
                logdetL += np.sum(np.log(np.diag(Ls[k])))
        off = 2 * self.na
        for I in range(self.npsr):
            for k in range(self.n_dm):
                for c in range(2):
                    v = kdm[I, k]
                    ak = a[I, off + 2 * k + c]
                    lp_a += -0.5 * ak * ak / v - 0.5 * math.log(2 * math.pi * v)
                    logdetL += 0.5 * math.log(v)
        chi2 = self.chi2_terms(x).sum()
        return -0.5 * chi2 + self.data_constant() + lp_a + logdetL + self.log_prior_theta(x)

    # -- gradient (analytic chain, pinned by central differences) -----------------
    def grad(self, x, theta_only_idx=None, beta: float = 1.0) -> np.ndarray:
        """d logp / dx.  z-block: g_z = L_k^T F^T N~^-1 r - z.  Hyper-parameters: the
        chain rule through a = L(phi(eta)) z with the forward-mode Cholesky tangent for
        each spectral parameter.  CW parameters: (N~^-1 r)^T dh/dtheta with dh/dtheta
        from complex-step differentiation of ``cw_signal`` (exact to rounding).
        beta: gradient of the tempered posterior of Eq. (tempered_post), every
        likelihood derivative (d logp / d a and the CW term) scaled by beta."""
        x = np.asarray(x, dtype=np.float64)
        if self.transform_kind == "curn":
            return self._grad_curn(x, beta)
        g = np.zeros(self.D)
        if not math.isfinite(self.log_prior_theta(x)):
            return g
        z_ach, z_dm, th_rn, th_dm, th_gwb, th_cw = self.unpack(x)
        rs, a, Ls, (rho, kappa, kdm) = self.residuals(x)
        npsr, na, nd = self.npsr, self.na, self.n_dm
        ghat = np.zeros((npsr, self.P))
        wts = []
        for I in range(npsr):
            wt = ntilde_inv_woodbury(self.Nvar[I], self.psrs[I].M, rs[I])
            wts.append(wt)
            ghat[I] = beta * (self.get_F(I).T @ wt)              # d logp / d a_I
        o = self.lay
        gz = np.zeros((na, 2, npsr))
        for k in range(na):
            for c in range(2):
                gz[k, c] = Ls[k].T @ ghat[:, 2 * k + c] - z_ach[k, c]
        g[: o["z_dm"]] = gz.reshape(-1)
        if nd:
            gzd = np.zeros((npsr, nd, 2))
            for I in range(npsr):
                for k in range(nd):
                    for c in range(2):
                        gzd[I, k, c] = (math.sqrt(kdm[I, k]) * ghat[I, 2 * na + 2 * k + c]
                                        - z_dm[I, k, c])
            g[o["z_dm"]: o["dz"]] = gzd.reshape(-1)
        # d logp / d rho_k and d logp / d kappa_Ik via dL = chol_tangent(L, dPhi)
        d_rho = np.zeros(na)
        d_kap = np.zeros((npsr, na))
        for k in range(na):
            Lk = Ls[k]
            def dir_deriv(dPhi):
                dL = chol_tangent(Lk, dPhi)
                return sum(ghat[:, 2 * k + c] @ (dL @ z_ach[k, c]) for c in range(2))
            if k < self.n_gwb:
                d_rho[k] = dir_deriv(self.Gamma)
            if k < self.n_rn:
                for I in range(npsr):
                    E = np.zeros((npsr, npsr))
                    E[I, I] = 1.0
                    d_kap[I, k] = dir_deriv(E)
        ks = np.arange(1, na + 1)
        lnf = np.log(ks / self.T / F_YR)
        # rho = A^2 ... f^-gamma: d rho/d log10A = 2 ln10 rho, d rho/d gamma = -ln(f/f_yr) rho;
        # free spectrum rho_k = 10^theta_k: d rho_k / d theta_k = ln10 rho_k
        if self.gwb_free:
            g[o["th_gwb"]: o["th_gwb"] + self.n_gwb] = (d_rho * LN10 * rho)[: self.n_gwb]
        else:
            g[o["th_gwb"]] = np.sum(d_rho * 2 * LN10 * rho)
            g[o["th_gwb"] + 1] = np.sum(d_rho * (-lnf) * rho)
        for I in range(npsr):
            if self.rn_free:
                g[o["th_rn"] + self.n_rn * I: o["th_rn"] + self.n_rn * (I + 1)] = \
                    (d_kap[I] * LN10 * kappa[I])[: self.n_rn]
            else:
                g[o["th_rn"] + 2 * I] = np.sum(d_kap[I] * 2 * LN10 * kappa[I])
                g[o["th_rn"] + 2 * I + 1] = np.sum(d_kap[I] * (-lnf) * kappa[I])
        if nd:
            kd = np.arange(1, nd + 1)
            lnfd = np.log(kd / self.T / F_YR)
            for I in range(npsr):
                # a = sqrt(kdm) z  =>  d logp / d kdm = ghat z / (2 sqrt(kdm))
                gz_dm = ghat[I, 2 * na:].reshape(nd, 2)
                dk = (gz_dm * z_dm[I]).sum(1) / (2.0 * np.sqrt(kdm[I]))
                g[o["th_dm"] + 2 * I] = np.sum(dk * 2 * LN10 * kdm[I])
                g[o["th_dm"] + 2 * I + 1] = np.sum(dk * (-lnfd) * kdm[I])
        if self.cw:
            h = 1e-30
            for j in range(8 + 2 * npsr):
                pulsars = range(npsr) if j < 8 else [(j - 8) // 2]
                acc = 0.0
                for I in pulsars:
                    th8, dist, pph = self.cw_th(th_cw, I)
                    th8c = np.array(th8, dtype=complex)
                    dist_c, pph_c = complex(dist), complex(pph)
                    if j < 8:
                        th8c[j] += 1j * h
                    elif (j - 8) % 2 == 0:
                        dist_c += 1j * h
                    else:
                        pph_c += 1j * h
                    ds = np.imag(cw_signal(self.t_rel[I], self.psrs[I].pos, th8c, dist_c, pph_c)) / h
                    acc += beta * (wts[I] @ ds)  # r = dt - F a - h  =>  d(-chi2/2) = +w~ . dh
                g[o["th_cw"] + j] = acc
            for I in range(npsr):
                g[o["th_cw"] + 8 + 2 * I] += -(th_cw[8 + 2 * I] - self.psrs[I].dist_kpc) / DIST_SIGMA_KPC ** 2
        return g

    # -- brute-force and alternative forms for pins -------------------------------
    def dense_marginal(self, x) -> float:
        """Time-domain Gaussian marginal likelihood with the Fourier coefficients and
        the timing-model offsets integrated out (flat prior on the offsets):
        log N(dt; 0, C) with C = N + F phi F^T and the standard TM marginal,
        -1/2 dt^T (C^-1 - C^-1 M (M^T C^-1 M)^-1 M^T C^-1) dt - 1/2 log det 2 pi C
        - 1/2 log det(M^T C^-1 M) + (m/2) log 2 pi.  Dense over all TOAs."""
        z_ach, z_dm, th_rn, th_dm, th_gwb, th_cw = self.unpack(x)
        rho, kappa, kdm = self.spectra(th_rn, th_dm, th_gwb)
        npsr, na, nd = self.npsr, self.na, self.n_dm
        ns = [p.n for p in self.psrs]
        offs = np.concatenate([[0], np.cumsum(ns)])
        ntot = offs[-1]
        Ptot = npsr * self.P
        Fbig = np.zeros((ntot, Ptot))
        for I in range(npsr):
            Fbig[offs[I]: offs[I + 1], I * self.P:(I + 1) * self.P] = self.get_F(I)
        phi = np.zeros((Ptot, Ptot))
        for I in range(npsr):
            for J in range(npsr):
                for k in range(na):
                    v = rho[k] * self.Gamma[I, J] + (kappa[I, k] if I == J else 0.0)
                    for c in range(2):
                        phi[I * self.P + 2 * k + c, J * self.P + 2 * k + c] = v
            for k in range(nd):
                for c in range(2):
                    q = I * self.P + 2 * na + 2 * k + c
                    phi[q, q] = kdm[I, k]
        C = Fbig @ phi @ Fbig.T + np.diag(np.concatenate(self.Nvar))
        mtot = sum(p.M.shape[1] for p in self.psrs)
        Mbig = np.zeros((ntot, mtot))
        mo = 0
        for I, p in enumerate(self.psrs):
            Mbig[offs[I]: offs[I + 1], mo: mo + p.M.shape[1]] = p.M
            mo += p.M.shape[1]
        dt = np.concatenate([self.dt_ns[I] - (self.signal(th_cw, I) if self.cw else 0.0)
                             for I in range(npsr)])
        cf = sla.cho_factor(C, lower=True)
        Ci_dt = sla.cho_solve(cf, dt)
        Ci_M = sla.cho_solve(cf, Mbig)
        MCM = Mbig.T @ Ci_M
        quad = dt @ Ci_dt - (Mbig.T @ Ci_dt) @ np.linalg.solve(MCM, Mbig.T @ Ci_dt)
        logdetC = 2.0 * np.sum(np.log(np.diag(cf[0])))
        s2, ldM = np.linalg.slogdet(MCM)
        return (-0.5 * quad - 0.5 * (ntot * math.log(2 * math.pi) + logdetC) - 0.5 * ldM
                + 0.5 * mtot * math.log(2 * math.pi))

    def raw_posterior_exponent(self, a_all, x):
        """Exponent of Eq. (raw_posterior) at coefficients a_all[I][P] (theta from x):
        -1/2 (dt - F a)^T N~^-1 (dt - F a) - 1/2 a^T phi^-1 a."""
        _, _, th_rn, th_dm, th_gwb, _ = self.unpack(x)
        rho, kappa, kdm = self.spectra(th_rn, th_dm, th_gwb)
        q = 0.0
        for I in range(self.npsr):
            r = self.dt_ns[I] - self.get_F(I) @ a_all[I]
            q += r @ ntilde_inv_woodbury(self.Nvar[I], self.psrs[I].M, r)
        q += self._a_phi_a(a_all, rho, kappa, kdm)
        return -0.5 * q

    def _a_phi_a(self, a_all, rho, kappa, kdm):
        q = 0.0
        for k in range(self.na):
            Phi = self.phi_bin(rho[k], kappa[:, k])
            for c in range(2):
                ak = a_all[:, 2 * k + c]
                q += ak @ np.linalg.solve(Phi, ak)
        for I in range(self.npsr):
            for k in range(self.n_dm):
                for c in range(2):
                    q += a_all[I, 2 * self.na + 2 * k + c] ** 2 / kdm[I, k]
        return q

    def gram_posterior_exponent(self, a_all, x):
        """Exponent of Eq. (stochastic_posterior): -1/2 (a - ahat)^T Sigma^-1 (a - ahat)
        + 1/2 ahat^T Sigma^-1 ahat with Sigma^-1 = F^T N~^-1 F + phi^-1 and
        ahat = Sigma F^T N~^-1 dt (the dt^T N~^-1 dt term dropped)."""
        _, _, th_rn, th_dm, th_gwb, _ = self.unpack(x)
        rho, kappa, kdm = self.spectra(th_rn, th_dm, th_gwb)
        npsr, P = self.npsr, self.P
        Ptot = npsr * P
        FNF = np.zeros((Ptot, Ptot))
        FNd = np.zeros(Ptot)
        for I in range(npsr):
            F = self.get_F(I)
            NF = ntilde_inv_woodbury(self.Nvar[I], self.psrs[I].M, F)
            FNF[I * P:(I + 1) * P, I * P:(I + 1) * P] = F.T @ NF
            FNd[I * P:(I + 1) * P] = NF.T @ self.dt_ns[I]
        phi = np.zeros((Ptot, Ptot))
        for I in range(npsr):
            for J in range(npsr):
                for k in range(self.na):
                    v = rho[k] * self.Gamma[I, J] + (kappa[I, k] if I == J else 0.0)
                    for c in range(2):
                        phi[I * P + 2 * k + c, J * P + 2 * k + c] = v
            for k in range(self.n_dm):
                for c in range(2):
                    q = I * P + 2 * self.na + 2 * k + c
                    phi[q, q] = kdm[I, k]
        Sinv = FNF + np.linalg.inv(phi)
        ahat = np.linalg.solve(Sinv, FNd)
        av = a_all.reshape(-1)
        d = av - ahat
        return -0.5 * d @ Sinv @ d + 0.5 * ahat @ Sinv @ ahat


# --------------------------------------------------------------------------- #
# Counter-based random numbers (Salmon, Moraes, Dror, Shaw, "Parallel random
# numbers: as easy as 1, 2, 3", SC'11): Philox4x32 with 10 rounds.
# --------------------------------------------------------------------------- #
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
MASK32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    c0, c1, c2, c3 = (int(v) & MASK32 for v in ctr)
    k0, k1 = (int(v) & MASK32 for v in key)
    for r in range(10):
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
        if r < 9:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
    return (c0, c1, c2, c3)


def u01(w: int) -> float:
    """uint32 -> (0, 1): (w + 1/2) 2^-32."""
    return (w + 0.5) * 2.0 ** -32


def hmc_normals(seed: int, iteration: int, chain: int, D: int) -> np.ndarray:
    """Momentum draw for one chain: Philox block j has counter (j, chain, it_lo, it_hi),
    key (seed_lo, seed_hi); each block's words (w0, w1, w2, w3) give two Box-Muller
    pairs (w0, w1) and (w2, w3): n = sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b)."""
    out = np.zeros(D)
    nblk = (D + 3) // 4
    key = (seed & MASK32, (seed >> 32) & MASK32)
    for j in range(nblk):
        w = philox4x32_10((j, chain, iteration & MASK32, (iteration >> 32) & MASK32), key)
        for q in range(2):
            ua, ub = u01(w[2 * q]), u01(w[2 * q + 1])
            rad = math.sqrt(-2.0 * math.log(ua))
            for s, v in enumerate((rad * math.cos(2 * math.pi * ub), rad * math.sin(2 * math.pi * ub))):
                idx = 4 * j + 2 * q + s
                if idx < D:
                    out[idx] = v
    return out


def hmc_uniform(seed: int, iteration: int, chain: int) -> float:
    """Metropolis uniform: word 0 of the Philox block with counter (0xFFFFFFFF, chain, it)."""
    key = (seed & MASK32, (seed >> 32) & MASK32)
    w = philox4x32_10((MASK32, chain, iteration & MASK32, (iteration >> 32) & MASK32), key)
    return u01(w[0])


def hmc_trajectory(logp_grad, x0, logp0, grad0, step, n_leapfrog, p0, u, inv_mass=None, bounds=None):
    """One HMC transition (App. "Hamiltonian Monte Carlo"): Euclidean-Gaussian kinetic
    energy 1/2 p^T M^-1 p (Eq. Gaussian_momentum), H = -logp + K (Eq. Hamiltonian),
    n_leapfrog leapfrog steps of Hamilton's equations (Eq. Hamilton's_eq), accepted
    with probability min(1, exp(H0 - H1)) (Eq. HMC_acceptance) if u < that.
    bounds = (lo, hi): the coordinates with a finite box move in
    v = logit((x - lo) / (hi - lo)), x = lo + (hi - lo) sigmoid(v), and the target there is
    logp(x(v)) + sum log((hi - lo) s (1 - s)), s = sigmoid(v) (change of variables of a
    box-bounded parameter); the momentum and inv_mass refer to v for those coordinates.
    Returns (x, logp, grad, accepted)."""
    im = np.ones_like(x0) if inv_mass is None else inv_mass
    if bounds is None:
        lo = np.full_like(x0, -np.inf)
        hi = np.full_like(x0, np.inf)
    else:
        lo, hi = bounds
    m = np.isfinite(lo) & np.isfinite(hi)
    w = hi[m] - lo[m]

    def to_v(x):
        v = x.copy()
        t = (x[m] - lo[m]) / w
        v[m] = np.log(t) - np.log1p(-t)
        return v

    def to_x(v):
        x = v.copy()
        x[m] = lo[m] + w / (1.0 + np.exp(-v[m]))
        return x

    def log_jac(v):
        s = 1.0 / (1.0 + np.exp(-v[m]))
        return float(np.sum(np.log(w) + np.log(s) + np.log1p(-s)))

    def grad_v(g, v):
        s = 1.0 / (1.0 + np.exp(-v[m]))
        gv = g.copy()
        gv[m] = g[m] * w * s * (1.0 - s) + (1.0 - 2.0 * s)
        return gv

    v = to_v(x0)
    p = p0.copy()
    lp, g = logp0, grad0.copy()
    H0 = -(logp0 + log_jac(v)) + 0.5 * np.sum(p0 * p0 * im)
    for _ in range(n_leapfrog):
        p = p + 0.5 * step * grad_v(g, v)
        v = v + step * im * p
        lp, g = logp_grad(to_x(v))
        p = p + 0.5 * step * grad_v(g, v)
    H1 = -(lp + log_jac(v)) + 0.5 * np.sum(p * p * im) if math.isfinite(lp) else math.inf
    acc = math.log(u) < (H0 - H1)
    if acc:
        return to_x(v), lp, g, True
    return x0.copy(), logp0, grad0.copy(), False


# --------------------------------------------------------------------------- #
# Near-posterior evaluation points (Eq. PTA_standard_transform_curn): per pulsar,
# Sigma_CURN^-1 = F^T N~^-1 F + phi_CURN^-1 with phi_CURN the prior covariance
# without inter-pulsar correlations, a_hat = Sigma_CURN F^T N~^-1 (dt - h), and
# a = a_hat + L_CURN eps.  Returned in the z coordinates of the prior-whitened
# transform, z = L_k^-1 a per frequency bin.
# --------------------------------------------------------------------------- #
def curn_point(orc: Oracle, x, eps_scale: float = 1.0, seed: int = 0):
    x = np.asarray(x, dtype=np.float64).copy()
    rng = np.random.default_rng(seed)
    z_ach, z_dm, th_rn, th_dm, th_gwb, th_cw = orc.unpack(x)
    rho, kappa, kdm = orc.spectra(th_rn, th_dm, th_gwb)
    a = np.zeros((orc.npsr, orc.P))
    for I in range(orc.npsr):
        F = orc.get_F(I)
        NF = ntilde_inv_woodbury(orc.Nvar[I], orc.psrs[I].M, F)
        phi = np.zeros(orc.P)
        for k in range(orc.na):
            phi[2 * k: 2 * k + 2] = rho[k] + kappa[I, k]
        for k in range(orc.n_dm):
            phi[2 * orc.na + 2 * k: 2 * orc.na + 2 * k + 2] = kdm[I, k]
        Sinv = F.T @ NF + np.diag(1.0 / phi)
        d = orc.dt_ns[I] - (orc.signal(th_cw, I) if orc.cw else 0.0)
        Lc = np.linalg.cholesky(Sinv)                 # Sinv = Lc Lc^T
        ahat = sla.cho_solve((Lc, True), NF.T @ d)
        # L_CURN eps with L_CURN L_CURN^T = Sinv^-1: solve Lc^T v = eps
        a[I] = ahat + eps_scale * sla.solve_triangular(Lc.T, rng.normal(size=orc.P), lower=False)
    Ls = [np.linalg.cholesky(orc.phi_bin(rho[k], kappa[:, k])) for k in range(orc.na)]
    z = np.zeros(orc.Dz)
    za = np.zeros((orc.na, 2, orc.npsr))
    for k in range(orc.na):
        for c in range(2):
            za[k, c] = sla.solve_triangular(Ls[k], a[:, 2 * k + c], lower=True)
    z[: orc.lay["z_dm"]] = za.reshape(-1)
    if orc.n_dm:
        zd = np.zeros((orc.npsr, orc.n_dm, 2))
        for I in range(orc.npsr):
            for k in range(orc.n_dm):
                zd[I, k] = a[I, 2 * orc.na + 2 * k: 2 * orc.na + 2 * k + 2] / math.sqrt(kdm[I, k])
        z[orc.lay["z_dm"]: orc.Dz] = zd.reshape(-1)
    x[: orc.Dz] = z
    return x
