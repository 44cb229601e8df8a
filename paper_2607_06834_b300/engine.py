"""Python front end of the C ABI: a context built from a pulsar array, the batched
log posterior + gradient, HMC trajectories, and a torch.autograd.Function.

Every numerical step runs in the CUDA library; this module only marshals
arguments (torch tensors for device memory and the current stream)."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import abi


class PTAError(RuntimeError):
    pass


def _dptr(t: torch.Tensor | None):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


class Engine:
    """One finalized context.  ``arr`` exposes ``pulsars`` (toas_s, freqs_mhz, resid_s,
    sigma_s, backend, efac, equad_s, M, pos, dist_kpc) and n_gwb, n_rn, n_dm, cw."""

    def __init__(self, arr, precision: str = "fp32", device: int = 0):
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        spectrum = (1 if getattr(arr, "gwb_free", False) else 0) | (2 if getattr(arr, "rn_free", False) else 0)
        desc = abi.ModelDesc(arr.n_gwb, arr.n_rn, arr.n_dm, int(bool(arr.cw)), abi.PREC[precision], 1400.0,
                             spectrum)
        h = C.c_void_p()
        rc = abi.lib.pta_create(C.byref(h), C.byref(desc))
        if rc != 0:
            raise PTAError(f"pta_create failed ({rc})")
        self._h = h
        self.precision = precision
        self.transform = "prior"
        keep = []
        for p in arr.pulsars:
            arrs = dict(
                toas_s=np.ascontiguousarray(p.toas_s, dtype=np.float64),
                freqs_mhz=np.ascontiguousarray(p.freqs_mhz, dtype=np.float64),
                resid_s=np.ascontiguousarray(p.resid_s, dtype=np.float64),
                sigma_s=np.ascontiguousarray(p.sigma_s, dtype=np.float64),
                backend=np.ascontiguousarray(p.backend, dtype=np.int32),
                efac=np.ascontiguousarray(p.efac, dtype=np.float64),
                equad_s=np.ascontiguousarray(p.equad_s, dtype=np.float64),
                M=np.ascontiguousarray(p.M, dtype=np.float64))
            keep.append(arrs)
            pd = abi.PulsarDesc()
            pd.n, pd.m, pd.n_backend = p.M.shape[0], p.M.shape[1], len(p.efac)
            for k in ("toas_s", "freqs_mhz", "resid_s", "sigma_s", "efac", "equad_s", "M"):
                setattr(pd, k, arrs[k].ctypes.data_as(C.POINTER(C.c_double)))
            pd.backend = arrs["backend"].ctypes.data_as(C.POINTER(C.c_int32))
            pd.pos = (C.c_double * 3)(*[float(v) for v in p.pos])
            pd.dist_kpc = float(p.dist_kpc)
            self._check(abi.lib.pta_add_pulsar(self._h, C.byref(pd)), "pta_add_pulsar")
        self._check(abi.lib.pta_finalize(self._h, C.c_void_p(torch.cuda.current_stream().cuda_stream)),
                    "pta_finalize")
        lay = abi.Layout()
        self._check(abi.lib.pta_layout(self._h, C.byref(lay)), "pta_layout")
        self.layout = {f: getattr(lay, f) for f, _ in abi.Layout._fields_}
        self.D = lay.d

    def _check(self, rc, what):
        if rc != 0:
            msg = abi.lib.pta_last_error(self._h).decode()
            raise PTAError(f"{what} failed ({rc}): {msg}")

    def close(self):
        if getattr(self, "_h", None):
            abi.lib.pta_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision: str):
        self._check(abi.lib.pta_set_precision(self._h, abi.PREC[precision]), "pta_set_precision")
        self.precision = precision

    def autotune(self, B: int):
        """Time every FP32 TOA-kernel tile shape that fits this model on B chains and
        keep the fastest.  Returns (chosen entry, {entry: ms per launch})."""
        n = toa_config_count()
        ms = (C.c_double * n)()
        chosen = C.c_int(-1)
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        self._check(abi.lib.pta_autotune(self._h, int(B), stream, C.byref(chosen), ms, n), "pta_autotune")
        return chosen.value, {i: ms[i] for i in range(n) if ms[i] >= 0}

    def set_beta(self, beta):
        """Per-chain inverse temperatures for the tempered likelihood (tensor of B
        values, any device), or None to switch tempering off.  The library copies them
        on the current stream."""
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        if beta is None:
            self._check(abi.lib.pta_set_beta(self._h, 0, None, stream), "pta_set_beta")
            return
        b = beta.to(dtype=torch.float64).contiguous()
        self._beta_keep = b  # alive until the stream has copied it
        self._check(abi.lib.pta_set_beta(self._h, int(b.numel()), C.c_void_p(b.data_ptr()), stream),
                    "pta_set_beta")

    def set_transform(self, transform: str):
        """Standardizing transform of the coefficients: "prior" (a = L_phi z per
        frequency bin, the default) or "curn" (a = ahat_CURN + L_CURN z per pulsar)."""
        self._check(abi.lib.pta_set_transform(self._h, abi.TRANSFORM[transform]), "pta_set_transform")
        self.transform = transform

    def set_cholesky(self, mode: str):
        """Arithmetic of the dense-bin per-frequency Cholesky, its inverse and adjoint:
        "dw" (double-word float pairs on the FP32 pipes, the default) or "fp64".  FP64
        precision mode and the CURN transform always use FP64."""
        self._check(abi.lib.pta_set_cholesky(self._h, abi.CHOLESKY[mode]), "pta_set_cholesky")
        self.cholesky = mode

    def param_bounds(self):
        """(lo, hi) float64 arrays of the prior support of each coordinate (+-inf where
        unbounded); the HMC trajectory moves the bounded ones in logit space."""
        lo = np.empty(self.D, dtype=np.float64)
        hi = np.empty(self.D, dtype=np.float64)
        self._check(abi.lib.pta_param_bounds(self._h, C.c_void_p(lo.ctypes.data), C.c_void_p(hi.ctypes.data)),
                    "pta_param_bounds")
        return lo, hi

    def set_toa_config(self, cfg: int):
        self._check(abi.lib.pta_set_toa_config(self._h, int(cfg)), "pta_set_toa_config")

    def logp_constant(self) -> float:
        c = C.c_double()
        self._check(abi.lib.pta_logp_constant(self._h, C.byref(c)), "pta_logp_constant")
        return c.value

    def logp_and_grad(self, x: torch.Tensor, want_grad: bool = True, out=None):
        """x [B, D] float32 on the device -> (logp [B] f64, grad [B, D] f32 | None, status [B] i32)."""
        assert x.dtype == torch.float32 and x.is_cuda and x.is_contiguous() and x.shape[-1] == self.D
        B = x.shape[0]
        if out is None:
            logp = torch.empty(B, dtype=torch.float64, device=x.device)
            grad = torch.empty_like(x) if want_grad else None
            status = torch.empty(B, dtype=torch.int32, device=x.device)
        else:
            logp, grad, status = out
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        self._check(abi.lib.pta_logp_and_grad(self._h, B, _dptr(x), _dptr(logp), _dptr(grad), _dptr(status),
                                              stream), "pta_logp_and_grad")
        return logp, grad, status

    def hmc_trajectory(self, x, logp, grad, step, n_leapfrog, seed, iteration, inv_mass=None, accepted=None):
        """In-place HMC transition of the state (x, logp, grad); returns accept flags [B] i32."""
        B = x.shape[0]
        if accepted is None:
            accepted = torch.empty(B, dtype=torch.int32, device=x.device)
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        self._check(abi.lib.pta_hmc_trajectory(self._h, B, _dptr(x), _dptr(logp), _dptr(grad), _dptr(step),
                                               _dptr(inv_mass), int(n_leapfrog), int(seed), int(iteration),
                                               _dptr(accepted), stream), "pta_hmc_trajectory")
        return accepted


def toa_config_count() -> int:
    n = 0
    while abi.lib.pta_toa_config_info(n, None, None, None, None) == 0:
        n += 1
    return n


def toa_config_info(cfg: int) -> dict:
    v = [C.c_int() for _ in range(4)]
    if abi.lib.pta_toa_config_info(int(cfg), *[C.byref(x) for x in v]) != 0:
        raise IndexError(cfg)
    return dict(chains_per_cta=v[0].value, toas_per_tile=v[1].value, rows_per_thread=v[2].value,
                order=v[3].value)


class LogPosterior(torch.autograd.Function):
    """logp(x) with the library's hand-written adjoint as the backward: forward runs
    one fused evaluation and stores the gradient; backward scales it by grad_output."""

    @staticmethod
    def forward(ctx, x, engine):
        logp, grad, status = engine.logp_and_grad(x.detach().contiguous(), want_grad=True)
        ctx.save_for_backward(grad)
        return logp

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (g.to(grad.dtype)[:, None] * grad, None)
