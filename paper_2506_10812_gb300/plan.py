"""Torch-facing wrapper of the C ABI.

PyTorch supplies device memory and the CUDA stream only; every step of the
computation runs in ``libsg.so``.  Arguments are checked and passed as raw
pointers (argument marshalling only).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N

_OUT_KEYS = ("phi_g", "gr_g", "gphi_g", "phi_d", "gr_d", "gphi_d")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Plan:
    """A self-gravity plan for one grid and one pair of aspect ratios.

    Parameters follow the paper's problem: ``nr`` x ``nphi`` log-polar cells
    between the radial edges ``r_in``, ``r_out``; aspect ratios ``h_g`` and
    (optional, bi-fluid) ``h_d``; gravitational constant ``G``.  ``method``
    is ``"fft"`` (constant aspect ratios, App. C convolution), ``"direct"``
    (pair sum, optionally with scale-height fields ``H_g``, ``H_d``) or
    ``"semispectral"`` (Fourier transform in phi and direct sum in r, for
    scale heights that depend on r only: ``H_g``, ``H_d`` with constant rows,
    or the aspect ratios)."""

    def __init__(self, nr, nphi, r_in, r_out, h_g, h_d=None, G=1.0, dtype=torch.float32,
                 method="fft", H_g=None, H_d=None, check_finite=False, device=None):
        self._lib = N.load()
        dev = torch.device("cuda") if device is None else torch.device(device)
        if dev.type != "cuda":
            raise ValueError("the library runs on a CUDA device only")
        self.device = dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())
        if dtype not in (torch.float32, torch.float64):
            raise ValueError("dtype must be torch.float32 or torch.float64")
        self.dtype = dtype
        self.nr, self.nphi = int(nr), int(nphi)
        self.r_in, self.r_out = float(r_in), float(r_out)
        self.h_g = float(h_g) if h_g is not None else 0.0
        self.h_d = float(h_d) if h_d else 0.0
        self.G = float(G)
        self.method = method
        self.bifluid = self.h_d > 0 or H_d is not None
        p = N.SgParams()
        p.nr, p.nphi = self.nr, self.nphi
        p.r_in, p.r_out = self.r_in, self.r_out
        p.h_g, p.h_d = self.h_g, self.h_d
        self._H = []
        for name, H in (("H_g_field", H_g), ("H_d_field", H_d)):
            if H is not None:
                H = self._check(H, name)
                self._H.append(H)
                setattr(p, name, H.data_ptr())
        p.G = self.G
        p.dtype = N.SG_F64 if dtype == torch.float64 else N.SG_F32
        p.method = {"fft": N.SG_METHOD_FFT, "direct": N.SG_METHOD_DIRECT,
                    "semispectral": N.SG_METHOD_SEMISPECTRAL}[method]
        p.flags = N.SG_CHECK_FINITE if check_finite else 0
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self._lib.sg_plan_create(ctypes.byref(h), ctypes.byref(p), self._stream())
        N.check(st, None, "sg_plan_create")
        self._h = h
        self._H = []   # the plan keeps its own copies

    # ------------------------------------------------------------------
    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _check(self, t, name):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.device != self.device:
            raise ValueError(f"{name} must be on {self.device}, got {t.device}")
        if t.dtype != self.dtype:
            raise ValueError(f"{name} must be {self.dtype}, got {t.dtype}")
        if tuple(t.shape) != (self.nr, self.nphi):
            raise ValueError(f"{name} must have shape ({self.nr}, {self.nphi}), got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def _inputs(self, sigma_g, sigma_d):
        sigma_g = self._check(sigma_g, "sigma_g")
        if self.bifluid:
            if sigma_d is None:
                raise ValueError("bi-fluid plan needs sigma_d")
            sigma_d = self._check(sigma_d, "sigma_d")
        else:
            sigma_d = None
        return sigma_g, sigma_d

    def _alloc(self, keys):
        return {k: torch.empty((self.nr, self.nphi), dtype=self.dtype, device=self.device) for k in keys}

    def _keys(self, outputs):
        comps = tuple(outputs)
        fl = ("g", "d") if self.bifluid else ("g",)
        return [f"{c}_{f}" for f in fl for c in comps]

    # ------------------------------------------------------------------
    def solve(self, sigma_g, sigma_d=None, outputs=("phi", "gr", "gphi"), out=None):
        """Phi, g_r, g_phi of every target fluid (dict keyed ``phi_g``,
        ``gr_g``, ``gphi_g``, ``phi_d`` ...).  ``out``: optional dict of
        preallocated tensors."""
        sigma_g, sigma_d = self._inputs(sigma_g, sigma_d)
        res = dict(out) if out is not None else self._alloc(self._keys(outputs))
        for k, v in res.items():
            self._check(v, k)
        ptrs = [_ptr(res.get(k)) for k in _OUT_KEYS]
        with torch.cuda.device(self.device):
            st = self._lib.sg_solve(self._h, _ptr(sigma_g), _ptr(sigma_d), *ptrs, self._stream())
        N.check(st, self._h, "sg_solve")
        return res

    def potential(self, sigma_g, sigma_d=None):
        sigma_g, sigma_d = self._inputs(sigma_g, sigma_d)
        res = self._alloc(self._keys(("phi",)))
        with torch.cuda.device(self.device):
            st = self._lib.sg_potential(self._h, _ptr(sigma_g), _ptr(sigma_d), _ptr(res.get("phi_g")),
                                        _ptr(res.get("phi_d")), self._stream())
        N.check(st, self._h, "sg_potential")
        return res

    def accel(self, sigma_g, sigma_d=None):
        sigma_g, sigma_d = self._inputs(sigma_g, sigma_d)
        res = self._alloc(self._keys(("gr", "gphi")))
        with torch.cuda.device(self.device):
            st = self._lib.sg_accel(self._h, _ptr(sigma_g), _ptr(sigma_d), _ptr(res.get("gr_g")),
                                    _ptr(res.get("gphi_g")), _ptr(res.get("gr_d")), _ptr(res.get("gphi_d")),
                                    self._stream())
        N.check(st, self._h, "sg_accel")
        return res

    def indirect(self, sigma_g, sigma_d=None):
        """Indirect-term sums (App. E) per source fluid: float64 tensor
        [[A_g, B_g], ([A_d, B_d])] on the plan's device."""
        sigma_g, sigma_d = self._inputs(sigma_g, sigma_d)
        out = torch.empty((2 if self.bifluid else 1, 2), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            st = self._lib.sg_indirect(self._h, _ptr(sigma_g), _ptr(sigma_d), _ptr(out), self._stream())
        N.check(st, self._h, "sg_indirect")
        return out

    def kernel_table(self, pair=N.SG_PAIR_GG, comp=N.SG_COMP_R):
        """Real-space lattice kernel [2 nr, nphi] of one ordered pair (App. C)."""
        out = torch.empty((2 * self.nr, self.nphi), dtype=self.dtype, device=self.device)
        with torch.cuda.device(self.device):
            st = self._lib.sg_kernel_table(self._h, int(pair), int(comp), _ptr(out), self._stream())
        N.check(st, self._h, "sg_kernel_table")
        return out

    def solve_host(self, sigma_g, sigma_d=None, outputs=("phi", "gr", "gphi"), out=None):
        """Same as ``solve`` with host (numpy / CPU tensor) buffers; the
        library copies in, solves and copies back (synchronous)."""
        npdt = np.float64 if self.dtype == torch.float64 else np.float32
        keys = self._keys(outputs)
        if out is None:
            out = {k: np.empty((self.nr, self.nphi), dtype=npdt) for k in keys}

        def hptr(a, name):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                if a.device.type != "cpu" or a.dtype != self.dtype or not a.is_contiguous():
                    raise ValueError(f"{name}: need a contiguous CPU tensor of {self.dtype}")
                return ctypes.c_void_p(a.data_ptr())
            if a.dtype != npdt or not a.flags.c_contiguous or a.shape != (self.nr, self.nphi):
                raise ValueError(f"{name}: need a C-contiguous {npdt.__name__} array ({self.nr}, {self.nphi})")
            return ctypes.c_void_p(a.ctypes.data)

        if self.bifluid and sigma_d is None:
            raise ValueError("bi-fluid plan needs sigma_d")
        ptrs = [hptr(out.get(k), k) for k in _OUT_KEYS]
        with torch.cuda.device(self.device):
            st = self._lib.sg_solve_host(self._h, hptr(sigma_g, "sigma_g"),
                                         hptr(sigma_d if self.bifluid else None, "sigma_d"), *ptrs,
                                         self._stream())
        N.check(st, self._h, "sg_solve_host")
        return out

    def set_column_engine(self, engine):
        """Column-pass engine: "fft32" (default) or a tensor-core DFT engine
        ("dft_fp16x3", "dft_bf16x3", "dft_fp16", "dft_bf16")."""
        with torch.cuda.device(self.device):
            st = self._lib.sg_set_column_engine(self._h, N.ENGINES[engine])
        N.check(st, self._h, "sg_set_column_engine")

    @property
    def tiles(self):
        """Launch tiles: {"rows_fwd": 2|4, "rows_inv": 2|4, "cols_staging": "all"|"step"}."""
        t = N.SgTiles()
        N.check(self._lib.sg_get_tiles(self._h, ctypes.byref(t)), self._h, "sg_get_tiles")
        names = {v: k for k, v in N.COLS_STAGING.items()}
        return {"rows_fwd": t.rows_fwd, "rows_inv": t.rows_inv, "cols_staging": names[t.cols_staging]}

    def set_tiles(self, rows_fwd=None, rows_inv=None, cols_staging=None):
        """Set any of the launch tiles (the others keep their values)."""
        cur = self.tiles
        t = N.SgTiles(rows_fwd if rows_fwd is not None else cur["rows_fwd"],
                      rows_inv if rows_inv is not None else cur["rows_inv"],
                      N.COLS_STAGING[cols_staging if cols_staging is not None else cur["cols_staging"]])
        with torch.cuda.device(self.device):
            st = self._lib.sg_set_tiles(self._h, ctypes.byref(t))
        N.check(st, self._h, "sg_set_tiles")

    def sync(self):
        with torch.cuda.device(self.device):
            st = self._lib.sg_sync(self._h, self._stream())
        N.check(st, self._h, "sg_sync")

    def launches_per_solve(self, outputs=("phi", "gr", "gphi")):
        mask = 0
        for b in range(2 if self.bifluid else 1):
            for c, name in enumerate(("phi", "gr", "gphi")):
                if name in outputs:
                    mask |= 1 << (3 * b + c)
        return int(self._lib.sg_launches_per_solve(self._h, mask))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
