"""FP64 CPU oracle for the thin-disc self-gravity field -- TEST INFRASTRUCTURE.

This package is the plain, slow, obviously-correct reference that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import it; the product path
never does.  It shares no code with the CUDA library and imports nothing from
it.

Paper: Rendon Restrepo, Rometsch, Ziegler & Gressel (2025), "Self-gravity in
thin protoplanetary discs 1: the smoothing-length approximation versus the
exact self-gravity kernel".

Two evaluations of the same finite sum are provided:

``direct``  the definition, Sec. 2.2 Eq. "volume force 2D" (divided by
            Sigma_b) with Eq. "SG force kernel exact" and Eq. "mean root
            square height", and Sec. 5.6 Eq. "grav. potential 2D", summed
            over all source cells (self cell excluded), in C with
            Kahan-compensated FP64 accumulation (``sg_oracle.c``).
``indirect`` the indirect-term sums A, B of App. E (Sec. 5.4).
``fft64``   the paper's fast algorithm, Sec. 5.2 and App. C: the convolution
            kernels K_r, K_phi on the log-polar lattice, radial zero padding
            to 2 N_r, FP64 FFTs (numpy).  The potential uses the same
            lattice form of Eq. "grav. potential 2D".

Discretisation reading (the paper does not state one): radial cell edges
r_in, r_out, log-spaced; centres u_i = ln r_in + (i + 1/2) du, phi_j =
(j + 1/2) dphi; cell mass Sigma r^2 du dphi (midpoint rule); the self cell
is excluded for every fluid pair.  Under this reading ``direct`` and
``fft64`` are the same sum and agree to FP64 rounding.

Outputs are accelerations (force per unit mass of the target fluid) summed
over the source fluids, and the potential Phi^{gb} + Phi^{db}.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(closed forms, limits, quadrature of the paper's general kernel, brute force
with mpmath); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None

SQRT_PI = np.sqrt(np.pi)


def build(force: bool = False) -> str:
    """Compile ``sg_oracle.c`` with gcc (FP64, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _get_lib():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_k0e_D.argtypes = [ctypes.c_int64, dp, dp, dp]
        lib.oracle_k0e_D.restype = None
        lib.oracle_direct_pair.argtypes = [ctypes.c_int64, dp, dp, dp, dp,
                                           ctypes.c_int64, dp, dp, dp, i64p,
                                           ctypes.c_double, dp, dp, dp]
        lib.oracle_direct_pair.restype = None
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Scaled Bessel functions and the pointwise kernels
# --------------------------------------------------------------------------
def k0e_D(x):
    """Return (e^x K0(x), e^x [K1(x) - K0(x)]) by trapezoidal quadrature of
    the integral representation DLMF 10.32.9 (see ``sg_oracle.c``).  App. A
    of the paper: F_0(x) = e^{x/4} K0(x/4), F_1(x) = D(x/4) / 2."""
    x = _c64(x)
    shp = x.shape
    x = x.ravel()
    k0 = np.empty_like(x)
    d = np.empty_like(x)
    _get_lib().oracle_k0e_D(x.size, _dp(x), _dp(k0), _dp(d))
    return k0.reshape(shp), d.reshape(shp)


def kernel_K(s, Ha, Hb):
    """Sec. 2.2, Eq. "SG force kernel exact": K_ab(s) for source scale height
    Ha and target scale height Hb (Eq. "mean root square height")."""
    s = np.asarray(s, dtype=np.float64)
    Hab2 = 0.5 * (np.asarray(Ha, dtype=np.float64) ** 2 + np.asarray(Hb, dtype=np.float64) ** 2)
    d = s / np.sqrt(Hab2)
    X = d * d / 8.0
    _, D = k0e_D(X)
    return (1.0 / SQRT_PI) / Hab2 * (d / 8.0) * D


def kernel_P(s, Ha, Hb):
    """Sec. 5.6, Eq. "grav. potential 2D" integrand without -Sigma_a:
    e^X K0(X) / (2 sqrt(pi) H_ab)."""
    s = np.asarray(s, dtype=np.float64)
    Hab = np.sqrt(0.5 * (np.asarray(Ha, dtype=np.float64) ** 2 + np.asarray(Hb, dtype=np.float64) ** 2))
    d = s / Hab
    k0, _ = k0e_D(d * d / 8.0)
    return k0 / (2.0 * SQRT_PI * Hab)


# --------------------------------------------------------------------------
# Grid
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Grid:
    """Log-polar grid: nr cells log-spaced between the radial edges r_in,
    r_out; nphi cells uniform in phi (Sec. 4.1, App. C)."""
    nr: int
    nphi: int
    r_in: float
    r_out: float

    @property
    def du(self):
        return np.log(self.r_out / self.r_in) / self.nr

    @property
    def dphi(self):
        return 2.0 * np.pi / self.nphi

    @property
    def r(self):
        return self.r_in * np.exp((np.arange(self.nr) + 0.5) * self.du)

    @property
    def phi(self):
        return (np.arange(self.nphi) + 0.5) * self.dphi

    def mesh(self):
        return np.meshgrid(self.r, self.phi, indexing="ij")


def _scale_height(grid, H, h):
    if H is not None:
        H = _c64(H)
        assert H.shape == (grid.nr, grid.nphi)
        return H
    R, _ = grid.mesh()
    return h * R


# --------------------------------------------------------------------------
# Direct pair sum (the definition)
# --------------------------------------------------------------------------
def direct_points(grid, sigmas, Hs, tx, ty, tH, tskip=None, G=1.0):
    """Direct sum at arbitrary target points.

    sigmas, Hs: lists over source fluids of [nr, nphi] surface densities and
    scale heights.  tx, ty, tH: target positions and the target fluid's scale
    height there.  Returns (phi, gx, gy), summed over the source fluids."""
    lib = _get_lib()
    R, P = grid.mesh()
    sx = _c64((R * np.cos(P)).ravel())
    sy = _c64((R * np.sin(P)).ravel())
    tx, ty, tH = _c64(tx).ravel(), _c64(ty).ravel(), _c64(tH).ravel()
    n = tx.size
    phi = np.zeros(n)
    gx = np.zeros(n)
    gy = np.zeros(n)
    skip = None
    if tskip is not None:
        skip = np.ascontiguousarray(tskip, dtype=np.int64).ravel()
    for sig, H in zip(sigmas, Hs):
        m = _c64((_c64(sig) * R * R * grid.du * grid.dphi).ravel())
        sH = _c64(H).ravel()
        lib.oracle_direct_pair(sx.size, _dp(sx), _dp(sy), _dp(m), _dp(sH),
                               n, _dp(tx), _dp(ty), _dp(tH),
                               None if skip is None else skip.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               float(G), _dp(phi), _dp(gx), _dp(gy))
    return phi, gx, gy


def direct(grid, sigma_g, sigma_d=None, h_g=None, h_d=None, H_g=None, H_d=None,
           G=1.0, targets=None):
    """Direct O(N^2) sum on the grid (Sec. 2.2 and Sec. 5.6 equations).

    Scale heights: either constant aspect ratios h_g, h_d (H = h r) or
    general fields H_g, H_d of shape [nr, nphi].  ``targets``: optional flat
    cell indices (sampled mode).  Returns a dict with keys phi_g, gr_g,
    gphi_g (and phi_d, gr_d, gphi_d when sigma_d is given), each [nr, nphi]
    or, in sampled mode, 1-D over ``targets``."""
    Hg = _scale_height(grid, H_g, h_g)
    sigmas, Hs = [sigma_g], [Hg]
    fluids = [("g", Hg)]
    if sigma_d is not None:
        Hd = _scale_height(grid, H_d, h_d)
        sigmas.append(sigma_d)
        Hs.append(Hd)
        fluids.append(("d", Hd))
    R, P = grid.mesh()
    idx = np.arange(grid.nr * grid.nphi) if targets is None else np.asarray(targets, dtype=np.int64)
    x = (R * np.cos(P)).ravel()[idx]
    y = (R * np.sin(P)).ravel()[idx]
    c = np.cos(P).ravel()[idx]
    s = np.sin(P).ravel()[idx]
    out = {}
    for name, Hb in fluids:
        phi, gx, gy = direct_points(grid, sigmas, Hs, x, y, Hb.ravel()[idx], tskip=idx, G=G)
        gr = gx * c + gy * s                  # e_r = (cos phi, sin phi)
        gp = -gx * s + gy * c                 # e_phi = (-sin phi, cos phi)
        if targets is None:
            phi, gr, gp = (a.reshape(grid.nr, grid.nphi) for a in (phi, gr, gp))
        out["phi_" + name], out["gr_" + name], out["gphi_" + name] = phi, gr, gp
    return out


# --------------------------------------------------------------------------
# FFT convolution (Sec. 5.2, App. C)
# --------------------------------------------------------------------------
def conv_tables(grid, h_a, h_b):
    """Convolution kernels on the lattice Delta = u - u' = k du (k taken
    circularly in [-nr, nr), the lag -nr entry unused and zero) and
    psi = phi - phi' = j dphi, for source aspect ratio h_a, target h_b.

    App. C: h_ab^2(Delta) = (h_a^2 e^-Delta + h_b^2 e^Delta) / 2 (the printed
    H_ab/(r r') is read as H_ab^2/(r r')), d^2 = 2 (cosh Delta - cos psi) /
    h_ab^2, written cancellation-free as 4 [sinh^2(Delta/2) + sin^2(psi/2)] /
    h_ab^2.  With D = e^X (K1 - K0)(X), X = d^2/8 (so L/(pi d^2) =
    D/(8 sqrt(pi))):
        K_r   = e^{-3 Delta/2} (e^Delta - cos psi) D / (8 sqrt(pi) h_ab^3)
        K_phi = e^{-3 Delta/2}  sin psi          D / (8 sqrt(pi) h_ab^3)
        K_Phi = e^{-3 Delta/2}  e^X K0(X)          / (2 sqrt(pi) h_ab)
    so that g_r = -G du dphi sum Sigma_a K_r (no r prefactor), likewise g_phi,
    and Phi = -G r du dphi sum Sigma_a K_Phi.  Self term K(0, 0) := 0.
    Returns (K_Phi, K_r, K_phi), each [2 nr, nphi]."""
    nr, nphi = grid.nr, grid.nphi
    k = np.arange(2 * nr)
    k = np.where(k < nr, k, k - 2 * nr).astype(np.float64)
    Dl = (k * grid.du)[:, None]
    psi = (np.arange(nphi) * grid.dphi)[None, :]
    hab2 = 0.5 * (h_a * h_a * np.exp(-Dl) + h_b * h_b * np.exp(Dl))
    sh = np.sinh(0.5 * Dl)
    sp2 = np.sin(0.5 * psi) ** 2
    d2 = 4.0 * (sh * sh + sp2) / hab2
    X = d2 / 8.0
    X[0, 0] = 1.0                       # placeholder, overwritten below
    k0, D = k0e_D(X)
    hab = np.sqrt(hab2)
    e32 = np.exp(-1.5 * Dl)
    KP = e32 * k0 / (2.0 * SQRT_PI * hab)
    Kr = e32 * (np.expm1(Dl) + 2.0 * sp2) * D / (8.0 * SQRT_PI * hab ** 3)
    Kp = e32 * np.sin(psi) * D / (8.0 * SQRT_PI * hab ** 3)
    for K in (KP, Kr, Kp):
        K[0, 0] = 0.0                   # self cell excluded
        K[nr, :] = 0.0                  # lag -nr never occurs
    return KP, Kr, Kp


def fft64_plan(grid, h_g=0.05, h_d=None, G=1.0):
    """Kernel spectra of every ordered (source, target) pair (Sec. 5.2: the
    kernel depends only on the grid and the aspect ratios, so it is
    transformed once)."""
    fl = [("g", h_g)] + ([("d", h_d)] if h_d is not None and h_d > 0 else [])
    spectra = {}
    for sname, ha in fl:
        for tname, hb in fl:
            spectra[(sname, tname)] = [np.fft.rfft2(t) for t in conv_tables(grid, ha, hb)]
    return {"grid": grid, "fluids": [f for f, _ in fl], "G": G, "spectra": spectra}


def fft64_apply(plan, sigma_g, sigma_d=None, workers=None):
    """FP64 zero-padded FFT convolution (Sec. 5.2: log grid, radial padding to
    2 nr; App. C kernels; bi-fluid sums over sources as in Sec. 5.2's
    multi-fluid equations, with one table per ordered pair).

    ``workers``: None runs numpy's FFTs on one thread (the parity reference);
    an integer runs the same FP64 transforms through scipy.fft on that many
    threads (for timing the oracle on all of a host's cores)."""
    if workers is None:
        rfft2, irfft2 = np.fft.rfft2, np.fft.irfft2
    else:
        import scipy.fft as sf

        def rfft2(a):
            return sf.rfft2(a, workers=workers)

        def irfft2(a, s):
            return sf.irfft2(a, s=s, workers=workers)
    grid = plan["grid"]
    nr, nphi = grid.nr, grid.nphi
    srcs = {"g": _c64(sigma_g)}
    if "d" in plan["fluids"]:
        srcs["d"] = _c64(sigma_d)
    spec = {}
    for name, sig in srcs.items():
        pad = np.zeros((2 * nr, nphi))
        pad[:nr] = sig
        spec[name] = rfft2(pad)
    out = {}
    r = grid.r[:, None]
    scale = -plan["G"] * grid.du * grid.dphi
    for tname in srcs:
        acc = [0.0, 0.0, 0.0]
        for sname in srcs:
            tabs = plan["spectra"][(sname, tname)]
            for c in range(3):
                acc[c] = acc[c] + spec[sname] * tabs[c]
        res = [irfft2(a, s=(2 * nr, nphi))[:nr] * scale for a in acc]
        out["phi_" + tname] = res[0] * r
        out["gr_" + tname] = res[1]
        out["gphi_" + tname] = res[2]
    return out


def fft64(grid, sigma_g, sigma_d=None, h_g=0.05, h_d=None, G=1.0):
    """``fft64_apply(fft64_plan(...), ...)`` in one call."""
    return fft64_apply(fft64_plan(grid, h_g, h_d if sigma_d is not None else None, G), sigma_g, sigma_d)


# --------------------------------------------------------------------------
# Indirect term (Sec. 5.4, App. E)
# --------------------------------------------------------------------------
def indirect_kernel(d_a, H_a):
    """App. E: K_a(d_a) = (1/sqrt(pi)) H_a^-2 (d_a/4) e^{d_a^2/4} [K1 - K0](d_a^2/4),
    d_a = |r'| / H_a (note d^2/4, not the d^2/8 of the pair kernel)."""
    d_a = np.asarray(d_a, dtype=np.float64)
    H_a = np.asarray(H_a, dtype=np.float64)
    _, D = k0e_D(d_a * d_a / 4.0)
    return (1.0 / SQRT_PI) / (H_a * H_a) * (d_a / 4.0) * D


def indirect(grid, sigma_g, sigma_d=None, h_g=None, h_d=None, H_g=None, H_d=None, G=1.0):
    """App. E: A_a = sqrt(2) G sum_cells m_a K_a cos phi', B_a = the same with
    sin phi', for each source fluid a (gas first), so that the gradient of
    the indirect potential is (A cos phi + B sin phi) e_r +
    (-A sin phi + B cos phi) e_phi with A = sum_a A_a, B = sum_a B_a.
    Returns an array [[A_g, B_g], [A_d, B_d]] (one row for a gas-only disc)."""
    R, P = grid.mesh()
    out = []
    srcs = [(sigma_g, _scale_height(grid, H_g, h_g))]
    if sigma_d is not None:
        srcs.append((sigma_d, _scale_height(grid, H_d, h_d)))
    for sig, H in srcs:
        m = _c64(sig) * R * R * grid.du * grid.dphi
        w = np.sqrt(2.0) * G * m * indirect_kernel(R / H, H)
        out.append([float(np.sum(w * np.cos(P))), float(np.sum(w * np.sin(P)))])
    return np.array(out)


# --------------------------------------------------------------------------
# Error metrics (readings: rel-L2 per field; max error normalised by the
# field's maximum, as the paper normalises its L-infinity errors, Sec. 4.4)
# --------------------------------------------------------------------------
def rel_l2(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))


def rel_max(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.abs(x - ref).max() / np.abs(ref).max())
