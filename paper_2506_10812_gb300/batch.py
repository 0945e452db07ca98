"""Torch-facing wrapper of the batch entry points of ``include/sg.h``: many
independent discs (FFT plans of uneven grids) solved by one persistent
kernel launch replayed from a CUDA graph.  Argument marshalling only."""
from __future__ import annotations

import ctypes

import torch

from . import _native as N
from .plan import _OUT_KEYS


class Batch:
    """Bind ``plans`` and their device buffers.

    ``sigma_g[k]``, ``sigma_d[k]`` (None for a gas-only plan) and ``outs[k]``
    (dict keyed like ``Plan.solve``'s result; missing keys are not computed)
    must stay alive and at the same addresses for the batch's lifetime.
    ``threads`` (256 / 512), ``ctas_per_sm``, ``order`` ("pipelined" /
    "staged") and ``specialize`` (compile-time transforms for the lengths the
    per-disc path specialises) fix the persistent kernel's launch; ``streams``
    > 0 selects the other engine, every disc's sg_solve chain on that many
    streams of one graph.  ``autotune`` times every candidate of both engines
    and keeps the fastest."""

    def __init__(self, plans, sigma_g, sigma_d, outs, threads=0, ctas_per_sm=0, order="pipelined",
                 specialize=False, autotune=False, check_finite=False, host_gate=False, timeout_ms=0.0,
                 streams=0):
        self._lib = N.load()
        n = len(plans)
        if not (len(sigma_g) == len(sigma_d) == len(outs) == n) or n < 1:
            raise ValueError("plans, sigma_g, sigma_d and outs need one entry per disc")
        self.plans = list(plans)
        self.device = plans[0].device
        self._keep = []
        sg = (ctypes.c_void_p * n)()
        sd = (ctypes.c_void_p * n)()
        op = (ctypes.c_void_p * (6 * n))()
        for k, pl in enumerate(plans):
            g, d = pl._inputs(sigma_g[k], sigma_d[k])
            sg[k] = g.data_ptr()
            sd[k] = d.data_ptr() if d is not None else None
            self._keep += [g, d]
            for key, t in outs[k].items():
                if key not in _OUT_KEYS:
                    raise ValueError(f"unknown output key {key}")
                pl._check(t, key)
                op[6 * k + _OUT_KEYS.index(key)] = t.data_ptr()
                self._keep.append(t)
        o = N.SgBatchOpts()
        o.threads, o.ctas_per_sm = int(threads), int(ctas_per_sm)
        o.order = {"pipelined": N.SG_BATCH_ORDER_PIPELINED, "staged": N.SG_BATCH_ORDER_STAGED}[order]
        o.specialize = 1 if specialize else 0
        o.autotune = 1 if autotune else 0
        o.flags = (N.SG_CHECK_FINITE if check_finite else 0) | (N.SG_BATCH_HOST_GATE if host_gate else 0)
        o.timeout_ms = float(timeout_ms)
        o.streams = int(streams)
        hp = (ctypes.c_void_p * n)(*[pl._h.value for pl in plans])
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self._lib.sg_batch_create(ctypes.byref(h), hp, n, sg, sd, op, ctypes.byref(o), self._stream())
        N.check(st, None, "sg_batch_create")
        self._h = h

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def solve(self):
        """Every disc, one graph launch (asynchronous)."""
        with torch.cuda.device(self.device):
            N.check(self._lib.sg_batch_solve(self._h, self._stream()), what="sg_batch_solve", batch_handle=self._h)

    def solve_loop(self):
        """The per-disc baseline: sg_solve on every plan in turn."""
        with torch.cuda.device(self.device):
            N.check(self._lib.sg_batch_solve_loop(self._h, self._stream()), what="sg_batch_solve_loop",
                    batch_handle=self._h)

    def release(self):
        N.check(self._lib.sg_batch_release(self._h), what="sg_batch_release", batch_handle=self._h)

    def sync(self):
        with torch.cuda.device(self.device):
            N.check(self._lib.sg_batch_sync(self._h, self._stream()), what="sg_batch_sync", batch_handle=self._h)

    def config(self):
        o = N.SgBatchOpts()
        grid, ntasks, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        N.check(self._lib.sg_batch_config(self._h, ctypes.byref(o), ctypes.byref(grid), ctypes.byref(ntasks),
                                          ctypes.byref(ms)), what="sg_batch_config", batch_handle=self._h)
        return {"threads": o.threads, "ctas_per_sm": o.ctas_per_sm,
                "order": ("pipelined", "staged")[o.order], "specialize": bool(o.specialize),
                "autotuned": bool(o.autotune), "streams": o.streams,
                "grid": grid.value, "tasks": ntasks.value, "tuned_ms": ms.value, "timeout_ms": o.timeout_ms}

    def tune_results(self):
        """[(config dict, ms per solve)] of every autotune candidate."""
        n = self._lib.sg_batch_tune_results(self._h, 0, None, None)
        cfgs = (N.SgBatchOpts * max(n, 1))()
        ms = (ctypes.c_float * max(n, 1))()
        self._lib.sg_batch_tune_results(self._h, n, cfgs, ms)
        return [({"streams": c.streams} if c.streams else
                 {"threads": c.threads, "ctas_per_sm": c.ctas_per_sm, "order": ("pipelined", "staged")[c.order],
                  "specialize": bool(c.specialize)}, float(m)) for c, m in zip(cfgs[:n], ms[:n])]

    def tile_trials(self):
        """[trial dict] of every launch-tile candidate the autotuner timed:
        disc, shape (nr, nphi, nsrc), tiles, median ms of one solve of that
        disc, and whether the shape's discs now use it."""
        n = self._lib.sg_batch_tile_trials(self._h, 0, None)
        out = (N.SgTileTrial * max(n, 1))()
        self._lib.sg_batch_tile_trials(self._h, n, out)
        names = {v: k for k, v in N.COLS_STAGING.items()}
        return [{"disc": t.disc, "nr": t.nr, "nphi": t.nphi, "nsrc": t.nsrc,
                 "tiles": {"rows_fwd": t.tiles.rows_fwd, "rows_inv": t.tiles.rows_inv,
                           "cols_staging": names[t.tiles.cols_staging]},
                 "ms": float(t.ms), "chosen": bool(t.chosen)} for t in out[:n]]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sg_batch_destroy(self._h)
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
