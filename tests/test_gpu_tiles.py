"""GPU tests of the per-plan launch tiles (rows per CTA of the tensor-copy row
transforms, kernel-spectrum staging of the column pass): every tile set
reproduces the default solve to FP32 rounding, gas-only and gas + dust,
through the device and the host-buffer entry points (bit for bit between
the two at equal tiles), up to the 2048 x 4096 disc; a non-default set still
meets the FP32 tolerance against the FP64 oracle; the argument checks; and
the batch autotuner's per-shape tile trials.

Tiles are not bit-identical: each kernel variant is compiled on its own, and
the compiler fuses the FFT's and the products' multiply-adds differently in
each (measured: relative L2 differences up to 2e-7 on the 2048 x 4096 disc).
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
from paper_2506_10812_gb300 import _native as N
from paper_2506_10812_gb300 import build as B
from paper_2506_10812_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL32 = (1e-5, 1e-4)
TILES = [dict(rows_fwd=rf, rows_inv=ri, cols_staging=st)
         for rf, ri, st in itertools.product((2, 4), (2, 4), ("all", "step"))]


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    B.build()
    N.load()
    oracle.build()


def make_plan(d, dtype=torch.float32, method="fft"):
    from paper_2506_10812_gb300 import Plan
    return Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, d.h_d, G=d.G, dtype=dtype, method=method,
                device="cuda:0")


def device_inputs(d, dtype=torch.float32):
    sg = torch.tensor(d.sigma_g, dtype=dtype, device="cuda:0")
    sd = None if d.sigma_d is None else torch.tensor(d.sigma_d, dtype=dtype, device="cuda:0")
    return sg, sd


def solve_all(pl, sg, sd):
    """phi, g_r, g_phi of every target fluid, keyed phi_g ... gphi_d."""
    o = pl.solve(sg, sd)
    torch.cuda.synchronize()
    return {k: v.clone() for k, v in o.items()}


def rel(a, b):
    return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))


def close_to(a, b):
    """Equal to FP32 rounding: relative L2 <= 1e-6, max error <= 1e-5 of the
    largest value."""
    return rel(a, b) <= 1e-6 and float((a - b).abs().max()) <= 1e-5 * float(b.abs().max())


@pytest.mark.parametrize("nr,nphi,bifluid", [(64, 512, False), (128, 1024, True), (256, 4096, True),
                                             (1024, 2048, True), (2048, 4096, False), (2048, 4096, True)])
def test_every_tile_set_matches_default(nr, nphi, bifluid):
    """Every tile set against the default (the 2048 x 4096 disc included,
    gas-only and gas + dust; the gas + dust all-at-once staging there needs
    194 KB of shared memory per block); a repeated solve with the same tiles
    is bit-identical."""
    d = inputs.ragged_noise(nr, nphi, offset=300 + nr, bifluid=bifluid)
    pl = make_plan(d)
    try:
        default = pl.tiles
        assert default["rows_fwd"] == 4 and default["rows_inv"] == 2
        want_step = bifluid or nr == 2048
        assert default["cols_staging"] == ("step" if want_step else "all")
        sg, sd = device_inputs(d)
        ref = solve_all(pl, sg, sd)
        for t in TILES:
            pl.set_tiles(**t)
            assert pl.tiles == t
            got = solve_all(pl, sg, sd)
            again = solve_all(pl, sg, sd)
            for k in ref:
                assert close_to(got[k], ref[k]), (t, k, rel(got[k], ref[k]))
                assert torch.equal(again[k], got[k]), (t, k)
        pl.set_tiles(**default)
        assert pl.tiles == default
        back = solve_all(pl, sg, sd)
        for k in ref:
            assert torch.equal(back[k], ref[k]), k
    finally:
        pl.close()


def test_host_entry_point_with_other_tiles():
    """The host-buffer solve transforms row chunks with the plan's tiles
    (chunk starts on a tile boundary): bit for bit the device solve with the
    same tiles."""
    d = inputs.ragged_noise(256, 2048, offset=321, bifluid=True)
    pl = make_plan(d)
    try:
        sg, sd = device_inputs(d)
        for t in (dict(rows_fwd=2, rows_inv=4, cols_staging="all"), dict(rows_fwd=4, rows_inv=4, cols_staging="step")):
            pl.set_tiles(**t)
            ref = solve_all(pl, sg, sd)
            got = pl.solve_host(sg.cpu(), sd.cpu())
            torch.cuda.synchronize()
            for k in ref:
                assert torch.equal(torch.as_tensor(got[k]), ref[k].cpu()), (t, k)
    finally:
        pl.close()


def test_non_default_tiles_meet_oracle_tolerance():
    d = inputs.ragged_noise(128, 1024, offset=333, bifluid=True)
    d.sigma_g = d.sigma_g.astype(np.float32).astype(np.float64)
    d.sigma_d = d.sigma_d.astype(np.float32).astype(np.float64)
    pl = make_plan(d)
    try:
        pl.set_tiles(rows_fwd=2, rows_inv=4, cols_staging="all")
        sg, sd = device_inputs(d)
        got = solve_all(pl, sg, sd)
        g = oracle.Grid(d.nr, d.nphi, d.r_in, d.r_out)
        o64 = oracle.fft64(g, d.sigma_g, d.sigma_d, h_g=d.h_g, h_d=d.h_d, G=d.G)
        for k, v in got.items():
            x = v.double().cpu().numpy()
            ref = o64[k]
            assert oracle.rel_l2(x, ref) <= TOL32[0] and oracle.rel_max(x, ref) <= TOL32[1], k
    finally:
        pl.close()


def test_tile_argument_checks():
    d = inputs.ragged_noise(64, 512, offset=340, bifluid=False)
    pl = make_plan(d)
    try:
        for bad in (dict(rows_fwd=3), dict(rows_inv=8), dict(rows_fwd=0)):
            with pytest.raises(N.SgError) as e:
                pl.set_tiles(**bad)
            assert e.value.status == N.SG_ERR_ARG
        t = N.SgTiles(4, 2, 2)
        import ctypes
        assert pl._lib.sg_set_tiles(pl._h, ctypes.byref(t)) == N.SG_ERR_ARG
        assert pl._lib.sg_set_tiles(pl._h, None) == N.SG_ERR_ARG
        assert pl._lib.sg_set_tiles(None, ctypes.byref(t)) == N.SG_ERR_ARG
        assert pl._lib.sg_get_tiles(pl._h, None) == N.SG_ERR_ARG
        assert pl.tiles == dict(rows_fwd=4, rows_inv=2, cols_staging="all")   # unchanged by the rejects
    finally:
        pl.close()
    p64 = make_plan(d, dtype=torch.float64)
    try:
        assert p64.tiles["cols_staging"] == "all"
        with pytest.raises(N.SgError) as e:
            p64.set_tiles(cols_staging="step")
        assert e.value.status == N.SG_ERR_UNSUPPORTED
        p64.set_tiles(rows_fwd=2)            # recorded; FP64 rows run their own kernels
        sg, sd = device_inputs(d, torch.float64)
        got = solve_all(p64, sg, sd)
        assert all(torch.isfinite(v).all() for v in got.values())
    finally:
        p64.close()
    pd = make_plan(d, method="direct")
    try:
        with pytest.raises(N.SgError) as e:
            pd.set_tiles(rows_fwd=2)
        assert e.value.status == N.SG_ERR_UNSUPPORTED
    finally:
        pd.close()


def test_batch_autotune_tile_trials():
    """The autotuner times every tile candidate per plan shape on the first
    disc of that shape (8 where the row transforms use tensor copies, the 2
    stagings elsewhere), gives every disc of the shape the fastest, and the
    batch equals the per-disc solve with those tiles (bit for bit on the
    stream engine)."""
    from paper_2506_10812_gb300 import Batch
    shapes = [(64, 512, False), (128, 1024, True), (64, 512, False), (16, 64, False), (128, 1024, True)]
    discs = [inputs.ragged_noise(nr, nphi, offset=350 + k, bifluid=bf) for k, (nr, nphi, bf) in enumerate(shapes)]
    plans = [make_plan(d) for d in discs]
    try:
        ins = [device_inputs(d) for d in discs]
        ref = [solve_all(pl, sg, sd) for pl, (sg, sd) in zip(plans, ins)]
        outs = [{k: torch.full((d.nr, d.nphi), float("nan"), device="cuda:0") for k in r} for d, r in zip(discs, ref)]
        with Batch(plans, [sg for sg, _ in ins], [sd for _, sd in ins], outs, autotune=True) as b:
            trials = b.tile_trials()
            by_disc = {}
            for t in trials:
                by_disc.setdefault(t["disc"], []).append(t)
            assert sorted(by_disc) == [0, 1, 3]            # first disc of each shape
            assert len(by_disc[0]) == 8 and len(by_disc[1]) == 8 and len(by_disc[3]) == 2
            for k, ts in by_disc.items():
                assert all(t["ms"] > 0 for t in ts)
                chosen = [t for t in ts if t["chosen"]]
                assert len(chosen) == 1
                assert chosen[0]["ms"] == min(t["ms"] for t in ts)
                for j, pl in enumerate(plans):
                    if shapes[j] == shapes[k]:
                        assert pl.tiles == chosen[0]["tiles"], (k, j)
            b.solve()
            b.sync()
            ref = [solve_all(pl, sg, sd) for pl, (sg, sd) in zip(plans, ins)]   # with the tuned tiles
            persistent = b.config()["streams"] == 0
            for k in range(len(discs)):
                for x, v in outs[k].items():
                    if persistent:      # its own row transforms: equal to FP32 rounding
                        assert rel(v, ref[k][x]) <= 1e-6, (k, x)
                    else:
                        assert torch.equal(v, ref[k][x]), (k, x)
    finally:
        for pl in plans:
            pl.close()
