"""GPU tests of the batched solve (many independent discs, one persistent
launch under a CUDA graph, or every disc's launch chain on forked streams of
one graph): against the per-disc solve, against the FP64 oracle, across
launch configurations, with output subsets, the autotuner over both engines,
and the bounded device waits (host gate withheld -> SG_ERR_TIMEOUT, context
still usable).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_10812_gb300 import _native as N
from paper_2506_10812_gb300 import build as B
from paper_2506_10812_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL32 = (1e-5, 1e-4)
KEYS = ("phi_g", "gr_g", "gphi_g", "phi_d", "gr_d", "gphi_d")


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    B.build()
    N.load()
    oracle.build()


def rounded(d):
    import copy
    e = copy.copy(d)
    e.sigma_g = d.sigma_g.astype(np.float32).astype(np.float64)
    if d.sigma_d is not None:
        e.sigma_d = d.sigma_d.astype(np.float32).astype(np.float64)
    return e


class Setup:
    """Plans, device inputs and two sets of outputs (batched, per-disc)."""

    def __init__(self, discs, dtype=torch.float32, keys=None):
        from paper_2506_10812_gb300 import Plan
        dev = torch.device("cuda:0")
        self.discs = discs
        self.plans = [Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, d.h_d, G=d.G, dtype=dtype, device=dev)
                      for d in discs]
        self.sg = [torch.tensor(d.sigma_g, dtype=dtype, device=dev) for d in discs]
        self.sd = [None if d.sigma_d is None else torch.tensor(d.sigma_d, dtype=dtype, device=dev)
                   for d in discs]
        self.keys = []
        for k, d in enumerate(discs):
            ks = [x for x in KEYS if d.sigma_d is not None or x.endswith("_g")]
            if keys is not None:
                ks = [x for x in ks if x in keys(k)]
            self.keys.append(ks)
        self.out = [{x: torch.full((d.nr, d.nphi), float("nan"), dtype=dtype, device=dev) for x in ks}
                    for d, ks in zip(discs, self.keys)]

    def batch(self, **kw):
        from paper_2506_10812_gb300 import Batch
        return Batch(self.plans, self.sg, self.sd, self.out, **kw)

    def per_disc(self):
        res = []
        for pl, g, d, ks in zip(self.plans, self.sg, self.sd, self.keys):
            o = pl.solve(g, d)
            res.append({x: o[x] for x in ks})
        torch.cuda.synchronize()
        return res

    def close(self):
        for p in self.plans:
            p.close()


def uneven(n=7, offset=50):
    shapes = [(8, 32), (16, 64), (64, 256), (128, 128), (32, 1024), (256, 512), (16, 2048)]
    discs = []
    for k in range(n):
        nr, nphi = shapes[k % len(shapes)]
        d = inputs.ragged_noise(nr, nphi, offset=offset + k, bifluid=(k % 2 == 0), h=0.04 + 0.01 * k)
        discs.append(rounded(d))
    return discs


def rel(a, b):
    return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))


def test_batch_matches_per_disc_and_oracle():
    """Uneven gas and gas + dust discs (every final radix, tiny to 2048-long
    rows): batched equals the per-disc solve, and both meet the FP32
    tolerance against the FP64 oracle."""
    S = Setup(uneven())
    try:
        with S.batch() as b:
            b.solve()
            b.sync()
            ref = S.per_disc()
            for k, d in enumerate(S.discs):
                g = oracle.Grid(d.nr, d.nphi, d.r_in, d.r_out)
                o64 = oracle.fft64(g, d.sigma_g, d.sigma_d, h_g=d.h_g, h_d=d.h_d, G=d.G)
                for x in S.keys[k]:
                    got = S.out[k][x]
                    assert rel(got, ref[k][x]) <= 1e-6, (k, x)
                    v = got.double().cpu().numpy()
                    e2, em = oracle.rel_l2(v, o64[x]), oracle.rel_max(v, o64[x])
                    assert e2 <= TOL32[0] and em <= TOL32[1], (k, x, e2, em)
    finally:
        S.close()


def test_batch_fp64_equals_per_disc():
    S = Setup(uneven(5, offset=70), dtype=torch.float64)
    try:
        with S.batch() as b:
            b.solve()
            b.sync()
            ref = S.per_disc()
            for k in range(len(S.discs)):
                for x in S.keys[k]:
                    assert rel(S.out[k][x], ref[k][x]) <= 1e-13, (k, x)
    finally:
        S.close()


def test_launch_configurations_are_bit_identical():
    """Every (threads, ctas_per_sm, order) runs the same transforms: results
    are bit-identical whatever the schedule."""
    S = Setup(uneven(6, offset=90))
    try:
        first = None
        for threads in (256, 512):
            for order in ("pipelined", "staged"):
                for cps in (1, 0):
                    with S.batch(threads=threads, order=order, ctas_per_sm=cps) as b:
                        cfg = b.config()
                        assert cfg["threads"] == threads and cfg["order"] == order
                        for t in (x for o in S.out for x in o.values()):
                            t.fill_(float("nan"))
                        b.solve()
                        b.solve()
                        b.sync()
                        cur = [{x: o[x].clone() for x in o} for o in S.out]
                    if first is None:
                        first = cur
                    else:
                        for a, c in zip(first, cur):
                            for x in a:
                                assert torch.equal(a[x], c[x]), (threads, order, cps, x)
    finally:
        S.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_stream_engine_equals_per_disc_solve(dtype):
    """The stream engine captures every disc's sg_solve chain on forked
    streams of one graph: its outputs equal the per-disc solve bit for bit
    (output subsets, one stream, several, more streams than discs), over
    repeated solves."""
    keys = lambda k: KEYS if k % 3 else ("gr_g", "phi_d")
    S = Setup(uneven(), dtype=dtype, keys=keys)
    try:
        ref = S.per_disc()
        for streams in (1, 3, 16):
            for o in S.out:
                for t in o.values():
                    t.fill_(float("nan"))
            with S.batch(streams=streams) as b:
                cfg = b.config()
                assert cfg["streams"] == streams and cfg["grid"] == 0 and cfg["tasks"] == 3 * len(S.discs)
                b.solve()
                b.solve()
                b.sync()
            for k in range(len(S.discs)):
                for x in S.keys[k]:
                    assert torch.equal(S.out[k][x], ref[k][x]), (streams, k, x)
    finally:
        S.close()


def test_autotune_times_both_engines():
    S = Setup(uneven(4, offset=90))
    try:
        ref = S.per_disc()
        with S.batch(autotune=True) as b:
            tried = b.tune_results()
            assert any("streams" in c for c, _ in tried) and any("threads" in c for c, _ in tried)
            cfg = b.config()
            best = min(ms for _, ms in tried)
            assert cfg["autotuned"] and cfg["tuned_ms"] == pytest.approx(best)
            b.solve()
            b.sync()
        for k in range(4):
            for x in S.keys[k]:
                assert rel(S.out[k][x], ref[k][x]) <= 1e-6, (k, x)
    finally:
        S.close()


def test_stream_engine_rejects_host_gate():
    S = Setup(uneven(2))
    try:
        with pytest.raises(N.SgError) as e:
            S.batch(streams=2, host_gate=True)
        assert e.value.status == N.SG_ERR_ARG
        with pytest.raises(N.SgError) as e:
            S.batch(streams=65)
        assert e.value.status == N.SG_ERR_ARG
    finally:
        S.close()


@pytest.mark.parametrize("streams", [0, 2])
def test_batch_rejects_misaligned_buffers(streams):
    """Both engines move element pairs: a buffer aligned to one element only
    is rejected at create (SG_ERR_ARG), before anything is launched."""
    S = Setup(uneven(2))
    try:
        d = S.discs[1]
        base = torch.zeros(d.nr * d.nphi + 2, device="cuda:0")
        S.out[1]["gr_g"] = base[1:1 + d.nr * d.nphi].view(d.nr, d.nphi)
        with pytest.raises(N.SgError) as e:
            S.batch(streams=streams)
        assert e.value.status == N.SG_ERR_ARG
    finally:
        S.close()


def test_stream_engine_reports_nonfinite_outputs():
    """The stream engine's per-disc chains write their status into the
    batch's flag: a NaN input gives SG_ERR_NONFINITE at sg_batch_sync, and
    the flag is cleared for the next solve."""
    S = Setup(uneven(3, offset=70))
    try:
        with S.batch(streams=2, check_finite=True) as b:
            b.solve()
            b.sync()
            S.sg[1][3, 5] = float("nan")
            b.solve()
            with pytest.raises(N.SgError) as e:
                b.sync()
            assert e.value.status == N.SG_ERR_NONFINITE
            S.sg[1][3, 5] = 1.0
            b.solve()
            b.sync()
    finally:
        S.close()


def test_specialized_transforms():
    """The length-specialised kernel: within FP32 rounding of sg_solve and of
    the generic batch (sg_solve's tensor-copy row transforms reduce the row
    mean and form the R2C twiddles in another order), and bit-identical
    across launch configurations."""
    discs = [rounded(inputs.lognormal_bifluid(1024, 2048, St=0.1, offset=170)),
             rounded(inputs.lognormal_bifluid(512, 1024, St=1.0, offset=171)),
             rounded(inputs.lognormal_gas(256, 4096, offset=172))]
    S = Setup(discs)
    try:
        ref = S.per_disc()
        with S.batch() as b:
            b.solve()
            b.sync()
            generic = [{x: o[x].clone() for x in o} for o in S.out]
        first = None
        for threads, order in ((256, "staged"), (512, "pipelined")):
            with S.batch(specialize=True, threads=threads, order=order) as b:
                assert b.config()["specialize"]
                b.solve()
                b.sync()
                cur = [{x: o[x].clone() for x in o} for o in S.out]
            if first is None:
                first = cur
            for a, c in zip(first, cur):
                for x in a:
                    assert torch.equal(a[x], c[x]), (threads, order, x)
        for k in range(3):
            for x in S.keys[k]:
                assert rel(first[k][x], generic[k][x]) <= 1e-6, (k, x)
                assert rel(first[k][x], ref[k][x]) <= 1e-6, (k, x)
    finally:
        S.close()


def test_output_subsets_and_input_updates():
    """Per-disc output subsets (some discs only g_r of the gas, one disc
    nothing of the dust); rewriting the bound inputs changes the next solve."""
    sel = {0: ("gr_g",), 1: ("phi_g", "gphi_g"), 2: ("gr_g", "gr_d", "gphi_d"), 3: ("phi_g", "gr_g", "gphi_g")}
    S = Setup(uneven(4, offset=110), keys=lambda k: sel[k])
    try:
        with S.batch() as b:
            b.solve()
            b.sync()
            ref = S.per_disc()
            for k in range(4):
                assert set(S.out[k]) == set(sel[k])
                for x in sel[k]:
                    assert rel(S.out[k][x], ref[k][x]) <= 1e-6, (k, x)
            for t in S.sg + S.sd:          # the field is linear in both sources
                if t is not None:
                    t.mul_(2.0)
            b.solve()
            b.sync()
            for k in range(4):
                for x in sel[k]:
                    assert rel(S.out[k][x], 2.0 * ref[k][x]) <= 1e-6, (k, x)
    finally:
        S.close()


def test_host_gate_timeout_then_recovery():
    """A bounded device wait: with the host gate withheld every block gives
    up after timeout_ms and sg_batch_sync reports SG_ERR_TIMEOUT; the same
    batch then runs normally once the gate is released."""
    S = Setup(uneven(3, offset=130))
    try:
        with S.batch(host_gate=True, timeout_ms=50.0) as b:
            b.solve()
            with pytest.raises(N.SgError) as ei:
                b.sync()
            assert ei.value.status == N.SG_ERR_TIMEOUT
            b.solve()
            b.release()
            b.sync()
            ref = S.per_disc()
            for k in range(3):
                for x in S.keys[k]:
                    assert rel(S.out[k][x], ref[k][x]) <= 1e-6, (k, x)
        with S.batch() as b:
            with pytest.raises(N.SgError) as ei:
                b.release()
            assert ei.value.status == N.SG_ERR_ARG
    finally:
        S.close()


def test_finite_check_and_argument_errors():
    from paper_2506_10812_gb300 import Batch, Plan
    S = Setup(uneven(3, offset=150))
    try:
        S.sg[1][3, 5] = float("nan")
        with S.batch(check_finite=True) as b:
            b.solve()
            with pytest.raises(N.SgError) as ei:
                b.sync()
            assert ei.value.status == N.SG_ERR_NONFINITE
            b.sync()                      # the flag was cleared
        dev = torch.device("cuda:0")
        d = S.discs[0]
        p64 = Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, d.h_d, dtype=torch.float64, device=dev)
        pdir = Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, d.h_d, method="direct", device=dev)
        try:
            g64 = torch.zeros((d.nr, d.nphi), dtype=torch.float64, device=dev)
            with pytest.raises(N.SgError) as ei:
                Batch([S.plans[0], p64], [S.sg[0], g64], [S.sd[0], g64.clone()], [{}, {}])
            assert ei.value.status == N.SG_ERR_ARG
            with pytest.raises(N.SgError) as ei:
                Batch([pdir], [S.sg[0]], [S.sd[0]], [{}])
            assert ei.value.status == N.SG_ERR_ARG
            with pytest.raises(N.SgError) as ei:
                Batch([S.plans[0]], [S.sg[0]], [S.sd[0]], [{}], threads=128)
            assert ei.value.status == N.SG_ERR_ARG
        finally:
            p64.close()
            pdir.close()
    finally:
        S.close()


def test_full_batch_workload():
    """The 64-disc workload bench.py times (grids 128x256 .. 1024x2048, gas +
    dust, FP32): the autotuned batch equals the per-disc launch loop on every
    output of every disc (bit for bit when the stream engine wins), and so does
    the persistent kernel to FP32 rounding; the smallest and one mid-size disc
    against the FP64 oracle."""
    discs = [rounded(d) for d in inputs.batch_discs()]
    S = Setup(discs)
    snap = lambda: [{x: o[x].clone() for x in o} for o in S.out]
    try:
        with S.batch(autotune=True) as b:
            cfg = b.config()
            assert cfg["autotuned"] and cfg["tuned_ms"] > 0
            tried = b.tune_results()
            assert len(tried) >= 4 and min(ms for _, ms in tried) == pytest.approx(cfg["tuned_ms"])
            b.solve()
            b.sync()
            got = snap()
            b.solve_loop()
            b.sync()
            loop = snap()
        for k in range(len(discs)):
            for x in S.keys[k]:
                assert rel(got[k][x], loop[k][x]) <= 1e-6, (k, x)
                if cfg["streams"]:
                    assert torch.equal(got[k][x], loop[k][x]), (k, x)
        with S.batch(threads=256, ctas_per_sm=2, order="staged", specialize=True) as b:
            b.solve()
            b.sync()
            for k in range(len(discs)):
                for x in S.keys[k]:
                    assert rel(S.out[k][x], loop[k][x]) <= 1e-6, ("persistent", k, x)
        small = min(range(len(discs)), key=lambda k: discs[k].nr)
        mid = next(k for k in range(len(discs)) if discs[k].nr == 512)
        for k in (small, mid):
            d = discs[k]
            g = oracle.Grid(d.nr, d.nphi, d.r_in, d.r_out)
            o64 = oracle.fft64(g, d.sigma_g, d.sigma_d, h_g=d.h_g, h_d=d.h_d, G=d.G)
            for x in S.keys[k]:
                v = got[k][x].double().cpu().numpy()
                e2, em = oracle.rel_l2(v, o64[x]), oracle.rel_max(v, o64[x])
                assert e2 <= TOL32[0] and em <= TOL32[1], (k, x, e2, em)
    finally:
        S.close()
