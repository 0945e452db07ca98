"""The benchmark's traffic model and argument parsing, on the CPU: the byte
counts behind every roofline fraction bench.py reports, derived here per cell
from what each pass reads and writes."""
import argparse

import pytest

import bench


@pytest.mark.parametrize("nr,nphi", [(2048, 4096), (1024, 2048), (256, 512)])
def test_gas_model_per_cell(nr, nphi):
    """Gas only with Phi, g_r, g_phi (FP32): the column pass reads 4 B/cell of
    row spectra and 3 x 4 B/cell of kernel spectra and writes 3 x 4 B/cell;
    the step adds 4 (source) + 4 (row spectra written) + 12 (column output read
    back) + 12 (outputs) B/cell; the compulsory traffic is source + kernel
    spectra + outputs.  The kernel spectra hold one extra column (m = nphi/2)."""
    cells, extra = nr * nphi, 3 * 8 * nr
    col, step, comp = bench.solve_model_bytes(nr, nphi, 1, 3)
    assert col == 28 * cells + extra
    assert step == 60 * cells + extra
    assert comp == 28 * cells + extra


def test_bifluid_and_accel_only_per_cell():
    nr, nphi = 512, 1024
    cells = nr * nphi
    # gas + dust with Phi: 8 sources, 16 row spectra, 48 kernel spectra, 48 column output, 24 outputs
    _, step, comp = bench.solve_model_bytes(nr, nphi, 2, 3)
    assert step == 144 * cells + 12 * 8 * nr
    assert comp == 80 * cells + 12 * 8 * nr
    # gas, accelerations only: 4 + 4 + 4 + 8 + 8 + 8 + 8 = 44 B/cell
    _, step, _ = bench.solve_model_bytes(nr, nphi, 1, 2)
    assert step == 44 * cells + 2 * 8 * nr


@pytest.mark.parametrize("nr,nphi,nsrc", [(1024, 2048, 2), (128, 256, 2), (2048, 4096, 1)])
def test_batch_model_agrees_with_solve_model(nr, nphi, nsrc):
    """The batch line's per-disc model counts the kernel spectra at their
    stored pitch (nr + 2 slots); otherwise it is the same sum."""
    _, step, _ = bench.solve_model_bytes(nr, nphi, nsrc, 3)
    b = bench.step_model_bytes(nr, nphi, nsrc, 3 * nsrc)
    pad = 8 * nsrc * 3 * nsrc * (nphi // 2 + 1) * 2
    assert b == step + pad


def test_outputs_option():
    ns = lambda v: argparse.Namespace(outputs=v)
    assert bench.outputs_of(ns("phi,gr,gphi")) == ("phi", "gr", "gphi")
    assert bench.outputs_of(ns("gr, gphi")) == ("gr", "gphi")
    for bad in ("", "gr,gr", "phi,xx"):
        with pytest.raises(SystemExit):
            bench.outputs_of(ns(bad))


def test_profiled_traffic_matches_the_workload():
    """The column pass's DRAM traffic comes from the ncu summary of the same
    workload only: gas or gas + dust at 2048 x 4096 with all three components
    on the FP32 FFT engine; any other size, output set or engine reports none.
    Each committed summary carries the source hash it was captured on, and
    the gas and gas + dust kernels differ, so the two figures differ."""
    base = dict(engine="fft32", nr=2048, nphi=4096, outputs="phi,gr,gphi")
    gas = bench.profiled_traffic(argparse.Namespace(bifluid=False, **base))
    dust = bench.profiled_traffic(argparse.Namespace(bifluid=True, **base))
    if gas is not None and dust is not None:
        assert dust > gas
    for change in (dict(nr=1024, nphi=2048), dict(outputs="gr,gphi"), dict(engine="tc_bf16x3")):
        args = argparse.Namespace(bifluid=False, **dict(base, **change))
        assert bench.profiled_traffic(args) is None


def test_direct_mode_is_an_option():
    import sys
    argv = sys.argv
    try:
        sys.argv = ["bench.py", "--direct", "--steps", "3"]
        args = bench.parse()
    finally:
        sys.argv = argv
    assert args.direct and args.steps == 3 and not args.batch and not args.surrogate


def test_reference_arm_line():
    """`bench.py --impl reference` runs the FP64 oracle on the host cores on
    this arm's workload and prints one JSON line of the bench contract: the
    same metric, unit and config as the main line, its CPU baseline (all
    cores and one core) and an e2e object without host-device bytes."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["dtype"] == "f64"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["nr"] == 2048 and d["config"]["nphi"] == 4096 and "2048x4096" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] == os.cpu_count()
    assert cb["single_core"]["cores"] == 1 and cb["single_core"]["value"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
