"""Host-side logic of bench.py (no GPU): the algorithmic bytes per cell of
each stage and the roofline arithmetic of the reported JSON line."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


LAUNCHES = {"prim": 1, "flux_pcm": 3, "emf": 2, "update_half": 1, "recon": 3, "flux_hlld": 3, "update_full": 1}


def test_counted_bytes_per_step(bench):
    """2400 B/cell per FP64 (or double-float) step, 1340 B/cell FP32-bulk."""
    for T, total in ((8, 2400), (4, 1340)):
        sb = bench.stage_bytes(T)
        assert sum(sb[k] * n for k, n in LAUNCHES.items()) == total


def _prof(ms_per_launch, steps):
    return {k: (ms_per_launch[k] * n * steps, n * steps) for k, n in LAUNCHES.items()} | {"dt": (0.01, steps)}


def test_roofline_of_a_counted_stage(bench):
    """The dominant stage with ncu counters: FP64-pipe operations per launch
    over the live launch time against 601.3 G op/s; traffic = ncu DRAM bytes
    per cell x cells; the HBM views of the stage and of the step."""
    n3 = 256 ** 3
    ms = {"prim": 3.5, "flux_pcm": 7.7, "emf": 3.0, "update_half": 2.8, "recon": 10.9, "flux_hlld": 7.7,
          "update_full": 1.5}
    r = bench.roofline_of(_prof(ms, 10), "fp64", n3, 6791.4, "measured", "plmc")
    assert r["kernel"] == "recon" and r["bound"] == "alu"
    ops, flop, winst, dram = bench.COUNTERS["plmc"]["fp64"]["recon"]
    assert r["fp64_pipe"]["achieved"] == pytest.approx(ops * n3 / 10.9e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(max(r["fp64_pipe"]["frac"], r["issue"]["frac"]), rel=1e-9)
    assert r["traffic"] == round(dram * n3)
    assert r["hbm"]["achieved"] == pytest.approx(176 * n3 / 10.9e-3 / 1e9, rel=1e-3)
    step_s = sum(ms[k] * n for k, n in LAUNCHES.items()) * 1e-3 + 0.001e-3
    assert r["step_hbm"]["frac_counted"] == pytest.approx(n3 / step_s * 2400 / 1e9 / 6791.4, rel=1e-3)
    assert sum(r["stage_share"].values()) == pytest.approx(1.0, abs=1e-3)


def test_roofline_without_counters_is_hbm_bound(bench):
    """A dominant stage without counters (here the PCM predictor, changed
    since its capture) is reported against HBM with no traffic figure."""
    n3 = 128 ** 3
    ms = {"prim": 0.5, "flux_pcm": 3.0, "emf": 0.4, "update_half": 0.4, "recon": 2.4, "flux_hlld": 1.0,
          "update_full": 0.2}
    assert "flux_pcm" not in bench.COUNTERS["ppmc"]["fp64"]
    r = bench.roofline_of(_prof(ms, 2), "fp64", n3, 6791.4, "measured", "ppmc")
    assert r["kernel"] == "flux_pcm"
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None
    assert r["frac"] == pytest.approx(120 * n3 / 3.0e-3 / 1e9 / 6791.4, abs=1e-4)  # (rounded to 4 places)


def test_ppmc_reconstruction_is_bound_by_the_fp64_pipe(bench):
    """The 512^3 PPMC headline's dominant stage: counted FP64-pipe operations
    per launch over the launch time against the measured pipe rate."""
    n3 = 512 ** 3
    ms = {"prim": 32.2, "flux_pcm": 59.7, "emf": 23.8, "update_half": 21.8, "recon": 158.0, "flux_hlld": 59.6,
          "update_full": 12.2}
    r = bench.roofline_of(_prof(ms, 10), "fp64", n3, 6762.3, "measured", "ppmc")
    ops = bench.COUNTERS["ppmc"]["fp64"]["recon"][0]
    assert r["kernel"] == "recon" and r["bound"] == "alu"
    assert r["frac"] == pytest.approx(ops * n3 / 158.0e-3 / 1e9 / bench.FP64_PIPE_GINST, rel=1e-3)


def test_partial_counters_give_no_step_dram_figure(bench):
    """Double-float: the dominant stage has counters, the primitive and update
    stages (changed after the capture) do not, so the stage's own figures
    are reported and the step-level ncu DRAM figure is left out."""
    n3 = 256 ** 3
    ms = {"prim": 0.9, "flux_pcm": 3.0, "emf": 0.9, "update_half": 0.6, "recon": 6.2, "flux_hlld": 3.9,
          "update_full": 0.4}
    assert "prim" not in bench.COUNTERS["plmc"]["fp64_df"] and "recon" in bench.COUNTERS["plmc"]["fp64_df"]
    r = bench.roofline_of(_prof(ms, 10), "fp64_df", n3, 6791.4, "measured", "plmc")
    assert r["kernel"] == "recon" and r["bound"] == "alu" and r["traffic"] is not None
    assert "ncu_dram_bytes_per_cell" not in r["step_hbm"]
