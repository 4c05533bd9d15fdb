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
    r = bench.roofline_of(_prof(ms, 10), "fp64", n3, 6791.4, "measured", "ppmc")
    assert r["kernel"] == "recon" and r["bound"] == "alu"
    ops, flop, winst, dram = bench.COUNTERS["ppmc"]["fp64"]["recon"]
    assert r["fp64_pipe"]["achieved"] == pytest.approx(ops * n3 / 10.9e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(max(r["fp64_pipe"]["frac"], r["issue"]["frac"]), rel=1e-9)
    assert r["traffic"] == round(dram * n3)
    assert r["hbm"]["achieved"] == pytest.approx(176 * n3 / 10.9e-3 / 1e9, rel=1e-3)
    step_s = sum(ms[k] * n for k, n in LAUNCHES.items()) * 1e-3 + 0.001e-3
    assert r["step_hbm"]["frac_counted"] == pytest.approx(n3 / step_s * 2400 / 1e9 / 6791.4, rel=1e-3)
    assert sum(r["stage_share"].values()) == pytest.approx(1.0, abs=1e-3)
    # the step's ncu DRAM bytes per cell exactly when every stage has counters
    tab = bench.COUNTERS["ppmc"]["fp64"]
    if all(k in tab for k in LAUNCHES):
        assert r["step_hbm"]["ncu_dram_bytes_per_cell"] == pytest.approx(
            sum(tab[k][3] * n for k, n in LAUNCHES.items()), abs=0.1)
    else:
        assert "ncu_dram_bytes_per_cell" not in r["step_hbm"]
    tab32 = bench.COUNTERS["ppmc"]["fp32_bulk"]
    r32 = bench.roofline_of(_prof(ms, 10), "fp32_bulk", n3, 6791.4, "measured", "ppmc")
    assert r32["step_hbm"]["ncu_dram_bytes_per_cell"] == pytest.approx(
        sum(tab32[k][3] * n for k, n in LAUNCHES.items()), abs=0.1)


def test_roofline_without_counters_is_hbm_bound(bench):
    """A dominant stage without counters (the PLMC reconstruction, changed
    since its capture) is reported against HBM with no traffic figure, and
    the step-level ncu DRAM figure is left out."""
    n3 = 128 ** 3
    ms = {"prim": 0.5, "flux_pcm": 1.0, "emf": 0.4, "update_half": 0.4, "recon": 3.0, "flux_hlld": 1.0,
          "update_full": 0.2}
    assert "recon" not in bench.COUNTERS["plmc"]["fp64"]
    r = bench.roofline_of(_prof(ms, 2), "fp64", n3, 6791.4, "measured", "plmc")
    assert r["kernel"] == "recon"
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None
    assert r["frac"] == pytest.approx(176 * n3 / 3.0e-3 / 1e9 / 6791.4, abs=1e-4)  # (rounded to 4 places)
    assert "ncu_dram_bytes_per_cell" not in r["step_hbm"]


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


def test_issue_bound_stage_of_the_fp32_bulk_step(bench):
    """FP32-bulk: the dominant float reconstruction has no FP64 work, so its
    roofline is the warp-instruction issue rate against 4 per clock per SM."""
    n3 = 512 ** 3
    ms = {"prim": 5.8, "flux_pcm": 2.0, "emf": 1.6, "update_half": 7.3, "recon": 4.3, "flux_hlld": 2.3,
          "update_full": 5.3}
    r = bench.roofline_of(_prof(ms, 10), "fp32_bulk", n3, 6762.3, "measured", "ppmc")
    assert r["kernel"] == "recon" and r["bound"] == "alu"
    ops, flop, winst, dram = bench.COUNTERS["ppmc"]["fp32_bulk"]["recon"]
    assert ops == 0.0 and r["fp64_pipe"]["achieved"] == 0.0
    assert r["unit"] == "G warp-inst/s issued"
    assert r["achieved"] == pytest.approx(winst * n3 / 4.3e-3 / 1e9, rel=1e-3)
    assert r["traffic"] == round(dram * n3)
