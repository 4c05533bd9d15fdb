"""GPU parity of the double-float mode (MHD_FP64_DF) against the CPU oracle.

The mode runs reconstruction, HLLD, edge fields and the update increments in
float pairs (about 2^-47 relative error per operation) and keeps the state,
the pressure recovery and the accumulation in double, so it is held to the
FP64 targets: per-stage outputs within 1e-12 of the field scale, the step
within rel L1 1e-12 per field after 10 steps, conservation and div B at the
FP64 bounds, and a uniform state bit-identical.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2402_05240_gb300 import inputs as I  # noqa: E402
from tests.helpers import rel_l1  # noqa: E402

RAGGED = (37, 21, 19)
P = "fp64_df"


@pytest.fixture(scope="module")
def mhd():
    from paper_2402_05240_gb300 import build
    build.build()
    from paper_2402_05240_gb300 import mhd as m
    return m


def turb(n, seed=3, kmax=4):
    return I.turbulent_box(I.Box(*n), seed_v=seed, seed_b=seed + 1, kmax=kmax)


def cuda(U):
    return torch.from_numpy(np.ascontiguousarray(U)).cuda()


def maxrel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


def test_primitives_and_dt(mhd):
    U = turb(RAGGED)
    sim = mhd.Sim(*RAGGED, cfl=0.3, precision=P)
    W = sim.primitives(cuda(U)).cpu().numpy()
    orc = O.Oracle(*RAGGED)
    ref = orc.primitives(U)
    for f in range(8):
        # the primitives are computed in double and stored as float pairs
        assert maxrel(W[f], ref[f]) < 2e-14, f
    dt = sim.dt(cuda(U))
    assert abs(dt - orc.dt(U, 0.3)) <= 1e-13 * dt


@pytest.mark.parametrize("recon", ["pcm", "plmc", "ppmc"])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_recon_states(mhd, recon, axis):
    U = turb(RAGGED)
    sim = mhd.Sim(*RAGGED, recon=recon, precision=P)
    WL, WR = sim.recon(cuda(U), axis)
    rL, rR = O.Oracle(*RAGGED).recon(U, axis, recon)
    for q in range(7):
        scale = max(np.max(np.abs(rL[q])), 1.0)
        assert np.max(np.abs(WL.cpu().numpy()[q] - rL[q])) < 1e-12 * scale, (q, "L")
        assert np.max(np.abs(WR.cpu().numpy()[q] - rR[q])) < 1e-12 * scale, (q, "R")


@pytest.mark.parametrize("recon", ["pcm", "plmc", "ppmc"])
def test_fluxes(mhd, recon):
    U = turb(RAGGED)
    F = mhd.Sim(*RAGGED, recon=recon, precision=P).fluxes(cuda(U)).cpu().numpy()
    ref = O.Oracle(*RAGGED, recon=recon).fluxes(U)
    for a in range(3):
        for q in range(7):
            scale = max(np.max(np.abs(ref[a, q])), 1e-3)
            assert np.max(np.abs(F[a, q] - ref[a, q])) < 1e-12 * scale, (a, q)


def test_edges(mhd):
    U = turb(RAGGED)
    orc = O.Oracle(*RAGGED)
    F = orc.fluxes(U, "plmc")
    E = mhd.Sim(*RAGGED, precision=P).edges(cuda(U), cuda(F)).cpu().numpy()
    assert maxrel(E, orc.edges(U, F)) < 1e-12


def run_gpu(mhd, U0, n, nsteps, cfl, **kw):
    sim = mhd.Sim(*n, cfl=cfl, precision=P, **kw)
    U = cuda(U0)
    dts = torch.zeros(nsteps, dtype=torch.float64, device="cuda")
    sim.run(U, nsteps, dts)
    torch.cuda.synchronize()
    sim.status()
    return U.cpu().numpy(), dts.cpu().numpy()


@pytest.mark.parametrize("recon", ["pcm", "plmc", "ppmc"])
def test_turbulent_ragged(mhd, recon):
    U0 = turb(RAGGED, seed=7)
    got, dts = run_gpu(mhd, U0, RAGGED, 10, 0.3, recon=recon)
    ref, _ = O.Oracle(*RAGGED, recon=recon).run(U0, 10, dts=list(dts))
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-12), err


def test_linear_wave_32(mhd):
    n = (32, 32, 32)
    U0, _ = I.linear_wave(I.Box(*n), amp=1e-6)
    got, dts = run_gpu(mhd, U0, n, 10, 0.4, recon="plmc")
    ref, _ = O.Oracle(*n, recon="plmc").run(U0, 10, dts=list(dts))
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-12), err
    # the 1e-6 wave itself, not only the background, is carried at FP64 accuracy
    bg = I.uniform(I.Box(*n), 1.0, (0, 0, 0), 0.6, (1.0, np.sqrt(2.0), 0.5))
    assert np.sum(np.abs(got - ref)) / np.sum(np.abs(ref - bg)) < 1e-7


@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
def test_uniform_state_bit_identical(mhd, recon):
    n = (33, 9, 6)
    U0 = I.uniform(I.Box(*n), 1.3, (0.4, -0.2, 0.3), 0.7, (0.6, -0.8, 0.2))
    got, _ = run_gpu(mhd, U0, n, 10, 0.4, recon=recon)
    assert np.array_equal(got, U0)


def test_conservation_and_divb(mhd):
    n = (48, 32, 24)
    U0 = turb(n, seed=13)
    sim = mhd.Sim(*n, cfl=0.3, precision=P)
    U = cuda(U0)
    _, t0 = sim.diagnostics(U)
    sim.run(U, 10)
    d1, t1 = sim.diagnostics(U)
    scale = np.array([np.sum(np.abs(U0[f])) for f in range(8)])
    assert np.all(np.abs(np.array(t1) - np.array(t0)) <= 1e-13 * scale)
    assert d1 * (1.0 / 24) / np.max(np.abs(U0[5:])) < 1e-13


def test_matches_fp64_mode(mhd):
    """The two FP64-accurate modes agree with each other at the 1e-12 level
    on the same dt sequence (both are within 1e-12 of the oracle)."""
    n = (40, 24, 20)
    U0 = turb(n, seed=21)
    out = []
    dts = None
    for prec in ("fp64", P):
        sim = mhd.Sim(*n, cfl=0.3, recon="ppmc", precision=prec)
        U = cuda(U0)
        if dts is None:
            d = torch.zeros(10, dtype=torch.float64, device="cuda")
            sim.run(U, 10, d)
            dts = d.cpu().numpy().tolist()
        else:
            for dt in dts:
                sim.step(U, dt)
        torch.cuda.synchronize()
        sim.status()
        out.append(U.cpu().numpy())
    assert np.all(rel_l1(out[1], out[0]) <= 1e-12)


def test_adjoint_matches_the_fp64_adjoint(mhd):
    """The double-float adjoint step agrees with the FP64 adjoint to the
    FP64 tolerance, and passes the dot-product test against the oracle's
    dual-number JVP of the step."""
    n = (16, 12, 10)
    U0 = turb(n, seed=5)
    rng = np.random.default_rng(2)
    gnp = rng.normal(size=U0.shape)
    g = cuda(gnp)
    res = []
    for prec in ("fp64", P):
        sim = mhd.Sim(*n, cfl=0.3, recon="plmc", precision=prec)
        res.append(sim.adjoint_step(cuda(U0), 2e-3, g).cpu().numpy())
    scale = np.abs(res[0]).reshape(8, -1).max(axis=1)[:, None, None, None] + 1e-300
    assert np.max(np.abs(res[1] - res[0]) / scale) < 1e-11
    # <J v, g> = <v, J^T g> with J v from the oracle's dual numbers
    v = rng.normal(size=U0.shape) * 1e-3
    Jv = O.Oracle(*n, recon="plmc").step_jvp(U0, v, 2e-3)[1]
    lhs, rhs = float(np.sum(Jv * gnp)), float(np.sum(v * res[1]))
    assert abs(lhs - rhs) <= 1e-10 * float(np.sum(np.abs(Jv * gnp))), (lhs, rhs)


def test_full_size_256_sampled(mhd):
    """256^3 turbulent box: 2 steps, then a third checked at sampled cells
    against the oracle on each cell's periodic neighbourhood."""
    from tests.test_gpu_parity import _subbox_step
    n = (256, 256, 256)
    U0 = I.turbulent_box(I.Box(*n), seed_v=1, seed_b=2)
    sim = mhd.Sim(*n, cfl=0.3, recon="plmc", precision=P)
    U = cuda(U0)
    del U0
    sim.run(U, 2)
    before = U.cpu().numpy()
    dt = sim.dt(U)
    sim.step(U, dt)
    after = U.cpu().numpy()
    rng = np.random.default_rng(1)
    cells = [tuple(int(x) for x in rng.integers(0, 256, 3)) for _ in range(16)] + [(0, 0, 0), (255, 255, 255)]
    for c in cells:
        ref = _subbox_step(before, c, dt, "plmc")
        got = after[:, c[0], c[1], c[2]]
        scale = np.abs(ref) + np.array([1, 1, 1, 1, 1, 0.5, 0.5, 0.5])
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (c, got - ref)


@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
def test_blast_with_quiet_regions(mhd, recon):
    """The strongly magnetised blast (uniform B along x): transverse fields
    and velocities start at exactly zero and grow from rounding to values of
    1e-20 and below, where float pairs run out of exponent range (their
    squares underflow).  The step stays finite and within 1e-12 of the
    oracle."""
    n = (24, 20, 16)
    U0 = I.blast(I.Box(*n), seed=4)
    got, dts = run_gpu(mhd, U0, n, 10, 0.3, recon=recon, rho_floor=1e-4, p_floor=1e-6)
    assert np.all(np.isfinite(got))
    ref, _ = O.Oracle(*n, recon=recon, rho_floor=1e-4, p_floor=1e-6).run(U0, 10, dts=list(dts))
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-12), err
