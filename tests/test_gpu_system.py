"""The paper's periodic system problems (Sec. 3.1) run on the GPU step.

* Linear waves (Sec. 3.1.1): all four MHD waves on the B = (1, 1.5, 0)
  background, one period on N x 16 x 16; second-order convergence of the L2
  norm of the per-variable L1 errors, PPM more accurate than PLM, and the
  same error for every axis and both directions of travel.
* Circularly polarised Alfven wave (Sec. 3.1.2): second-order convergence
  of the travelling wave on 2N x N x N.
* Advecting field loop (Sec. 3.1.3): div B at round-off through two periods,
  magnetic energy loss that shrinks with resolution.
* Orszag-Tang vortex (Sec. 3.1.6): parity with the oracle over the first
  steps, conservation and div B through t = 0.5.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2402_05240_gb300 import inputs as I  # noqa: E402
from tests.helpers import rel_l1  # noqa: E402

BG = dict(rho=1.0, pres=0.6, b=(1.0, 1.5, 0.0))  # P = 1/gamma
WAVES = {"fast": "fast+", "alfven": "alfven+", "slow": "slow+", "entropy": "entropy"}


@pytest.fixture(scope="module")
def mhd():
    from paper_2402_05240_gb300 import build
    build.build()
    from paper_2402_05240_gb300 import mhd as m
    return m


def cuda(U):
    return torch.from_numpy(np.ascontiguousarray(U)).cuda()


def wave_state(n, wave, sign=+1, axis=0):
    """Linear wave along `axis` on n cells (16 across), travelling in +/-."""
    name = WAVES[wave]
    if sign < 0 and name != "entropy":
        name = name[:-1] + "-"
    vel = (1.0, 0.0, 0.0) if wave == "entropy" else (0.0, 0.0, 0.0)
    if wave == "entropy" and sign < 0:
        vel = (-1.0, 0.0, 0.0)
    U, speed = I.linear_wave(I.Box(n, 16, 16), amp=1e-6, rho=BG["rho"], vel=vel, pres=1.0 / (5.0 / 3.0),
                             b=BG["b"], wave=name)
    for _ in range(axis):
        U = I.cycle_axes(U)
    return U, abs(speed)


def wave_error(mhd, n, wave, recon, sign=+1, axis=0):
    U0, speed = wave_state(n, wave, sign, axis)
    nz, ny, nx = U0.shape[1:]
    sim = mhd.Sim(nx, ny, nz, cfl=0.4, recon=recon)
    U = cuda(U0)
    t, _ = sim.evolve(U, 1.0 / speed)
    sim.status()
    assert t == 1.0 / speed
    return I.l1_error_norm(U.cpu().numpy(), U0)


@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
@pytest.mark.parametrize("wave", list(WAVES))
def test_linear_wave_second_order(mhd, wave, recon):
    # N = 16 is pre-asymptotic for the PLM Alfven wave (slope 1.4 from 16 to 32)
    errs = [wave_error(mhd, n, wave, recon) for n in (32, 64, 128)]
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(slopes) >= 1.8, (errs, slopes)


@pytest.mark.parametrize("wave", list(WAVES))
def test_ppm_more_accurate_than_plm(mhd, wave):
    e_plm = wave_error(mhd, 32, wave, "plmc")
    e_ppm = wave_error(mhd, 32, wave, "ppmc")
    assert e_ppm < 0.5 * e_plm, (e_plm, e_ppm)


@pytest.mark.parametrize("wave", list(WAVES))
def test_linear_wave_same_error_every_axis_and_direction(mhd, wave):
    errs = [wave_error(mhd, 32, wave, "plmc", sign, axis) for axis in (0, 1, 2) for sign in (+1, -1)]
    assert max(errs) - min(errs) <= 1e-6 * max(errs), errs


def cpaw_error(mhd, n, recon):
    box, U0 = I.cpaw(n)
    sim = mhd.Sim(box.nx, box.ny, box.nz, box.lx, box.ly, box.lz, cfl=0.4, recon=recon)
    U = cuda(U0)
    t, _ = sim.evolve(U, 1.0)
    sim.status()
    d, _ = sim.diagnostics(U)
    return I.l1_error_norm(U.cpu().numpy(), U0), d * box.dx / np.max(np.abs(U0[5:]))


@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
def test_cpaw_second_order(mhd, recon):
    res = [cpaw_error(mhd, n, recon) for n in (8, 16, 32)]
    errs = [r[0] for r in res]
    slope = math.log2(errs[1] / errs[2])
    assert slope >= 1.7, (errs, slope)
    assert max(r[1] for r in res) < 1e-13


def field_loop_run(mhd, n, recon="plmc"):
    box, U0 = I.field_loop(n)
    sim = mhd.Sim(box.nx, box.ny, box.nz, box.lx, box.ly, box.lz, cfl=0.4, recon=recon)
    U = cuda(U0)

    def b2_mean(V):
        bx = 0.5 * (V[5] + torch.roll(V[5], 1, dims=2))
        by = 0.5 * (V[6] + torch.roll(V[6], 1, dims=1))
        bz = 0.5 * (V[7] + torch.roll(V[7], 1, dims=0))
        return float(torch.mean(bx * bx + by * by + bz * bz))

    e0 = b2_mean(U)
    divs = []
    for _ in range(4):  # two periods in quarters; each evolve call advances 0.5
        sim.evolve(U, 0.5)
        d, _ = sim.diagnostics(U)
        divs.append(d * box.dx)
    sim.status()
    return b2_mean(U) / e0, max(divs), float(np.max(np.abs(U0[5:])))


def test_field_loop_divergence_and_dissipation(mhd):
    r16, div16, b16 = field_loop_run(mhd, 16)
    r32, div32, b32 = field_loop_run(mhd, 32)
    # div B stays at round-off through two periods (Sec. 3.1.3)
    assert div16 < 1e-13 * b16 and div32 < 1e-13 * b32, (div16, div32)
    # the loop loses magnetic energy, less at higher resolution
    assert 0.0 < r16 < r32 < 1.0, (r16, r32)


def test_orszag_tang_matches_oracle(mhd):
    box, U0 = I.orszag_tang(32, nz=4)
    sim = mhd.Sim(box.nx, box.ny, box.nz, cfl=0.4, recon="plmc")
    U = cuda(U0)
    dts = torch.zeros(10, dtype=torch.float64, device="cuda")
    sim.run(U, 10, dts)
    sim.status()
    ref, _ = O.Oracle(box.nx, box.ny, box.nz, recon="plmc").run(U0, 10, dts=list(dts.cpu().numpy()))
    assert np.all(rel_l1(U.cpu().numpy(), ref) <= 1e-12)


@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
def test_orszag_tang_to_half_time(mhd, recon):
    box, U0 = I.orszag_tang(64, nz=4)
    sim = mhd.Sim(box.nx, box.ny, box.nz, cfl=0.4, recon=recon)
    U = cuda(U0)
    d0, t0 = sim.diagnostics(U)
    t, n = sim.evolve(U, 0.5)
    sim.status()
    assert t == 0.5 and n > 100
    d1, t1 = sim.diagnostics(U)
    V = U.cpu().numpy()
    scale = np.array([np.sum(np.abs(U0[f])) for f in range(8)])
    assert np.all(np.abs(np.array(t1) - np.array(t0)) <= 1e-12 * scale + 1e-13)
    assert d1 * box.dx / np.max(np.abs(U0[5:])) < 1e-12
    W = O.Oracle(box.nx, box.ny, box.nz).primitives(V)
    assert W[0].min() > 0 and W[4].min() > 0
    # the flow is uniform along z
    assert np.max(np.abs(V - V[:, :1])) <= 1e-12 * np.max(np.abs(V))


@pytest.mark.parametrize("problem", ["cpaw", "field_loop"])
def test_system_problem_matches_oracle(mhd, problem):
    """Parity on the CPAW and on a generic field loop (off-centre, with a
    weak oblique background field).  The paper's loop has exact ties for the
    PPM limiter: cells equal in exact arithmetic by symmetry differ in the
    last bit, and where B vanishes or one of its components does, some
    characteristic differences are exactly 0 in exact arithmetic but come
    out as +-1e-20 from the oracle's numerically inverted eigenvectors.  The
    extremum test (q_i - q_{i-1})(q_{i+1} - q_i) <= 0 then takes either
    branch, both valid, with results that differ at the size of the data.
    Generic data has no such ties."""
    if problem == "cpaw":
        box, U0 = I.cpaw(8)
    else:
        box, U0 = I.field_loop(8, centre=(0.0123, -0.0217, 0.0311), b0=(3.1e-5, 4.7e-5, 8.3e-5))
    sim = mhd.Sim(box.nx, box.ny, box.nz, box.lx, box.ly, box.lz, cfl=0.4, recon="ppmc")
    U = cuda(U0)
    dts = torch.zeros(10, dtype=torch.float64, device="cuda")
    sim.run(U, 10, dts)
    sim.status()
    orc = O.Oracle(box.nx, box.ny, box.nz, recon="ppmc", lx=box.lx, ly=box.ly, lz=box.lz)
    ref, _ = orc.run(U0, 10, dts=list(dts.cpu().numpy()))
    err = rel_l1(U.cpu().numpy(), ref)
    assert np.all(err <= 1e-12), (err, np.abs(U.cpu().numpy() - ref).reshape(8, -1).max(axis=1))
