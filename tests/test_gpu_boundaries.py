"""Outflow (zero-gradient) boundaries on the GPU step: parity with the outflow
oracle, and the paper's Riemann problems (Sec. 3.1.4) and blast wave
(Sec. 3.1.5)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2402_05240_gb300 import inputs as I  # noqa: E402
from tests.helpers import rel_l1  # noqa: E402


@pytest.fixture(scope="module")
def mhd():
    from paper_2402_05240_gb300 import build
    build.build()
    from paper_2402_05240_gb300 import mhd as m
    return m


def cuda(U):
    return torch.from_numpy(np.ascontiguousarray(U)).cuda()


BC_XY = ("outflow", "outflow", "periodic")


@pytest.mark.parametrize("precision", ["fp64", "fp64_df"])
@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
def test_outflow_parity_turbulent(mhd, recon, precision):
    """Structure reaches the boundaries: a turbulent state with outflow on x
    and y (periodic z), 8 steps with device dt, against the outflow oracle
    (whose ghost depth differs from the library's)."""
    n = (30, 20, 12)
    U0 = I.turbulent_box(I.Box(*n), seed_v=21, seed_b=22, kmax=4)
    sim = mhd.Sim(*n, cfl=0.3, recon=recon, precision=precision, bc=BC_XY)
    U = cuda(U0)
    dts = torch.zeros(8, dtype=torch.float64, device="cuda")
    sim.run(U, 8, dts)
    sim.status()
    orc = O.OutflowOracle(*n, BC_XY, recon=recon)
    d = dts.cpu().numpy()
    assert abs(d[0] - orc.dt(U0, 0.3)) <= 1e-13 * d[0]
    ref, _ = orc.run(U0, 8, dts=list(d))
    err = rel_l1(U.cpu().numpy(), ref)
    assert np.all(err <= 1e-12), err


def test_outflow_step_dt_and_evolve_agree(mhd):
    n = (24, 16, 8)
    U0 = I.turbulent_box(I.Box(*n), seed_v=5, seed_b=6, kmax=3)
    bc = ("outflow", "periodic", "outflow")
    sim = mhd.Sim(*n, cfl=0.3, recon="plmc", bc=bc)
    orc = O.OutflowOracle(*n, bc, recon="plmc")
    U = cuda(U0)
    dt = sim.dt(U)
    assert abs(dt - orc.dt(U0, 0.3)) <= 1e-13 * dt
    sim.step(U, dt)
    assert np.all(rel_l1(U.cpu().numpy(), orc.step(U0, dt)) <= 1e-13)
    V = cuda(U0)
    t, nsteps = sim.evolve(V, 0.01)
    assert t == 0.01
    ref, tr, k = U0, 0.0, 0
    while tr < 0.01:  # CFL steps, the last one shortened to land on t = 0.01
        dt = orc.dt(ref, 0.3)
        if dt >= 0.01 - tr:
            dt = 0.01 - tr
        ref = orc.step(ref, dt)
        tr = 0.01 if dt == 0.01 - tr else tr + dt
        k += 1
    assert k == nsteps
    assert np.all(rel_l1(V.cpu().numpy(), ref) <= 1e-11)


def test_outflow_rejected_by_periodic_only_entry_points(mhd):
    n = (8, 8, 8)
    U = cuda(I.uniform(I.Box(*n), 1.0, (0, 0, 0), 1.0, (0.1, 0.2, 0.3)))
    sim = mhd.Sim(*n, bc=("outflow", "periodic", "periodic"))
    with pytest.raises(mhd.MHDError):
        sim.adjoint_step(U, 1e-3, torch.ones_like(U))
    with pytest.raises(mhd.MHDError):
        sim.recon(U, 0)


@pytest.mark.parametrize("name", list(I.RIEMANN))
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_riemann_parity(mhd, name, axis):
    """Each Riemann problem along each axis, 64 x 4 x 4 (axes cycled), PPMC,
    12 steps against the outflow oracle.  The Einfeldt problem is symmetric
    about the discontinuity (zero mass flux there in exact arithmetic, which
    rounding turns into either sign for the edge-field upwinding); its right
    state is skewed by 1e-3 to make the data generic."""
    skew = 1e-3 if name == "einfeldt" else 0.0
    box, U0, gamma, _ = I.riemann(name, n=64, ntrans=4, skew=skew)
    bc = ["periodic"] * 3
    bc[axis] = "outflow"
    for _ in range(axis):
        U0 = I.cycle_axes(U0)
    nz, ny, nx = U0.shape[1:]
    sim = mhd.Sim(nx, ny, nz, gamma=gamma, cfl=0.4, recon="ppmc", bc=tuple(bc))
    U = cuda(U0)
    dts = torch.zeros(12, dtype=torch.float64, device="cuda")
    sim.run(U, 12, dts)
    sim.status()
    orc = O.OutflowOracle(nx, ny, nz, tuple(bc), gamma=gamma, recon="ppmc")
    ref, _ = orc.run(U0, 12, dts=list(dts.cpu().numpy()))
    err = rel_l1(U.cpu().numpy(), ref)
    assert np.all(err <= 1e-12), err


def run_riemann(mhd, name, axis=0, mirror=False, n=512, dts=None):
    """Runs to t_max with CFL dts (returned), or with the given dts."""
    box, U0, gamma, t_max = I.riemann(name, n=n, ntrans=16, mirror=mirror)
    bc = ["periodic"] * 3
    bc[axis] = "outflow"
    for _ in range(axis):
        U0 = I.cycle_axes(U0)
    nz, ny, nx = U0.shape[1:]
    sim = mhd.Sim(nx, ny, nz, gamma=gamma, cfl=0.4, recon="ppmc", bc=tuple(bc))
    U = cuda(U0)
    if dts is None:
        dts, t = [], 0.0
        while t < t_max:
            dt = min(sim.dt(U), t_max - t)
            sim.step(U, dt)
            dts.append(dt)
            t += dt
    else:
        for dt in dts:
            sim.step(U, dt)
    sim.status()
    V = U.cpu().numpy()
    for _ in range((3 - axis) % 3):
        V = I.cycle_axes(V)
    return V, gamma, dts


@pytest.mark.parametrize("name", list(I.RIEMANN))
def test_riemann_paper_resolution(mhd, name):
    """512 x 16 x 16 to t_max (the paper's setup): positive density and
    pressure, uniform across the transverse directions, the same solution
    along y and z as along x, and for the mirrored problem."""
    V, gamma, dts = run_riemann(mhd, name)
    W = O.Oracle(512, 16, 16, gamma=gamma).primitives(V)
    assert W[0].min() > 0 and W[4].min() > 0
    assert np.max(np.abs(V - V[:, :1, :1, :])) == 0.0
    # Same dt sequence along y and z and for the mirrored problem: only the
    # rounding differs (the order of three-term sums over the components),
    # and ~500 steps of PPM grow it: a few 1e-9 on the Dai-Woodward problem,
    # up to 6e-8 in the transverse fields of Ryu-Jones 4d, whose left state
    # has B_t = 0 exactly -- there the eigenvectors take the beta = (1,1)/sqrt2
    # convention, which couples the two transverse directions, and the
    # coupled components then grow from summation-order rounding.
    for axis in (1, 2):
        Va, _, _ = run_riemann(mhd, name, axis=axis, dts=dts)
        assert np.all(rel_l1(Va, V) <= 1e-7), axis
    if name == "einfeldt":
        return  # symmetric about x = 1/2: its own mirror image, decided at exact ties
    Vm, _, _ = run_riemann(mhd, name, mirror=True, dts=dts)
    m = Vm[..., ::-1].copy()
    m[1] = -m[1]
    m[5] = -Vm[5][..., ::-1]
    assert np.all(rel_l1(m, V) <= 1e-7)


def test_blast_parity(mhd):
    """Parity on the blast with its centre moved off the symmetry point (the
    centred blast has zero mass fluxes on its symmetry planes in exact
    arithmetic, which rounding turns into either sign for the upwinding)."""
    box, U0 = I.blast_paper(16, 24, 16, centre=(0.5123, 0.7377, 0.4911))
    sim = mhd.Sim(box.nx, box.ny, box.nz, box.lx, box.ly, box.lz, cfl=0.4, recon="ppmc")
    U = cuda(U0)
    dts = torch.zeros(8, dtype=torch.float64, device="cuda")
    sim.run(U, 8, dts)
    sim.status()
    orc = O.Oracle(box.nx, box.ny, box.nz, recon="ppmc", lx=box.lx, ly=box.ly, lz=box.lz)
    ref, _ = orc.run(U0, 8, dts=list(dts.cpu().numpy()))
    assert np.all(rel_l1(U.cpu().numpy(), ref) <= 1e-12)


def test_blast_reduced(mhd):
    """The strongly magnetised blast (Sec. 3.1.5) at 64 x 96 x 64 to t = 0.2,
    periodic: conservation, div B at round-off, positivity.  (The method as
    read is not exactly symmetric under point inversion: the oracle shows the
    same 1e-4 asymmetry after two steps, so no symmetry is asserted.)"""
    box, U0 = I.blast_paper(64, 96, 64)
    sim = mhd.Sim(box.nx, box.ny, box.nz, box.lx, box.ly, box.lz, cfl=0.4, recon="plmc")
    U = cuda(U0)
    _, t0 = sim.diagnostics(U)
    t, n = sim.evolve(U, 0.2)
    sim.status()
    d1, t1 = sim.diagnostics(U)
    assert t == 0.2 and n > 50
    scale = np.array([np.sum(np.abs(U0[f])) for f in range(8)])
    assert np.all(np.abs(np.array(t1) - np.array(t0)) <= 1e-12 * scale + 1e-12)
    assert d1 * box.dx < 1e-12
    V = U.cpu().numpy()
    W = O.Oracle(box.nx, box.ny, box.nz, lx=box.lx, ly=box.ly, lz=box.lz).primitives(V)
    assert W[0].min() > 0 and W[4].min() > 0
