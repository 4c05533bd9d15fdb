"""GPU adjoint (vector-Jacobian products) against the oracle's forward-mode
derivatives (dual numbers): dot-product tests <J v, w> = <v, J^T w> for the
HLLD solver, the reconstruction and the whole step.  Tolerances: FP64 1e-10
relative; FP32-bulk 1e-3 relative to the FP64 reference derivative."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2402_05240_gb300 import inputs as I  # noqa: E402

G = 5.0 / 3.0


@pytest.fixture(scope="module")
def mhd():
    from paper_2402_05240_gb300 import build
    build.build()
    from paper_2402_05240_gb300 import mhd as m
    return m


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def face_states(n, seed):
    """Random face states over the solver's regimes: generic, supersonic either
    way, B_n = 0, B_t = 0 and strong fields."""
    rng = np.random.default_rng(seed)
    wl = np.column_stack([rng.uniform(0.3, 2, n), rng.normal(0, 1, n), rng.normal(0, 1, n), rng.normal(0, 1, n),
                          rng.uniform(0.2, 2, n), rng.normal(0, 1, n), rng.normal(0, 1, n)])
    wr = np.column_stack([rng.uniform(0.3, 2, n), rng.normal(0, 1, n), rng.normal(0, 1, n), rng.normal(0, 1, n),
                          rng.uniform(0.2, 2, n), rng.normal(0, 1, n), rng.normal(0, 1, n)])
    bn = rng.normal(0, 1, n)
    k = n // 6
    wl[:k, 1] += 8.0
    wr[:k, 1] += 8.0            # supersonic to the right
    wl[k:2 * k, 1] -= 8.0
    wr[k:2 * k, 1] -= 8.0       # supersonic to the left
    bn[2 * k:3 * k] = 0.0       # no rotational states
    wl[3 * k:4 * k, 5:] = 0.0
    wr[3 * k:4 * k, 5:] = 0.0   # no transverse field
    bn[4 * k:5 * k] *= 4.0      # strong normal field
    return wl, wr, bn


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32_bulk", 2e-3), ("fp64_df", 1e-10)])
def test_hlld_vjp_dot_product(mhd, precision, tol):
    n = 3000
    wl, wr, bn = face_states(n, 1)
    rng = np.random.default_rng(2)
    gf = rng.normal(size=(n, 7))
    dwl = rng.normal(size=(n, 7))
    dwr = rng.normal(size=(n, 7))
    dbn = rng.normal(size=n)
    out = [torch.zeros((n, 7), dtype=torch.float64, device="cuda") for _ in range(3)]
    gbn = torch.zeros(n, dtype=torch.float64, device="cuda")
    mhd.mhd_stage_hlld_vjp(G, mhd.PRECISION[precision], cuda(wl), cuda(wr), cuda(bn), cuda(gf), out[0], out[1], gbn,
                           out[2])
    torch.cuda.synchronize()
    gwl, gwr, f = (x.cpu().numpy() for x in out)
    gbn = gbn.cpu().numpy()
    bad = 0
    for t in range(n):
        fo, df = O.hlld_jvp(G, wl[t], wr[t], bn[t], dwl[t], dwr[t], dbn[t])
        lhs = float(df @ gf[t])
        rhs = float(dwl[t] @ gwl[t] + dwr[t] @ gwr[t] + dbn[t] * gbn[t])
        scale = np.abs(df) @ np.abs(gf[t]) + 1e-30
        if abs(lhs - rhs) > tol * scale:
            bad += 1
        if precision == "fp64":
            assert np.max(np.abs(f[t] - fo)) <= 1e-13 * (1 + np.max(np.abs(fo)))
    # FP32 branch decisions can differ from the FP64 reference on a few near-tie faces
    assert bad <= (0 if precision == "fp64" else n // 500), bad


def turb(n, seed, kmax=4):
    return I.turbulent_box(I.Box(*n), seed_v=seed, seed_b=seed + 1, kmax=kmax)


def generic(n, seed, kmax=4):
    """Turbulent box with smooth random density and pressure variations.

    The plain turbulent box has exactly uniform rho and P, so its entropy-wave
    characteristic slopes are pure rounding noise and the limiter branch
    (a_L a_R > 0) there is decided by noise: the derivative is not defined at
    such points.  Dot-product tests need a state away from limiter kinks.
    """
    box = I.Box(*n)
    U = turb(n, seed, kmax)
    W = O.Oracle(*n).primitives(U)
    rng = np.random.default_rng(seed + 100)
    x, y, z = box.centres()
    ph = rng.uniform(0, 2 * np.pi, 6)
    rho = W[0] * (1 + 0.2 * np.sin(2 * np.pi * x + ph[0]) * np.cos(2 * np.pi * y + ph[1]) * np.sin(2 * np.pi * z + ph[2]))
    p = W[4] * (1 + 0.2 * np.cos(2 * np.pi * x + ph[3]) * np.sin(2 * np.pi * y + ph[4]) * np.cos(2 * np.pi * z + ph[5]))
    return I.assemble(box, rho, (W[1], W[2], W[3]), p, (U[5], U[6], U[7]))


@pytest.mark.parametrize("recon", ["pcm", "plmc", "ppmc"])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_recon_vjp_dot_product(mhd, recon, axis):
    n = (21, 13, 11)
    U = generic(n, 31)
    rng = np.random.default_rng(3 + axis)
    dU = rng.normal(size=U.shape)
    gWL = rng.normal(size=(7,) + U.shape[1:])
    gWR = rng.normal(size=(7,) + U.shape[1:])
    WL, WR, dWL, dWR = O.Oracle(*n, recon=recon).recon_jvp(U, dU, axis)
    sim = mhd.Sim(*n, recon=recon)
    gU = sim.recon_vjp(cuda(U), axis, cuda(gWL), cuda(gWR)).cpu().numpy()
    lhs = np.sum(dWL * gWL) + np.sum(dWR * gWR)
    rhs = np.sum(dU * gU)
    scale = np.sum(np.abs(dWL * gWL)) + np.sum(np.abs(dWR * gWR))
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs)


@pytest.mark.parametrize("recon,precision,tol", [("pcm", "fp64", 1e-10), ("plmc", "fp64", 1e-10),
                                                 ("ppmc", "fp64", 1e-10), ("plmc", "fp32_bulk", 1e-3),
                                                 ("ppmc", "fp32_bulk", 1e-3), ("plmc", "fp64_df", 1e-10),
                                                 ("ppmc", "fp64_df", 1e-10)])
def test_adjoint_step_dot_product(mhd, recon, precision, tol):
    n = (26, 18, 14)
    U = turb(n, 41)
    orc = O.Oracle(*n, recon=recon)
    dt = orc.dt(U, 0.3)
    rng = np.random.default_rng(5)
    dU = rng.normal(size=U.shape)
    g = rng.normal(size=U.shape)
    _, JdU = orc.step_jvp(U, dU, dt)
    sim = mhd.Sim(*n, recon=recon, precision=precision)
    gU = sim.adjoint_step(cuda(U), dt, cuda(g)).cpu().numpy()
    lhs = float(np.sum(JdU * g))
    rhs = float(np.sum(dU * gU))
    scale = float(np.sum(np.abs(JdU * g)))
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, abs(lhs - rhs) / scale)


def test_adjoint_step_with_floors(mhd):
    """Floors that bind change the derivative; the adjoint follows them."""
    n = (16, 8, 8)
    box = I.Box(*n)
    x, _, _ = box.centres()
    vx = np.broadcast_to(np.where(x < 0.5, -3.0, 3.0), box.shape)
    rng0 = np.random.default_rng(9)
    rho0 = 1.0 + 0.1 * rng0.uniform(size=box.shape)
    p0 = 1e-3 * (1.0 + 0.1 * rng0.uniform(size=box.shape))
    vt = 0.1 * rng0.normal(size=(2,) + box.shape)
    U = I.assemble(box, rho0, (vx, vt[0], vt[1]), p0, (0.2, 0.1, 0.05))
    pf = 5e-4
    orc = O.Oracle(*n, rho_floor=1e-3, p_floor=pf, recon="plmc")
    U0, _ = orc.run(U, 3, cfl=0.3)
    # cells the previous steps left exactly at the floor sit on the kink of
    # max(P, P_floor); lift them to 1.5 P_floor so the derivative is defined
    W = O.Oracle(*n, rho_floor=1e-30, p_floor=-1e30).primitives(U0)
    W[4] = np.maximum(W[4], 1.5 * pf)
    U1 = I.assemble(box, W[0], (W[1], W[2], W[3]), W[4], (U0[5], U0[6], U0[7]))
    dt = orc.dt(U1, 0.3)
    orc.floor_counts[1] = 0
    orc.step(U1, dt)
    assert orc.floor_counts[1] > 0  # the pressure floor binds in the differentiated step
    rng = np.random.default_rng(6)
    dU = rng.normal(size=U.shape)
    g = rng.normal(size=U.shape)
    _, JdU = orc.step_jvp(U1, dU, dt)
    sim = mhd.Sim(*n, rho_floor=1e-3, p_floor=pf, recon="plmc")
    gU = sim.adjoint_step(cuda(U1), dt, cuda(g)).cpu().numpy()
    lhs, rhs = float(np.sum(JdU * g)), float(np.sum(dU * gU))
    assert abs(lhs - rhs) <= 1e-9 * float(np.sum(np.abs(JdU * g)))


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk", "fp64_df"])
@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
def test_adjoint_finite_on_quiet_regions(mhd, precision, recon):
    """The blast (uniform B along x) leaves cells with velocities and
    transverse fields of order 1e-33 around O(1) density and pressure: the
    reverse limiter formulas must not square such differences (they underflow,
    in FP32 at once) and the cotangent must stay finite."""
    n = (32, 32, 32)
    U0 = cuda(I.blast(I.Box(*n), seed=4))
    sim = mhd.Sim(*n, cfl=0.3, recon=recon, precision=precision, rho_floor=1e-4, p_floor=1e-6)
    sim.run(U0, 5)
    dt = sim.dt(U0)
    gU = sim.adjoint_step(U0, dt, torch.ones_like(U0))
    assert bool(torch.isfinite(gU).all())


@pytest.mark.parametrize("recon,precision,tol", [("plmc", "fp64", 1e-10), ("ppmc", "fp64", 1e-10),
                                                 ("pcm", "fp64", 1e-10), ("plmc", "fp64_df", 1e-10),
                                                 ("ppmc", "fp32_bulk", 1e-3)])
def test_adjoint_step_cfl_dot_product(mhd, recon, precision, tol):
    """The step at the CFL dt of its own start state: <J dU, g> from the
    oracle's dual numbers (the dt's derivative included) equals <dU, J^T g>
    from mhd_adjoint_step_cfl; the fixed-dt adjoint misses the dt term by far
    more than the FP64 tolerance; dt is mhd_dt's and g_dt = <g, dstep/d dt>
    matches a central difference of the oracle in dt."""
    n = (26, 18, 14)
    U = generic(n, 43)
    orc = O.Oracle(*n, recon=recon)
    rng = np.random.default_rng(15)
    dU = rng.normal(size=U.shape)
    g = rng.normal(size=U.shape)
    _, JdU, dt_o = orc.step_cfl_jvp(U, dU, 0.3)
    sim = mhd.Sim(*n, cfl=0.3, recon=recon, precision=precision)
    gU, dt, gdt = sim.adjoint_step_cfl(cuda(U), cuda(g))
    gU = gU.cpu().numpy()
    assert dt == sim.dt(cuda(U))
    assert abs(dt - dt_o) <= (1e-14 if precision != "fp32_bulk" else 1e-6) * dt
    lhs = float(np.sum(JdU * g))
    rhs = float(np.sum(dU * gU))
    scale = float(np.sum(np.abs(JdU * g)))
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, abs(lhs - rhs) / scale)
    gU0 = sim.adjoint_step(cuda(U), dt, cuda(g)).cpu().numpy()
    # the dt term is about 2e-4 of the scale here: resolved at the FP64 tolerance
    assert abs(float(np.sum(dU * gU0)) - lhs) > (100 * tol * scale if tol < 1e-6 else 0.0)
    if precision == "fp64":
        delta = 1e-6
        Sp = orc.step(U, dt * (1 + delta))
        Sm = orc.step(U, dt * (1 - delta))
        fd = float(np.sum(g * (Sp - Sm))) / (2 * delta * dt)
        # (smooth rho and P: no limiter switch within dt (1 +- 1e-6))
        assert abs(gdt - fd) <= 1e-6 * abs(fd), (gdt, fd)


def test_adjoint_step_cfl_deterministic(mhd):
    n = (40, 24, 20)
    U = cuda(turb(n, 44))
    g = cuda(np.random.default_rng(3).normal(size=(8, n[2], n[1], n[0])))
    sim = mhd.Sim(*n, cfl=0.3, recon="ppmc")
    a = sim.adjoint_step_cfl(U, g)
    b = sim.adjoint_step_cfl(U, g)
    assert torch.equal(a[0], b[0]) and a[1:] == b[1:]
