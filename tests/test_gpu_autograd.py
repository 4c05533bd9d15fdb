"""Gradients of a rollout through torch.autograd (adjoint steps with step-level
checkpointing) against central finite differences of the GPU forward, the
configuration of the adjoint benchmark at reduced size: turbulent box, PLMC,
loss = magnetic energy at the final step, gradients with respect to the
initial velocity (fixed rho, P) and the initial face field."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2402_05240_gb300 import inputs as I  # noqa: E402

G = 5.0 / 3.0


@pytest.fixture(scope="module")
def mods():
    from paper_2402_05240_gb300 import build
    build.build()
    from paper_2402_05240_gb300 import autograd as A
    from paper_2402_05240_gb300 import mhd
    return mhd, A


def setup_state(n, seed=3, kmax=4):
    U = I.turbulent_box(I.Box(*n), seed_v=seed, seed_b=seed + 1, kmax=kmax)
    rho = U[0]
    vel = U[1:4] / rho
    # pressure from the generator's recipe (uniform P = 1)
    pres = np.ones_like(rho)
    return rho, vel, pres, U[5:8]


def setup_generic(n, seed=3, kmax=2):
    """As setup_state with smooth density and pressure variations, so that no
    limiter sits on its kink (the recipe's uniform rho, P puts the entropy
    wave's characteristic slopes at exactly zero)."""
    rho, vel, pres, bf = setup_state(n, seed, kmax)
    box = I.Box(*n)
    x, y, z = box.centres()
    rho = rho * (1 + 0.2 * np.sin(2 * np.pi * (x + 0.1)) * np.cos(2 * np.pi * (y + 0.3)))
    pres = pres * (1 + 0.2 * np.cos(2 * np.pi * (x + 0.2)) * np.sin(2 * np.pi * (z + 0.4)))
    return rho, vel, np.ascontiguousarray(pres), bf


def loss_of(A, sim, n, rho, vel, pres, bface, nsteps, dts, k=None):
    U0 = A.conserved_from(rho, vel, pres, bface, G)
    Un = A.rollout(sim, U0, nsteps, dts=dts, checkpoint_every=k)
    nx, ny, nz = n
    return A.magnetic_energy(Un, 1.0 / (nx * ny * nz))


def div_free_direction(n, rng):
    """dB = curl dA of a random edge vector potential (discrete divergence 0)."""
    nx, ny, nz = n
    ax, ay, az = (rng.normal(size=(nz, ny, nx)) for _ in range(3))
    dx, dy, dz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    bx = (az - np.roll(az, 1, axis=1)) / dy - (ay - np.roll(ay, 1, axis=0)) / dz
    by = (ax - np.roll(ax, 1, axis=0)) / dz - (az - np.roll(az, 1, axis=2)) / dx
    bz = (ay - np.roll(ay, 1, axis=2)) / dx - (ax - np.roll(ax, 1, axis=1)) / dy
    d = np.stack([bx, by, bz])
    return d / np.max(np.abs(d))


@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
@pytest.mark.parametrize("state,eps", [("generic", 1e-7), ("turbulent", 1e-7)])
def test_rollout_gradient_vs_finite_differences(mods, recon, state, eps):
    """Central differences along 16 random directions (half velocity, half
    divergence-free face field).  With eps = 1e-6 the perturbed runs cross
    limiter and upwind switches in practically every direction at this size
    (the difference quotients at eps and 2 eps disagree); eps = 1e-7 keeps
    the rounding error of the quotient near 1e-5 and rarely crosses one.
    Directions whose quotients at eps and 2 eps disagree are redrawn."""
    mhd, A = mods
    n = (20, 16, 12)
    nsteps = 3
    rho, vel, pres, bf = setup_generic(n) if state == "generic" else setup_state(n, kmax=2)
    sim = mhd.Sim(*n, cfl=0.3, recon=recon)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    # record the dt sequence once, then hold it fixed (D-16)
    U0 = A.conserved_from(t(rho), t(vel), t(pres), t(bf), G)
    dts = []
    Ut = U0.clone()
    for _ in range(nsteps):
        dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
        mhd.mhd_run(sim.ctx, Ut, 1, dt_dev)
        dts.append(float(dt_dev.item()))
    v = t(vel).requires_grad_(True)
    b = t(bf).requires_grad_(True)
    L = loss_of(A, sim, n, t(rho), v, t(pres), b, nsteps, dts, k=2)
    L.backward()
    gv, gb = v.grad.cpu().numpy(), b.grad.cpu().numpy()
    rng = np.random.default_rng(11)
    ok = 0
    worst = 0.0
    for trial in range(16):
        if trial % 2 == 0:
            dv = rng.normal(size=vel.shape)
            dv /= np.max(np.abs(dv))
            db = np.zeros_like(bf)
        else:
            dv = np.zeros_like(vel)
            db = div_free_direction(n, rng)
        adj = float(np.sum(gv * dv) + np.sum(gb * db))

        def fd(eps):
            with torch.no_grad():
                lp = loss_of(A, sim, n, t(rho), t(vel + eps * dv), t(pres), t(bf + eps * db), nsteps, dts)
                lm = loss_of(A, sim, n, t(rho), t(vel - eps * dv), t(pres), t(bf - eps * db), nsteps, dts)
            return (float(lp) - float(lm)) / (2 * eps)

        f1, f2 = fd(eps), fd(2 * eps)
        if abs(f1 - f2) > 3e-5 * max(abs(f1), 1e-12):
            continue  # a limiter / upwind switch lies between the two evaluations: redraw
        ok += 1
        err = abs(f1 - adj) / max(abs(f1), 1e-12)
        worst = max(worst, err)
    assert ok >= 10, ok
    assert worst <= 1e-4, worst


def test_rollout_dt_grad_dot_product_and_finite_differences(mods):
    """rollout(dt_grad=True): each step's CFL dt is differentiated through its
    start state.  (1) Dot test of the 3-step gradient against the oracle's
    dual-number chain of CFL-coupled steps (1e-10); the fixed-dt gradient
    misses it.  (2) Central differences of the loss whose every run takes its
    own CFL dts, along 8 random directions (redrawn where the quotients at
    eps and 2 eps disagree)."""
    import oracle as O
    mhd, A = mods
    n = (20, 16, 12)
    nsteps = 3
    rho, vel, pres, bf = setup_generic(n)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    sim = mhd.Sim(*n, cfl=0.3, recon="plmc")
    U0 = A.conserved_from(t(rho), t(vel), t(pres), t(bf), G).cpu().numpy()
    rng = np.random.default_rng(21)
    gN = rng.normal(size=U0.shape)
    grads = {}
    for dt_grad in (True, False):
        U = t(U0).requires_grad_(True)
        L = torch.sum(A.rollout(sim, U, nsteps, checkpoint_every=2, dt_grad=dt_grad) * t(gN))
        L.backward()
        grads[dt_grad] = U.grad.cpu().numpy()
    orc = O.Oracle(*n, recon="plmc")
    v = rng.normal(size=U0.shape)
    V, dV = U0.copy(), v.copy()
    for _ in range(nsteps):
        V, dV, _ = orc.step_cfl_jvp(V, dV, 0.3)
    lhs = float(np.sum(gN * dV))
    scale = float(np.sum(np.abs(gN * dV)))
    assert abs(lhs - float(np.sum(v * grads[True]))) <= 1e-10 * scale
    assert abs(lhs - float(np.sum(v * grads[False]))) > 1e-8 * scale

    vv = t(vel).requires_grad_(True)
    b = t(bf).requires_grad_(True)
    U = A.conserved_from(t(rho), vv, t(pres), b, G)
    L = A.magnetic_energy(A.rollout(sim, U, nsteps, checkpoint_every=2, dt_grad=True), 1.0 / (n[0] * n[1] * n[2]))
    L.backward()
    gv, gb = vv.grad.cpu().numpy(), b.grad.cpu().numpy()
    ok, worst = 0, 0.0
    for trial in range(8):
        dv = rng.normal(size=vel.shape) if trial % 2 == 0 else np.zeros_like(vel)
        db = np.zeros_like(bf) if trial % 2 == 0 else div_free_direction(n, rng)
        if trial % 2 == 0:
            dv /= np.max(np.abs(dv))
        adj = float(np.sum(gv * dv) + np.sum(gb * db))

        def fd(eps):
            with torch.no_grad():
                lp = loss_of(A, sim, n, t(rho), t(vel + eps * dv), t(pres), t(bf + eps * db), nsteps, None)
                lm = loss_of(A, sim, n, t(rho), t(vel - eps * dv), t(pres), t(bf - eps * db), nsteps, None)
            return (float(lp) - float(lm)) / (2 * eps)

        f1, f2 = fd(1e-7), fd(2e-7)
        if abs(f1 - f2) > 3e-5 * max(abs(f1), 1e-12):
            continue
        ok += 1
        worst = max(worst, abs(f1 - adj) / max(abs(f1), 1e-12))
    assert ok >= 5, ok
    assert worst <= 1e-4, worst


def test_checkpointing_does_not_change_the_gradient(mods):
    mhd, A = mods
    n = (16, 12, 10)
    rho, vel, pres, bf = setup_state(n, seed=7)
    sim = mhd.Sim(*n, cfl=0.3, recon="plmc")
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    dts = [2e-3, 2.1e-3, 1.9e-3, 2e-3, 2.2e-3, 1.8e-3]
    grads = []
    for k in (None, 1, 2, 4):
        v = t(vel).requires_grad_(True)
        L = loss_of(A, sim, n, t(rho), v, t(pres), t(bf), len(dts), dts, k=k)
        L.backward()
        grads.append(v.grad.cpu().numpy())
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])


def test_fp32_bulk_gradient_close_to_fp64(mods):
    mhd, A = mods
    n = (20, 16, 12)
    rho, vel, pres, bf = setup_state(n, seed=13)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    dts = [2e-3] * 4
    out = []
    for precision in ("fp64", "fp32_bulk"):
        sim = mhd.Sim(*n, cfl=0.3, recon="plmc", precision=precision)
        v = t(vel).requires_grad_(True)
        b = t(bf).requires_grad_(True)
        L = loss_of(A, sim, n, t(rho), v, t(pres), b, len(dts), dts, k=2)
        L.backward()
        out.append((v.grad.cpu().numpy(), b.grad.cpu().numpy()))
    g32 = np.concatenate([out[1][0].ravel(), out[1][1].ravel()])
    g64 = np.concatenate([out[0][0].ravel(), out[0][1].ravel()])
    assert np.linalg.norm(g32 - g64) / np.linalg.norm(g64) <= 1e-3
    # the velocity gradient is small (the loss is magnetic): looser relative bound
    assert np.linalg.norm(out[1][0] - out[0][0]) / np.linalg.norm(out[0][0]) <= 1e-2
    assert math.isfinite(float(np.sum(out[1][0])))


def test_rollout_adjoint_128_cubed_20_steps(mods):
    """The adjoint configuration at full size: 128^3 turbulent box (the
    benchmark recipe), PLMC, 20 steps at the recorded dts.  (1) Dot test of
    the 20-step adjoint chain against the oracle's dual-number JVP of the
    same 20 steps along 2 seeded directions (a velocity-like and a
    divergence-free face-field one): <g_20, J v> = <J^T g_20, v>.  Central
    differences are no check at this size: 2M cells x 20 steps put a limiter
    or upwind switch between x + eps d and x - eps d for every direction
    tried.  (2) The FP32-bulk rollout gradient of the magnetic energy agrees
    with the FP64 one to 1e-3."""
    import oracle as O
    mhd, A = mods
    n = (128, 128, 128)
    nsteps = 20
    U0 = I.turbulent_box(I.Box(*n), seed_v=1, seed_b=2)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    sim = mhd.Sim(*n, cfl=0.3, recon="plmc")
    Ut = t(U0)
    dts, states = [], [U0]
    for _ in range(nsteps):
        d = torch.zeros(1, dtype=torch.float64, device="cuda")
        mhd.mhd_run(sim.ctx, Ut, 1, d)
        dts.append(float(d.item()))
        states.append(Ut.cpu().numpy())
    rng = np.random.default_rng(5)
    gN = rng.normal(size=U0.shape)
    g = t(gN)
    for s in range(nsteps - 1, -1, -1):
        g = sim.adjoint_step(t(states[s]), dts[s], g)
    g0 = g.cpu().numpy()
    orc = O.Oracle(*n, recon="plmc")
    for trial in range(2):
        v = np.zeros_like(U0)
        if trial == 0:
            v[1:4] = rng.normal(size=(3,) + U0.shape[1:]) * 1e-2
        else:
            v[5:8] = div_free_direction(n, rng) * 1e-2
        V, dV = U0, v
        for s in range(nsteps):
            V, dV = orc.step_jvp(V, dV, dts[s])
        lhs, rhs = float(np.sum(gN * dV)), float(np.sum(g0 * v))
        assert abs(lhs - rhs) <= 1e-8 * float(np.sum(np.abs(gN * dV))), (trial, lhs, rhs)
    # FP32-bulk against FP64 rollout gradients of the magnetic energy
    rho, vel, bf = U0[0], U0[1:4] / U0[0], U0[5:8]
    pres = np.ones_like(rho)
    grads = {}
    for precision in ("fp64", "fp32_bulk"):
        s = sim if precision == "fp64" else mhd.Sim(*n, cfl=0.3, recon="plmc", precision=precision)
        vv = t(vel).requires_grad_(True)
        b = t(bf).requires_grad_(True)
        L = loss_of(A, s, n, t(rho), vv, t(pres), b, nsteps, dts, k=5)
        L.backward()
        grads[precision] = np.concatenate([vv.grad.cpu().numpy().ravel(), b.grad.cpu().numpy().ravel()])
    assert np.linalg.norm(grads["fp32_bulk"] - grads["fp64"]) / np.linalg.norm(grads["fp64"]) <= 1e-3
