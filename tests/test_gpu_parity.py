"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: FP64 step rel L1 <= 1e-12 per field after 10 steps (the stated
target); per-stage FP64 outputs element-wise within 1e-12 relative to the
field scale; FP32-bulk step rel L1 <= 1e-5 against the FP64 oracle.
Sizes span several 32 x 4 thread tiles with ragged tails.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2402_05240_gb300 import inputs as I  # noqa: E402
from tests.helpers import rel_l1  # noqa: E402

RAGGED = (37, 21, 19)


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
    a = np.asarray(a)
    b = np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ------------------------------------------------------------------ stages --
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("fp32_bulk", 1e-6)])
def test_primitives(mhd, precision, tol):
    U = turb(RAGGED)
    sim = mhd.Sim(*RAGGED, precision=precision)
    W = sim.primitives(cuda(U)).cpu().numpy()
    ref = O.Oracle(*RAGGED).primitives(U)
    for f in range(8):
        assert maxrel(W[f], ref[f]) < tol, f


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_dt(mhd, precision):
    U = turb(RAGGED)
    sim = mhd.Sim(*RAGGED, cfl=0.3, precision=precision)
    dt = sim.dt(cuda(U))
    ref = O.Oracle(*RAGGED).dt(U, 0.3)
    assert abs(dt - ref) <= (1e-14 if precision == "fp64" else 1e-6) * ref


def _energy_for_pressure(U, p, gamma=5.0 / 3.0):
    """Sets E so that the pressure recovered from U is p (face-averaged B)."""
    bcc = [0.5 * (U[5 + a] + np.roll(U[5 + a], 1, axis=2 - a)) for a in range(3)]
    ke = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
    U[4] = p / (gamma - 1.0) + ke + 0.5 * (bcc[0] ** 2 + bcc[1] ** 2 + bcc[2] ** 2)


@pytest.mark.parametrize("case", ["float_overflow", "float_underflow", "near_ties"])
def test_dt_extreme_states(mhd, case):
    """The FP64 CFL maximum selects its candidate cells from float estimates
    of the rates; states whose float estimates overflow, underflow or tie
    still give the oracle's dt (the exact per-cell maximum)."""
    n = RAGGED
    rng = np.random.default_rng(7)
    if case == "float_overflow":
        U = turb(n)
        # one strong face field: B_cc of two cells ~ 2e19, B^2 beyond float range
        U[5, 3, 5, 7] = 4e19
        _energy_for_pressure(U, 1.0)
    elif case == "float_underflow":
        U = turb(n)
        U[0] = 1e-30 * (1.0 + 0.5 * rng.random(U[0].shape))
        U[1:4] *= 1e-33
        U[5:8] = 1e-20 * (1.0 + rng.random(U[5:8].shape))  # B^2 ~ 1e-40 underflows in float
        _energy_for_pressure(U, 1e-35)
    else:
        U = I.uniform(I.Box(*n), 1.0, (1.0, 0.0, 0.0), 0.6, (0.3, 0.2, 0.1))
        U[1] *= 1.0 + 1e-13 * rng.standard_normal(U[1].shape)
        _energy_for_pressure(U, 0.6)
    sim = mhd.Sim(*n, cfl=0.3, rho_floor=1e-300, p_floor=1e-300)
    dt = sim.dt(cuda(U))
    ref = O.Oracle(*n, rho_floor=1e-300, p_floor=1e-300).dt(U, 0.3)
    assert abs(dt - ref) <= 1e-14 * ref, (case, dt, ref)


@pytest.mark.parametrize("recon", ["pcm", "plmc", "ppmc", "plm_prim"])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_recon_states(mhd, recon, axis):
    U = turb(RAGGED)
    sim = mhd.Sim(*RAGGED, recon=recon)
    WL, WR = sim.recon(cuda(U), axis)
    rL, rR = O.Oracle(*RAGGED).recon(U, axis, recon)
    for q in range(7):
        scale = np.max(np.abs(rL[q])) + 1e-300
        assert np.max(np.abs(WL.cpu().numpy()[q] - rL[q])) < 1e-12 * max(scale, 1.0), (q, "L")
        assert np.max(np.abs(WR.cpu().numpy()[q] - rR[q])) < 1e-12 * max(scale, 1.0), (q, "R")


@pytest.mark.parametrize("recon", ["pcm", "plmc", "ppmc"])
def test_fluxes(mhd, recon):
    U = turb(RAGGED)
    sim = mhd.Sim(*RAGGED, recon=recon)
    F = sim.fluxes(cuda(U)).cpu().numpy()
    ref = O.Oracle(*RAGGED, recon=recon).fluxes(U)
    for a in range(3):
        for q in range(7):
            scale = max(np.max(np.abs(ref[a, q])), 1e-3)
            assert np.max(np.abs(F[a, q] - ref[a, q])) < 1e-12 * scale, (a, q)


def test_edges(mhd):
    U = turb(RAGGED)
    orc = O.Oracle(*RAGGED)
    F = orc.fluxes(U, "plmc")
    E = mhd.Sim(*RAGGED).edges(cuda(U), cuda(F)).cpu().numpy()
    ref = orc.edges(U, F)
    assert maxrel(E, ref) < 1e-13


# -------------------------------------------------------------- full step --
def run_gpu(mhd, U0, n, nsteps, cfl, **kw):
    sim = mhd.Sim(*n, cfl=cfl, **kw)
    U = cuda(U0)
    dts = torch.zeros(nsteps, dtype=torch.float64, device="cuda")
    sim.run(U, nsteps, dts)
    torch.cuda.synchronize()
    sim.status()
    return U.cpu().numpy(), dts.cpu().numpy()


def test_config0_linear_wave_fp64(mhd):
    """32^3 fast wave, B = (1, sqrt2, 0.5), PLMC, CFL 0.4, 10 steps."""
    n = (32, 32, 32)
    U0, _ = I.linear_wave(I.Box(*n), amp=1e-6)
    got, dts = run_gpu(mhd, U0, n, 10, 0.4, recon="plmc")
    orc = O.Oracle(*n, recon="plmc")
    assert abs(dts[0] - orc.dt(U0, 0.4)) <= 1e-14 * dts[0]
    ref, _ = orc.run(U0, 10, dts=list(dts))
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-12), err
    # the wave itself (perturbation) agrees too, not only the background
    pert = np.sum(np.abs(got - ref)) / np.sum(np.abs(ref - I.uniform(I.Box(*n), 1.0, (0, 0, 0), 0.6,
                                                                           (1.0, math.sqrt(2), 0.5))))
    assert pert < 1e-8


@pytest.mark.parametrize("recon", ["pcm", "plmc", "ppmc", "plm_prim"])
def test_turbulent_ragged_fp64(mhd, recon):
    U0 = turb(RAGGED, seed=7)
    got, dts = run_gpu(mhd, U0, RAGGED, 10, 0.3, recon=recon)
    ref, _ = O.Oracle(*RAGGED, recon=recon).run(U0, 10, dts=list(dts))
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
def test_turbulent_fp32_bulk(mhd, recon):
    n = (40, 24, 20)
    U0 = turb(n, seed=9)
    got, dts = run_gpu(mhd, U0, n, 10, 0.3, recon=recon, precision="fp32_bulk")
    ref, _ = O.Oracle(*n, recon=recon).run(U0, 10, dts=list(dts))
    err = rel_l1(got, ref)
    assert np.all(err <= 1e-5), err


def test_step_returns_next_dt_and_floor_counts(mhd):
    n = (16, 12, 8)
    U0 = turb(n, seed=12)
    sim = mhd.Sim(*n, cfl=0.3)
    U = cuda(U0)
    nxt = sim.step(U, 1e-3, want_next_dt=True)
    ref = O.Oracle(*n).step(U0, 1e-3)
    assert abs(nxt - O.Oracle(*n).dt(ref, 0.3)) <= 1e-14 * nxt
    assert sim.dt(U) == nxt
    assert sim.floor_count() == (0, 0)


def test_fixed_dt_step_matches_run(mhd):
    n = (16, 12, 8)
    U0 = turb(n, seed=11)
    sim = mhd.Sim(*n, cfl=0.3)
    U = cuda(U0)
    dt = sim.dt(U)
    sim.step(U, dt)
    ref = O.Oracle(*n).step(U0, dt)
    assert np.all(rel_l1(U.cpu().numpy(), ref) <= 1e-13)


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk", "fp64_df"])
@pytest.mark.parametrize("n,steps", [((40, 28, 21), 3), ((20, 12, 5), 2)])
def test_run_host_equals_copy_run_copy(mhd, precision, n, steps):
    """mhd_run_host (the host-buffer entry point): the state (floors
    included, set high enough to fire) and the simulated time equal those of
    a copy, mhd_run and a copy back, bit for bit, from pinned, pageable and
    mhd_host_alloc (huge-page) host memory, in every precision."""
    U0 = turb(n, seed=11)
    ref_sim = mhd.Sim(*n, cfl=0.3, recon="ppmc", precision=precision, rho_floor=0.9, p_floor=0.5)
    ref = cuda(U0)
    dts = torch.zeros(steps, dtype=torch.float64, device="cuda")
    ref_sim.run(ref, steps, dts)
    ref_sim.status()
    for kind in ("pinned", "pageable", "host_buffer"):
        sim = mhd.Sim(*n, cfl=0.3, recon="ppmc", precision=precision, rho_floor=0.9, p_floor=0.5)
        host = torch.from_numpy(U0.copy())
        if kind == "pinned":
            host = host.pin_memory()
        elif kind == "host_buffer":
            hb = mhd.host_buffer(*host.shape)
            hb.copy_(host)
            host = hb
        t = mhd.mhd_run_host(sim.ctx, host, steps)
        assert torch.equal(host, ref.cpu()), (precision, n, steps, kind)
        assert t == float(dts.sum().item()) or abs(t - float(dts.sum().item())) <= 1e-15 * t
        sim.close()
    ref_sim.close()


def test_host_alloc_and_free(mhd):
    """mhd_host_alloc gives registered host memory that copies both ways and
    frees; size 0 and a NULL output are argument errors; freeing NULL is a
    no-op."""
    p = ctypes.c_void_p()
    assert mhd.LIB.mhd_host_alloc(0, ctypes.byref(p)) == mhd.MHD_ERR_ARG
    assert mhd.LIB.mhd_host_alloc(64, None) == mhd.MHD_ERR_ARG
    assert mhd.LIB.mhd_host_free(None) == mhd.MHD_OK
    nbytes = 3 * (1 << 20) + 8  # not a multiple of the huge page size
    assert mhd.LIB.mhd_host_alloc(nbytes, ctypes.byref(p)) == mhd.MHD_OK and p.value
    host = torch.frombuffer((ctypes.c_uint8 * nbytes).from_address(p.value), dtype=torch.uint8)
    host.copy_(torch.arange(nbytes, dtype=torch.int64).remainder(251).to(torch.uint8))
    dev = host.to("cuda", non_blocking=True)
    back = torch.empty_like(host)
    back.copy_(dev)
    assert torch.equal(back, host)
    del host
    assert mhd.LIB.mhd_host_free(p) == mhd.MHD_OK
    t = mhd.host_buffer(2, 3)
    assert t.shape == (2, 3) and t.dtype == torch.float64


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
def test_uniform_state_bit_identical(mhd, precision, recon):
    n = (33, 9, 6)
    U0 = I.uniform(I.Box(*n), 1.3, (0.4, -0.2, 0.3), 0.7, (0.6, -0.8, 0.2))
    got, _ = run_gpu(mhd, U0, n, 10, 0.4, recon=recon, precision=precision)
    assert np.array_equal(got, U0)


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_conservation_and_divb(mhd, precision):
    n = (48, 32, 24)
    U0 = turb(n, seed=13)
    sim = mhd.Sim(*n, cfl=0.3, precision=precision)
    U = cuda(U0)
    d0, t0 = sim.diagnostics(U)
    sim.run(U, 10)
    d1, t1 = sim.diagnostics(U)
    scale = np.array([np.sum(np.abs(U0[f])) for f in range(8)])
    assert np.all(np.abs(np.array(t1) - np.array(t0)) <= 1e-13 * scale)
    assert d1 * (1.0 / 24) / np.max(np.abs(U0[5:])) < 1e-13
    od, ot = O.Oracle(*n).diagnostics(U0)
    assert abs(d0 - od) <= 1e-15 * max(od, 1.0)
    np.testing.assert_allclose(t0, ot, rtol=1e-12, atol=1e-12 * np.max(scale))


# ---------------------------------------------------- full size, sampled --
def _subbox_step(U, c, dt, recon, r=8):
    """Oracle step on the periodic (2r+1)^3 neighbourhood of cell c; the centre
    depends only on cells within the one-step stencil radius (< r), so the
    wrap of the sub-box does not reach it."""
    nz, ny, nx = U.shape[1:]
    k, j, i = c
    ks = [(k + d) % nz for d in range(-r, r + 1)]
    js = [(j + d) % ny for d in range(-r, r + 1)]
    is_ = [(i + d) % nx for d in range(-r, r + 1)]
    sub = np.ascontiguousarray(U[:, ks][:, :, js][:, :, :, is_])
    m = 2 * r + 1
    orc = O.Oracle(m, m, m, dx=1.0 / nx, dy=1.0 / ny, dz=1.0 / nz, recon=recon)
    return orc.step(sub, dt)[:, r, r, r]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_bulk", 1e-5)])
def test_full_size_256_sampled(mhd, precision, tol):
    """256^3 turbulent box (the benchmark workload): 2 GPU steps, then a third
    step checked against the oracle at sampled cells, plus the invariants."""
    n = (256, 256, 256)
    U0 = I.turbulent_box(I.Box(*n), seed_v=1, seed_b=2)
    sim = mhd.Sim(*n, cfl=0.3, recon="plmc", precision=precision)
    U = cuda(U0)
    del U0
    sim.run(U, 2)
    before = U.cpu().numpy()
    dt = sim.dt(U)
    sim.step(U, dt)
    after = U.cpu().numpy()
    rng = np.random.default_rng(0)
    cells = [tuple(int(x) for x in rng.integers(0, 256, 3)) for _ in range(24)] + [(0, 0, 0), (255, 255, 255)]
    for c in cells:
        ref = _subbox_step(before, c, dt, "plmc")
        got = after[:, c[0], c[1], c[2]]
        scale = np.abs(ref) + np.array([1, 1, 1, 1, 1, 0.5, 0.5, 0.5])
        assert np.all(np.abs(got - ref) <= tol * scale), (c, got - ref)
    d, _ = sim.diagnostics(U)
    assert d * (1.0 / 256) / np.max(np.abs(after[5:])) < 1e-12


# ------------------------------------------------------------- error paths --
def test_error_codes(mhd):
    n = (8, 8, 8)
    U0 = I.uniform(I.Box(*n), 1.0, (0, 0, 0), 1.0, (0.1, 0.2, 0.3))
    sim = mhd.Sim(*n)
    U = cuda(U0)
    with pytest.raises(mhd.MHDError) as e:
        sim.step(U, -1.0)
    assert e.value.code == mhd.MHD_ERR_DT
    with pytest.raises(mhd.MHDError) as e:
        sim.step(U, float("nan"))
    assert e.value.code == mhd.MHD_ERR_DT
    bad = U0.copy()
    bad[0, 3, 3, 3] = float("nan")
    Ub = cuda(bad)
    with pytest.raises(mhd.MHDError) as e:
        sim.dt(Ub)
    assert e.value.code == mhd.MHD_ERR_NONFINITE
    bad = U0.copy()
    bad[0, 1, 2, 3] = -1.0
    Ub = cuda(bad)
    sim.step(Ub, 1e-3)
    code, _ = mhd.mhd_status(sim.ctx)
    assert code == mhd.MHD_ERR_NONFINITE
    # the context stays usable after an error
    sim.step(U, 1e-3)
    assert mhd.mhd_status(sim.ctx)[0] == mhd.MHD_OK


def test_floors_trigger_and_count(mhd):
    """A cell driven below the pressure floor is reset and counted (D-12)."""
    n = (16, 8, 8)
    box = I.Box(*n)
    x, _, _ = box.centres()
    vx = np.broadcast_to(np.where(x < 0.5, -3.0, 3.0), box.shape)  # strong rarefaction
    U0 = I.assemble(box, 1.0, (vx, np.zeros(box.shape), np.zeros(box.shape)), 1e-3, (0.0, 0.0, 0.0))
    pf = 5e-4
    sim = mhd.Sim(*n, cfl=0.3, rho_floor=1e-3, p_floor=pf)
    U = cuda(U0)
    dts = torch.zeros(5, dtype=torch.float64, device="cuda")
    sim.run(U, 5, dts)
    counts = sim.status()
    orc = O.Oracle(*n, rho_floor=1e-3, p_floor=pf)
    ref, _ = orc.run(U0, 5, dts=list(dts.cpu().numpy()))
    assert counts[1] > 0
    assert counts[1] == orc.floor_counts[1] and counts[0] == orc.floor_counts[0]
    assert np.all(rel_l1(U.cpu().numpy(), ref) <= 1e-12)


# ------------------------------------------------------------- edge sizes --
@pytest.mark.parametrize("n", [(4, 4, 4), (5, 4, 7), (4, 6, 5)])
@pytest.mark.parametrize("recon", ["pcm", "plmc", "ppmc"])
def test_smallest_grids(mhd, n, recon):
    """Grids at the 4-cell minimum per axis: one step's stencil (5 cells with
    PPMC) wraps around the periodic box more than once."""
    U0 = turb(n, seed=17, kmax=1)
    sim = mhd.Sim(*n, cfl=0.3, recon=recon)
    U = cuda(U0)
    dts = torch.zeros(5, dtype=torch.float64, device="cuda")
    sim.run(U, 5, dts)
    torch.cuda.synchronize()
    sim.status()
    ref, _ = O.Oracle(*n, recon=recon).run(U0, 5, dts=list(dts.cpu().numpy()))
    assert np.all(rel_l1(U.cpu().numpy(), ref) <= 1e-12)


def test_longest_z_axis(mhd):
    """nz = 65535, the largest extent the launch grid's z dimension takes,
    with 4 x 4 cells per plane."""
    n = (4, 4, 65535)
    U0 = turb(n, seed=19, kmax=2)
    sim = mhd.Sim(*n, cfl=0.3, recon="plmc")
    U = cuda(U0)
    dts = torch.zeros(2, dtype=torch.float64, device="cuda")
    sim.run(U, 2, dts)
    torch.cuda.synchronize()
    sim.status()
    ref, _ = O.Oracle(*n, recon="plmc").run(U0, 2, dts=list(dts.cpu().numpy()))
    assert np.all(rel_l1(U.cpu().numpy(), ref) <= 1e-12)


@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp64_df", 1e-12), ("fp32_bulk", 1e-5)])
def test_zero_field(mhd, recon, precision, tol):
    """B = 0 everywhere (the hydrodynamic limit of Sec. 2.1): HLLD without
    rotational states, B_n = B_t = 0 in every eigensystem (the
    beta = (1,1)/sqrt2 convention, c_s = c_a = 0), zero edge fields.  One step
    against the oracle; then six steps keep B exactly 0 on the GPU.  (The
    oracle's numerically inverted eigenvectors leave ~1e-17 of B after a step,
    and B_t/|B_t| of that noise replaces the (1,1)/sqrt2 convention in the next
    reconstruction: with c_s = c_a = 0 the basis of the degenerate waves is
    arbitrary and the limited slopes depend on it (reading D-28), so the two
    runs part at O(slope) from the second step.)"""
    n = (24, 20, 18)
    box = I.Box(*n)
    U0 = I.turbulent_box(box, seed_v=23, seed_b=24, kmax=4, b0=(0.0, 0.0, 0.0), db_rms=0.0)
    W = O.Oracle(*n).primitives(U0)
    x, y, z = box.centres()
    rho = W[0] * (1 + 0.2 * np.sin(2 * np.pi * (x + 0.13)) * np.cos(2 * np.pi * (y + 0.31)))
    pres = W[4] * (1 + 0.2 * np.cos(2 * np.pi * (x + 0.27)) * np.sin(2 * np.pi * (z + 0.41)))
    zero = np.zeros_like(rho)
    U0 = I.assemble(box, rho, (W[1], W[2], W[3]), np.ascontiguousarray(pres), (zero, zero, zero))
    sim = mhd.Sim(*n, cfl=0.3, recon=recon, precision=precision)
    orc = O.Oracle(*n, recon=recon)
    dt = orc.dt(U0, 0.3)
    U = cuda(U0)
    sim.step(U, dt)
    torch.cuda.synchronize()
    sim.status()
    got = U.cpu().numpy()
    ref = orc.step(U0, dt)
    assert np.max(np.abs(ref[5:])) < 1e-15
    err = rel_l1(got, ref)[:5]
    assert np.all(err <= tol), err
    sim.run(U, 5)
    torch.cuda.synchronize()
    sim.status()
    got = U.cpu().numpy()
    assert np.all(got[5:] == 0.0) and np.all(np.isfinite(got))


def test_diagnostics_totals_are_compensated(mhd):
    """The totals of the conservation diagnostics carry the rounding errors of
    their additions: a field of +-2^52-sized values that cancel to ~1e5 is
    summed to the exactly rounded total (math.fsum) within 1e-6, where plain
    pairwise summation is off by ~100."""
    n = (64, 32, 32)
    N = n[0] * n[1] * n[2]
    rng = np.random.default_rng(31)
    b = rng.integers(-2 ** 52, 2 ** 52, size=N // 2).astype(np.float64)
    x = np.concatenate([b, -b + rng.uniform(-1, 1, size=N // 2) * 1e3])
    rng.shuffle(x)
    U = turb(n, seed=3)
    U[1] = x.reshape(U[1].shape)
    sim = mhd.Sim(*n)
    _, tot = sim.diagnostics(cuda(U))
    ref = math.fsum(x)
    assert abs(float(np.sum(x)) - ref) > 10.0  # the case defeats plain summation
    assert abs(tot[1] - ref) <= 1e-6, (tot[1], ref)
    for f in (0, 4, 5, 6, 7):
        assert abs(tot[f] - math.fsum(U[f].ravel())) <= 1e-12 * math.fsum(np.abs(U[f]).ravel())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_bulk", 2e-5)])
def test_full_size_512_ppmc_sampled(mhd, precision, tol):
    """512^3 turbulent box with PPMC (the benchmark workload): one GPU step
    checked against the oracle at sampled cells, FP64 at 1e-12 and FP32-bulk
    at 2e-5 of each value's scale (float reconstruction and Riemann solver,
    one step)."""
    n = (512, 512, 512)
    U0 = I.turbulent_box(I.Box(*n), seed_v=1, seed_b=2)
    sim = mhd.Sim(*n, cfl=0.3, recon="ppmc", precision=precision)
    U = cuda(U0)
    dt = sim.dt(U)
    sim.step(U, dt)
    torch.cuda.synchronize()
    sim.status()
    rng = np.random.default_rng(7)
    cells = [tuple(int(x) for x in rng.integers(0, 512, 3)) for _ in range(12)] + [(0, 0, 0), (511, 511, 511)]
    idx = tuple(torch.tensor(v, device="cuda") for v in zip(*cells))
    got = U[:, idx[0], idx[1], idx[2]].cpu().numpy()
    del U, sim
    for m, c in enumerate(cells):
        ref = _subbox_step(U0, c, dt, "ppmc")
        scale = np.abs(ref) + np.array([1, 1, 1, 1, 1, 0.5, 0.5, 0.5])
        assert np.all(np.abs(got[:, m] - ref) <= tol * scale), (c, got[:, m] - ref)
