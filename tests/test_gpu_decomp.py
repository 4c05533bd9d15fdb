"""Virtual subdomains on one GPU: a grid split into 2 x 2 x 2 (and 3 x 1 x 2)
subdomains, each stepped by mhd_step_sub from the global state (periodic
halo gathered by the kernel), reproduces the monolithic step bit for bit;
the minimum of the subdomains' mhd_dt_sub is the monolithic dt."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2402_05240_gb300 import inputs as I  # noqa: E402

N = (36, 28, 20)


@pytest.fixture(scope="module")
def mhd():
    from paper_2402_05240_gb300 import build
    build.build()
    from paper_2402_05240_gb300 import mhd as m
    return m


@pytest.mark.parametrize("precision", ["fp64", "fp64_df", "fp32_bulk"])
@pytest.mark.parametrize("recon,parts", [("plmc", (2, 2, 2)), ("ppmc", (3, 1, 2))])
def test_subdomains_reproduce_monolithic_steps(mhd, recon, parts, precision):
    from paper_2402_05240_gb300 import decomp
    U0 = I.turbulent_box(I.Box(*N), seed_v=41, seed_b=42, kmax=5)
    mono = mhd.Sim(*N, cfl=0.3, recon=recon, precision=precision)
    plan = decomp.plan(N, parts)
    bc = tuple("halo" if parts[a] > 1 else "periodic" for a in range(3))
    subs = [mhd.Sim(*p.size, lx=p.size[0] / N[0], ly=p.size[1] / N[1], lz=p.size[2] / N[2], cfl=0.3,
                    recon=recon, precision=precision, bc=bc) for p in plan]
    Um = torch.from_numpy(U0).cuda()
    Ud = Um.clone()
    for _ in range(4):
        dt = mono.dt(Um)
        dts = [mhd.mhd_dt_sub(s.ctx, Ud, p.offset) for s, p in zip(subs, plan)]
        assert min(dts) == dt
        mono.step(Um, dt)
        Unew = torch.empty_like(Ud)
        for s, p in zip(subs, plan):
            mhd.mhd_step_sub(s.ctx, Ud, p.offset, dt, Unew)
        Ud = Unew
    torch.cuda.synchronize()
    mono.status()
    for s in subs:
        s.status()
    assert torch.equal(Ud, Um)


def test_halo_extended_block_input(mhd):
    """mhd_step_sub on a subdomain's own halo-extended block (offset = halo,
    the form a rank receives after the exchange) equals the global gather."""
    from paper_2402_05240_gb300 import decomp
    U0 = torch.from_numpy(I.turbulent_box(I.Box(*N), seed_v=43, seed_b=44, kmax=5)).cuda()
    parts = (2, 2, 1)
    p = decomp.plan(N, parts)[3]
    h = decomp.HALO
    sim = mhd.Sim(*p.size, lx=p.size[0] / N[0], ly=p.size[1] / N[1], lz=p.size[2] / N[2], cfl=0.3,
                  recon="ppmc", bc=("halo", "halo", "periodic"))
    (ox, oy, oz), (nx, ny, nz) = p.offset, p.size
    ix = torch.arange(ox - h, ox + nx + h, device="cuda") % N[0]
    iy = torch.arange(oy - h, oy + ny + h, device="cuda") % N[1]
    ext = U0[:, :, iy][:, :, :, ix].contiguous()
    out = torch.zeros_like(ext)
    mhd.mhd_step_sub(sim.ctx, ext, (h, h, 0), 1e-3, out)
    full = torch.zeros_like(U0)
    mhd.mhd_step_sub(sim.ctx, U0, p.offset, 1e-3, full)
    torch.cuda.synchronize()
    assert torch.equal(out[:, :, h:h + ny, h:h + nx], full[:, :, oy:oy + ny, ox:ox + nx])
