"""Domain decomposition over ranks on the CPU (gloo): the halo exchange and
the dt all-reduce of paper_2402_05240_gb300.decomp, with the oracle's step on
each rank's halo-extended block, reproduce the monolithic oracle run bit for
bit (2, 3 and 4 ranks, every decomposed axis, edges and corners included)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

GLOBAL_N = (24, 16, 18)  # nx, ny, nz
STEPS = 3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _state():
    from paper_2402_05240_gb300 import inputs as I
    return I.turbulent_box(I.Box(*GLOBAL_N), seed_v=31, seed_b=32, kmax=4)


def _worker(rank, world, port, parts, recon, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["OMP_NUM_THREADS"] = "1"
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2402_05240_gb300 import decomp
    U = _state()
    part = decomp.plan(GLOBAL_N, parts)[rank]
    (ox, oy, oz), (nx, ny, nz) = part.offset, part.size
    sub = decomp.Subdomain(part, parts, torch.from_numpy(U[:, oz:oz + nz, oy:oy + ny, ox:ox + nx].copy()))
    d = [1.0 / n for n in GLOBAL_N]

    def oracle_for(ext):
        ez, ey, ex = ext.shape[1:]
        return O.Oracle(ex, ey, ez, dx=d[0], dy=d[1], dz=d[2], recon=recon)

    def step_fn(ext, halo, dt, out):
        hx, hy, hz = halo
        V = oracle_for(ext).step(ext.numpy(), dt)
        out[:, hz:hz + nz, hy:hy + ny, hx:hx + nx] = torch.from_numpy(V[:, hz:hz + nz, hy:hy + ny, hx:hx + nx])

    def dt_fn(ext, halo):
        import ctypes
        hx, hy, hz = halo
        o = oracle_for(ext)
        E = np.ascontiguousarray(ext.numpy())
        lo = (ctypes.c_int * 3)(hx, hy, hz)
        hi = (ctypes.c_int * 3)(hx + nx, hy + ny, hz + nz)
        return o.lib.oracle_dt_box(ctypes.byref(o.p), O._ptr(E), 0.3, lo, hi)

    dts = [sub.step(step_fn, dt_fn=dt_fn) for _ in range(STEPS)]
    np.save(os.path.join(outdir, f"part{rank}.npy"), sub.interior.numpy())
    np.save(os.path.join(outdir, f"dts{rank}.npy"), np.array(dts))
    dist.barrier()
    dist.destroy_process_group()


# with 2 parts on an axis both neighbours are the same rank; 3 parts make
# a ring with distinct lower and upper neighbours
@pytest.mark.parametrize("parts,recon", [((2, 1, 1), "plmc"), ((1, 2, 1), "ppmc"), ((1, 1, 2), "plmc"),
                                         ((2, 2, 1), "ppmc"), ((3, 1, 1), "plmc"), ((3, 1, 1), "ppmc")])
def test_decomposed_run_equals_monolithic(tmp_path, parts, recon):
    import torch.multiprocessing as mp

    import oracle as O
    from paper_2402_05240_gb300 import decomp
    world = parts[0] * parts[1] * parts[2]
    mp.start_processes(_worker, args=(world, _free_port(), parts, recon, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    U = _state()
    ref, ref_dts = O.Oracle(*GLOBAL_N, recon=recon).run(U, STEPS, cfl=0.3)
    got = np.empty_like(ref)
    for p in decomp.plan(GLOBAL_N, parts):
        (ox, oy, oz), (nx, ny, nz) = p.offset, p.size
        got[:, oz:oz + nz, oy:oy + ny, ox:ox + nx] = np.load(tmp_path / f"part{p.rank}.npy")
        assert np.array_equal(np.load(tmp_path / f"dts{p.rank}.npy"), np.array(ref_dts))
    assert np.array_equal(got, ref)


def test_plan_covers_the_grid_once():
    from paper_2402_05240_gb300 import decomp
    parts = (3, 2, 2)
    n = (40, 17, 16)
    seen = np.zeros((n[2], n[1], n[0]), int)
    plan = decomp.plan(n, parts)
    for p in plan:
        (ox, oy, oz), (nx, ny, nz) = p.offset, p.size
        seen[oz:oz + nz, oy:oy + ny, ox:ox + nx] += 1
        for a in range(3):  # neighbours are symmetric
            assert plan[p.lo[a]].hi[a] == p.rank and plan[p.hi[a]].lo[a] == p.rank
    assert np.all(seen == 1)
    with pytest.raises(ValueError):
        decomp.plan((12, 16, 16), (2, 1, 1))  # 6-cell subdomains are thinner than the halo
