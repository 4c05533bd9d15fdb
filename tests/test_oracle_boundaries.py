"""Pins of the outflow-boundary oracle (Sec. 3.1.4 setup: zero-gradient ghost
cells filled once per step).  CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_2402_05240_gb300 import inputs as I


@pytest.mark.parametrize("recon", ["plmc", "ppmc"])
def test_uniform_state_unchanged_with_outflow(recon):
    n = (12, 6, 5)
    U = I.uniform(I.Box(*n), 1.3, (0.4, -0.2, 0.3), 0.7, (0.6, -0.8, 0.2))
    o = O.OutflowOracle(*n, ("outflow", "periodic", "outflow"), recon=recon)
    V, _ = o.run(U, 3, cfl=0.4)
    assert np.array_equal(U, V)


def test_result_independent_of_ghost_depth_beyond_the_stencil(monkeypatch):
    """With more ghost cells than one step's dependency radius (5 cells) the
    interior is bit-identical for any depth; with too few it is not."""
    n = (20, 12, 10)
    U = I.turbulent_box(I.Box(*n), seed_v=3, seed_b=4, kmax=3)
    res = {}
    for g in (2, 6, 10):
        monkeypatch.setattr(O, "GHOST", g)
        o = O.OutflowOracle(*n, ("outflow", "outflow", "periodic"), recon="ppmc")
        res[g], _ = o.run(U, 2, dts=[2e-3, 2e-3])
    assert np.array_equal(res[6], res[10])
    assert not np.array_equal(res[2], res[10])


def test_riemann_far_field_and_transverse_uniformity():
    box, U, gamma, _ = I.riemann("brio_wu", n=64, ntrans=4)
    o = O.OutflowOracle(64, 4, 4, ("outflow", "periodic", "periodic"), gamma=gamma, recon="plmc")
    V, dts = o.run(U, 3, cfl=0.4)
    # uniform along y and z
    assert np.array_equal(V, np.broadcast_to(V[:, :1, :1, :], V.shape))
    # one step reaches at most 5 cells: after 3 steps the outer 16 cells, and
    # the zero-gradient ghosts beyond them, keep their states bit for bit
    assert np.array_equal(V[..., :16], U[..., :16]) and np.array_equal(V[..., -16:], U[..., -16:])
    # the middle has evolved
    assert not np.array_equal(V[..., 28:36], U[..., 28:36])


def test_riemann_mirror_symmetry():
    """The mirrored problem (x -> 1 - x, v_x, B_x -> -v_x, -B_x) evolves into
    the mirror image of the solution."""
    n = 48
    out = []
    for mirror in (False, True):
        box, U, gamma, _ = I.riemann("dai_woodward", n=n, ntrans=4, mirror=mirror)
        o = O.OutflowOracle(n, 4, 4, ("outflow", "periodic", "periodic"), gamma=gamma, recon="plmc")
        out.append(o.run(U, 8, dts=[1e-3] * 8)[0])
    a, b = out
    m = b[..., ::-1].copy()
    m[1] = -m[1]   # m_x
    m[5] = -b[5][..., ::-1]  # B_x on faces: uniform here, the sign flips
    scale = np.abs(a).max(axis=(1, 2, 3), keepdims=True) + 1e-300
    assert np.max(np.abs(m - a) / scale) < 1e-12
