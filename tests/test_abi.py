"""CPU checks of the C ABI library: it loads, exports every declared symbol and
validates configurations without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:int|void|const char\*)\s+\**(mhd_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_05240_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_step_api():
    names = declared_functions()
    for required in ("mhd_init", "mhd_step", "mhd_dt", "mhd_adjoint_step", "mhd_run", "mhd_destroy"):
        assert required in names


def test_every_entry_point_is_documented():
    """Each declaration in include/*.h has its own comment directly above it
    that either cites the passage it computes (Sec., Eq., Step or a reading
    D-n) or states that the paper has no counterpart."""
    cite = re.compile(r"Sec\.|Eq\.|Steps? \d|D-\d+|not in the paper|paper has no counterpart")
    seen = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        for m in re.finditer(r"^(?:int|void|const char\*)\s+\**(mhd_\w+)\s*\(", txt, flags=re.M):
            before = txt[:m.start()].rstrip()
            assert before.endswith("*/"), f"{h}: {m.group(1)} has no comment directly above it"
            comment = re.sub(r"\s*\n\s*\*?\s*", " ", before[before.rfind("/*"):])
            assert cite.search(comment), f"{h}: {m.group(1)} cites no passage: {comment[:120]}"
            seen.add(m.group(1))
    assert seen == set(declared_functions())


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_config_validation_without_gpu():
    from paper_2402_05240_gb300 import mhd
    ok = mhd.mhd_config(32, 32, 32, 1 / 32, 1 / 32, 1 / 32, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20)
    assert mhd.mhd_workspace_bytes(ok) > 32 ** 3 * 8 * 8
    fp32 = mhd.mhd_config(32, 32, 32, 1 / 32, 1 / 32, 1 / 32, 5 / 3, 0.4, 1, 1, 1e-20, 1e-20)
    assert mhd.mhd_workspace_bytes(fp32) < mhd.mhd_workspace_bytes(ok)
    bad = [
        mhd.mhd_config(0, 32, 32, 1, 1, 1, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20),  # empty
        mhd.mhd_config(3, 32, 32, 1, 1, 1, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20),  # below minimum
        mhd.mhd_config(8, 8, 8, 0, 1, 1, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20),  # dx = 0
        mhd.mhd_config(8, 8, 8, 1, 1, 1, 1.0, 0.4, 1, 0, 1e-20, 1e-20),  # gamma = 1
        mhd.mhd_config(8, 8, 8, 1, 1, 1, 5 / 3, 0.0, 1, 0, 1e-20, 1e-20),  # cfl = 0
        mhd.mhd_config(8, 8, 8, 1, 1, 1, 5 / 3, 0.4, 7, 0, 1e-20, 1e-20),  # recon
        mhd.mhd_config(8, 8, 8, 1, 1, 1, 5 / 3, 0.4, 1, 5, 1e-20, 1e-20),  # precision
        mhd.mhd_config(8, 8, 8, 1, 1, 1, 5 / 3, 0.4, 1, 0, 0.0, 1e-20),  # floor
        mhd.mhd_config(8, 8, 8, 1, 1, 1, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20, (ctypes.c_int * 3)(0, 3, 0)),  # bc
        mhd.mhd_config(8, 8, 8, 1, 1, 1, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20, (ctypes.c_int * 3)(1, 2, 0)),  # outflow+halo
        mhd.mhd_config(4, 4, 65536, 1, 1, 1, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20),  # nz above the launch grid's z limit
        mhd.mhd_config(65536, 32769, 4, 1, 1, 1, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20),  # nx ny above 2^31
        mhd.mhd_config(4, 4, 65530, 1, 1, 1, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20,
                       (ctypes.c_int * 3)(0, 0, 1)),  # padded nz above the z limit
        mhd.mhd_config(2048, 2048, 512, 1, 1, 1, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20),  # 2^31 cells: 32-bit indices
        mhd.mhd_config(2048, 2032, 512, 1, 1, 1, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20,
                       (ctypes.c_int * 3)(0, 1, 0)),  # 2^31 cells with the ghost cells of an outflow axis
    ]
    for cfg in bad:
        with pytest.raises(mhd.MHDError) as e:
            mhd.mhd_workspace_bytes(cfg)
        assert e.value.code == mhd.MHD_ERR_ARG
    # an outflow axis pads the grid by MHD_GHOST cells per side and adds the padded state
    out = mhd.mhd_config(32, 32, 32, 1 / 32, 1 / 32, 1 / 32, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20,
                         (ctypes.c_int * 3)(1, 0, 0))
    ratio = mhd.mhd_workspace_bytes(out) / mhd.mhd_workspace_bytes(ok)
    assert 48 / 32 < ratio < 48 / 32 * (1 + 8 * 8 / (49 * 8)) + 0.01
    # the largest grid the 32-bit cell indices allow is accepted
    big = mhd.mhd_config(2048, 2048, 511, 1, 1, 1, 5 / 3, 0.4, 1, 1, 1e-20, 1e-20)
    assert mhd.mhd_workspace_bytes(big) > 2048 * 2048 * 511 * 64


def test_host_alloc_argument_errors_without_gpu(lib):
    """mhd_host_alloc refuses a zero size and a NULL output before any CUDA
    call; mhd_host_free(NULL) is a no-op."""
    vp = ctypes.c_void_p
    lib.mhd_host_alloc.argtypes = [ctypes.c_size_t, ctypes.POINTER(vp)]
    lib.mhd_host_alloc.restype = ctypes.c_int
    lib.mhd_host_free.argtypes = [vp]
    lib.mhd_host_free.restype = ctypes.c_int
    p = vp()
    assert lib.mhd_host_alloc(0, ctypes.byref(p)) == -1 and p.value is None
    assert lib.mhd_host_alloc(64, None) == -1
    assert lib.mhd_host_free(None) == 0


def test_null_arguments_rejected(lib):
    lib.mhd_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
    lib.mhd_step.restype = ctypes.c_int
    assert lib.mhd_step(None, None, 0.1, None) == -1
    vp = ctypes.c_void_p
    lib.mhd_adjoint_step.argtypes = [vp, vp, ctypes.c_double, vp, vp]
    lib.mhd_adjoint_step.restype = ctypes.c_int
    assert lib.mhd_adjoint_step(None, None, 1e-3, None, None) == -1
    lib.mhd_adjoint_step_cfl.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.mhd_adjoint_step_cfl.restype = ctypes.c_int
    assert lib.mhd_adjoint_step_cfl(None, None, None, None, None, None) == -1
    lib.mhd_strerror.restype = ctypes.c_char_p
    assert lib.mhd_strerror(-4).startswith(b"non-finite")


def test_binding_checks_buffers_before_the_library_sees_them():
    """The library takes raw pointers and cannot see sizes; the binding
    refuses a wrong dtype, device, layout or size with an exception (not an
    assert, which python -O would strip) before any call."""
    import torch
    from paper_2402_05240_gb300 import mhd
    f64 = torch.float64
    with pytest.raises(TypeError):
        mhd._ptr([1.0, 2.0], name="U")
    with pytest.raises(TypeError):
        mhd._ptr(torch.zeros(8, dtype=torch.float32), name="U")
    with pytest.raises(ValueError):
        mhd._ptr(torch.zeros(8, dtype=f64), name="U")  # host tensor where a CUDA one is needed
    with pytest.raises(ValueError):
        mhd._ptr(torch.zeros(4, 4, dtype=f64).t(), name="U_host", cuda=False)  # not contiguous
    with pytest.raises(ValueError):
        mhd._ptr(torch.zeros(8, dtype=f64), 9, "U_host", cuda=False)
    assert mhd._ptr(torch.zeros(9, dtype=f64), 9, "U_host", cuda=False).value is not None
    # a context's cells come from its registration (made by mhd_init); a fake
    # registration stands in for one here and no library call is reached
    fake = ctypes.c_void_p(0x1000)
    mhd._CTX[fake.value] = (4 * 5 * 6, 0)
    try:
        assert mhd._cells(fake) == (120, 0)
        with pytest.raises(ValueError):
            mhd.mhd_run_host(fake, torch.zeros(8 * 120 - 1, dtype=f64), 1)
        with pytest.raises(ValueError):
            mhd.mhd_step_sub(fake, torch.zeros(8, 6, 5, 4, dtype=f64), (0, 0, 0), 1e-3,
                             torch.zeros(8, 6, 5, 5, dtype=f64))
        with pytest.raises(ValueError):
            mhd.mhd_dt_sub(fake, torch.zeros(7, 6, 5, 4, dtype=f64), (0, 0, 0))
    finally:
        del mhd._CTX[fake.value]
    assert mhd._cells(fake) == (None, None)


def test_static_diagnostics_scratch_holds_the_layout_the_kernels_write(lib):
    """The allocation-free diagnostics write 9 results, then 9 partials and 8
    compensation terms per 1024-cell block; for its largest grid (512^3 cells,
    131072 blocks) its file-scope device array must hold 9 + 17 * 131072
    doubles.  The host shadow of a __device__ array has the array's size, so
    the symbol table of the built library shows it without a GPU."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    from paper_2402_05240_gb300 import build
    out = subprocess.run([nm, "-S", "-C", build.LIB], capture_output=True, text=True, check=True).stdout
    sizes = [int(ln.split()[1], 16) for ln in out.splitlines() if ln.endswith("g_diag_scratch")]
    assert len(sizes) == 1, out[:2000]
    blocks = -(-512 ** 3 // 1024)
    assert sizes[0] == 8 * (9 + 17 * blocks)
