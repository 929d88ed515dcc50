"""The C-ABI library builds for sm_103a, loads, exports every symbol include/vl2mhd.h declares, and
validates its arguments on the host (no GPU needed for any call made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_06651_gb300 import build, vl2

    build.build()
    return vl2.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "vl2mhd.h")).read()
    return sorted(set(re.findall(r"^\s*(?:vl2_status|const char\*)\s+(vl2_\w+)\s*\(", text, re.M)))


def test_header_declares_the_abi():
    names = declared_symbols()
    for n in ("vl2_mesh_create", "vl2_block_layout", "vl2_set_prims", "vl2_step", "vl2_fill_ghosts", "vl2_new_dt",
              "vl2_get_cons", "vl2_divb_norm"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_export(lib):
    from paper_2005_06651_gb300 import vl2

    assert set(declared_symbols()) <= set(vl2.EXPORTS) | {"vl2_profile", "vl2_profile_read", "vl2_launch_count"}


def _params(**kw):
    from paper_2005_06651_gb300 import vl2

    p = vl2.Params()
    p.nx[:] = kw.get("nx", (32, 32, 32))
    p.mb[:] = kw.get("mb", (16, 16, 16))
    p.ng = kw.get("ng", 2)
    p.xmin[:] = (0.0, 0.0, 0.0)
    p.xmax[:] = kw.get("xmax", (1.0, 1.0, 1.0))
    p.gamma = kw.get("gamma", 5.0 / 3.0)
    p.cfl = 0.3
    p.riemann = kw.get("riemann", 1)
    p.precision = kw.get("precision", 0)
    p.bc[:] = kw.get("bc", (0,) * 6)
    p.dfloor = p.pfloor = 1e-12
    p.adjoint = kw.get("adjoint", 0)
    p.recon = kw.get("recon", 0)
    p.nscalars = kw.get("nscalars", 0)
    p.ct_delta = kw.get("ct_delta", 0.0)
    return p


def test_workspace_bytes_and_argument_checks(lib):
    n = ctypes.c_size_t()
    assert lib.vl2_workspace_bytes(ctypes.byref(_params()), ctypes.byref(n)) == 0
    # 8 blocks of (16+5 -> 24) x 21 x 21 padded cells, 48 double arrays, plus staging
    assert n.value >= 8 * 24 * 21 * 21 * 48 * 8
    bad = [dict(nx=(30, 32, 32)), dict(ng=1), dict(ng=4), dict(gamma=1.0), dict(riemann=5), dict(precision=7),
           dict(bc=(0, 1, 0, 0, 0, 0)), dict(nx=(0, 32, 32)), dict(xmax=(0.0, 1.0, 1.0)), dict(recon=7),
           dict(recon=2, ng=2), dict(adjoint=1, ng=3), dict(adjoint=1, ng=3, recon=2), dict(nscalars=-1),
           dict(nscalars=17), dict(adjoint=1, nscalars=1), dict(ct_delta=-1.0),
           dict(ct_delta=float("nan")), dict(adjoint=1, recon=3), dict(recon=5), dict(recon=4, ng=2),
           dict(riemann=3), dict(adjoint=1, riemann=2)]
    for kw in bad:
        assert lib.vl2_workspace_bytes(ctypes.byref(_params(**kw)), ctypes.byref(n)) == 1, kw
        assert lib.vl2_last_error(None)
    # three ghost layers (with PLM or PPM) enlarge the padded boxes
    for kw in (dict(ng=3), dict(ng=3, recon=2)):
        m = ctypes.c_size_t()
        assert lib.vl2_workspace_bytes(ctypes.byref(_params(**kw)), ctypes.byref(m)) == 0, kw
        assert m.value > n.value
    out = ctypes.c_void_p()
    # misaligned or null workspace is rejected before any CUDA call
    assert lib.vl2_mesh_create(ctypes.byref(_params()), ctypes.c_void_p(0), ctypes.c_size_t(1 << 30),
                               ctypes.byref(out)) == 1
    assert lib.vl2_mesh_create(ctypes.byref(_params()), ctypes.c_void_p(1 << 20), ctypes.c_size_t(10),
                               ctypes.byref(out)) == 6
    assert lib.vl2_step(None, ctypes.c_double(0.1)) == 1


def test_full_size_workspace_fits_one_gb300(lib):
    n = ctypes.c_size_t()
    assert lib.vl2_workspace_bytes(ctypes.byref(_params(nx=(256,) * 3, mb=(32,) * 3)), ctypes.byref(n)) == 0
    assert n.value < 20e9
    assert lib.vl2_workspace_bytes(ctypes.byref(_params(nx=(512,) * 3, mb=(32,) * 3)), ctypes.byref(n)) == 0
    assert n.value < 200e9


def test_totals_noalloc_binding_rejects_mis_shaped_tensors():
    """The binding checks every shape before anything reaches the device (a wrong shape would make the kernel
    read past a buffer); CPU tensors of the right shapes stop at the CUDA check."""
    import torch

    from paper_2005_06651_gb300 import vl2

    nz, ny, nx = 4, 3, 5
    f64 = torch.float64
    u = torch.zeros((5, nz, ny, nx), dtype=f64)
    b1, b2, b3 = (torch.zeros(s, dtype=f64) for s in ((nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)))
    out = torch.zeros(8, dtype=f64)
    with pytest.raises(ValueError, match="b1 must have shape"):
        vl2.totals_noalloc(u, torch.zeros((nz, ny, nx), dtype=f64), b2, b3, (1.0, 1.0, 1.0), out)
    with pytest.raises(ValueError, match="b3 must have shape"):
        vl2.totals_noalloc(u, b1, b2, torch.zeros((nz, ny, nx), dtype=f64), (1.0, 1.0, 1.0), out)
    with pytest.raises(ValueError, match="u must have shape"):
        vl2.totals_noalloc(u[:4], b1, b2, b3, (1.0, 1.0, 1.0), out)
    with pytest.raises(ValueError, match="at least 8"):
        vl2.totals_noalloc(u, b1, b2, b3, (1.0, 1.0, 1.0), torch.zeros(7, dtype=f64))
    with pytest.raises(ValueError, match="CUDA tensor"):
        vl2.totals_noalloc(u, b1, b2, b3, (1.0, 1.0, 1.0), out)
