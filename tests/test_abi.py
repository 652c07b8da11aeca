"""The C-ABI library loads and exports every entry point include/sq.h declares;
host-side argument validation rejects bad input before touching the GPU.
No compute call is made here (runs without a GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sq.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1708_07913_gb300 import build, sq
    build()
    return sq.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sq_[a-z_]+)\s*\(", src)))


def test_header_declares_the_path_calls():
    names = _declared()
    for need in ("sq_setup_grid", "sq_spectral_bounds", "sq_moments", "sq_fermi_level", "sq_density_energy",
                 "sq_destroy", "sq_strerror"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1708_07913_gb300 import sq
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in sq.EXPORTS, name


def test_strerror(lib):
    from paper_1708_07913_gb300 import sq
    assert sq.sq_strerror(0) == "ok"
    assert "invalid" in sq.sq_strerror(sq.SQ_EINVAL)
    assert sq.sq_strerror(999) == "unknown status"


@pytest.mark.parametrize("kw", [
    dict(n1=0), dict(h=-1.0), dict(h=float("nan")), dict(npl=6), dict(npl=0), dict(npl=1024),
    dict(precision=7), dict(r_cut=-1.0), dict(fd_half_order=0),
])
def test_setup_rejects_bad_arguments(lib, kw):
    from paper_1708_07913_gb300 import sq
    args = dict(n1=8, n2=8, n3=8, h=0.5, fd_half_order=6, r_cut=2.0, npl=8, precision=0)
    args.update(kw)
    ctx = C.c_void_p(123)
    rc = lib.sq_setup_grid(C.byref(ctx), args["n1"], args["n2"], args["n3"], args["h"], args["fd_half_order"],
                           args["r_cut"], args["npl"], args["precision"], 0, None, 0, None, None)
    assert rc == sq.SQ_EINVAL
    assert ctx.value is None


def test_setup_rejects_unsupported_requests(lib):
    from paper_1708_07913_gb300 import sq
    ctx = C.c_void_p()
    # region side above 31
    assert lib.sq_setup_grid(C.byref(ctx), 8, 8, 8, 0.5, 6, 8.0, 8, 0, 0, None, 0, None, None) == sq.SQ_EUNSUPPORTED
    # FP64 regions above 25^3
    assert lib.sq_setup_grid(C.byref(ctx), 8, 8, 8, 0.5, 6, 6.5, 8, 0, 0, None, 0, None, None) == sq.SQ_EUNSUPPORTED
    # FD order other than 12
    assert lib.sq_setup_grid(C.byref(ctx), 8, 8, 8, 0.5, 4, 2.0, 8, 0, 0, None, 0, None, None) == sq.SQ_EUNSUPPORTED
    # two s channels / mismatched widths
    two_s = (sq.ProjType * 2)(sq.ProjType(0, 0.5, 1.5, 4.5), sq.ProjType(0, 0.2, 1.5, 4.5))
    pos = np.zeros(3)
    assert lib.sq_setup_grid(C.byref(ctx), 8, 8, 8, 0.5, 6, 2.0, 8, 0, 1, pos.ctypes.data_as(C.POINTER(C.c_double)),
                             2, two_s, None) == sq.SQ_EUNSUPPORTED


def test_setup_rejects_missing_positions_and_nonfinite_atoms(lib):
    from paper_1708_07913_gb300 import sq
    ctx = C.c_void_p()
    one = (sq.ProjType * 1)(sq.ProjType(0, 0.5, 1.5, 4.5))
    assert lib.sq_setup_grid(C.byref(ctx), 8, 8, 8, 0.5, 6, 2.0, 8, 0, 2, None, 1, one, None) == sq.SQ_EINVAL
    pos = np.array([0.0, 1.0, np.inf])
    assert lib.sq_setup_grid(C.byref(ctx), 8, 8, 8, 0.5, 6, 2.0, 8, 0, 1, pos.ctypes.data_as(C.POINTER(C.c_double)),
                             1, one, None) == sq.SQ_EINVAL


def test_calls_reject_null_context(lib):
    from paper_1708_07913_gb300 import sq
    assert lib.sq_spectral_bounds(None, None, None, None, 10, 0.01) == sq.SQ_EINVAL
    assert lib.sq_moments(None, None, None, None, None) == sq.SQ_EINVAL
    mu = C.c_double()
    assert lib.sq_fermi_level(None, None, None, None, 1.0, 0.1, C.byref(mu)) == sq.SQ_EINVAL
    assert lib.sq_density_energy(None, None, None, None, 0.0, 0.1, None, None, None, None) == sq.SQ_EINVAL
    assert lib.sq_sync(None) == sq.SQ_EINVAL
    assert lib.sq_launch_count(None) == -1
    lib.sq_destroy(None)
    assert lib.sq_nl_forces(None, None, None, None, 0.0, 0.1, None) == sq.SQ_EINVAL
    assert lib.sq_nl_forces_nodes(None, None, None, None, 0.0, 0.1, None, 0, None) == sq.SQ_EINVAL
    res, it = C.c_double(), C.c_int()
    assert lib.sq_kerker(None, None, None, 1.0, 0.2, 1e-10, 100, None, C.byref(res), C.byref(it)) == sq.SQ_EINVAL
    assert lib.sq_mixer_set_period(None, 3, 0) == sq.SQ_EINVAL
    assert lib.sq_poisson(None, None, None, 1e-10, 10, None, None) == sq.SQ_EINVAL
    assert lib.sq_mixer_step(None, None, None, None, None) == sq.SQ_EINVAL


def test_cnn_host_checks(lib):
    """Parameter count of the warm-start network and the checks made before
    any CUDA call (no GPU needed)."""
    from paper_1708_07913_gb300 import sq
    from oracle import cnn_oracle
    p = cnn_oracle.init_params(0)
    assert lib.sq_cnn_param_count(32) == sum(p[k].size for k in cnn_oracle.TRAINED) == 32577
    assert lib.sq_cnn_param_count(16) == -1
    net = C.c_void_p()
    assert lib.sq_cnn_create(C.byref(net), 16, 1, None) == sq.SQ_EUNSUPPORTED and not net.value
    assert lib.sq_cnn_create(C.byref(net), 32, 2, None) == sq.SQ_EINVAL
    assert lib.sq_cnn_create(None, 32, 1, None) == sq.SQ_EINVAL
    L = C.c_double()
    assert lib.sq_cnn_forward(None, 4, 4, 4, None, None) == sq.SQ_EINVAL
    assert lib.sq_cnn_backward(None, 4, 4, 4, None, None, None, 0, C.byref(L)) == sq.SQ_EINVAL
    assert lib.sq_cnn_adam_step(None, 1e-3, 0.9, 0.999, 1e-8, 1.0) == sq.SQ_EINVAL
    assert lib.sq_cnn_set_params(None, None, 0.0, 1.0, 1.0) == sq.SQ_EINVAL
    lib.sq_cnn_destroy(None)


def test_warm_start_driver_imports():
    from paper_1708_07913_gb300 import warmstart
    assert callable(warmstart.training_pairs) and callable(warmstart.compare)


def test_package_fails_loudly_without_library(tmp_path):
    from paper_1708_07913_gb300 import sq
    with pytest.raises(RuntimeError):
        sq.load(str(tmp_path / "missing.so"))
