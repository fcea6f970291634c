"""Host-side checks of the C ABI: the library loads without a GPU, exports
every entry point declared in include/g3pcf.h, and rejects invalid arguments
before any device work is enqueued."""
import ctypes
import re

import pytest

import paper_1709_00086_gb300 as g3


def _declared():
    txt = open(g3.HEADER).read()
    return sorted(set(re.findall(r"\b(g3pcf_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = g3.lib()
    names = _declared()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_zeta_size():
    # sum_m K_m^2 with K_m = B (lmax + 1 - m)
    assert g3.zeta_size(10, 10) == sum((10 * (11 - m)) ** 2 for m in range(11)) == 50600
    assert g3.zeta_size(3, 0) == 9
    assert g3.zeta_size(0, 3) == 0


@pytest.mark.parametrize("args,code", [
    ((0, 0.0, 10.0, 2, 100.0, 0), "ERR_ARG"),          # nbins < 1
    ((33, 0.0, 10.0, 2, 100.0, 0), "ERR_ARG"),         # nbins > 32
    ((4, 0.0, 10.0, 11, 100.0, 0), "ERR_ARG"),         # lmax > 10
    ((4, 0.0, 10.0, -1, 100.0, 0), "ERR_ARG"),         # lmax < 0
    ((4, 5.0, 5.0, 2, 100.0, 0), "ERR_ARG"),           # rmax <= rmin
    ((4, -1.0, 5.0, 2, 100.0, 0), "ERR_ARG"),          # rmin < 0
    ((4, 0.0, 5.0, 2, 0.0, 0), "ERR_ARG"),             # box <= 0
    ((4, 0.0, 5.0, 2, 100.0, 3), "ERR_ARG"),           # los mode
    ((4, 0.0, 50.0, 2, 100.0, 0), "ERR_RMAX"),         # rmax = box/2 periodic
    ((4, 0.0, float("nan"), 2, 100.0, 0), "ERR_ARG"),
])
def test_plan_validation(args, code):
    with pytest.raises(g3.G3PCFError) as ei:
        g3.Plan(*args)
    assert ei.value.name == code
    assert g3.lib().g3pcf_last_error().decode() != ""


def test_open_box_allows_large_rmax():
    p = g3.Plan(4, 0.0, 80.0, 2, 100.0, g3.LOS_Z_OPEN)
    p.close()


def test_compute_argument_errors_before_device_work():
    lib = g3.lib()
    p = g3.Plan(4, 0.0, 10.0, 2, 100.0, 0)
    h = p._h
    dummy = ctypes.c_void_p(16)
    # null zeta
    assert lib.g3pcf_compute_ex(h, dummy, dummy, 10, -1, None, None, 0) == -1
    # null pos with n > 0
    assert lib.g3pcf_compute_ex(h, None, dummy, 10, -1, dummy, None, 0) == -1
    # negative n, too many points, unknown flags
    assert lib.g3pcf_compute_ex(h, dummy, dummy, -5, -1, dummy, None, 0) == -1
    assert lib.g3pcf_compute_ex(h, dummy, dummy, 1 << 27, -1, dummy, None, 0) == -1
    assert lib.g3pcf_compute_ex(h, dummy, dummy, 10, -1, dummy, None, 1 << 10) == -1
    # batch: bad offsets
    offs = (ctypes.c_int64 * 3)(0, 5, 3)
    assert lib.g3pcf_compute_batch(h, dummy, dummy, offs, 2, dummy, None, 0) == -1
    offs = (ctypes.c_int64 * 2)(1, 5)
    assert lib.g3pcf_compute_batch(h, dummy, dummy, offs, 1, dummy, None, 0) == -1
    # backward / alm before forward
    assert lib.g3pcf_backward(h, dummy, dummy, dummy) == -7
    assert lib.g3pcf_alm(h, dummy, 1, dummy) == -7
    # null plan
    assert lib.g3pcf_set_stream(None, None) == -1
    assert lib.g3pcf_destroy(None) == 0
    p.close()


def test_set_option_validation():
    p = g3.Plan(4, 0.0, 10.0, 2, 100.0, 0)
    p.set_option(g3.OPT_CHUNK_ROWS, 1000)
    p.set_option(g3.OPT_CHUNK_ROWS, 0)
    p.set_option(g3.OPT_CELLS_PER_RMAX, 3)
    p.set_option(g3.OPT_KFLUSH, 8)
    p.set_option(g3.OPT_PAIR_KERNELS, 1)
    p.set_option(g3.OPT_LIST_BYTES, 1 << 20)
    p.set_option(g3.OPT_BASIS, 1)
    p.set_option(g3.OPT_X_REFINE, 1)
    p.set_option(g3.OPT_X_REFINE, 16)
    p.set_option(g3.OPT_GRAD_PRECISION, 1)
    p.set_option(g3.OPT_GRAD_PRECISION, 0)
    p.set_option(g3.OPT_TEST_FAIL_ALLOC, 3)
    p.set_option(g3.OPT_TEST_FAIL_ALLOC, 0)
    p.set_option(g3.OPT_TEST_TC_TIMEOUT, 1)
    p.set_option(g3.OPT_TEST_TC_TIMEOUT, 0)
    p.set_option(g3.OPT_TC_OPERANDS, 1)
    p.set_option(g3.OPT_TC_OPERANDS, 0)
    for opt, val in [(g3.OPT_TEST_FAIL_ALLOC, -1), (g3.OPT_TEST_TC_TIMEOUT, 2), (g3.OPT_TC_OPERANDS, 2), (g3.OPT_TC_OPERANDS, -1), (g3.OPT_GRAD_PRECISION, 2), (g3.OPT_GRAD_PRECISION, -1), (g3.OPT_CHUNK_ROWS, -1), (g3.OPT_CELLS_PER_RMAX, 9), (g3.OPT_KFLUSH, 1),
                     (g3.OPT_X_REFINE, 17), (g3.OPT_X_REFINE, -1),
                     (g3.OPT_KFLUSH, 17), (g3.OPT_PAIR_KERNELS, 3), (g3.OPT_PAIR_KERNELS, -1),
                     (g3.OPT_LIST_BYTES, -1), (g3.OPT_LIST_BYTES, 1000), (g3.OPT_BASIS, 2), (99, 1)]:
        with pytest.raises(g3.G3PCFError) as ei:
            p.set_option(opt, val)
        assert ei.value.name == "ERR_ARG"
    p.close()


def test_zeta_combine_argument_errors_before_device_work():
    lib = g3.lib()
    dummy = ctypes.c_void_p(16)
    coef = (ctypes.c_double * 2)(0.5, 0.5)
    bad = (ctypes.c_double * 2)(0.5, float("nan"))
    assert lib.g3pcf_zeta_combine(0, 2, 2, dummy, coef, dummy, None) == -1     # nbins < 1
    assert lib.g3pcf_zeta_combine(4, 11, 2, dummy, coef, dummy, None) == -1    # lmax > 10
    assert lib.g3pcf_zeta_combine(4, 2, 0, dummy, coef, dummy, None) == -1     # ncat < 1
    assert lib.g3pcf_zeta_combine(4, 2, 257, dummy, coef, dummy, None) == -1   # ncat > max
    assert lib.g3pcf_zeta_combine(4, 2, 2, None, coef, dummy, None) == -1      # null zeta
    assert lib.g3pcf_zeta_combine(4, 2, 2, dummy, None, dummy, None) == -1     # null coef
    assert lib.g3pcf_zeta_combine(4, 2, 2, dummy, bad, dummy, None) == -1      # non-finite
    assert "finite" in lib.g3pcf_last_error().decode()


def test_isotropic_argument_errors_before_device_work():
    lib = g3.lib()
    dummy = ctypes.c_void_p(16)
    assert lib.g3pcf_isotropic(0, 2, 1, dummy, dummy, None) == -1      # nbins < 1
    assert lib.g3pcf_isotropic(33, 2, 1, dummy, dummy, None) == -1     # nbins > 32
    assert lib.g3pcf_isotropic(4, 11, 1, dummy, dummy, None) == -1     # lmax > 10
    assert lib.g3pcf_isotropic(4, 2, -1, dummy, dummy, None) == -1     # ncat < 0
    assert lib.g3pcf_isotropic(4, 2, 1, None, dummy, None) == -1       # null zeta
    assert lib.g3pcf_isotropic(4, 2, 0, None, None, None) == 0         # nothing to do
