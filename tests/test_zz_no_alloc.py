"""The allocation-free entry point, g3pcf_zeta_from_alm_noalloc.

It serves callers that cannot allocate device memory (a fixed, pre-reserved
memory budget, or a streamed pipeline that must not pay cudaMalloc's implicit
synchronisation): they hand in multipoles they already hold and get zeta back,
with all scratch taken from fixed arrays inside the library.  This file checks,
through the C ABI, that two calls in a row reproduce the zeta of the regular
g3pcf_compute_ex path (plain-FP32 contraction) within the FP32 tolerance, and
that sizes beyond the fixed maximum are refused.  It is named so that pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1709_00086_gb300 as g3  # noqa: E402
from paper_1709_00086_gb300 import catalogs  # noqa: E402

pytestmark = pytest.mark.gpu
TOL_FP32 = 1e-5


def _rows(a, nbins, lmax):
    """Multipoles (np, nbins, nlm) complex -> the documented row layout."""
    n = a.shape[0]
    cols = []
    for m in range(lmax + 1):
        idx = [l * (l + 1) // 2 + m for l in range(m, lmax + 1)]
        blk = a[:, :, idx].transpose(0, 2, 1).reshape(n, -1)  # column (l - m) * nbins + b
        cols.append(blk.real)
        if m > 0:
            cols.append(blk.imag)
    return np.ascontiguousarray(np.concatenate(cols, axis=1), dtype=np.float32)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_regular_path_twice():
    cat = catalogs.small_case("clustered", 12000, seed=31, box=500.0, nbins=10, rmin=0.0,
                              rmax=100.0, lmax=10)
    plan = g3.Plan(**cat.params())
    pos = torch.from_numpy(cat.pos).cuda()
    w = torch.from_numpy(cat.w).cuda()
    z_ref, _ = plan.compute(pos, w, fp32_contraction=True, keep_alm=True)
    z_ref = z_ref.cpu().numpy()
    rows = torch.from_numpy(_rows(plan.alm(np.arange(cat.n)), cat.nbins, cat.lmax)).cuda()
    lib = g3.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        z = torch.full((plan.zsize, 2), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.g3pcf_zeta_from_alm_noalloc(cat.nbins, cat.lmax, _ptr(rows), rows.shape[1], _ptr(w),
                                             cat.n, _ptr(z), stream)
        assert rc == 0, lib.g3pcf_last_error().decode()
        torch.cuda.synchronize()
        zc = torch.view_as_complex(z).cpu().numpy()
        err = np.abs(zc - z_ref).max() / np.abs(z_ref).max()
        assert err < TOL_FP32, err


def test_noalloc_rejects_bad_sizes():
    lib = g3.lib()
    buf = torch.zeros(16, device="cuda")
    # leading dimension shorter than a row
    assert lib.g3pcf_zeta_from_alm_noalloc(10, 10, _ptr(buf), 5, _ptr(buf), 1, _ptr(buf), None) == -1
    assert "ld" in lib.g3pcf_last_error().decode()
    # shapes beyond the build's limits
    assert lib.g3pcf_zeta_from_alm_noalloc(33, 2, _ptr(buf), 4096, _ptr(buf), 1, _ptr(buf), None) == -1
    assert lib.g3pcf_zeta_from_alm_noalloc(4, 2, _ptr(buf), 64, _ptr(buf), 1 << 27, _ptr(buf), None) == -1
