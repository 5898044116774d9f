"""lgf_measure_static, the measurement entry point that allocates nothing.

It serves callers that must not allocate device memory where they measure
(a host application whose device memory belongs to its own pool allocator,
or monitoring code between the steps of a time-critical loop, where
cudaMalloc/cudaFree could fail or synchronise the device).  Its scratch is a
fixed array inside the library that every call shares, so two calls in a row
must each give the same answer as the handle-based path: the reduction
ticket left by one call must not leak into the next.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""

import numpy as np
import pytest

from paper_1206_0675_gb300 import fields, lgf

pytestmark = pytest.mark.gpu


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def handle_path(ext, U):
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        F, th = lat.measure()
        D = lat.get_divergence()
    return F, th, D


def static_path(torch, ext, Ut, out_D, out_ft):
    st = lgf.lgf_measure_static(ext, Ut.data_ptr(), out_D.data_ptr(), out_ft.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == lgf.LGF_OK
    torch.cuda.synchronize()
    ft = out_ft.cpu().numpy()
    return float(ft[0]), float(ft[1]), out_D.cpu().numpy()


@pytest.mark.parametrize("ext", [(8, 8, 8, 8), (3, 4, 6, 9)])
def test_static_measure_matches_handle_path_twice(ext):
    import torch
    assert torch.cuda.is_available()
    lx, ly, lz, lt = ext
    outs_D = torch.empty((lt, lz, ly, lx, 3, 3), dtype=torch.complex128, device="cuda")
    out_ft = torch.empty(2, dtype=torch.float64, device="cuda")
    for seed in (0, 1):  # two calls in a row on different fields
        U = fields.random_links(ext, eps=0.7, seed=seed)
        Fh, thh, Dh = handle_path(ext, U)
        Ut = torch.from_numpy(U).cuda()
        F, th, D = static_path(torch, ext, Ut, outs_D, out_ft)
        assert rel(F, Fh) < 1e-14
        assert rel(th, thh) < 1e-13
        assert np.max(np.abs(D - Dh)) < 1e-13
    # the same field again after another one: the shared scratch keeps no state
    F2, th2, _ = static_path(torch, ext, Ut, outs_D, out_ft)
    assert F2 == F and th2 == th


def test_static_measure_rejects_oversized_lattice():
    import torch
    buf = torch.zeros(2, dtype=torch.float64, device="cuda")
    ext = (128, 128, 128, 9)  # 18.9 M sites > LGF_STATIC_MAX_SITES; rejected before any launch
    assert np.prod(ext) > lgf.LGF_STATIC_MAX_SITES
    st = lgf.lgf_measure_static(ext, buf.data_ptr(), 0, buf.data_ptr(), 0)
    assert st == lgf.LGF_E_UNSUPPORTED
    assert lgf.lgf_measure_static(ext, 0, 0, 0, 0) == lgf.LGF_E_ARG
