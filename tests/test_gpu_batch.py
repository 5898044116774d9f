"""Batched fixing of configurations of uneven shapes (lgf_batch_*).

The batch runs the same kernels as a single-configuration handle (one launch
per shape and step kernel, with a configuration index), so every
configuration must reach exactly the same iteration count, F and theta as
when it is fixed alone; one configuration is also checked against the CPU
oracle's iteration count.
"""

import numpy as np
import pytest

from oracle import lgf_oracle as O
from paper_1206_0675_gb300 import fields, lgf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available()
    lgf.load_library()


def single_fix(ext, U, tol, max_iter):
    with lgf.Lattice(ext, "fp64") as lat:
        lat.set_links(U)
        return lat.fix(tol, max_iter, 0.08)


def test_batch_matches_single_handles_and_oracle():
    exts = [(4, 4, 4, 4)] * 3 + [(6, 4, 4, 6)] * 2 + [(8, 8, 8, 8), (3, 4, 6, 9)]
    eps = [0.9, 0.5, 1.0, 0.8, 0.6, 0.7, 0.9]
    Us = [fields.random_links(e, ep, 40 + i) for i, (e, ep) in enumerate(zip(exts, eps))]
    tol, max_iter = 1e-12, 4000
    with lgf.Batch(exts) as b:
        desc = b.describe()
        assert sum(c["n"] for c in desc) == len(exts) and len(desc) == 4
        for i, U in enumerate(Us):
            b.set_links(i, U)
        it, F, th, conv = b.fix(tol, max_iter)
        U5 = b.get_links(5)
    assert conv and np.all(th < tol)
    for i, (e, U) in enumerate(zip(exts, Us)):
        it1, F1, th1, conv1 = single_fix(e, U, tol, max_iter)
        assert it[i] == it1, i
        assert abs(F[i] - F1) <= 1e-14 * abs(F1)
        assert abs(th[i] - th1) <= 1e-12 * th1
    ref = O.fix(Us[5], tol=tol, max_iter=max_iter, track_G=False)
    assert abs(it[5] - ref["iters"]) <= max(1, 0.02 * ref["iters"])
    assert abs(F[5] - ref["F"][-1]) < 1e-10
    assert abs(O.plaquette(U5) - O.plaquette(Us[5])) < 1e-12


def test_batch_retires_configurations_independently():
    """A configuration already below tol never moves; max_iter stops the rest."""
    exts = [(4, 4, 4, 4)] * 2
    U_fixed = O.identity_links(exts[0])
    U_rough = fields.random_links(exts[1], 1.0, 3)
    with lgf.Batch(exts) as b:
        b.set_links(0, U_fixed)
        b.set_links(1, U_rough)
        it, F, th, conv = b.fix(1e-30, 7)
        assert not conv
        assert it[0] == 0 and F[0] == 1.0 and it[1] == 7
        assert np.array_equal(b.get_links(0), U_fixed)


@pytest.mark.slow
def test_batch64_uneven_workload():
    """The 64-configuration workload (16 x 8^4, 16 x 12^4, 16 x 16^4, 8 x 16^3x32, 8 x 24^4,
    eps uniform in [0.3, 1.0], seeds 0-63) retired at theta < 1e-14."""
    exts = fields.BATCH64_EXTENTS
    Us = [fields.random_links(e, fields.batch_eps(i), i) for i, e in enumerate(exts)]
    with lgf.Batch(exts) as b:
        for i, U in enumerate(Us):
            b.set_links(i, U)
        it, F, th, conv = b.fix(1e-14, 30000)
        last = b.get_links(63)
    assert conv and np.all(th < 1e-14)
    for i in (0, 16, 32, 48, 63):
        it1, F1, th1, _ = single_fix(exts[i], Us[i], 1e-14, 30000)
        assert it[i] == it1 and abs(F[i] - F1) <= 1e-14 * abs(F1)
    assert abs(O.plaquette(last) - O.plaquette(Us[63])) < 1e-12
