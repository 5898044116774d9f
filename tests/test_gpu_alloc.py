"""Device memory from a caller-supplied allocator (lgf_create_with_allocator).

The handle's buffers are taken from PyTorch's caching allocator through the
C callbacks; the fix must be bit-identical to one on a handle whose buffers
come from CUDA's stream-ordered allocator, and every buffer must go back on
lgf_destroy.  Allocation failures are made on the host: a callback that
returns NULL, or memory that is not 256-byte aligned."""

import ctypes

import numpy as np
import pytest

from paper_1206_0675_gb300 import fields
from paper_1206_0675_gb300 import lgf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    lgf.load_library()
    return torch


@pytest.mark.parametrize("prec,store12", [("fp64", False), ("mixed", True)])
def test_torch_allocator_matches_stream_ordered(torch, prec, store12):
    ext = (8, 6, 4, 12)
    U = fields.random_links(ext, eps=0.9, seed=4)
    out = []
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    for alloc in (None, "torch"):
        with lgf.Lattice(ext, prec, store12=store12, track_G=True, allocator=alloc) as lat:
            if alloc == "torch":
                # links, divergence, g, G, staging ... all counted by torch
                assert torch.cuda.memory_allocated() - base >= 4 * 18 * 8 * int(np.prod(ext))
            lat.set_links(U)
            Fh, Th = lat.set_trace(41)
            it, F, th, conv = lat.fix(1e-14, 40, 0.08)
            out.append((it, F, th, Fh.copy(), Th.copy(), lat.get_links(), lat.get_transform()))
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    a, b = out
    assert a[0] == b[0] and a[1] == b[1] and a[2] == b[2]
    for x, y in zip(a[3:], b[3:]):
        assert np.array_equal(x, y)


def test_allocator_failures_are_reported(torch):
    ext = (4, 4, 4, 4)
    calls = {"n": 0}

    def fail_alloc(nbytes, stream, ctx):
        calls["n"] += 1
        return None

    def no_free(ptr, nbytes, stream, ctx):
        raise AssertionError("nothing was allocated")

    al = lgf.LgfAllocator(lgf.ALLOC_FN(fail_alloc), lgf.FREE_FN(no_free), None)
    with pytest.raises(lgf.LgfError) as e:
        lgf.lgf_create_with_allocator(ext, lgf.LGF_FP64, 0, torch.cuda.current_stream().cuda_stream, al)
    assert e.value.status == lgf.LGF_E_NOMEM and calls["n"] == 1

    held = {}

    def odd_alloc(nbytes, stream, ctx):
        p = torch.cuda.caching_allocator_alloc(int(nbytes) + 256, stream=int(stream or 0))
        held[p + 8] = p
        return p + 8          # 8 bytes off a 256-byte boundary

    def odd_free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(held.pop(ptr))

    al2 = lgf.LgfAllocator(lgf.ALLOC_FN(odd_alloc), lgf.FREE_FN(odd_free), None)
    with pytest.raises(lgf.LgfError) as e:
        lgf.lgf_create_with_allocator(ext, lgf.LGF_FP64, 0, torch.cuda.current_stream().cuda_stream, al2)
    assert e.value.status == lgf.LGF_E_ARG
    assert not held   # the rejected buffer went back

    lib = lgf.load_library()
    h = ctypes.c_void_p()
    half = lgf.LgfAllocator(lgf.ALLOC_FN(fail_alloc), lgf.FREE_FN(), None)   # no free function
    ext4 = (ctypes.c_int32 * 4)(*ext)
    assert lib.lgf_create_with_allocator(ext4, lgf.LGF_FP64, 0, None, ctypes.byref(half), ctypes.byref(h)) == \
        lgf.LGF_E_ARG
