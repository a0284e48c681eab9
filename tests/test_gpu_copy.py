"""vd_copy: the library's SM copy between device memory and page-locked host
memory, at every alignment class and for sizes around the vector width."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SIZES = [1, 3, 15, 16, 17, 31, 1000, 65_537, 1_000_003]
OFFSETS = [(0, 0), (1, 1), (3, 7), (4, 8), (5, 6), (16, 0), (0, 9)]


def _bytes(n, seed):
    return torch.from_numpy(np.random.default_rng(seed).integers(0, 256, n, dtype=np.uint8))


@pytest.mark.parametrize("kind", ["h2d", "d2h", "d2d"])
def test_copy_matches_source_at_every_alignment(kind):
    from paper_2605_06408_gb300 import vd

    lib = vd.load_library()
    for n in SIZES:
        for so, do in OFFSETS:
            src_all = _bytes(n + 32, n + so)
            dst_all = torch.full((n + 32,), 0xAB, dtype=torch.uint8)
            if kind == "h2d":
                src_all, dst_all = src_all.pin_memory(), dst_all.cuda()
            elif kind == "d2h":
                src_all, dst_all = src_all.cuda(), dst_all.pin_memory()
            else:
                src_all, dst_all = src_all.cuda(), dst_all.cuda()
            src, dst = src_all[so:so + n], dst_all[do:do + n]
            rc = lib.vd_copy(ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(src.data_ptr()), n,
                             vd._stream_ptr(torch.device("cuda", 0)))
            assert rc == vd.VD_OK
            torch.cuda.synchronize()
            got, want = dst_all.cpu(), src_all.cpu()
            assert torch.equal(got[do:do + n], want[so:so + n]), (kind, n, so, do)
            # nothing written outside the range
            assert bool((got[:do] == 0xAB).all()) and bool((got[do + n:] == 0xAB).all()), (kind, n, so, do)


def test_copy_binding_round_trip_of_build_sized_arrays():
    from paper_2605_06408_gb300 import vd

    x = torch.rand(1_000_001, 3)
    h = x.pin_memory()
    d = torch.empty_like(x, device="cuda")
    vd.copy_(d, h)
    back = torch.empty_like(x).pin_memory()
    vd.copy_(back, d)
    torch.cuda.synchronize()
    assert torch.equal(back, x)
    i = torch.arange(12_345_679, dtype=torch.int32, device="cuda")
    hi = torch.empty(12_345_679, dtype=torch.int32).pin_memory()
    vd.copy_(hi, i)
    torch.cuda.synchronize()
    assert torch.equal(hi, torch.arange(12_345_679, dtype=torch.int32))


def test_copy_rejects_pageable_host_memory():
    from paper_2605_06408_gb300 import vd

    lib = vd.load_library()
    d = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    pageable = np.ones(1024, dtype=np.uint8)
    rc = lib.vd_copy(ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(pageable.ctypes.data), 1024,
                     vd._stream_ptr(torch.device("cuda", 0)))
    assert rc == vd.VD_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        vd.copy_(d, torch.ones(1024, dtype=torch.uint8))
