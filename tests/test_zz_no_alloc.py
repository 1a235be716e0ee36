"""ffa_fold_noalloc: the fold for callers that cannot allocate device memory
(it keeps its scratch plane in a fixed device array inside the library).

Checked through the C ABI against ffa_fold, which takes caller-provided
scratch, on two calls in a row (the shared array keeps the previous call's
contents).  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_05581_gb300 import ffa
    return ffa


def _fold_ref(F, z, prec, p0, md, m):
    import torch
    dt = torch.float32 if prec == F.FOLD_F32 else torch.int32
    plane = torch.empty((m, p0), dtype=dt, device=z.device)
    tmp = torch.empty_like(plane)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    F._check(F._lib.ffa_fold(F._ptr(z), prec, p0, md, m, F._ptr(plane), F._ptr(tmp), s))
    return plane


def _fold_noalloc(F, z, prec, p0, md, m):
    import torch
    dt = torch.float32 if prec == F.FOLD_F32 else torch.int32
    plane = torch.empty((m, p0), dtype=dt, device=z.device)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    F._check(F._lib.ffa_fold_noalloc(F._ptr(z), prec, p0, md, m, F._ptr(plane), s))
    return plane


@pytest.mark.parametrize("prec", ["f32", "i8"])
def test_noalloc_fold_matches_fold_twice(F, prec):
    import torch
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(123)
    p = F.FOLD_F32 if prec == "f32" else F.FOLD_I8
    # two different shapes in a row: the second call finds the first's contents
    for p0, md, m in [(390, 168, 256), (4097, 1000, 1024)]:
        n = md * p0 + 7
        if p == F.FOLD_F32:
            z = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).to(dev)
        else:
            z = torch.from_numpy(rng.integers(-127, 128, n).astype(np.int8)).to(dev)
        got = _fold_noalloc(F, z, p, p0, md, m)
        ref = _fold_ref(F, z, p, p0, md, m)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_noalloc_fold_rejects_oversized(F):
    import torch
    dev = torch.device("cuda", 0)
    z = torch.zeros(16, dtype=torch.float32, device=dev)
    m, p0 = 8192, F.NOALLOC_FOLD_MAX_ELEMS // 8192 + 1
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = F._lib.ffa_fold_noalloc(F._ptr(z), F.FOLD_F32, p0, 1, m, F._ptr(z), s)
    assert st == F.ERR_UNSUPPORTED
    assert b"FFA_NOALLOC_FOLD_MAX_ELEMS" in F._lib.ffa_last_error()
    # m_rows * p0 beyond int64 would wrap in a plain product: still rejected
    st = F._lib.ffa_fold_noalloc(F._ptr(z), F.FOLD_F32, 1 << 24, 1, 1 << 40, F._ptr(z), s)
    assert st == F.ERR_UNSUPPORTED


def test_noalloc_fold_allocates_nothing(F):
    """A warm call changes neither the caching allocator's count nor the
    device's free memory (the output plane is allocated before measuring)."""
    import torch
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(5)
    p0, md, m = 1000, 700, 1024
    z = torch.from_numpy(rng.standard_normal(md * p0).astype(np.float32)).to(dev)
    first = _fold_noalloc(F, z, F.FOLD_F32, p0, md, m)  # warm: set-up and kernels loaded
    plane = torch.empty_like(first)
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated(dev)
    free0, _ = torch.cuda.mem_get_info(dev)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    F._check(F._lib.ffa_fold_noalloc(F._ptr(z), F.FOLD_F32, p0, md, m, F._ptr(plane), s))
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated(dev) == alloc0
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert torch.equal(plane, first)
