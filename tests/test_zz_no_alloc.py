"""The allocation-free interpolative decomposition (hbs_row_id_static).

Callers that may not allocate device memory during a call (a fixed memory budget, code
that cannot wait on cudaMalloc/cudaFree, a foreign allocator) use hbs_row_id_static.  It
must give the same decomposition as hbs_row_id, call after call, although every call
reuses the same fixed working array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import dev, require_lib


def _low_rank(m, n, seed):
    rng = np.random.default_rng(seed)
    r = 60
    u = rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r))
    v = rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n))
    sig = 10.0 ** (-np.arange(r) / 3.0)
    return (u * sig) @ v  # Mt (m x n): columns are the rows of M


def _run(fn, mt_host, m, n, tol):
    import torch
    mt = dev(np.asfortranarray(mt_host).ravel(order="F"))
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    t = torch.zeros(min(m, n) * n, dtype=torch.complex128, device="cuda")
    k = fn(mt, m, n, tol, perm, t)
    return k, perm.cpu().numpy(), t.cpu().numpy()[: k * (n - k)]


def _device_memory_counters():
    """(free device bytes from cudaMemGetInfo, used bytes of the device's default stream-ordered
    memory pool, bytes held by torch's caching allocator).  Any device allocation by the call
    under test moves the first (cudaMalloc reserves at least 2 MiB) or the second (cudaMallocAsync)."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    used = None
    try:
        cu = ctypes.CDLL("libcuda.so.1")
        devh = ctypes.c_int()
        pool = ctypes.c_void_p()
        val = ctypes.c_uint64()
        if (cu.cuDeviceGet(ctypes.byref(devh), torch.cuda.current_device()) == 0
                and cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), devh) == 0
                and cu.cuMemPoolGetAttribute(pool, 7, ctypes.byref(val)) == 0):  # USED_MEM_CURRENT
            used = int(val.value)
    except OSError:
        pass
    return free, used, torch.cuda.memory_reserved()


@pytest.mark.gpu
def test_static_scratch_id_allocates_nothing():
    """After a first call (which looks up the fixed array's address), further calls leave the
    device's free memory, its default memory pool and torch's allocator exactly as they were."""
    hbs = require_lib()
    import torch
    mt_host = _low_rank(96, 6000, 9)
    mt = dev(np.asfortranarray(mt_host).ravel(order="F"))
    perm = torch.zeros(6000, dtype=torch.int32, device="cuda")
    t = torch.zeros(96 * 6000, dtype=torch.complex128, device="cuda")
    inputs = [mt.clone() for _ in range(4)]  # Mt is overwritten: one copy per call, made up front
    hbs.row_id_static(inputs[0], 96, 6000, 1e-12, perm, t)
    torch.cuda.synchronize()
    before = _device_memory_counters()
    for a in inputs[1:]:
        hbs.row_id_static(a, 96, 6000, 1e-12, perm, t)
    torch.cuda.synchronize()
    after = _device_memory_counters()
    assert abs(after[0] - before[0]) < (1 << 20), (before, after)
    assert after[1] == before[1], (before, after)


@pytest.mark.gpu
def test_static_scratch_id_matches_one_cta_id_small_n():
    """For n <= 4096 hbs_row_id runs the one-CTA-per-matrix pivoted QR while the static entry
    point runs the multi-CTA one: the two must still give the same rank, skeleton order and T."""
    hbs = require_lib()
    for m, n, seed in ((48, 1000, 11), (90, 4096, 12), (64, 300, 13)):
        mt = _low_rank(m, n, seed)
        k0, p0, t0 = _run(hbs.row_id, mt, m, n, 1e-12)
        for _ in range(2):
            k, p, t = _run(hbs.row_id_static, mt, m, n, 1e-12)
            assert k == k0, (m, n, k, k0)
            assert np.array_equal(p, p0), (m, n)
            assert np.allclose(t, t0, rtol=1e-11, atol=1e-11 * np.abs(t0).max())


@pytest.mark.gpu
def test_static_scratch_id_matches_allocating_id_twice():
    hbs = require_lib()
    m, n, tol = 96, 6000, 1e-12  # n > 4096: both entry points run the multi-CTA pivoted QR
    mt = _low_rank(m, n, 7)
    k0, p0, t0 = _run(hbs.row_id, mt, m, n, tol)
    assert 20 < k0 < m
    for _ in range(2):  # two calls in a row share the same working array
        k, p, t = _run(hbs.row_id_static, mt, m, n, tol)
        assert k == k0
        assert np.array_equal(p, p0)
        assert np.allclose(t, t0, rtol=1e-12, atol=1e-12 * np.abs(t0).max())
    # a different, smaller problem next: state left by the previous call must not leak
    mt2 = _low_rank(40, 5000, 8)
    k0, p0, t0 = _run(hbs.row_id, mt2, 40, 5000, tol)
    k, p, t = _run(hbs.row_id_static, mt2, 40, 5000, tol)
    assert k == k0 and np.array_equal(p, p0)
    assert np.allclose(t, t0, rtol=1e-12, atol=1e-12 * np.abs(t0).max())


def test_static_scratch_id_rejects_oversize_n():
    """n beyond the fixed capacity is refused on the host, before any GPU work."""
    import os
    from paper_1301_1247_gb300 import build, hbs
    if not os.path.exists(hbs.LIB_PATH):
        build.build()
    L = hbs.lib()
    rank = ctypes.c_int()
    fake = ctypes.c_void_p(16)
    st = L.hbs_row_id_static(fake, 8, hbs.ROW_ID_STATIC_MAX_N + 1, 1e-12, ctypes.byref(rank), fake, fake, None)
    assert st == 1
    assert b"HBS_ROW_ID_STATIC_MAX_N" in L.hbs_last_error()
