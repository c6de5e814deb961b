"""The allocation-free sampling/selection entry point gives the same elite set as the
allocating path.

Callers that cannot allocate device memory while they plan (a control loop that must not
stall on cudaMalloc, a plug-in inside a framework that owns the GPU's memory) use
spasm_place_select_static, whose intermediates live in a fixed device array of the library.
This test calls it twice in a row through the C ABI and compares each result with
spasm_place_sample + spasm_select_topk + a gather of the same particles.  It lives in a file
of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_2510_07674_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _device_memory():
    """(used, reserved) bytes of the device's default memory pool -- where the library's
    stream-ordered allocations come from -- and the free bytes cudaMemGetInfo reports."""
    rt = None
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            continue
    if rt is None:
        pytest.skip("no CUDA runtime library to query the memory pool")
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    used, reserved = ctypes.c_uint64(), ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, 7, ctypes.byref(used)) == 0        # UsedMemCurrent
    assert rt.cudaMemPoolGetAttribute(pool, 5, ctypes.byref(reserved)) == 0    # ReservedMemCurrent
    free, _ = torch.cuda.mem_get_info()
    return used.value, reserved.value, free


def test_static_scratch_matches_allocating_path_twice():
    from paper_2510_07674_gb300 import spasm as S
    wl = scenes.make_problem("tower10", seed=3)
    pr = S.Problem(wl)
    B, n, m = pr.B, 16384, 4096
    for attempt in (0, 1):   # two calls in a row share (and overwrite) the scratch array
        x_el = torch.full((4 * B, m), float("nan"), device="cuda")
        c_el = torch.full((m,), float("nan"), device="cuda")
        S.spasm_place_select_static(pr, n, attempt, m, x_el, c_el)

        x = torch.empty(4 * B, n, device="cuda")
        cost = torch.empty(n, device="cuda")
        S.spasm_place_sample(pr, n, attempt, x, cost)
        idx = torch.empty(m, dtype=torch.int32, device="cuda")
        S.spasm_select_topk(pr, n, cost, m, idx)
        torch.cuda.synchronize()
        ref_x = x[:, idx.long()]
        ref_c = cost[idx.long()]
        np.testing.assert_allclose(c_el.cpu().numpy(), ref_c.cpu().numpy(), rtol=1e-6, atol=0)
        np.testing.assert_allclose(x_el.cpu().numpy(), ref_x.cpu().numpy(), rtol=1e-6, atol=0)
        assert np.all(np.diff(c_el.cpu().numpy()) >= 0)


def test_static_scratch_allocates_nothing_after_the_first_call():
    """The first call on a device is the set-up (it looks up the array and may load the
    library's device code); after it, a call changes neither the default pool's used or
    reserved bytes nor the device's free memory."""
    from paper_2510_07674_gb300 import spasm as S
    wl = scenes.make_problem("tower10", seed=4)
    pr = S.Problem(wl)
    B, n, m = pr.B, 16384, 4096
    x_el = torch.empty(4 * B, m, device="cuda")
    c_el = torch.empty(m, device="cuda")
    S.spasm_place_select_static(pr, n, 0, m, x_el, c_el)   # set-up call
    torch.cuda.synchronize()
    before = _device_memory()
    for attempt in (1, 2):
        S.spasm_place_select_static(pr, n, attempt, m, x_el, c_el)
    torch.cuda.synchronize()
    after = _device_memory()
    assert after == before, (before, after)
    assert np.all(np.isfinite(c_el.cpu().numpy()))


def test_static_scratch_rejects_sizes_beyond_its_array():
    from paper_2510_07674_gb300 import spasm as S
    wl = scenes.make_problem("tower10", seed=3, B=16)
    pr = S.Problem(wl)
    n, m = 32768, 64   # 4*16*32768 floats alone exceed the 2^20-float array
    x_el = torch.empty(4 * 16, m, device="cuda")
    c_el = torch.empty(m, device="cuda")
    with pytest.raises(S.SpasmError) as e:
        S.spasm_place_select_static(pr, n, 0, m, x_el, c_el)
    assert e.value.status == -1 and "static scratch" in str(e.value)
