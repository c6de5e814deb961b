"""Failure paths, exercised without a GPU fault.

* A bounded device wait that runs out: one CTA waits, through the same bounded wait the
  kernels' table staging uses, on an mbarrier whose expected bytes no copy delivers (no copy
  is issued, so nothing is in flight).  The kernel returns, the next synchronising call
  reports SPASM_ERR_DEVICE with the timeout, and the context stays usable.
* An allocation that fails: a host-side fake makes the nth device allocation of
  spasm_create_problem fail; creation reports SPASM_ERR_NOMEM and returns every byte it had
  taken to the memory pool.
"""
import ctypes

import numpy as np
import pytest

from paper_2510_07674_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _S():
    from paper_2510_07674_gb300 import spasm as S
    return S


def _pool_used() -> int:
    rt = None
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            continue
    if rt is None:
        pytest.skip("no CUDA runtime library to query the memory pool")
    torch.cuda.synchronize()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    used = ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, 7, ctypes.byref(used)) == 0   # UsedMemCurrent
    return used.value


def test_bounded_wait_timeout_is_reported_and_the_context_survives():
    S = _S()
    wl = scenes.make_problem("tower1", seed=0)
    pr = S.Problem(wl)
    try:
        S.spasm_synchronize(pr)                      # clean before
        S.spasm_inject_wait_timeout(pr, 1000)
        with pytest.raises(S.SpasmError) as e:
            S.spasm_synchronize(pr)
        assert e.value.status == -6 and "bounded device wait" in str(e.value)
        with pytest.raises(S.SpasmError):            # sticky: the problem keeps reporting it
            S.spasm_synchronize(pr)
    finally:
        pr.close()
    # the GPU context is intact: a fresh problem solves
    pr2 = S.Problem(wl)
    try:
        S.spasm_optimize(pr2)
        r = S.spasm_result(pr2)
        assert r["n_found"] > 0 and r["success"].all()
        S.spasm_synchronize(pr2)
    finally:
        pr2.close()


@pytest.mark.parametrize("nth", [0, 3, 17, 29])
def test_injected_allocation_failure_reports_nomem_without_leak(nth):
    S = _S()
    wl = scenes.make_problem("tower4", seed=0)
    S.Problem(wl).close()                            # warm the pool and the module
    before = _pool_used()
    S.spasm_inject_alloc_failure(nth)
    try:
        with pytest.raises(S.SpasmError) as e:
            S.Problem(wl)
        assert e.value.status == -2 and "injected" in str(e.value)
    finally:
        S.spasm_inject_alloc_failure(-1)
    assert _pool_used() == before
    pr = S.Problem(wl)                                # allocation works again
    pr.close()
    assert _pool_used() == before
