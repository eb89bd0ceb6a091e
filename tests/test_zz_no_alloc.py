"""dwos_eval_static: the allocation-free variant of dwos_eval.

Callers whose device memory belongs to another allocator or a fixed budget,
or whose loops cannot absorb cudaMalloc's implicit synchronisation, cannot let
a library allocate; this entry point keeps its scratch in a fixed array inside
the library.  It must return what
dwos_eval returns for the same walks, call after call (the array is reused and
keeps the previous call's contents), and refuse requests larger than its
array.  The file name sorts last so that pytest collects it last: a run that
stops at the first failure (-x) has then already run every other test.  The
tests depend on no earlier test: they pass alone in a fresh process, and after
the rest of the suite, whatever the array held before.
"""
import ctypes

import numpy as np
import pytest

from paper_2405_12964_gb300 import scenes

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12964_gb300 import build
    build.build()
    from paper_2405_12964_gb300 import dwos
    return torch, dwos


def _static(torch, dwos, s, xq, W, grad):
    n = xq.shape[0]
    dd = dict(device=s.device, dtype=torch.float64)
    u, se = torch.full((n,), -1.0, **dd), torch.full((n,), -1.0, **dd)
    du = torch.full((n, s.n_param), -1.0, **dd) if grad else None
    dse = torch.full((n, s.n_param), -1.0, **dd) if grad else None
    s._stream()
    st = dwos.lib().dwos_eval_static(s._h, n, _ptr(xq), W, _ptr(u), _ptr(se), _ptr(du), _ptr(dse))
    assert st == 0, dwos.lib().dwos_last_error(s._h).decode()
    torch.cuda.synchronize()
    return u, se, du, dse


def test_static_eval_matches_eval_on_two_calls_in_a_row(env):
    torch, dwos = env
    s = dwos.Solver(0)
    sc = scenes.disk_scene("screened_1", n_query=24)
    s.load_scene(sc)
    cases = [(sc.query, 512, True), (sc.query[5:21], 1024, False)]
    for q, W, grad in cases:
        xq = torch.tensor(q, dtype=torch.float32, device=s.device)
        u, se, du, dse = _static(torch, dwos, s, xq, W, grad)
        ref = s.eval(xq, W, grad=grad)
        torch.cuda.synchronize()
        # same kernels on the same Philox walks: equal to FP64 reduction order
        assert np.allclose(u.cpu().numpy(), ref["u"].cpu().numpy(), rtol=1e-12, atol=1e-12)
        assert np.allclose(se.cpu().numpy(), ref["u_se"].cpu().numpy(), rtol=1e-9, atol=1e-12)
        if grad:
            assert np.allclose(du.cpu().numpy(), ref["du"].cpu().numpy(), rtol=1e-9, atol=1e-12)
            assert np.allclose(dse.cpu().numpy(), ref["du_se"].cpu().numpy(), rtol=1e-9, atol=1e-12)


def test_static_eval_rejects_requests_beyond_its_array(env):
    torch, dwos = env
    s = dwos.Solver(0)
    sc = scenes.disk_scene("screened_1", n_query=64)
    s.load_scene(sc)
    xq = torch.tensor(sc.query, dtype=torch.float32, device=s.device)
    u = torch.empty(64, device=s.device, dtype=torch.float64)
    st = dwos.lib().dwos_eval_static(s._h, 64, _ptr(xq), 8192, _ptr(u), None, None, None)
    assert st == 1
    assert b"DWOS_STATIC_MAX_WALKS" in dwos.lib().dwos_last_error(s._h)
