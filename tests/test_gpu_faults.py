"""Failure handling through the C ABI, with every failure made on the host or by
a bounded wait that runs out: nothing here faults, traps or hangs the GPU.

* bad inputs are refused with DWOS_ERR_INVALID_ARG before any walk runs:
  non-finite vertices or Jacobians, element ids out of range, degenerate
  elements (zero length / zero area), an empty mesh, sigma < 0 or NaN, bad
  query points, oversized requests, empty or inconsistent batches; host and
  device copies of the arrays are checked alike;
* a distance query whose node-fetch bound runs out ends with
  DWOS_ERR_STEP_LIMIT and the context keeps working;
* the tensor-core kernel's bounded mbarrier wait gives up on a barrier that
  nothing arrives at and reports DWOS_ERR_TIMEOUT; the network keeps working.
"""
import numpy as np
import pytest

from paper_2405_12964_gb300 import scenes

pytestmark = pytest.mark.gpu

INVALID, STEP_LIMIT, TIMEOUT = 1, 4, 5


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12964_gb300 import build
    build.build()
    from paper_2405_12964_gb300 import dwos
    return torch, dwos


def _raises(dwos, status, fn, *a, **k):
    with pytest.raises(dwos.DwosError) as ei:
        fn(*a, **k)
    assert ei.value.status == status, str(ei.value)
    return str(ei.value)


def test_bad_boundaries_are_refused(env):
    torch, dwos = env
    sc = scenes.star_box_scene(n_seg=256, n_query=4, walks=16)
    s = dwos.Solver(0)
    for on_device in (False, True):
        def load(vert, elem, jac=None):
            if on_device:        # the binding passes device copies (mem = device)
                return s.set_boundary(vert, elem, jac)
            import ctypes
            v = np.ascontiguousarray(vert, np.float32)
            e = np.ascontiguousarray(elem, np.int32)
            j = None if jac is None else np.ascontiguousarray(jac, np.float32)
            P = 0 if j is None else j.shape[2]
            s._check(dwos.lib().dwos_set_boundary(
                s._h, v.shape[1], v.shape[0], v.ctypes.data_as(ctypes.c_void_p), e.shape[0],
                e.ctypes.data_as(ctypes.c_void_p), P, None if j is None else j.ctypes.data_as(ctypes.c_void_p),
                dwos.MEM_HOST))
        v = sc.vert.copy()
        v[7, 1] = np.nan
        _raises(dwos, INVALID, load, v, sc.elem, sc.jac)
        j = sc.jac.copy()
        j[9, 0, 3] = np.inf
        _raises(dwos, INVALID, load, sc.vert, sc.elem, j)
        e = sc.elem.copy()
        e[5, 1] = sc.vert.shape[0]
        _raises(dwos, INVALID, load, sc.vert, e, sc.jac)
        e = sc.elem.copy()
        e[11, 1] = e[11, 0]                       # zero-length segment
        assert "degenerate" in _raises(dwos, INVALID, load, sc.vert, e, sc.jac)
        tri = np.array([[0.0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0]])
        _raises(dwos, INVALID, load, tri, np.array([[0, 1, 2]], np.int32))   # collinear: zero area
        load(tri, np.array([[0, 1, 3]], np.int32))                            # a proper triangle loads
    with pytest.raises((dwos.DwosError, IndexError, ValueError)):
        s.set_boundary(np.zeros((0, 2)), np.zeros((0, 2), np.int32))         # empty mesh


def test_bad_pde_options_and_queries_are_refused(env):
    torch, dwos = env
    sc = scenes.disk_scene("screened_1", n_query=8)
    s = dwos.Solver(0)
    s.load_scene(sc)
    _raises(dwos, INVALID, s.set_pde, -1.0, 0.0)
    _raises(dwos, INVALID, s.set_pde, float("nan"), 0.0)
    _raises(dwos, INVALID, s.set_pde, 1.0, float("inf"))
    _raises(dwos, INVALID, s.set_options, K=0)
    _raises(dwos, INVALID, s.set_options, max_steps=1 << 24)
    s.set_options(K=1, max_steps=1 << 14)
    s.set_pde(4.0, 0.0)
    # non-finite query points: refused up front from host memory ...
    import ctypes
    q = sc.query.astype(np.float32).copy()
    q[3, 0] = np.nan
    u = np.zeros(8)
    st = dwos.lib().dwos_eval(s._h, 8, q.ctypes.data_as(ctypes.c_void_p), 16, u.ctypes.data_as(ctypes.c_void_p),
                              None, None, None, dwos.MEM_HOST)
    assert st == INVALID
    # ... and reported by the walk kernel for device memory (at the next sync)
    s.eval(q, 16)
    _raises(dwos, INVALID, s.sync)
    # the context still works
    out = s.eval(sc.query, 64)
    s.sync()
    assert np.all(np.isfinite(out["u"].cpu().numpy()))
    # oversized and malformed requests: more than 2^40 walks in one call
    big = np.zeros((1024, 2), np.float32)
    ub = np.zeros(1024)
    st = dwos.lib().dwos_eval(s._h, 1024, big.ctypes.data_as(ctypes.c_void_p), (1 << 31) - 1,
                              ub.ctypes.data_as(ctypes.c_void_p), None, None, None, dwos.MEM_HOST)
    assert st == INVALID and b"too many walks" in dwos.lib().dwos_last_error(s._h)
    st = dwos.lib().dwos_eval(s._h, -1, None, 16, None, None, None, None, dwos.MEM_HOST)
    assert st == INVALID


def test_bad_batches_are_refused(env):
    torch, dwos = env
    import ctypes
    h = ctypes.c_void_p()
    jobs = (dwos.BatchJob * 1)()
    assert dwos.lib().dwos_batch_create(ctypes.byref(h), jobs, 0, None) == INVALID
    sc = scenes.disk_scene("screened_1", n_query=4)
    s = dwos.Solver(0)
    s.load_scene(sc)
    with pytest.raises(dwos.DwosError) as ei:
        dwos.Batch([(s, sc.query, 12, np.zeros(4), 0)])        # 12 walks: not a multiple of B = 8
    assert ei.value.status == INVALID
    with pytest.raises(dwos.DwosError) as ei:
        dwos.Batch([(s, np.zeros((0, 2)), 16, np.zeros(0), 0)])  # empty job
    assert ei.value.status == INVALID
    with pytest.raises(dwos.DwosError) as ei:
        dwos.Batch([(s, np.array([[3.0, 0.0]]), 16, np.zeros(1), 0)])   # point outside the disk
    assert ei.value.status == 8


def test_traversal_bound_running_out_is_reported(env):
    torch, dwos = env
    for sc in (scenes.star_box_scene(n_seg=4096, n_query=16, walks=64),
               scenes.sh_sphere_scene(freq=24, n_query=16, walks=32)):
        for traversal in (0, 3):
            s = dwos.Solver(0)
            s.load_scene(sc, traversal=traversal)
            ref = s.eval(sc.query, sc.walks)["u"].cpu().numpy()
            s.set_traversal_budget(1)               # one node fetch per query: the searches give up
            s.eval(sc.query, sc.walks)
            _raises(dwos, STEP_LIMIT, s.sync)
            # the walks ended (no hang) and the context works again with the default bound
            s.set_traversal_budget(0)
            again = s.eval(sc.query, sc.walks)["u"].cpu().numpy()
            s.sync()
            assert np.array_equal(again, ref)


def test_tensor_core_wait_running_out_is_reported(env):
    torch, dwos = env
    net = dwos.ControlVariateNet(seed=3)
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, size=(512, 2)).astype(np.float32)
    t = np.stack([x[:, 0], x[:, 1]], 1).astype(np.float32)
    m = np.ones_like(t)
    before = net.loss_grad(x, t, m)[1].cpu().numpy()
    for polls in (1, 1000):
        _raises(dwos, TIMEOUT, net.wait_probe, polls)
    # reported once; the network trains and evaluates as before
    after = net.loss_grad(x, t, m)[1].cpu().numpy()
    net.sync()
    assert np.array_equal(before, after)
    net.train_step(x, t, m, lr=1e-3)
    net.sync()
