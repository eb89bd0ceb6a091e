"""The optimisers and the walk schedule of the optimisation loop (Sec. 5,
Sec. 5.2), on the CPU.

* Vector Adam (Ling et al. 2022) keeps one second moment per d-vector, from
  the squared norm of its gradient.  For d = 1 that is Adam (checked against
  the Adam class step by step); for d > 1 its trajectory is equivariant under
  rotations of the gradients, which Adam's per-coordinate moment is not (the
  same check run on Adam fails, so the check has teeth); its first step
  moves each vector by lr along its gradient.
* Eq. (update_rule): WPP_t = WPP_0 exp(log(WPP_T / WPP_0) t / T), read with t / T.
"""
import numpy as np

from paper_2405_12964_gb300 import optimize


def _rot(a):
    return np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])


def test_vector_adam_is_adam_for_scalars():
    rng = np.random.default_rng(1)
    x0 = rng.normal(size=7)
    a = optimize.Adam(x0, lr=3e-3)
    v = optimize.VectorAdam(x0[:, None], lr=3e-3)
    for _ in range(40):
        g = rng.normal(size=7) * rng.uniform(0.1, 10.0)
        a.step(g)
        v.step(g[:, None])
        assert np.allclose(v.theta[:, 0], a.theta, rtol=1e-13, atol=1e-15)


def _trajectory(opt_cls, x0, grads, flat=False):
    o = opt_cls(x0.ravel() if flat else x0, lr=1e-2)
    out = []
    for g in grads:
        o.step(g.ravel() if flat else g)
        out.append(np.array(o.theta).reshape(x0.shape))
    return np.array(out)


def test_vector_adam_steps_rotate_with_the_gradients():
    rng = np.random.default_rng(2)
    x0 = rng.normal(size=(5, 2))
    grads = [rng.normal(size=(5, 2)) * np.array([[3.0, 0.2]]) for _ in range(30)]   # anisotropic
    R = _rot(0.7)
    t1 = _trajectory(optimize.VectorAdam, x0, grads)
    t2 = _trajectory(optimize.VectorAdam, x0 @ R.T, [g @ R.T for g in grads])
    assert np.allclose(t1 @ R.T, t2, rtol=1e-12, atol=1e-12)
    # Adam's per-coordinate second moment breaks the symmetry
    a1 = _trajectory(optimize.Adam, x0, grads, flat=True)
    a2 = _trajectory(optimize.Adam, x0 @ R.T, [g @ R.T for g in grads], flat=True)
    assert np.abs(a1 @ R.T - a2).max() > 1e-3


def test_vector_adam_first_step_has_length_lr():
    rng = np.random.default_rng(3)
    x0 = rng.normal(size=(6, 3))
    g = rng.normal(size=(6, 3))
    o = optimize.VectorAdam(x0, lr=2e-3)
    x1 = o.step(g)
    d = x0 - x1
    assert np.allclose(np.linalg.norm(d, axis=1), 2e-3, rtol=1e-6)
    assert np.allclose(d / np.linalg.norm(d, axis=1, keepdims=True), g / np.linalg.norm(g, axis=1, keepdims=True))


def test_wpp_schedule_follows_update_rule():
    assert optimize.wpp_schedule(0, 100, 16, 256) == 16
    assert optimize.wpp_schedule(100, 100, 16, 256) == 256
    assert optimize.wpp_schedule(50, 100, 16, 256) == 64      # geometric midpoint
    assert optimize.wpp_schedule(1, 600, 2, 128, multiple=2) == 2
    assert optimize.wpp_schedule(600, 600, 2, 128, multiple=2) == 128
    assert optimize.wpp_schedule(300, 600, 2, 128, multiple=2) == 16
