"""Reverse-mode scatter with vertex flags.

Vertices whose Jacobian rows (and dg rows) are all zero cannot change the
parameter gradient, so the scatter leaves them out unless the vertex gradient
is returned.  On the same walks the parameter gradient must not depend on
that choice, and the vertex gradient must still reach the fixed vertices (the
box around the star has zero Jacobian rows but collects most shell hits).
"""
import numpy as np
import pytest

from paper_2405_12964_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Solver():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12964_gb300 import build
    build.build()
    from paper_2405_12964_gb300.dwos import Solver as S
    return S


@pytest.mark.parametrize("which", ["star_box", "sh_sphere"])
def test_parameter_gradient_does_not_depend_on_the_vertex_flags(Solver, which):
    sc = scenes.star_box_scene(n_query=64, walks=512) if which == "star_box" else \
        scenes.sh_sphere_scene(freq=20, n_query=32, walks=256)
    uref = np.zeros(sc.query.shape[0]) if which == "sh_sphere" else sc.u_ref
    s = Solver(0)
    s.load_scene(sc)
    loss_a, g_a = s.grad_l2(sc.query, uref, sc.walks, walk_id_base=7)
    loss_b, g_b, gv = s.grad_l2(sc.query, uref, sc.walks, walk_id_base=7, vertex_grad=True)
    g_a, g_b, gv = g_a.cpu().numpy(), g_b.cpu().numpy(), gv.cpu().numpy()
    assert float(loss_a) == float(loss_b)
    # the same walks: only the FP64 summation order of the scatter differs
    assert np.allclose(g_a, g_b, rtol=1e-9, atol=1e-12 * np.abs(g_b).max())
    jac = np.asarray(sc.jac).reshape(gv.shape[0], -1)
    fixed = np.all(jac == 0.0, axis=1)
    assert fixed.any() and (~fixed).any()
    # the fixed vertices still collect their terms when the vertex gradient is asked for
    assert np.abs(gv[fixed]).sum() > 0.0
