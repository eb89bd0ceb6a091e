"""3D thermal design check (reduced size): the adjoint gradient of
L = 1/2 sum_p (u_p(theta) - uref_p)^2 through DWoSFunction (differential walks,
scatter, adjoint GEMV) agrees with central finite differences of the forward
estimator under common random numbers (Sec. 5.1 compares the differential
estimate with finite differences the same way).

Geometry: SH-perturbed icosphere (l <= 8, 81 coefficients) inside the box
[-2,2]^3, sigma = 1, source 0.5, g = 1 on the object and 0 on the box.
"""
import numpy as np
import pytest

from paper_2405_12964_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12964_gb300 import build
    build.build()
    from paper_2405_12964_gb300 import dwos
    sc = scenes.sh_sphere_scene(freq=24, n_query=96, walks=1024, coef_std=0.05)
    s = dwos.Solver(0)
    s.load_scene(sc)
    s.set_boundary(sc.reference_vertices(), sc.elem, sc.jac)
    s.set_dirichlet_mapped(sc.g_vert)
    xq = torch.tensor(sc.query, dtype=torch.float32, device="cuda")
    s.set_params(np.zeros(sc.n_param))
    uref = s.eval(xq, 4 * sc.walks)["u"].detach().clone()       # target at theta = 0
    return torch, dwos, sc, s, xq, uref


def test_adjoint_gradient_matches_central_differences(setup):
    torch, dwos, sc, s, xq, uref = setup
    theta0 = torch.tensor(sc.theta0, dtype=torch.float64)
    R, W, h = 4, sc.walks, 1e-3
    g_adj, g_fd = [], []
    for r in range(R):
        s.set_options(seed=0x12964 + 17 * r)
        th = theta0.clone().requires_grad_(True)
        u = dwos.solve(th, s, xq, W, backward_walks=W, backward_base=(1 << 40) + r * (1 << 30))
        L = 0.5 * ((u - uref) ** 2).sum()
        L.backward()
        g_adj.append(th.grad.numpy().copy())
        fd = np.zeros(sc.n_param)
        for j in range(sc.n_param):
            Ls = []
            for sgn in (1.0, -1.0):
                tj = sc.theta0.copy()
                tj[j] += sgn * h
                s.set_params(tj)
                uj = s.eval(xq, W)["u"]                  # same walk ids and seed: common random numbers
                Ls.append(0.5 * float(((uj - uref) ** 2).sum()))
            fd[j] = (Ls[0] - Ls[1]) / (2 * h)
        g_fd.append(fd)
    s.set_options(seed=0x12964)
    A, F = np.array(g_adj), np.array(g_fd)
    ma, mf = A.mean(0), F.mean(0)
    sa, sf = A.std(0, ddof=1) / np.sqrt(R), F.std(0, ddof=1) / np.sqrt(R)
    scale = np.sqrt(np.mean(mf ** 2))
    cos = float(ma @ mf / (np.linalg.norm(ma) * np.linalg.norm(mf)))
    big = np.abs(mf) > 0.25 * np.abs(mf).max()
    z = np.abs(ma - mf) / np.sqrt(sa ** 2 + sf ** 2 + (0.08 * np.abs(mf)) ** 2 + (0.02 * scale) ** 2)
    assert cos > 0.9, cos
    assert np.all(z[big] < 4.5), (z[big], ma[big], mf[big])
    assert np.mean(z) < 2.0
