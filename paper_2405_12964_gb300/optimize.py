"""Gradient-based shape optimisation with differential walk on spheres.

The loop of the paper's experiments (Sec. 5.2, Sec. 6): at each iteration,
estimate dL/dtheta of L = 1/2 sum_p (u_p(theta) - uref_p)^2 with fresh walks
(U-statistic product estimator, Sec. 4.3), and take an Adam step (Sec. 5: lr
1e-3).  The number of walks per point follows the exponential annealing
schedule of Eq. (update_rule), read with t/T in the exponent.

Optionally a learned control variate (the library's tensor-core MLP) is trained
online on the walks' own estimates: (x1, estimate of u at x1) for the u head,
and for the du/dn head the nested walks' estimates and displacements (a
variance-minimising least-squares fit), and its spatial gradient at the observation
points is subtracted from every walk's estimate (dwos_grad_l2_cv); the nested
walks behind each du/dn estimate subtract (q n + t) . (x_end - x_off) with q the
du/dn head at the element and t the data's tangential gradient.  Both
corrections have mean zero, which keeps the gradient unbiased.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import torch

from . import dwos


def wpp_schedule(t: int, T: int, wpp0: int, wppT: int, multiple: int = 8) -> int:
    """Eq. (update_rule): WPP_t = WPP_0 exp(log(WPP_T / WPP_0) t / T), rounded to
    a multiple of the U-statistic batch size."""
    w = wpp0 * math.exp(math.log(wppT / wpp0) * t / max(T, 1))
    return max(multiple, int(round(w / multiple)) * multiple)


class Adam:
    """Adam (Kingma & Ba 2015) on a parameter vector."""

    def __init__(self, theta: np.ndarray, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8):
        self.theta = np.array(theta, dtype=np.float64)
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = np.zeros_like(self.theta)
        self.v = np.zeros_like(self.theta)
        self.t = 0

    def step(self, g: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        self.theta = self.theta - self.lr * mh / (np.sqrt(vh) + self.eps)
        return self.theta


class VectorAdam:
    """Vector Adam (Ling et al. 2022), the optimiser Sec. 5 uses for shape
    parameters such as vertex positions: Adam on an (n, d) array of d-vectors
    whose second moment is kept per vector, from the squared norm of its
    gradient, so that a step is the same whatever the frame the vectors are
    written in (Adam's per-coordinate second moment is not: it depends on the
    axes).  For d = 1 it is Adam."""

    def __init__(self, x: np.ndarray, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8):
        x = np.array(x, dtype=np.float64)
        self.shape = x.shape
        self.x = x.reshape(x.shape[0], -1) if x.ndim > 1 else x.reshape(1, -1)
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = np.zeros_like(self.x)
        self.v = np.zeros(self.x.shape[0])
        self.t = 0

    @property
    def theta(self) -> np.ndarray:
        return self.x.reshape(self.shape)

    def step(self, g: np.ndarray) -> np.ndarray:
        g = np.asarray(g, dtype=np.float64).reshape(self.x.shape)
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * np.sum(g * g, axis=1)
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        self.x = self.x - self.lr * mh / (np.sqrt(vh)[:, None] + self.eps)
        return self.theta


@dataclass
class History:
    loss: List[float] = field(default_factory=list)
    theta_err: List[float] = field(default_factory=list)
    wpp: List[int] = field(default_factory=list)
    seconds: List[float] = field(default_factory=list)
    var_ratio: List[float] = field(default_factory=list)     # median per-point Var(u with CV) / Var(u)
    mlp_loss: List[float] = field(default_factory=list)
    thetas: List[np.ndarray] = field(default_factory=list)   # the iterate after each step


class ControlVariateTrainer:
    """Online training of the control-variate network on walk samples."""

    def __init__(self, device: int = 0, seed: int = 0, lr: float = 2e-3, iters: int = 4, max_samples: int = 65536,
                 q_weight: float = 0.2, h: float = 0.02):
        self.net = dwos.ControlVariateNet(device, seed=seed)
        self.h = h                   # the solver's offset distance (du/dn = (g - u_off) / h)
        self.lr, self.iters, self.max_samples = lr, iters, max_samples
        self.q_weight = q_weight     # weight of the du/dn head's (normalised) variance loss against the u head's
        self.rng = np.random.default_rng(seed)

    def update(self, solver: "dwos.Solver", samples: torch.Tensor, debug: Optional[torch.Tensor]) -> torch.Tensor:
        """Train on one gradient step's walks.  The training rows (one per walk
        for the u head, one per walk for the du/dn head, thinned to at most
        max_samples by a common stride with a random offset) are built on the
        device by dwos_cv_training_set: the u head learns the walks' estimates
        at their first-step points; the du/dn head learns, at each hit point,
        the slope q that minimises the variance of the corrected nested mean
        u_plain - disp_t - q disp_n (a least-squares fit of r / disp_n with
        weights disp_n^2, r = u_plain - g(xbar) - disp_t; centring on g keeps
        the fit's noise at Var(u)).  Returns the last iteration's loss as a
        device tensor: nothing here waits for the GPU."""
        n_rows = samples.shape[0] * (2 if debug is not None else 1)
        stride = max(1, (n_rows + self.max_samples - 1) // self.max_samples)
        off = int(self.rng.integers(stride))
        x, t, m = solver.cv_training_set(samples, debug, stride, off, self.q_weight)
        loss = None
        for _ in range(self.iters):
            loss = self.net.train_step(x, t, m, lr=self.lr)
        return loss

    def grad_at(self, xq) -> torch.Tensor:
        _, g, _ = self.net.eval(xq)
        return g


def run(scene, theta_target: np.ndarray, theta_start: np.ndarray, steps: int = 200, lr: float = 1e-3,
        wpp0: int = 256, wppT: int = 1024, use_cv: bool = False, whole_walk: bool = True, seed: int = 1,
        device: int = 0, target_walks: int = 16384, trainer: Optional[ControlVariateTrainer] = None,
        train_every: int = 1):
    """Optimise theta to match the profile that theta_target produces at the
    scene's observation points (the network, if any, is trained on every
    train_every-th step's walks).  Returns (theta, History, trainer)."""
    s = dwos.Solver(device)
    s.load_scene(scene)
    s.set_boundary(scene.reference_vertices(), scene.elem, scene.jac)
    s.set_dirichlet_mapped(scene.g_vert, scene.dg_vert)
    xq = torch.tensor(scene.query, dtype=torch.float32, device=s.device)
    s.set_params(theta_target)
    uref = s.eval(xq, target_walks)["u"].to(torch.float32)
    opt = Adam(theta_start, lr=lr)
    hist = History()
    if use_cv and trainer is None:
        trainer = ControlVariateTrainer(device, seed=seed, h=scene.h)
    total = 0.0
    for it in range(steps):
        W = wpp_schedule(it + 1, steps, wpp0, wppT)
        s.set_params(opt.theta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cv_grad = trainer.grad_at(xq) if use_cv else None
        cv_elem = s.cv_table(trainer.net) if use_cv else None
        train = use_cv and it % train_every == 0
        out = s.grad_l2_cv(xq, uref, W, walk_id_base=(seed << 40) + it * (1 << 28), cv_grad=cv_grad,
                           whole_walk=whole_walk, cv_elem=cv_elem, samples=train, debug=train)
        g = out["grad"].cpu().numpy()
        if train:
            hist.mlp_loss.append(trainer.update(s, out["samples"], out["debug"]))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        total += dt
        opt.step(g)
        hist.loss.append(float(out["loss"][0]))
        hist.theta_err.append(float(np.linalg.norm(opt.theta - theta_target)))
        hist.thetas.append(opt.theta.copy())
        hist.wpp.append(W)
        hist.seconds.append(total)
        if use_cv:
            r = (out["u_se_cv"] / out["u_se"].clamp_min(1e-30)).cpu().numpy() ** 2
            hist.var_ratio.append(float(np.median(r)))
    if use_cv:
        trainer.net.sync()                               # reports a timed-out tensor-core wait, if any
        hist.mlp_loss = [float(l[0]) for l in hist.mlp_loss]
    return opt.theta, hist, trainer


def noisy_gradient_study(offset=(0.1, -0.06), iters: int = 600, lr: float = 1e-3, wpps=(2, 16, 128),
                         anneal=(2, 128), seeds=(1, 2, 3), target_walks: int = 16384, eval_every: int = 20,
                         eval_walks: int = 4096, device: int = 0, n_seg: int = 4096, n_query: int = 256):
    """The experiment of Sec. 5.2 (Fig. sgd) on the 2D shape-from-diffusion
    geometry: the star's position (a 2-vector, Vector Adam, lr 1e-3) is
    optimised from `offset` back to the origin, where the target profile was
    taken (target_walks per point), with a fixed number of differential walks
    per point (each of `wpps`) or the annealing schedule of Eq. (update_rule)
    from anneal[0] to anneal[1].  Each run records per iteration the position
    error |theta - theta*| and the seconds spent (the gradient estimate with
    its BVH rebuild, the read-back and the optimiser step; synchronised), and
    every eval_every iterations the loss 1/2 sum_p (u_p - uref_p)^2 from
    eval_walks walks per point (outside the timed region).  n_query
    observation points on the square |x|_inf = 0.6.  Returns a dict config ->
    list over seeds of {"err", "seconds", "loss_iter", "loss", "err0"}."""
    from . import scenes
    sc = scenes.translated_star_scene(n_seg=n_seg, n_query=n_query)
    s = dwos.Solver(device)
    s.load_scene(sc)
    s.set_boundary(sc.reference_vertices(), sc.elem, sc.jac)
    s.set_dirichlet_mapped(sc.g_vert)
    xq = torch.tensor(sc.query, dtype=torch.float32, device=s.device)
    target = np.zeros(2)
    s.set_params(target)
    uref = s.eval(xq, target_walks)["u"].to(torch.float32)
    configs = [("%d WPP" % w, w, w) for w in wpps] + [("annealed %d->%d WPP" % anneal, anneal[0], anneal[1])]
    out = {}
    for name, w0, wT in configs:
        runs = []
        for seed in seeds:
            opt = VectorAdam(np.asarray(offset, dtype=np.float64)[None, :], lr=lr)
            err, secs, loss_it, loss = [], [], [], []
            total = 0.0
            for it in range(iters):
                W = wpp_schedule(it + 1, iters, w0, wT, multiple=sc.B) if w0 != wT else w0
                if it % eval_every == 0:
                    s.set_params(opt.theta[0])
                    u = s.eval(xq, eval_walks)["u"]
                    loss_it.append(it)
                    loss.append(float(0.5 * torch.sum((u - uref.double()) ** 2)))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.set_params(opt.theta[0])
                _, g = s.grad_l2(xq, uref, W, walk_id_base=(seed << 44) + it * (1 << 24))
                opt.step(g.cpu().numpy()[None, :])
                total += time.perf_counter() - t0
                err.append(float(np.linalg.norm(opt.theta[0] - target)))
                secs.append(total)
            s.set_params(opt.theta[0])
            u = s.eval(xq, eval_walks)["u"]
            loss_it.append(iters)
            loss.append(float(0.5 * torch.sum((u - uref.double()) ** 2)))
            runs.append({"err": err, "seconds": secs, "loss_iter": loss_it, "loss": loss,
                         "err0": float(np.linalg.norm(np.asarray(offset) - target))})
        out[name] = runs
    return out


def thermal_design(target=(0.15, 0.05), start=(0.0, 0.0), iters: int = 200, lr: float = 5e-3, walks: int = 128,
                   target_walks: int = 8192, n_query: int = 32, seed: int = 1, device: int = 0):
    """The thermal design of Sec. 6.3 in 2D: move the heating wire of
    scenes.thermal_scene (Dirichlet g = 1) so that the temperature on the
    insulating slab's underside (Neumann part; query points on it) matches the
    profile the wire makes at `target`.  Differential walks on stars give
    dL/dtheta of L = 1/2 sum_p (u_p - uref_p)^2 (U-statistic estimator); the
    wire's position is one 2-vector, updated by Vector Adam.  Returns
    (theta, position errors, losses of the estimates)."""
    from . import scenes
    sc = scenes.thermal_scene(n_query=n_query)
    s = dwos.Solver(device)
    s.load_scene(sc)
    xq = torch.tensor(sc.query, dtype=torch.float32, device=s.device)
    tgt = np.asarray(target, dtype=np.float64)
    s.set_params(tgt)
    uref = s.eval(xq, target_walks)["u"].to(torch.float32)
    opt = VectorAdam(np.asarray(start, dtype=np.float64)[None, :], lr=lr)
    err, losses = [float(np.linalg.norm(opt.theta[0] - tgt))], []
    for it in range(iters):
        s.set_params(opt.theta[0])
        loss, g = s.grad_l2(xq, uref, walks, walk_id_base=(seed << 40) + it * (1 << 24))
        opt.step(g.cpu().numpy()[None, :])
        err.append(float(np.linalg.norm(opt.theta[0] - tgt)))
        losses.append(float(loss[0]))
    return opt.theta[0], err, losses


def thermal_design_3d(target=(0.12, -0.08, 0.05), start=(0.0, 0.0, 0.0), iters: int = 200, lr: float = 5e-3,
                      walks: int = 128, target_walks: int = 8192, n_side: int = 6, seed: int = 1, device: int = 0):
    """The thermal design of Sec. 6.3 in 3D: move the heating element of
    scenes.thermal_scene_3d (a Dirichlet sphere, g = 1) so that the temperature
    on the insulating slab's underside (the Neumann part; an n_side x n_side
    grid of query points on it) matches the profile the element makes at
    `target`.  Differential walks on stars give dL/dtheta of
    L = 1/2 sum_p (u_p - uref_p)^2 (U-statistic estimator); the element's
    position is one 3-vector, updated by Vector Adam.  Returns (theta, position
    errors, losses of the estimates)."""
    from . import scenes
    sc = scenes.thermal_scene_3d(n_side=n_side)
    s = dwos.Solver(device)
    s.load_scene(sc)
    xq = torch.tensor(sc.query, dtype=torch.float32, device=s.device)
    tgt = np.asarray(target, dtype=np.float64)
    s.set_params(tgt)
    uref = s.eval(xq, target_walks)["u"].to(torch.float32)
    opt = VectorAdam(np.asarray(start, dtype=np.float64)[None, :], lr=lr)
    err, losses = [float(np.linalg.norm(opt.theta[0] - tgt))], []
    for it in range(iters):
        s.set_params(opt.theta[0])
        loss, g = s.grad_l2(xq, uref, walks, walk_id_base=(seed << 40) + it * (1 << 24))
        opt.step(g.cpu().numpy()[None, :])
        err.append(float(np.linalg.norm(opt.theta[0] - tgt)))
        losses.append(float(loss[0]))
    return opt.theta[0], err, losses


def study_table(res: dict, iters=(50, 150, 300, 600), time_fracs=(0.1, 0.25, 0.5, 1.0)) -> dict:
    """Summary of noisy_gradient_study: per configuration the mean (over
    seeds) position error and loss at equal iterations, the seconds per
    iteration, and the position error at equal wall time (fractions of the
    fastest configuration's run, so that every configuration is still
    running; before its first iteration ends a run is at its start)."""
    t_min = min(np.mean([r["seconds"][-1] for r in runs]) for runs in res.values())
    rows = {}
    for name, runs in res.items():
        err = np.array([r["err"] for r in runs])
        secs = np.array([r["seconds"] for r in runs])
        li = np.array(runs[0]["loss_iter"])
        loss = np.array([r["loss"] for r in runs])
        row = {"seconds_per_iter": float(np.mean(secs[:, -1]) / secs.shape[1])}
        row["err_at_iter"] = {int(i): float(np.mean(err[:, min(i, err.shape[1]) - 1])) for i in iters}
        row["loss_at_iter"] = {int(i): float(np.mean(loss[:, int(np.argmin(np.abs(li - i)))])) for i in iters}
        at_t = {}
        for f in time_fracs:
            t = f * t_min
            vals = []
            for r, run in enumerate(runs):
                k = int(np.searchsorted(secs[r], t, side="right"))   # iterations finished by t
                vals.append(float(err[r, k - 1]) if k > 0 else float(run["err0"]))
            at_t["%.4f s" % t] = float(np.mean(vals))
        row["err_at_time"] = at_t
        rows[name] = row
    return rows


def gradient_rmse_x_time(scene, theta: np.ndarray, uref, walks: int, repeats: int = 16, net=None,
                         whole_walk: bool = True, nested: bool = True, main: bool = True, ref_walks: int = 65536,
                         device: int = 0, seed: int = 5):
    """RMSE of one gradient estimate (walks per point) against a reference
    (ref_walks per point, plain estimator), times the seconds one estimate
    takes: the figure that compares estimators at equal accuracy.  With a
    control-variate network the timed region includes its inference (the
    gradient at the points and the nested table), not its training."""
    s = dwos.Solver(device)
    s.load_scene(scene)
    s.set_boundary(scene.reference_vertices(), scene.elem, scene.jac)
    s.set_dirichlet_mapped(scene.g_vert, scene.dg_vert)
    s.set_params(theta)
    xq = torch.tensor(scene.query, dtype=torch.float32, device=s.device)
    ur = torch.as_tensor(uref, dtype=torch.float32, device=s.device)
    ref = []
    for r in range(4):
        ref.append(s.grad_l2_cv(xq, ur, ref_walks // 4, walk_id_base=(7 << 44) + r * (1 << 34))["grad"].cpu().numpy())
    g_ref = np.mean(ref, axis=0)
    est, times = [], []
    for r in range(repeats):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cv_grad = net.eval(xq)[1] if (net is not None and main) else None
        cv_elem = s.cv_table(net) if (net is not None and nested) else None
        out = s.grad_l2_cv(xq, ur, walks, walk_id_base=(seed << 44) + r * (1 << 30), cv_grad=cv_grad,
                           whole_walk=whole_walk, cv_elem=cv_elem)
        g = out["grad"].cpu().numpy()
        times.append(time.perf_counter() - t0)
        est.append(g)
    E = np.array(est)
    rmse = float(np.sqrt(np.mean((E - g_ref[None]) ** 2)))
    sec = float(np.median(times))
    return {"rmse": rmse, "seconds": sec, "rmse_x_seconds": rmse * sec,
            "rel_rmse": rmse / float(np.sqrt(np.mean(g_ref ** 2)))}
