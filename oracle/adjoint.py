"""FP64 adjoint oracle of the tracking step: gradients by automatic differentiation.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): only tests may use it.

The tracking cost over a horizon of H frames,
    L = sum_f sum_l w_force |c_f^(l) - o_f^(l)|^2   (+ contact-state terms, gradient 0),
is written here a second time, in plain PyTorch FP64 operations on one
environment (vectorised over sphere-link pairs and contacts), following the
same readings as inhand_oracle.c: the frame step f(s_t, u_t, theta) of
Sec. III-A, the pad forces and the cost of Sec. III-C. torch.autograd then
gives dL / d(initial pose tangent, mass, friction); nothing is derived by hand.

The projection of the contact impulse is not differentiable where the normal
impulse reaches zero or the tangential impulse reaches the Coulomb disk. The
adjoint therefore smooths the projection:
  * normal:  max(0, z)      -> derivative of softplus_beta, sigmoid(beta z);
  * disk:    z min(1, L/|z|) -> z smin(|z|, L)/|z| with
             smin(a, b) = (a + b - sqrt((a - b)^2 + (width b)^2)) / 2.
With smooth_forward=False (the default) the values are the exact projection
and only the derivatives are smoothed ("backward-only smoothing"); with
smooth_forward=True the values are smoothed too, which makes the whole
function smooth along contact-stable paths so that its gradient can be
checked against central finite differences. Contact membership (d < margin),
the capsule clamp, the palm's inside/outside and face choice and the bias
regimes are branch decisions: no derivative flows through them, and
branch_signature() reports them so that tests can pick branch-stable cases.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import fk as _fk, OracleScene, unit_inertia

DT = torch.float64


# ------------------------------------------------------------------ smoothing
class _Max0(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z, beta, smooth_forward):
        ctx.save_for_backward(z)
        ctx.beta = beta
        if smooth_forward:
            return torch.nn.functional.softplus(z, beta=beta)
        return torch.clamp(z, min=0.0)

    @staticmethod
    def backward(ctx, g):
        (z,) = ctx.saved_tensors
        return g * torch.sigmoid(ctx.beta * z), None, None


def _smin(a, b, width):
    return 0.5 * (a + b - torch.sqrt((a - b) ** 2 + (width * b) ** 2))


def _disk_smooth(z, L, width):
    nz = torch.sqrt((z * z).sum(-1, keepdim=True) + 1e-300)
    return z * (_smin(nz, L[..., None], width) / nz)


class _Disk(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z, L, width, smooth_forward):
        ctx.save_for_backward(z, L)
        ctx.width = width
        if smooth_forward:
            return _disk_smooth(z, L, width)
        nz = torch.sqrt((z * z).sum(-1, keepdim=True))
        scale = torch.where(nz > L[..., None], L[..., None] / torch.clamp(nz, min=1e-300), torch.ones_like(nz))
        return z * scale

    @staticmethod
    def backward(ctx, g):
        z, L = ctx.saved_tensors
        with torch.enable_grad():
            z2 = z.detach().requires_grad_(True)
            L2 = L.detach().requires_grad_(True)
            out = _disk_smooth(z2, L2, ctx.width)
            gz, gL = torch.autograd.grad(out, (z2, L2), g)
        return gz, gL, None, None


# ------------------------------------------------------------------ quaternions
def qmul(a, b):
    aw, ax, ay, az = a.unbind(-1)
    bw, bx, by, bz = b.unbind(-1)
    return torch.stack([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                        aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw], -1)


def qexp(w):
    """Unit quaternion of the rotation vector w (smooth at w = 0)."""
    th2 = (w * w).sum(-1)
    th = torch.sqrt(th2 + 1e-300)
    small = th2 < 1e-12
    s = torch.where(small, 0.5 - th2 / 48.0, torch.sin(0.5 * th) / th)
    c = torch.where(small, 1.0 - th2 / 8.0, torch.cos(0.5 * th))
    return torch.cat([c[..., None], w * s[..., None]], -1)


def qmat(q):
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def _skew(r):
    z = torch.zeros_like(r[..., 0])
    return torch.stack([torch.stack([z, -r[..., 2], r[..., 1]], -1),
                        torch.stack([r[..., 2], z, -r[..., 0]], -1),
                        torch.stack([-r[..., 1], r[..., 0], z], -1)], -2)


# ------------------------------------------------------------------ the model
class Model:
    """One environment's frame step and cost in FP64 torch (see the module doc)."""

    def __init__(self, scene, sim, shape: int = 0, beta: float = 1e3, width: float = 1e-3,
                 smooth_forward: bool = False, record_regimes: bool = False):
        self.osc = OracleScene(scene)
        self.scene = scene
        self.sim = sim
        rows = np.asarray(scene.shapes[shape], np.float64)
        cen = rows[:, :3].mean(0)
        self.body = torch.tensor(rows[:, :3] - cen, dtype=DT)          # (S, 3)
        self.rad = torch.tensor(rows[:, 3], dtype=DT)                  # (S,)
        self.Jinv = torch.tensor(np.linalg.inv(unit_inertia(self.osc, shape)), dtype=DT)
        self.beta, self.width, self.smooth = beta, width, smooth_forward
        self.record_regimes = record_regimes   # add the projections' active sets to the signature
        self.n_links = scene.n_links
        self.P = scene.n_pads
        self.h = sim.frame_dt / sim.substeps
        self.g = torch.tensor(sim.gravity, dtype=DT)
        self.signature = []

    # commanded link poses (constants) at the substep boundaries of frame f
    def link_poses(self, q_traj, f):
        ns = self.sim.substeps
        out = []
        for k in range(ns + 1):
            qk = q_traj[f].astype(np.float64) + (k / ns) * (q_traj[f + 1].astype(np.float64) - q_traj[f].astype(np.float64))
            out.append(torch.tensor(_fk(self.osc, qk), dtype=DT))
        return out

    def _pad_of(self, l, t):
        sc = self.scene
        for k in range(sc.n_pads):
            if int(sc.pad_link[k]) != l:
                continue
            if l == 0:
                return k
            if t >= sc.pad_s0[k] and (t < sc.pad_s1[k] or sc.pad_s1[k] >= 1.0):
                return k
        return -1

    def _contacts(self, x, R, lp0):
        """Narrowphase over every (sphere, link) pair: gaps, normals, lever arms, pads."""
        sc, cfg = self.scene, self.sim
        c_rel = self.body @ R.T                       # (S, 3)
        c = x[None] + c_rel
        d_all, n_all, t_all, info = [], [], [], []
        for l in range(self.n_links):
            a = lp0[l, :3]
            Rl = qmat(lp0[l, 3:])
            if l == 0:
                half = torch.tensor(sc.palm_half, dtype=DT)
                cl = (c - a) @ Rl                      # box coordinates
                k = torch.maximum(torch.minimum(cl, half), -half)
                inside = (cl.detach().abs() <= half).all(-1)
                diff = cl - k
                dist = torch.sqrt((diff * diff).sum(-1) + 1e-300)
                n_out = (diff / dist[:, None]) @ Rl.T
                d_out = dist - self.rad
                # faces in the order +x, -x, +y, -y, +z, -z (ties: lowest axis, + side first)
                depth = torch.stack([half[0] - cl[:, 0], half[0] + cl[:, 0], half[1] - cl[:, 1],
                                     half[1] + cl[:, 1], half[2] - cl[:, 2], half[2] + cl[:, 2]], -1)
                face = torch.argmin(depth.detach(), -1)
                dsel = depth.gather(1, face[:, None])[:, 0]
                normals = torch.tensor([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=DT)
                n_in = normals[face] @ Rl.T
                d_in = -dsel - self.rad
                d = torch.where(inside, d_in, d_out)
                n = torch.where(inside[:, None], n_in, n_out)
                t = torch.zeros_like(d)
                ins, fc = inside.tolist(), face.tolist()
                clamp_pat = ((cl.detach() > half) | (cl.detach() < -half)).tolist()
                for j in range(len(ins)):
                    info.append((j, l, ins[j], fc[j] if ins[j] else tuple(clamp_pat[j])))
            else:
                u = Rl[:, 0]
                L = sc.link_len
                ca = c - a
                t_raw = (ca @ u) / L
                t = torch.clamp(t_raw, 0.0, 1.0)
                diff = ca - t[:, None] * L * u[None]
                dist = torch.sqrt((diff * diff).sum(-1) + 1e-300)
                n = diff / dist[:, None]
                d = dist - self.rad - sc.link_rad
                tr_all = t_raw.detach().tolist()
                for j, tr in enumerate(tr_all):
                    info.append((j, l, tr < 0.0 or tr > 1.0, -1))
            d_all.append(d)
            n_all.append(n)
            t_all.append(t)
        d = torch.stack(d_all, 1).reshape(-1)          # pair index = j * n_links + l
        n = torch.stack(n_all, 1).reshape(-1, 3)
        t = torch.stack(t_all, 1).reshape(-1)
        S = self.body.shape[0]
        order = [j * self.n_links + l for j in range(S) for l in range(self.n_links)]
        info = {(jj, ll): (a, b) for (jj, ll, a, b) in info}
        d_val, t_val = d.detach(), t.detach()
        sel = [p for p in order if float(d_val[p]) < cfg.margin]
        idx = torch.tensor(sel, dtype=torch.long)
        r = (c_rel[:, None, :].expand(S, self.n_links, 3).reshape(-1, 3) - self.rad.repeat_interleave(self.n_links)[:, None] * n)
        links = [p % self.n_links for p in sel]
        pads = [self._pad_of(p % self.n_links, float(t_val[p])) for p in sel]
        sig = tuple((p, info[(p // self.n_links, p % self.n_links)]) for p in sel)
        return d[idx], n[idx], r[idx], links, pads, sig

    def _bias(self, d):
        cfg, h = self.sim, self.h
        spec = d / h
        rec = torch.clamp(cfg.beta * torch.clamp(d + cfg.slop, max=0.0) / h, min=-cfg.vmax)
        return torch.where(d > 0, spec, rec)

    def substep(self, x, q, v, w, m, mu, lp0, lp1, forces):
        cfg, h = self.sim, self.h
        v_pred = v + h * self.g
        w_pred = w
        R = qmat(q)
        W = R @ self.Jinv @ R.T / m
        d, n, r, links, pads, sig = self._contacts(x, R, lp0)
        nc = d.shape[0]
        regimes = tuple(int((dd > 0)) * 2 + int(dd + cfg.slop < 0) + 4 * int(
            cfg.beta * (dd + cfg.slop) / h < -cfg.vmax) for dd in d.detach().tolist())
        self.signature.append((sig, regimes))
        if nc > cfg.c_max:
            nc = 0
        if nc == 0:
            vv, ww = v_pred, w_pred
            lam = torch.zeros((0, 3), dtype=DT)
        else:
            S = _skew(r)
            K = torch.eye(3, dtype=DT)[None] / m - S @ W[None] @ S
            kn = torch.einsum("ki,kij,kj->k", n, K, n)
            kt = 0.5 * (K.diagonal(dim1=1, dim2=2).sum(-1) - kn)
            ikn, ikt = 1.0 / kn, 1.0 / kt
            b = self._bias(d)
            vl = []
            for k in range(nc):
                l = links[k]
                if l == 0:
                    vl.append(torch.zeros(3, dtype=DT))
                else:
                    A, B = lp0[l], lp1[l]
                    RA, RB = qmat(A[3:]), qmat(B[3:])
                    p = x + r[k]
                    pl = RA.T @ (p - A[:3])
                    vl.append(((B[:3] + RB @ pl) - p) / h)
            vl = torch.stack(vl)
            cc = vl - b[:, None] * n
            lam = torch.zeros((nc, 3), dtype=DT)
            for it in range(self.iters):
                vv = v_pred + lam.sum(0) / m
                ww = w_pred + W @ torch.cross(r, lam, dim=-1).sum(0)
                u = vv[None] + torch.cross(ww[None].expand_as(r), r, dim=-1) - cc
                un = (u * n).sum(-1)
                l_old = (lam * n).sum(-1)
                zn = l_old - un * ikn
                ln = _Max0.apply(zn, self.beta, self.smooth)
                zt = (lam - n * l_old[:, None]) - (u - n * un[:, None]) * ikt[:, None]
                if self.record_regimes:   # which side of each projection every contact is on
                    nz = torch.sqrt((zt.detach() ** 2).sum(-1))
                    self.signature.append(tuple((zn.detach() > 0).tolist()) +
                                          tuple((nz > (mu * ln).detach()).tolist()))
                lt = _Disk.apply(zt, mu * ln, self.width, self.smooth)
                lp = n * ln[:, None] + lt
                lam = lam + (lp - lam) / nc
            vv = v_pred + lam.sum(0) / m
            ww = w_pred + W @ torch.cross(r, lam, dim=-1).sum(0)
        x = x + h * vv
        q = qmul(qexp(h * ww), q)
        q = q / torch.sqrt((q * q).sum())
        for k in range(lam.shape[0]):
            if pads[k] >= 0:
                forces = forces.index_add(0, torch.tensor([pads[k]]), (-lam[k] / h)[None])
        return x, q, vv, ww, forces

    def frame(self, state, m, mu, q_traj, f, iters=None):
        x, q, v, w = state
        self.iters = self.sim.iters if iters is None else iters
        lps = self.link_poses(q_traj, f)
        forces = torch.zeros((self.P, 3), dtype=DT)
        for s in range(self.sim.substeps):
            x, q, v, w, forces = self.substep(x, q, v, w, m, mu, lps[s], lps[s + 1], forces)
        return (x, q, v, w), forces / self.sim.substeps

    def frame_cost(self, forces, obs):
        cfg = self.sim
        o = torch.as_tensor(obs, dtype=DT)
        cost = cfg.w_force * ((forces - o) ** 2).sum()
        on_f = (forces.detach() ** 2).sum(-1) > cfg.tau ** 2
        on_o = (o ** 2).sum(-1) > cfg.tau ** 2
        return cost + cfg.w_contact * (on_f != on_o).sum()


def horizon(scene, sim, pose7, vel6, theta, q_traj, frame0, H, obs, shape=0, iters=None,
            beta=1e3, width=1e-3, smooth_forward=False, delta=None, record_regimes=False):
    """Cost over frames [frame0, frame0 + H) and its gradient w.r.t. the
    initial state's position (3), rotation tangent (3, world frame, applied on
    the left), mass and friction. Returns (cost, grad[8] in the order x y z,
    rx ry rz, m, mu, final state (x, q, v, w), per-frame forces, branch
    signature). With `delta` given, no gradient is taken and the initial
    state is offset by it (for finite differences)."""
    model = Model(scene, sim, shape, beta, width, smooth_forward, record_regimes)
    dlt = torch.zeros(8, dtype=DT, requires_grad=True) if delta is None else torch.as_tensor(delta, dtype=DT)
    p = torch.as_tensor(pose7, dtype=DT)
    x = p[:3] + dlt[:3]
    q = qmul(qexp(dlt[3:6]), p[3:7])
    vv = torch.as_tensor(vel6, dtype=DT)
    v, w = vv[:3], vv[3:]
    m = torch.as_tensor(theta[0], dtype=DT) + dlt[6]
    mu = torch.as_tensor(theta[1], dtype=DT) + dlt[7]
    state = (x, q, v, w)
    total = torch.zeros((), dtype=DT)
    forces_all = []
    for k in range(H):
        state, forces = model.frame(state, m, mu, q_traj, frame0 + k, iters)
        forces_all.append(forces.detach().numpy().copy())
        total = total + model.frame_cost(forces, obs[k])
    grad = None
    if delta is None:
        if total.requires_grad:
            (grad,) = torch.autograd.grad(total, dlt, allow_unused=True)
        grad = np.zeros(8) if grad is None else grad.numpy()
    fin = np.concatenate([t.detach().numpy() for t in state])
    return float(total.detach()), grad, fin, np.array(forces_all), model.signature


# ------------------------------------------------------------------ refinement of the elites
def _qexp_np(w):
    """Unit quaternion (w x y z) of a rotation vector, numpy FP64."""
    th = float(np.linalg.norm(w))
    if th == 0.0:
        return np.array([1.0, 0.0, 0.0, 0.0])
    return np.concatenate([[math.cos(0.5 * th)], math.sin(0.5 * th) * np.asarray(w) / th])


def _qmul_np(a, b):
    return np.array([a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3],
                     a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
                     a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1],
                     a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0]])


def refine_step(pose7, theta, grad, eta, scale, m_range, mu_range):
    """One step of the refinement from the state (pose7, theta) with gradient
    `grad` (x y z, left rotation vector, m, mu): in coordinates scaled by eta
    the step is the steepest descent of length `scale`,
        s = eta * g,   dz = -scale * eta * s / |s|,
    applied as x += dz[0:3], R <- exp([dz[3:6]]x) R (world frame, on the
    left), m += dz[6], mu += dz[7], with m and mu clamped to the optimizer's
    ranges. A zero or non-finite |s| leaves the state where it is."""
    eta = np.asarray(eta, np.float64)
    s = eta * np.asarray(grad, np.float64)
    nrm = float(np.sqrt(np.sum(s * s)))
    dz = np.zeros(8)
    if nrm > 0.0 and math.isfinite(nrm):
        dz = -scale * eta * s / nrm
    p = np.asarray(pose7, np.float64).copy()
    p[:3] += dz[:3]
    q = _qmul_np(_qexp_np(dz[3:6]), p[3:7])
    p[3:7] = q / np.linalg.norm(q)
    th = np.asarray(theta, np.float64).copy()
    th[0] = min(max(th[0] + dz[6], m_range[0]), m_range[1])
    th[1] = min(max(th[1] + dz[7], mu_range[0]), mu_range[1])
    return p, th


def refine_rule(evaluate, pose7, theta, eta, steps, m_range, mu_range):
    """The refinement's accept/halve rule on one elite (an addition to the
    derivative-free update of Sec. III-D, run on the elites before it).

    evaluate(pose7, theta) -> (cost, grad[8], end) scores a window-start
    state over the window. Evaluation 0 is the elite's own state and is always
    kept; evaluation j >= 1 is the step from the best state so far with the
    current scale (starting at 1); it is kept when its cost is strictly lower
    than the best cost, otherwise the scale halves. After `steps` steps the
    best state, its cost, gradient and end state are returned together with the
    per-evaluation decisions."""
    scale = 1.0
    trial_p, trial_t = np.asarray(pose7, np.float64).copy(), np.asarray(theta, np.float64).copy()
    accepted, costs, scales, trials = [], [], [], []
    best = None
    for it in range(steps + 1):
        c, g, end = evaluate(trial_p, trial_t)
        costs.append(c)
        trials.append((trial_p, trial_t))
        keep = it == 0 or c < best["cost"]
        accepted.append(bool(keep))
        if keep:
            best = {"cost": c, "grad": np.asarray(g, np.float64), "pose7": trial_p, "theta": trial_t, "end": end}
        else:
            scale *= 0.5
        scales.append(scale)
        if it == steps:
            break
        trial_p, trial_t = refine_step(best["pose7"], best["theta"], best["grad"], eta, scale, m_range, mu_range)
    return {"c0": costs[0], "best_c": best["cost"], "accepted": accepted, "costs": costs, "scales": scales,
            "trials": trials, "pose7": best["pose7"], "theta": best["theta"], "end": best["end"], "grad": best["grad"],
            "improved": best["cost"] < costs[0]}


def refine_elite(scene, sim, opt, pose7, vel6, theta, q_traj, frame0, T, obs, steps=3, step_scale=0.5,
                 beta=1e3, width=1e-3, shape=0, iters=None):
    """Gradient refinement of one elite's window-start state over the window of
    T frames [frame0, frame0 + T): the window cost and its gradient come from
    horizon() (the same backward-only smoothing), the velocity stays the
    window-start velocity, eta = step_scale * floor_std per coordinate. When
    the best cost is lower than the unrefined one, the elite's state at the
    window's end becomes the simulation's state, with the best parameters and
    the best cost as its window sum (returned as "end", "theta", "best_c")."""
    eta = step_scale * np.asarray(opt.floor_std, np.float64)

    def evaluate(p, th):
        c, g, fin, _, _ = horizon(scene, sim, p, vel6, th, q_traj, frame0, T, obs, shape=shape, iters=iters,
                                  beta=beta, width=width)
        return c, g, fin

    return refine_rule(evaluate, pose7, theta, eta, steps, opt.m_range, opt.mu_range)
