"""FP64 reverse-mode reference for the gradient of the column conversion.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The objective is the outlet conversion of the column after T steps,

    J = 1 - Phi_out / Phi_in,   Phi = sum over a z plane of fluid nodes of u_z C

(u_z = j_z / rho of the stored populations, C = sum_j g_j), the quantity whose
sensitivity to the wettability motivates the paper's coating discussion
(Sec. 5.2).  Its parameters are the per-solid-node contact angle theta (degrees;
each wall node uses the weighted mean of ``cglbm.wall_contact_angle``) and the
inlet velocity u_in; the start state is held fixed.

``TorchStep`` restates ``cglbm.step`` pass by pass with PyTorch float64 CPU
tensors, so that autograd yields the exact derivative of the same discrete map.
Threshold and branch decisions (|grad rho^N| >= 1e-5, the n_+/n_- choice, the
reaction clamps) are taken from the forward values and are therefore frozen, as
in any discrete adjoint.  Square roots whose argument can be exactly zero in a
bulk region are guarded so that their derivative is not evaluated there.

Pins (tests): the forward agrees with ``cglbm.step`` to rounding, and the
autograd gradient agrees with FP64 central differences of ``cglbm`` itself.
"""
import math

import numpy as np
import torch

from . import cglbm as O
from .lattice import C19L, W19L, NORM19L, C7L, W7L, CS2, CS2_7, GRAD_EPS, SIN2_EPS, Q19

DT = torch.float64


def _safe_sqrt(x):
    pos = x > 0.0
    return torch.where(pos, torch.sqrt(torch.where(pos, x, torch.ones_like(x))), torch.zeros_like(x))


def _feq(rho, ux, uy, uz):
    uu = ux * ux + uy * uy + uz * uz
    out = []
    for i in range(Q19):
        cx, cy, cz = C19L[i]
        cu = cx * ux + cy * uy + cz * uz
        out.append(W19L[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)))
    return torch.stack(out)


def _geq(conc, ux, uy, uz):
    out = []
    for j in range(len(C7L)):
        cx, cy, cz = C7L[j]
        out.append(W7L[j] * conc * (1.0 + (cx * ux + cy * uy + cz * uz) / CS2_7))
    return torch.stack(out)


class TorchStep:
    """cglbm.step in PyTorch float64, differentiable in (f, theta, u_in)."""

    def __init__(self, geom, params):
        assert params.reaction_mode in (0, 1)
        self.g = geom
        self.p = params
        self.shape = geom.shape
        self.zm = O._zmode(geom.bc_z)
        self.column = params.bc_z == 1
        self.fluid = torch.from_numpy(geom.fluid)
        self.solid = torch.from_numpy(geom.solid)
        self.fl_f = self.fluid.to(DT)
        self.ns = torch.from_numpy(np.ascontiguousarray(geom.ns)).to(DT)
        self.ns_ok = torch.from_numpy(geom.ns_ok)
        self.wall = torch.from_numpy(geom.wall)
        self.solid_bnd = torch.from_numpy(geom.solid_bnd)
        self.nn = torch.from_numpy(geom.nn).to(DT)
        self.rmask = torch.from_numpy(geom.reactive).to(DT)

    # --- neighbour access (same index maps as cglbm.neighbor) ----------------
    def nb(self, a, d, zmode=None):
        zmode = self.zm if zmode is None else zmode
        shape = tuple(a.shape[-3:])
        idx = torch.from_numpy(O._neighbor_index(shape, tuple(int(v) for v in d), zmode))
        lead = tuple(a.shape[:-3])
        return a.reshape(lead + (-1,))[..., idx].reshape(a.shape)

    # --- wettability ---------------------------------------------------------
    def wall_theta(self, theta):
        s = self.solid.to(DT)
        num = torch.zeros(self.shape, dtype=DT)
        den = torch.zeros(self.shape, dtype=DT)
        for i in range(Q19 - 1):
            sn = self.nb(s, C19L[i])
            num = num + W19L[i] * sn * self.nb(theta, C19L[i])
            den = den + W19L[i] * sn
        return torch.where(den > 0.0, num / torch.where(den > 0.0, den, torch.ones_like(den)), torch.zeros_like(den))

    # --- a1 ------------------------------------------------------------------
    def _inlet_ghost(self, u_in):
        ny, nx = self.shape[1:]
        one = torch.ones((ny, nx), dtype=DT)
        zero = torch.zeros((ny, nx), dtype=DT)
        uz = u_in * one
        return torch.cat([_feq(one, zero, zero, uz), torch.zeros((Q19, ny, nx), dtype=DT),
                          _geq(self.p.c_in * one, zero, zero, uz)], dim=0)

    def _outlet_ghost(self, last, solid_last):
        fr, fp, g = last[0:19], last[19:38], last[38:45]
        fm = fr + fp
        rho = fm.sum(dim=0)
        rho_safe = torch.where(solid_last, torch.ones_like(rho), rho)
        v = [sum(C19L[i][a] * fm[i] for i in range(Q19) if C19L[i][a]) / rho_safe for a in range(3)]
        psi = fr.sum(dim=0) / rho_safe
        rout = torch.full_like(rho, self.p.rho_out)
        corr = _feq(rout, *v) - _feq(rho_safe, *v)
        ghost = torch.cat([fr + psi * corr, fp + (1.0 - psi) * corr, g], dim=0)
        z = torch.zeros_like(rho)
        rest = torch.cat([_feq(rout, z, z, z), torch.zeros_like(fp), torch.zeros_like(g)], dim=0)
        return torch.where(solid_last[None], rest, ghost)

    def stream(self, F, u_in):
        nz = self.shape[0]
        if self.column:
            gin = self._inlet_ghost(u_in)
            gout = self._outlet_ghost(F[:, nz - 1], self.solid[nz - 1])
        out = []
        for p in range(O.NPOP):
            c, op = O._velocity_set(p)
            c = tuple(int(v) for v in c)
            if p >= 38 and self.p.reaction_mode == 1:
                out.append(F[p])
                continue
            mc = (-c[0], -c[1], -c[2])
            pulled = self.nb(F[p], mc, "periodic")
            src_solid = self.nb(self.solid, mc, "periodic").clone()
            if self.column and c[2] == 1:
                row = self.nb(gin[p][None], (mc[0], mc[1], 0), "periodic")[0]
                pulled = torch.cat([row[None], pulled[1:]], dim=0)
                src_solid[0] = False
            if self.column and c[2] == -1:
                row = self.nb(gout[p][None], (mc[0], mc[1], 0), "periodic")[0]
                pulled = torch.cat([pulled[:-1], row[None]], dim=0)
                src_solid[nz - 1] = False
            out.append(torch.where(src_solid, F[op], pulled))
        return torch.stack(out) * self.fl_f

    # --- a3 - a6 -------------------------------------------------------------
    def color_at_solids(self, rhoN):
        l = self.fl_f
        num = torch.zeros_like(rhoN)
        den = torch.zeros_like(rhoN)
        for i in range(Q19):
            ln = self.nb(l, C19L[i])
            num = num + W19L[i] * self.nb(rhoN, C19L[i]) * ln
            den = den + W19L[i] * ln
        sb = self.solid_bnd
        return torch.where(sb, num / torch.where(sb, den, torch.ones_like(den)), rhoN)

    def gradient(self, phi):
        comps = [torch.zeros_like(phi) for _ in range(3)]
        for i in range(Q19):
            if not any(C19L[i]):
                continue
            v = self.nb(phi, C19L[i])
            for a in range(3):
                if C19L[i][a]:
                    comps[a] = comps[a] + (W19L[i] / CS2 * C19L[i][a]) * v
        return torch.stack(comps)

    def wetting(self, n, theta_wall):
        th = theta_wall * (math.pi / 180.0)
        cos_th, sin_th = torch.cos(th), torch.sin(th)
        ns = self.ns
        cos_tp = (ns * n).sum(dim=0)
        nz_n = (n * n).sum(dim=0) > 0.0
        ok = self.ns_ok & nz_n & (1.0 - cos_tp * cos_tp >= SIN2_EPS)
        cos_tp_s = torch.where(ok, cos_tp, torch.zeros_like(cos_tp))
        sin_tp = torch.sqrt(torch.where(ok, 1.0 - cos_tp_s * cos_tp_s, torch.ones_like(cos_tp)))
        cands = []
        for sgn in (1.0, -1.0):
            a_s = cos_th - sgn * sin_th * cos_tp_s / sin_tp
            a_n = sgn * sin_th / sin_tp
            cands.append(a_s * ns + a_n * n)
        d_plus = ((cands[0] - n) ** 2).sum(dim=0)
        d_minus = ((cands[1] - n) ** 2).sum(dim=0)
        chosen = torch.where((d_plus <= d_minus)[None], cands[0], cands[1])
        return torch.where(ok[None], chosen, n)

    def normals_at_solids(self, n):
        l = self.fl_f
        acc = [torch.zeros_like(n[0]) for _ in range(3)]
        for i in range(Q19):
            ln = self.nb(l, C19L[i])
            for a in range(3):
                acc[a] = acc[a] + W19L[i] * ln * self.nb(n[a], C19L[i])
        acc = torch.stack(acc)
        mag = _safe_sqrt((acc * acc).sum(dim=0))
        ok = self.solid_bnd & (mag >= GRAD_EPS)
        out = torch.where(self.fluid[None], n, torch.zeros_like(n))
        return torch.where(ok[None], acc / torch.where(mag > 0, mag, torch.ones_like(mag)), out)

    def curvature(self, n):
        D = torch.stack([self.gradient(n[b]) for b in range(3)], dim=1)   # D[a, b] = d_a n_b
        tr = D[0, 0] + D[1, 1] + D[2, 2]
        nDn = torch.einsum("a...,ab...,b...->...", n, D, n)
        return -(tr - nDn)

    # --- a8 ------------------------------------------------------------------
    def backtransform(self, fm, u):
        """T^{-1} (I - R) T f^m node by node (fm (19, N), u (3, N)), by a linear solve."""
        cb = torch.tensor(C19L, dtype=DT).T[None] - u.T[:, :, None]     # (N, 3, 19)
        x, y, z = cb[:, 0], cb[:, 1], cb[:, 2]
        one = torch.ones_like(x)
        T = torch.stack([one, x, y, z, x * x + y * y + z * z, x * x - y * y, y * y - z * z,
                         x * y, x * z, y * z, x * x * y, x * y * y, x * x * z, x * z * z,
                         y * y * z, y * z * z, x * x * y * y, x * x * z * z, y * y * z * z], dim=1)
        om = torch.zeros(Q19, dtype=DT)
        om[5:10] = 1.0 - 1.0 / self.p.tau
        k = torch.einsum("nmi,in->nm", T, fm) * om[None]
        return torch.linalg.solve(T, k[:, :, None])[:, :, 0].T

    # --- the step ------------------------------------------------------------
    def step(self, f, theta_wall, u_in):
        p = self.p
        fl = self.fluid
        F = self.stream(f, u_in)
        fr, fp, g = F[0:19], F[19:38], F[38:45]
        rho_r = fr.sum(dim=0)
        rho_p = fp.sum(dim=0)
        fm = fr + fp
        rho_m = rho_r + rho_p
        rms = torch.where(fl, rho_m, torch.ones_like(rho_m))
        u = torch.stack([sum(C19L[i][a] * fm[i] for i in range(Q19) if C19L[i][a]) for a in range(3)]) / rms
        u = torch.where(fl[None], u, torch.zeros_like(u))
        conc = g.sum(dim=0)
        rhoN = torch.where(fl, (rho_r - rho_p) / rms, torch.zeros_like(rms))
        rhoN = self.color_at_solids(rhoN)
        grad = self.gradient(rhoN)
        gmag = _safe_sqrt((grad * grad).sum(dim=0))
        has_n = fl & (gmag >= GRAD_EPS)
        n = torch.where(has_n[None], grad / torch.where(has_n, gmag, torch.ones_like(gmag)), torch.zeros_like(grad))
        n = self.wetting(n, theta_wall)
        n = torch.where(fl[None], n, torch.zeros_like(n))
        n_all = self.normals_at_solids(n)
        H = torch.where(has_n, self.curvature(n_all), torch.zeros_like(gmag))
        acc = torch.tensor(p.accel, dtype=DT).reshape(3, 1, 1, 1)
        du = 0.5 * p.sigma * H * gmag * n / rms + acc
        du = torch.where(fl[None], du, torch.zeros_like(du))
        idx = torch.from_numpy(np.nonzero(self.g.fluid.ravel())[0])
        bt_f = self.backtransform(fm.reshape(Q19, -1)[:, idx], u.reshape(3, -1)[:, idx])
        bt = torch.zeros((Q19, self.fluid.numel()), dtype=DT).index_copy(1, idx, bt_f).reshape((Q19,) + self.shape)
        v = u + du
        fm_star = _feq(rms, v[0], v[1], v[2]) + bt
        psi = rho_r / rms
        rec_amp = p.beta * rho_r * rho_p / rms
        fr_star = []
        for i in range(Q19):
            cx, cy, cz = C19L[i]
            cn = (cx * n[0] + cy * n[1] + cz * n[2]) / NORM19L[i] if NORM19L[i] > 0 else torch.zeros_like(psi)
            fr_star.append(psi * fm_star[i] + rec_amp * W19L[i] * cn)
        fr_star = torch.stack(fr_star)
        fp_star = fm_star - fr_star
        if p.reaction_mode == 1:
            delta = torch.clamp(p.xi * self.nn * self.rmask, max=1.0) * rho_r
        else:
            delta = torch.minimum(torch.minimum(p.k_rate * self.nn * self.rmask * conc * psi, conc), rho_r)
        delta = torch.where(fl, torch.clamp(delta, min=0.0), torch.zeros_like(delta))
        w19 = torch.tensor(W19L, dtype=DT).reshape(-1, 1, 1, 1)
        fr_star = fr_star - w19 * delta
        fp_star = fp_star + w19 * delta
        if p.reaction_mode == 1:
            g_star = g
        else:
            tau_g = p.diffusivity / CS2_7 + 0.5
            up = u + 0.5 * du
            g_star = g - (g - _geq(conc, up[0], up[1], up[2])) / tau_g - torch.tensor(W7L, dtype=DT).reshape(
                -1, 1, 1, 1) * delta
        return torch.cat([fr_star, fp_star, g_star], dim=0) * self.fl_f

    def conversion(self, f):
        """Column objective J = 1 - Phi_out / Phi_in of the stored populations."""
        fr, fp, g = f[0:19], f[19:38], f[38:45]
        rm = fr.sum(dim=0) + fp.sum(dim=0)
        rms = torch.where(self.fluid, rm, torch.ones_like(rm))
        jz = sum(C19L[i][2] * (fr[i] + fp[i]) for i in range(Q19) if C19L[i][2])
        phi = jz / rms * g.sum(dim=0) * self.fl_f
        return 1.0 - phi[-1].sum() / phi[0].sum()


def conversion_gradient(geom, params, f0, theta_deg, nsteps):
    """J after nsteps from f0, dJ/dtheta (per node, degrees^-1) and dJ/du_in, all FP64."""
    ts = TorchStep(geom, params)
    theta = torch.tensor(np.asarray(theta_deg, dtype=np.float64), requires_grad=True)
    u_in = torch.tensor(float(params.u_in), dtype=DT, requires_grad=True)
    f = torch.from_numpy(np.asarray(f0, dtype=np.float64).copy())
    tw = ts.wall_theta(theta)
    for _ in range(nsteps):
        f = ts.step(f, tw, u_in)
    J = ts.conversion(f)
    J.backward()
    return float(J.detach()), theta.grad.numpy().copy(), float(u_in.grad)


def conversion_forward(geom, params, f0, theta_deg, nsteps):
    """The same objective from the NumPy oracle (the function the gradient differentiates)."""
    g = O.Geometry(solid=geom.solid, bc_z=geom.bc_z, reactive_mask=geom.reactive_mask,
                   theta_deg=np.asarray(theta_deg, dtype=np.float64))
    st = O.State(f=np.asarray(f0, dtype=np.float64).copy())
    for _ in range(nsteps):
        st = O.step(st, g, params)
    return O.observables(st, g, params)["conversion"]
