"""Naive per-node evaluation of one time step (oracle cross-check).

TEST INFRASTRUCTURE ONLY.  A second, deliberately plain reading of the same
step as ``oracle.cglbm``: pure Python loops over one node at a time, every
neighbour quantity recomputed (memoised) from the pre-step populations, and the
collision written per component exactly as the operator split of
Eq. operator_decomposition states it,

    f^k + Omega^(1),k + (rho^k/rho^m) Omega^CM,   then recolouring Omega^(3),

with Omega^(1),k from Eq. operator_perturbation using Delta u^k = F^k / rho^k
(Eq. delta_u, Eq. continuum_surface_force) and Omega^CM = f^eq - f +
T^{-1}(I - R) T f (Eq. collision_operator) with an explicit matrix inverse.
``oracle.cglbm`` instead uses the summed form f^m* = f^eq(rho^m, u + du) +
T^{-1} k* and a linear solve, so agreement between the two checks that
algebra, the neighbour indexing of the whole-lattice passes and the ghost
planes.

It is also used to evaluate a sample of nodes of a full-size lattice: only the
neighbourhood (up to five lattice hops) of each sampled node is touched.
"""
import math

import numpy as np

from .lattice import (
    C19L, W19L, NORM19L, OPP19, C7L, W7L, OPP7, E92L, OMEGA92L, CS2, CS2_7,
    GRAD_EPS, SIN2_EPS,
)


class PointwiseStep:
    def __init__(self, F, solid, params, reactive=None, theta=None):
        self.F = np.asarray(F)   # any float dtype; every access converts to a Python float (FP64)
        self.solid = np.asarray(solid, dtype=bool)
        self.theta = None if theta is None else np.asarray(theta, dtype=np.float64)   # per solid node, degrees
        self.p = params
        self.nz, self.ny, self.nx = self.solid.shape
        self.reactive = None if reactive is None else np.asarray(reactive, dtype=bool)
        self.column = params.bc_z == 1
        self._pulled = {}
        self._rhoN = {}
        self._grad = {}
        self._normal = {}

    # -- indexing ------------------------------------------------------------
    def site(self, x, y, z):
        """Lattice site for the colour/geometry stencils: periodic x, y; z periodic or clamped."""
        x %= self.nx
        y %= self.ny
        if self.column:
            z = min(max(z, 0), self.nz - 1)
        else:
            z %= self.nz
        return (x, y, z)

    def is_solid(self, s):
        x, y, z = s
        return bool(self.solid[z, y, x])

    def is_wall(self, s):
        if self.is_solid(s):
            return False
        x, y, z = s
        return any(self.is_solid(self.site(x + c[0], y + c[1], z + c[2])) for c in C19L[:18])

    def nn(self, s):
        """Eq. nearest_solid_neighbors."""
        if self.is_solid(s):
            return 0
        x, y, z = s
        return sum(self.is_solid(self.site(x + c[0], y + c[1], z + c[2])) for c in C19L[:6])

    def r(self, s):
        if self.is_solid(s):
            return 0
        if self.reactive is not None:
            x, y, z = s
            return int(self.reactive[z, y, x])
        return 1 if self.nn(s) >= 1 else 0

    # -- streaming -----------------------------------------------------------
    def _feq_list(self, rho, u):
        uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
        out = []
        for i in range(19):
            c = C19L[i]
            cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2]
            out.append(W19L[i] * rho * (1 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2)))
        return out

    def _ghost_out(self, x, y, p):
        """Outlet ghost value of population p at (x, y, nz) from plane nz-1 of the input state."""
        x %= self.nx
        y %= self.ny
        z = self.nz - 1
        if self.solid[z, y, x]:
            if p < 19:
                return W19L[p] * self.p.rho_out
            return 0.0
        fr = [float(self.F[i, z, y, x]) for i in range(19)]
        fp = [float(self.F[19 + i, z, y, x]) for i in range(19)]
        if p >= 38:
            return float(self.F[p, z, y, x])
        fm = [a + b for a, b in zip(fr, fp)]
        rho = sum(fm)
        v = [sum(fm[i] * C19L[i][a] for i in range(19)) / rho for a in range(3)]
        psi = sum(fr) / rho
        i = p % 19
        corr = self._feq_list(self.p.rho_out, v)[i] - self._feq_list(rho, v)[i]
        if p < 19:
            return fr[i] + psi * corr
        return fp[i] + (1 - psi) * corr

    def _ghost_in(self, p):
        u = (0.0, 0.0, self.p.u_in)
        if p < 19:
            return self._feq_list(1.0, u)[p]
        if p < 38:
            return 0.0
        j = p - 38
        return W7L[j] * self.p.c_in * (1 + (C7L[j][2] * self.p.u_in) / CS2_7)

    def pulled(self, s):
        """Post-streaming populations at fluid site s (45 values)."""
        if s in self._pulled:
            return self._pulled[s]
        x, y, z = s
        out = []
        for p in range(45):
            if p < 38:
                c = C19L[p % 19]
                opp = (p - p % 19) + int(OPP19[p % 19])
            else:
                c = C7L[p - 38]
                opp = 38 + int(OPP7[p - 38])
            if p >= 38 and self.p.reaction_mode == 1:
                out.append(float(self.F[p, z, y, x]))
                continue
            sx, sy, sz = x - c[0], y - c[1], z - c[2]
            if self.column and sz < 0:
                out.append(self._ghost_in(p))
                continue
            if self.column and sz >= self.nz:
                out.append(self._ghost_out(sx, sy, p))
                continue
            src = (sx % self.nx, sy % self.ny, sz % self.nz)
            if self.is_solid(src):
                out.append(float(self.F[opp, z, y, x]))
            else:
                out.append(float(self.F[p, src[2], src[1], src[0]]))
        self._pulled[s] = out
        return out

    # -- colour field ----------------------------------------------------------
    def rhoN(self, s):
        if s in self._rhoN:
            return self._rhoN[s]
        x, y, z = s
        if not self.is_solid(s):
            f = self.pulled(s)
            rr, rp = sum(f[0:19]), sum(f[19:38])
            val = (rr - rp) / (rr + rp)
        else:
            num = den = 0.0
            for i in range(19):
                c = C19L[i]
                nb = self.site(x + c[0], y + c[1], z + c[2])
                if not self.is_solid(nb):
                    num += W19L[i] * self.rhoN(nb)
                    den += W19L[i]
            val = num / den if den > 0 else 0.0
        self._rhoN[s] = val
        return val

    def grad(self, s):
        if s in self._grad:
            return self._grad[s]
        x, y, z = s
        g = [0.0, 0.0, 0.0]
        for i in range(19):
            c = C19L[i]
            v = self.rhoN(self.site(x + c[0], y + c[1], z + c[2]))
            for a in range(3):
                g[a] += W19L[i] * c[a] * v / CS2
        self._grad[s] = g
        return g

    def ns(self, s):
        x, y, z = s
        acc = [0.0, 0.0, 0.0]
        for e, om in zip(E92L, OMEGA92L):
            if self.is_solid(self.site(x + e[0], y + e[1], z + e[2])):
                for a in range(3):
                    acc[a] += om * e[a]
        m = math.sqrt(sum(v * v for v in acc))
        if m == 0.0:
            return None
        return [v / m for v in acc]

    def normal(self, s):
        """Wetted interface normal at a fluid site; averaged normal at a solid site."""
        if s in self._normal:
            return self._normal[s]
        x, y, z = s
        if not self.is_solid(s):
            g = self.grad(s)
            m = math.sqrt(sum(v * v for v in g))
            if m < GRAD_EPS:
                n = [0.0, 0.0, 0.0]
            else:
                n = [v / m for v in g]
                if self.is_wall(s):
                    n = self._wet(s, n)
        else:
            acc = [0.0, 0.0, 0.0]
            for i in range(19):
                c = C19L[i]
                nb = self.site(x + c[0], y + c[1], z + c[2])
                if not self.is_solid(nb):
                    nn_ = self.normal(nb)
                    for a in range(3):
                        acc[a] += W19L[i] * nn_[a]
            m = math.sqrt(sum(v * v for v in acc))
            n = [v / m for v in acc] if m >= GRAD_EPS else [0.0, 0.0, 0.0]
        self._normal[s] = n
        return n

    def _wet(self, s, n):
        ns = self.ns(s)
        if ns is None:
            return n
        ct = sum(a * b for a, b in zip(ns, n))
        if 1.0 - ct * ct < SIN2_EPS:
            return n
        st = math.sin(math.acos(max(-1.0, min(1.0, ct))))
        th = math.radians(self.p.theta_deg if self.theta is None else self.wall_theta(s))
        best = None
        for sg in (1.0, -1.0):
            cand = [(math.cos(sg * th) - math.sin(sg * th) * ct / st) * ns[a] + math.sin(sg * th) / st * n[a]
                    for a in range(3)]
            d = sum((cand[a] - n[a]) ** 2 for a in range(3))
            if best is None or d < best[0]:
                best = (d, cand)
        return best[1]

    def wall_theta(self, s):
        """Weighted mean of the per-node contact angle over the solid D3Q19 neighbours of s."""
        x, y, z = s
        num = den = 0.0
        for i in range(18):
            c = C19L[i]
            nb = self.site(x + c[0], y + c[1], z + c[2])
            if self.is_solid(nb):
                num += W19L[i] * float(self.theta[nb[2], nb[1], nb[0]])
                den += W19L[i]
        return num / den

    def curvature(self, s):
        x, y, z = s
        n = self.normal(s)
        D = [[0.0] * 3 for _ in range(3)]   # D[a][b] = d_a n_b
        for i in range(19):
            c = C19L[i]
            nb = self.normal(self.site(x + c[0], y + c[1], z + c[2]))
            for a in range(3):
                for b in range(3):
                    D[a][b] += W19L[i] * c[a] * nb[b] / CS2
        proj = 0.0
        for a in range(3):
            for b in range(3):
                proj += ((1.0 if a == b else 0.0) - n[a] * n[b]) * D[a][b]
        return -proj

    # -- collision -------------------------------------------------------------
    @staticmethod
    def _T(u):
        T = np.zeros((19, 19))
        for i in range(19):
            x, y, z = (C19L[i][0] - u[0], C19L[i][1] - u[1], C19L[i][2] - u[2])
            T[:, i] = [1, x, y, z, x * x + y * y + z * z, x * x - y * y, y * y - z * z, x * y, x * z, y * z,
                       x * x * y, x * y * y, x * x * z, x * z * z, y * y * z, y * z * z,
                       x * x * y * y, x * x * z * z, y * y * z * z]
        return T

    def update(self, s):
        """Post-collision populations (45 values) and the reaction amount delta at fluid site s."""
        p = self.p
        f = self.pulled(s)
        fr, fp, g = f[0:19], f[19:38], f[38:45]
        rho = {"r": sum(fr), "p": sum(fp)}
        rho_m = rho["r"] + rho["p"]
        fm = [a + b for a, b in zip(fr, fp)]
        um = [sum(fm[i] * C19L[i][a] for i in range(19)) / rho_m for a in range(3)]
        conc = sum(g)
        gr = self.grad(s)
        gmag = math.sqrt(sum(v * v for v in gr))
        n = self.normal(s)
        H = self.curvature(s) if gmag >= GRAD_EPS else 0.0
        grad_wet = [gmag * v for v in n]
        # Omega^CM of the colour-blind populations (Eq. collision_operator)
        T = self._T(um)
        Rd = np.ones(19)
        Rd[5:10] = 1.0 / p.tau
        feq_m = self._feq_list(rho_m, um)
        om_cm = np.array(feq_m) - np.array(fm) + np.linalg.inv(T) @ (np.diag(1.0 - Rd) @ (T @ np.array(fm)))
        post = {}
        for k, fk in (("r", fr), ("p", fp)):
            if rho[k] != 0.0:
                Fk = [0.5 * p.sigma * H * grad_wet[a] * rho[k] / rho_m + rho[k] * p.accel[a] for a in range(3)]
                duk = [Fk[a] / rho[k] for a in range(3)]
                om1 = np.array(self._feq_list(rho[k], [um[a] + duk[a] for a in range(3)])) - \
                    np.array(self._feq_list(rho[k], um))
            else:
                om1 = np.zeros(19)
            post[k] = np.array(fk) + om1 + rho[k] / rho_m * om_cm
        fm_post = post["r"] + post["p"]
        # recolouring (Eq. operator_recoloring) on the colour-blind post-collision populations
        rec = np.array([p.beta * rho["r"] * rho["p"] / rho_m * W19L[i] *
                        (sum(C19L[i][a] * n[a] for a in range(3)) / NORM19L[i] if NORM19L[i] > 0 else 0.0)
                        for i in range(19)])
        fr_post = rho["r"] / rho_m * fm_post + rec
        fp_post = fm_post - fr_post
        # reaction
        nn, rr = self.nn(s), self.r(s)
        if p.reaction_mode == 1:
            delta = min(p.xi * nn * rr, 1.0) * rho["r"]
        else:
            psi = rho["r"] / rho_m
            delta = min(p.k_rate * nn * rr * conc * psi, conc, rho["r"])
        delta = max(delta, 0.0)
        fr_post = fr_post - np.array(W19L) * delta
        fp_post = fp_post + np.array(W19L) * delta
        if p.reaction_mode == 1:
            g_post = np.array(g)
        else:
            du = [0.5 * p.sigma * H * grad_wet[a] / rho_m + p.accel[a] for a in range(3)]
            uph = [um[a] + 0.5 * du[a] for a in range(3)]
            tau_g = p.diffusivity / CS2_7 + 0.5
            geq = [W7L[j] * conc * (1 + sum(C7L[j][a] * uph[a] for a in range(3)) / CS2_7) for j in range(7)]
            g_post = np.array([g[j] - (g[j] - geq[j]) / tau_g - W7L[j] * delta for j in range(7)])
        return np.concatenate([fr_post, fp_post, g_post]), delta
