"""A second, independent implementation of the method's step in vectorised NumPy,
written from the paper's equations (where the paper leaves a step open, the same
reading as the oracle: the source of Eq. 36 with c_j on the mobility part, the
closed-form charge of Eq. 50 with the previous field, half-way walls)
(test infrastructure: it checks the C oracle's transcription on tiny lattices).

Whole-lattice array operations replace the oracle's per-cell loops: neighbours
come from index arrays (x periodic; y periodic, or mirrored about the half-way
walls for stencils), streaming shifts whole planes and reflects what crosses a wall.
Only the fixed-iteration potential solve is implemented (the residual-controlled
stop is a host decision, covered elsewhere).  Optionally the two Nernst-Planck ion
species of Eq. 52 (the paper prints no lattice scheme for them; read as, per species, a D2Q9 set with
equilibrium w_j n (1 + c_j . v / cs2), v = u + z beta D E, the backward-difference
source of d/dt(n v), bounce-back walls; the charge they carry replaces the closure).
"""
from __future__ import annotations

import numpy as np

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])       # Eq. 31
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])
CS2 = 1.0 / 3.0


class Twin:
    def __init__(self, p: dict, phi, u=None, q=None, noise=None, ions=None):
        self.p = dict(p)
        self.ny, self.nx = int(p["ny"]), int(p["nx"])
        ny, nx = self.ny, self.nx
        g12, g13, g23 = p["gamma12"], p["gamma13"], p["gamma23"]
        self.lam = np.array([g12 + g13 - g23, g12 + g23 - g13, g13 + g23 - g12])   # Eq. 9
        self.m0 = CS2 * (p["tau_f"] - 0.5)
        self.tau_h = 0.5 + p["eps_ref"] / CS2
        self.tau_l = 0.5 + p["alpha"] / CS2
        self.phi = np.array(phi, dtype=float).copy()
        self.u = np.zeros((2, ny, nx)) if u is None else np.array(u, dtype=float).copy()
        self.q = np.zeros((ny, nx)) if q is None else np.array(q, dtype=float).copy()
        self.step_count = 0
        self._properties()
        # potential populations at equilibrium with the linear electrode profile (or 0)
        yy = (np.arange(ny) + 0.5)[:, None] * np.ones((1, nx))
        psi0 = p["V_bottom"] + (p["V_top"] - p["V_bottom"]) * yy / ny if p["bc_y"] == 2 else np.zeros((ny, nx))
        self.h = self._heq(psi0)
        self._solve_potential()
        self._chemical_potential()
        ux, uy = self.u
        f = np.empty((3, 9, ny, nx))
        for i in range(3):
            f[i] = self._feq(self.phi[i], self.mu[i], ux, uy)
        self.f = f
        self.g = self.rho[None] * self._s(ux, uy)                 # g_eq with p = 0
        self.l = self._leq(self.q, ux, uy)
        if noise is not None:
            nz = np.asarray(noise, dtype=float)
            self.g = self.g + nz[0]
            self.f = self.f + nz[1:4]
            self.l = self.l + nz[4]
        self.prev_phiu = np.zeros((3, 2, ny, nx))
        self.prev_qu = np.zeros((2, ny, nx))
        self.ion = None
        if ions is not None:
            # start the species: their charge, a potential solve, each set at equilibrium
            n = np.asarray(ions, dtype=float)
            self.q = p["ion_charge"] * (p["ion_z"][0] * n[0] + p["ion_z"][1] * n[1])
            self._solve_potential()
            self.ion = np.array([self._neq(k, n[k]) for k in range(2)])
            self.prev_nv = np.zeros((2, 2, ny, nx))

    def _drift(self, k):                        # v_k = u + z_k beta D_k E
        p = self.p
        m = p["ion_z"][k] * p["ion_beta"] * p["ion_D"][k]
        return self.u[0] + m * self.E[0], self.u[1] + m * self.E[1]

    def _neq(self, k, n):
        vx, vy = self._drift(k)
        return np.array([W[j] * n * (1 + (CX[j] * vx + CY[j] * vy) / CS2) for j in range(9)])

    # ---------------------------------------------------------------- lattice helpers
    def _rows(self, dy):
        y = np.arange(self.ny) + dy
        if self.p["bc_y"] == 0:
            return y % self.ny
        return np.where(y < 0, -1 - y, np.where(y >= self.ny, 2 * self.ny - 1 - y, y))

    def _nb(self, a, dx, dy):
        """a at (x + dx, y + dy): x periodic; y periodic or mirror ghosts."""
        return np.roll(a[self._rows(dy)], -dx, axis=1)

    def _grad(self, a):                                              # Eq. 33
        gx = sum(W[j] * CX[j] * self._nb(a, CX[j], CY[j]) for j in range(9)) / CS2
        gy = sum(W[j] * CY[j] * self._nb(a, CX[j], CY[j]) for j in range(9)) / CS2
        return gx, gy

    def _lap(self, a):                                               # Eq. 33
        return sum(2 * W[j] * (self._nb(a, CX[j], CY[j]) - a) for j in range(9)) / CS2

    def _stream(self, post, kind):
        """Push streaming of 9 planes; what leaves through a wall comes back to the
        same cell in the opposite direction: plain (kind 'bb'), with the moving-wall
        term (kind 'flow'), or anti-bounce-back to the electrode potential ('pot')."""
        ny = self.ny
        out = np.empty_like(post)
        walls = self.p["bc_y"] != 0
        for j in range(9):
            v = np.roll(post[j], CX[j], axis=1)
            if not walls or CY[j] == 0:
                out[j] = np.roll(v, CY[j], axis=0)
            elif CY[j] > 0:
                out[j][1:] = v[:-1]
            else:
                out[j][:-1] = v[1:]
        if walls:
            for j in range(9):
                if CY[j] == 0:
                    continue
                row = ny - 1 if CY[j] > 0 else 0       # cells whose link j crosses the wall
                top = CY[j] > 0
                v = post[j][row]
                if kind == "flow":
                    uw = self.p["u_wall_top"] if top else self.p["u_wall_bottom"]
                    v = v - 2.0 * W[j] * self.rho[row] * (CX[j] * uw) / CS2
                elif kind == "pot" and self.p["bc_y"] == 2:
                    vw = self.p["V_top"] if top else self.p["V_bottom"]
                    v = -v + 2.0 * W[j] * vw
                out[OPP[j]][row] = v
        return out

    # ---------------------------------------------------------------- closures
    def _properties(self):
        p = self.p
        ph = self.phi
        self.rho = sum(ph[i] * p["rho"][i] for i in range(3))                      # Eq. 29
        self.sig = sum(ph[i] * p["sigma"][i] for i in range(3))
        self.eps = sum(p["eps"][i] * ph[i] ** 2 * (3 - 2 * ph[i]) for i in range(3))   # Eq. 30
        self.lap = np.array([self._lap(ph[i]) for i in range(3)])
        self.geps = np.array(self._grad(self.eps))
        self.gsig = np.array(self._grad(self.sig))
        self.grho = np.array(self._grad(self.rho))

    def observables(self) -> dict:
        """The reductions over the last step's fields: phase masses, total charge, the
        parts of the free energy of Eq. 18 summed over cells (phase: bulk
        6 lambda_i phi_i^2 (1 - phi_i)^2 / D plus gradient 3 D lambda_i |grad phi_i|^2 / 8
        with the Eq. 33 gradient; electric eps |E|^2 / 2; kinetic rho |u|^2 / 2; charge
        alpha q^2 / (2 sigma) where sigma > 0), max |sum phi - 1|, and the deformation
        factors (a - b)/(a + b) of the indicators phi_inner and 1 - phi_matrix, with a
        and b twice the standard deviations of the indicator along y and x."""
        p, ph = self.p, self.phi
        D = p["width_D"]
        ny, nx = self.ny, self.nx
        out = {f"mass{i + 1}": float(ph[i].sum()) for i in range(3)}
        out["charge"] = float(self.q.sum())
        fphi = 0.0
        for i in range(3):
            gx, gy = self._grad(ph[i])
            fphi += float((6.0 * self.lam[i] / D * ph[i] ** 2 * (1 - ph[i]) ** 2
                           + 3.0 * D * self.lam[i] / 8.0 * (gx ** 2 + gy ** 2)).sum())
        out["F_phi"] = fphi
        eps = sum(p["eps"][i] * ph[i] ** 2 * (3 - 2 * ph[i]) for i in range(3))
        out["F_E"] = float((0.5 * eps * (self.E[0] ** 2 + self.E[1] ** 2)).sum())
        rho = sum(ph[i] * p["rho"][i] for i in range(3))
        out["F_u"] = float((0.5 * rho * (self.u[0] ** 2 + self.u[1] ** 2)).sum())
        sig = sum(ph[i] * p["sigma"][i] for i in range(3))
        safe = np.where(sig > 0, sig, 1.0)
        out["F_q"] = float(np.where(sig > 0, 0.5 * p["alpha"] / safe * self.q ** 2, 0.0).sum())
        out["max_sum_dev"] = float(np.abs(ph.sum(axis=0) - 1.0).max())
        y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
        for key, chi in (("D_inner", ph[p["inner_phase"] - 1]), ("D_outer", 1.0 - ph[p["matrix_phase"] - 1])):
            A = chi.sum()
            if not A > 0:
                out[key] = 0.0
                continue
            xm, ym = (chi * x).sum() / A, (chi * y).sum() / A
            a = 2.0 * np.sqrt(max(((chi * (y - ym) ** 2).sum() / A), 0.0))
            b = 2.0 * np.sqrt(max(((chi * (x - xm) ** 2).sum() / A), 0.0))
            out[key] = float((a - b) / (a + b)) if a + b > 0 else 0.0
        return out

    def _heq(self, psi):
        h = np.empty((9,) + psi.shape)
        h[0] = (W[0] - 1.0) * psi                                                   # Eq. 44
        for j in range(1, 9):
            h[j] = W[j] * psi
        return h

    def _solve_potential(self):
        p = self.p
        if not p["electric"]:
            self.E = np.array([np.full((self.ny, self.nx), p["E_ext"][0]), np.full((self.ny, self.nx), p["E_ext"][1])])
            self.psi = np.zeros((self.ny, self.nx))
            return
        th = self.tau_h
        ehat = self.eps - p["eps_ref"]
        den = ehat + CS2 * th
        varpi = np.array([0.0] + [1 / 8] * 8)
        for _ in range(p["poisson_fixed_iter"]):                                    # Eq. 43
            psi = self.h[1:].sum(0) / (1 - W[0])
            jx = np.tensordot(CX, self.h, 1)
            jy = np.tensordot(CY, self.h, 1)
            gx, gy = -jx / den, -jy / den
            heq = self._heq(psi)
            post = np.empty_like(self.h)
            for j in range(9):
                post[j] = (self.h[j] - (self.h[j] - heq[j]) / th
                           - (ehat / CS2) * W[j] * (CX[j] * gx + CY[j] * gy) / th + varpi[j] * self.q)
            self.h = self._stream(post, "pot")
        self.psi = self.h[1:].sum(0) / (1 - W[0])                                    # Eq. 45
        jx = np.tensordot(CX, self.h, 1)
        jy = np.tensordot(CY, self.h, 1)
        self.E = np.array([jx / den + p["E_ext"][0], jy / den + p["E_ext"][1]])

    def _chemical_potential(self):                                                  # Eq. 20
        D = self.p["width_D"]
        e2 = self.E[0] ** 2 + self.E[1] ** 2
        self.mu = np.array([24 / D * self.lam[i] * self.phi[i] * (self.phi[i] - 0.5) * (self.phi[i] - 1)
                            - 0.75 * D * self.lam[i] * self.lap[i]
                            - 0.5 * 6 * self.p["eps"][i] * self.phi[i] * (1 - self.phi[i]) * e2 for i in range(3)])

    def _s(self, ux, uy):                                                           # Eq. 40
        out = np.empty((9,) + ux.shape)
        uu = ux * ux + uy * uy
        for j in range(9):
            cu = CX[j] * ux + CY[j] * uy
            out[j] = W[j] * (cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2))
        return out

    def _feq(self, ph, mu, ux, uy):                                                 # Eq. 35
        out = np.empty((9,) + ph.shape)
        out[0] = ph - (1 - W[0]) * mu
        for j in range(1, 9):
            out[j] = W[j] * mu + W[j] * (CX[j] * ph * ux + CY[j] * ph * uy) / CS2
        return out

    def _leq(self, q, ux, uy):                                                      # Eq. 50
        out = np.empty((9,) + q.shape)
        for j in range(9):
            cu = CX[j] * ux + CY[j] * uy
            out[j] = W[j] * q * (1 + cu / CS2) if self.p["charge_convection"] else W[j] * q
        return out

    # ---------------------------------------------------------------- one time step
    def step(self, n: int = 1):
        for _ in range(n):
            self._one_step()
        return self

    def _one_step(self):
        p = self.p
        first = self.step_count == 0
        self.phi = self.f.sum(1)                                                    # S1
        qt = self.l.sum(0)
        self._properties()                                                          # S2, S3
        r = self.sig / self.eps
        Ex, Ey = self.E                                                             # E of the last step
        src = r * (self.geps[0] * Ex + self.geps[1] * Ey) - (self.gsig[0] * Ex + self.gsig[1] * Ey)
        if self.ion is None:
            self.q = (qt + 0.5 * src) / (1 + 0.5 * r)                               # S4 (reading R9)
        else:                                                                       # the ions' charge
            nion = self.ion.sum(1)
            self.q = p["ion_charge"] * (p["ion_z"][0] * nion[0] + p["ion_z"][1] * nion[1])
        self._solve_potential()                                                     # S5
        Ex, Ey = self.E
        R = -r * self.q + r * (self.geps[0] * Ex + self.geps[1] * Ey) - (self.gsig[0] * Ex + self.gsig[1] * Ey)
        self._chemical_potential()                                                  # S6
        gmu = np.array([self._grad(self.mu[i]) for i in range(3)])                 # S7
        Fx = -sum(self.phi[i] * gmu[i][0] for i in range(3)) + self.q * Ex         # S8
        Fy = -sum(self.phi[i] * gmu[i][1] for i in range(3)) + self.q * Ey
        g = self.g                                                                  # S9, Eq. 41
        ux = (np.tensordot(CX, g, 1) + 0.5 * Fx) / self.rho
        uy = (np.tensordot(CY, g, 1) + 0.5 * Fy) / self.rho
        ugr = ux * self.grho[0] + uy * self.grho[1]
        s = self._s(ux, uy)
        pr = CS2 / (1 - W[0]) * (g[1:].sum(0) + 0.5 * ugr + self.rho * s[0])
        self.u = np.array([ux, uy])
        self.pr = pr
        # S10: backward differences, zero on the first step (reading R10)
        phiu = np.array([[self.phi[i] * ux, self.phi[i] * uy] for i in range(3)])
        qu = np.array([self.q * ux, self.q * uy])
        dpu = np.zeros_like(phiu) if first else phiu - self.prev_phiu
        dqu = np.zeros_like(qu) if first else qu - self.prev_qu
        # S11: phase populations, mobility of Eq. 28, source read as R3
        tf, m0 = p["tau_f"], self.m0
        fpost = np.empty_like(self.f)
        for i in range(3):
            Y = np.zeros((2,) + ux.shape)
            for k in range(3):
                if k == i:
                    Mik = m0 * self.phi[i] * sum(self.phi[kk] for kk in range(3) if kk != i) - m0
                else:
                    Mik = -m0 * self.phi[i] * self.phi[k]
                Y = Y + Mik * gmu[k]
            A = dpu[i] / CS2 - Y / m0
            feq = self._feq(self.phi[i], self.mu[i], ux, uy)
            for j in range(9):
                Fj = W[j] * (CX[j] * A[0] + CY[j] * A[1])
                fpost[i, j] = self.f[i, j] - (self.f[i, j] - feq[j]) / tf + (1 - 1 / (2 * tf)) * Fj
        # S12: flow populations, Eq. 37-40 (local tau_g from the dynamic viscosity)
        if all(v > 0 for v in p["visc"]):
            eta = sum(self.phi[i] * p["visc"][i] for i in range(3))
            tg = 0.5 + eta / (self.rho * CS2)
        else:
            tg = p["tau_g"]
        gpost = np.empty_like(g)
        for j in range(9):
            geq = ((W[0] - 1) if j == 0 else W[j]) * pr / CS2 + self.rho * s[j]
            cu = CX[j] * ux + CY[j] * uy
            cgr = CX[j] * self.grho[0] + CY[j] * self.grho[1]
            cF = CX[j] * Fx + CY[j] * Fy
            G = W[j] * (ugr + cF / CS2 + (cu * cgr - CS2 * ugr) / CS2)
            gpost[j] = g[j] - (g[j] - geq) / tg + (1 - 1 / (2 * tg)) * G
        # S13: charge populations, Eq. 48-50
        tl = self.tau_l
        leq = self._leq(self.q, ux, uy)
        lpost = np.empty_like(self.l)
        for j in range(9):
            Sj = (1 - 1 / (2 * tl)) * W[j] * R
            Tj = ((1 - 1 / (2 * tl)) * W[j] * (CX[j] * dqu[0] + CY[j] * dqu[1]) / CS2
                  if p["charge_convection"] else 0.0)
            lpost[j] = self.l[j] - (self.l[j] - leq[j]) / tl + Sj + Tj
        # S14: streaming with the walls
        self.f = np.array([self._stream(fpost[i], "bb") for i in range(3)])
        self.g = self._stream(gpost, "flow")
        self.l = self._stream(lpost, "bb")
        if self.ion is not None:                                                    # Eq. 52 (ions)
            new = np.empty_like(self.ion)
            for k in range(2):
                tk = 0.5 + p["ion_D"][k] / CS2
                vx, vy = self._drift(k)
                nk = nion[k]
                nv = np.array([nk * vx, nk * vy])
                dnv = np.zeros_like(nv) if first else nv - self.prev_nv[k]
                neq = self._neq(k, nk)
                post = np.empty_like(self.ion[k])
                for j in range(9):
                    Tj = (1 - 1 / (2 * tk)) * W[j] * (CX[j] * dnv[0] + CY[j] * dnv[1]) / CS2
                    post[j] = self.ion[k, j] - (self.ion[k, j] - neq[j]) / tk + Tj
                new[k] = self._stream(post, "bb")
                self.prev_nv[k] = nv
            self.ion = new
        self.prev_phiu = phiu
        self.prev_qu = qu
        self.step_count += 1
