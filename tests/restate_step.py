"""An independent multi-precision restatement of one PonD time step, used only
to pin the C oracle on tiny grids.

It follows the same passages of the paper but reaches each quantity by a
different route than the oracle:

* frame transformation: the matrix form G = M(lambda')^-1 M(lambda) of
  Appendix B, solved in mpmath (tensor-product moments v_x^a v_y^b, a,b < q);
* equilibrium in a foreign frame: the lattice populations whose raw moments
  equal the Maxwell-Boltzmann ones (Sec. II.D, Eq. NonComovingEq), solved by
  the same matrix;
* phi_bar^+ and the face phi with the DUGKS coefficients combined in closed
  form ((2 tau - h) phi~ + 3 h phi^eq)/(2 tau + dt) and
  (2 tau phi_bar + h phi^eq)/(2 tau + h), h = dt/2;
* quasi-equilibrium: the total-order-3 Hermite content of f - f^eq and the
  first-order content of g - g^eq (Eq. eq::quasi_f rewritten by Hermite
  orthogonality).
"""
from __future__ import annotations

import math

import numpy as np


class Restated:
    def __init__(self, mp, cfg: dict, dps: int = 30):
        self.mp = mp
        mp.mp.dps = dps
        self.cfg = cfg
        self.D = cfg["D"]
        self.nx = cfg["nx"]
        self.ny = cfg["ny"] if self.D == 2 else 1
        self.Cv = mp.mpf(1) / (mp.mpf(cfg["gamma"]) - 1)
        self.tau = mp.mpf(cfg["tau"])
        self.dt = mp.mpf(cfg["dt"])
        self.dx = mp.mpf(cfg["dx"])
        self.lat = {q: self._lattice(q) for q in (3, 4)}
        self.noconv_faces = 0  # iterated face frames that did not converge
        self.face_evals = 0    # iterated face frame: faces evaluated,
        self.traces = 0        # interface traces made over them,
        self.max_traces = 0    # and the most at one face

    # Table I, from the node formulas
    def _lattice(self, q):
        mp = self.mp
        if q == 3:
            c = [-mp.sqrt(3), mp.mpf(0), mp.sqrt(3)]
            w = [mp.mpf(1) / 6, mp.mpf(2) / 3, mp.mpf(1) / 6]
        else:
            r1, r2 = mp.sqrt(3 - mp.sqrt(6)), mp.sqrt(3 + mp.sqrt(6))
            c = [-r2, -r1, r1, r2]
            w = [(3 - mp.sqrt(6)) / 12, (3 + mp.sqrt(6)) / 12, (3 + mp.sqrt(6)) / 12, (3 - mp.sqrt(6)) / 12]
        if self.D == 1:
            C = [(x, mp.mpf(0)) for x in c]
            W = list(w)
        else:
            C = [(c[j % q], c[j // q]) for j in range(q * q)]
            W = [w[j % q] * w[j // q] for j in range(q * q)]
        return q, C, W

    def _M(self, q, u, T):
        """Raw-moment matrix rows v_x^a v_y^b (a, b < q), Appendix B."""
        mp = self.mp
        _, C, _ = self.lat[q]
        sT = mp.sqrt(T)
        rows = [(a, b) for a in range(q) for b in range(q if self.D == 2 else 1)]
        M = mp.matrix(len(rows), len(C))
        for r, (a, b) in enumerate(rows):
            for j, (cx, cy) in enumerate(C):
                vx, vy = sT * cx + u[0], sT * cy + u[1]
                M[r, j] = vx**a * (vy**b if self.D == 2 else 1)
        return M, rows

    def transform(self, q, f, u, T, up, Tp):
        mp = self.mp
        Ms, _ = self._M(q, u, T)
        Mt, _ = self._M(q, up, Tp)
        return list(mp.lu_solve(Mt, Ms * mp.matrix(f)))

    def equilibrium(self, q, scale, u, T, up, Tp):
        """Populations in frame (up, Tp) with the Gaussian raw moments of (u, T)."""
        mp = self.mp
        Mt, rows = self._M(q, up, Tp)
        gm = lambda n, m, t: [mp.mpf(1), m, m * m + t, m**3 + 3 * m * t][n]
        rhs = mp.matrix([scale * gm(a, u[0], T) * (gm(b, u[1], T) if self.D == 2 else 1) for a, b in rows])
        return list(mp.lu_solve(Mt, rhs))

    def macro(self, f, g, u, T):
        mp = self.mp
        _, C4, _ = self.lat[4]
        sT = mp.sqrt(T)
        rho = sum(f)
        jx = sum((sT * cx + u[0]) * fi for (cx, cy), fi in zip(C4, f))
        jy = sum((sT * cy + u[1]) * fi for (cx, cy), fi in zip(C4, f))
        e2 = sum(((sT * cx + u[0]) ** 2 + (sT * cy + u[1]) ** 2) * fi for (cx, cy), fi in zip(C4, f)) / 2
        ux, uy = jx / rho, (jy / rho if self.D == 2 else mp.mpf(0))
        TT = (e2 + sum(g) - rho * (ux * ux + uy * uy) / 2) / (self.Cv * rho)
        return rho, [ux, uy], TT

    def _he(self, n, x):
        return [1, x, x * x - 1, x**3 - 3 * x][n]

    def qe_half(self, f, g, T):
        """Scale-free form: f += k W sum_{a+b=3} A_ab He_a He_b/(a! b!), A of f - rho W."""
        mp = self.mp
        pr = mp.mpf(self.cfg["prandtl"])
        if pr == 1:
            return f, g
        t1 = self.tau
        t2 = t1 / pr
        k = self.dt / 2 * (1 / t1 - 1 / t2)
        _, C4, W4 = self.lat[4]
        _, C3, W3 = self.lat[3]
        rho = sum(f)
        fneq = [fi - rho * wi for fi, wi in zip(f, W4)]
        gneq = [gi - (self.Cv - mp.mpf(self.D) / 2) * T * rho * wi for gi, wi in zip(g, W3)]
        orders = [(a, b) for a in range(4) for b in range(4 if self.D == 2 else 1) if a + b == 3]
        A = {ab: sum(x * self._he(ab[0], cx) * self._he(ab[1], cy) for x, (cx, cy) in zip(fneq, C4))
             for ab in orders}
        fo = [fi + k * wi * sum(A[(a, b)] * self._he(a, cx) * self._he(b, cy) / (math.factorial(a) * math.factorial(b))
                                for (a, b) in orders) for fi, wi, (cx, cy) in zip(f, W4, C4)]
        Bx = sum(x * cx for x, (cx, cy) in zip(gneq, C3))
        By = sum(x * cy for x, (cx, cy) in zip(gneq, C3))
        go = [gi + k * wi * (Bx * cx + By * cy) for gi, wi, (cx, cy) in zip(g, W3, C3)]
        return fo, go

    def _ghost(self, j, k):
        bc, nx, ny = self.cfg["bc"], self.nx, self.ny
        if j < 0 or j >= nx:
            side = 0 if j < 0 else 1
            if bc[side] == 2:
                return ("in", side)
            j = (j + nx if j < 0 else j - nx) if bc[side] == 0 else (0 if j < 0 else nx - 1)
        if self.D == 2 and (k < 0 or k >= ny):
            side = 2 if k < 0 else 3
            if bc[side] == 2:
                return ("in", side)
            k = (k + ny if k < 0 else k - ny) if bc[side] == 0 else (0 if k < 0 else ny - 1)
        return ("cell", j, k)

    def step(self, st):
        """st: dict of mp lists: f[(j,k)], g[(j,k)], u[(j,k)] (2-list), T[(j,k)]."""
        mp = self.mp
        D, nx, ny = self.D, self.nx, self.ny
        tau, dt, dx = self.tau, self.dt, self.dx
        h = dt / 2
        _, C4, W4 = self.lat[4]
        _, C3, W3 = self.lat[3]
        gfac = lambda T: (self.Cv - mp.mpf(D) / 2) * T
        cells = [(j, k) for k in range(ny) for j in range(nx)]
        f, g, u, T = dict(st["f"]), dict(st["g"]), dict(st["u"]), dict(st["T"])
        for c in cells:
            f[c], g[c] = self.qe_half(f[c], g[c], T[c])
        # every cell the faces touch, with ghosts resolved
        def cell_state(j, k):
            r = self._ghost(j, k)
            if r[0] == "cell":
                cc = (r[1], r[2])
                return f[cc], g[cc], u[cc], T[cc]
            s = self.cfg["inflow"][r[1]]
            rho, ux, uy, TT = [mp.mpf(x) for x in s]
            if D == 1:  # a 1D state has no u_y: the inflow's u_y slot is unused
                uy = mp.mpf(0)
            return ([rho * w for w in W4], [gfac(TT) * rho * w for w in W3], [ux, uy], TT)

        pplus = {}

        def phiplus(j, k):
            if (j, k) not in pplus:
                fc, gc, uc, Tc = cell_state(j, k)
                rho = sum(fc)
                fp = [((2 * tau - h) * x + 3 * h * rho * w) / (2 * tau + dt) for x, w in zip(fc, W4)]
                gp = [((2 * tau - h) * x + 3 * h * gfac(Tc) * rho * w) / (2 * tau + dt) for x, w in zip(gc, W3)]
                pplus[(j, k)] = (fp, gp, uc, Tc)
            return pplus[(j, k)]

        def limit(sl, sr):
            if sl * sr <= 0:
                return mp.mpf(0)
            if self.cfg["limiter"] == 1:
                return sl if abs(sl) < abs(sr) else sr
            return 2 * sl * sr / (sl + sr)

        def face(dirn, j, k):
            # stencil along the normal: offsets -1, 0, 1, 2 from the left cell
            def at(n, t=0):
                return (j - 1 + n, k + t) if dirn == 0 else (j + t, k - 1 + n)
            L, R = phiplus(*at(1)), phiplus(*at(2))
            uF = [(L[2][0] + R[2][0]) / 2, (L[2][1] + R[2][1]) / 2]
            TF = (L[3] + R[3]) / 2
            # iterated face frame (earlier predictor-corrector scheme): the face
            # frame is replaced by the interface state until they agree
            iterative = int(self.cfg.get("iterative", 0))
            n_iter = max(1, int(self.cfg.get("iter_max", 10))) if iterative else 1
            tol = mp.mpf(self.cfg.get("iter_tol", 1e-12))
            # an iterate with a nonphysical interface state ends the iteration;
            # the face then keeps the previous iterate
            converged = False
            prev = (uF, TF)
            ntrace = 0
            for it in range(n_iter):
                fb, gb = self._trace(dirn, at, phiplus, uF, TF, limit, C4, C3)
                ntrace += 1
                rho, ub, Tb = self.macro(fb, gb, uF, TF)
                if not (rho > 0 and Tb > 0):
                    if iterative and it > 0:
                        uF, TF = prev
                        fb, gb = self._trace(dirn, at, phiplus, uF, TF, limit, C4, C3)
                        ntrace += 1
                        rho, ub, Tb = self.macro(fb, gb, uF, TF)
                    break
                if not iterative:
                    break
                du = mp.sqrt((ub[0] - uF[0]) ** 2 + (ub[1] - uF[1]) ** 2)
                if max(du / mp.sqrt(TF), abs(Tb - TF) / TF) < tol:
                    converged = True
                    break
                if it + 1 < n_iter:
                    prev = (uF, TF)
                    uF = [ub[0], ub[1] if D == 2 else mp.mpf(0)]
                    TF = Tb
            if iterative:
                self.face_evals += 1
                self.traces += ntrace
                self.max_traces = max(self.max_traces, ntrace)
            if iterative and not converged:
                self.noconv_faces += 1
            if converged:
                feq = [rho * w for w in W4]
                geq = [gfac(Tb) * rho * w for w in W3]
            else:
                feq = self.equilibrium(4, rho, ub, Tb, uF, TF)
                geq = self.equilibrium(3, gfac(Tb) * rho, ub, Tb, uF, TF)
            pf = [(2 * tau * a + h * b) / (2 * tau + h) for a, b in zip(fb, feq)]
            pg = [(2 * tau * a + h * b) / (2 * tau + h) for a, b in zip(gb, geq)]
            return pf, pg, uF, TF

        xf = {(j, k): face(0, j, k) for k in range(ny) for j in range(-1, nx)}
        yf = {(j, k): face(1, j, k) for k in range(-1, ny) for j in range(nx)} if D == 2 else {}
        return self._update(cells, f, g, u, T, xf, yf, W4, W3, C4, C3, gfac)

    def _trace(self, dirn, at, phiplus, uF, TF, limit, C4, C3):
        """Stencil moved into the face frame {uF, TF} and the limited half-step
        trace of every population to the face (Eq. eq:InterfacePop)."""
        mp, D, dt, dx = self.mp, self.D, self.dt, self.dx
        cache = {}

        def tr(cell):
            if cell not in cache:
                fp, gp, uc, Tc = phiplus(*cell)
                cache[cell] = (self.transform(4, fp, uc, Tc, uF, TF), self.transform(3, gp, uc, Tc, uF, TF))
            return cache[cell]

        out = []
        for pop, (q, C) in enumerate(((4, C4), (3, C3))):
            vals = []
            for i, (cx, cy) in enumerate(C):
                vx, vy = mp.sqrt(TF) * cx + uF[0], mp.sqrt(TF) * cy + uF[1]
                vn, vt = (vx, vy) if dirn == 0 else (vy, vx)

                def one_sided(up):
                    s = 1 if up else 2
                    ps = tr(at(s))[pop][i]
                    pm = tr(at(s - 1))[pop][i]
                    pp = tr(at(s + 1))[pop][i]
                    sig = limit((ps - pm) / dx, (pp - ps) / dx)
                    val = ps + ((dx / 2 if up else -dx / 2) - vn * dt / 2) * sig
                    if D == 2:
                        # transverse neighbours of the upwind cell
                        cs = at(s)
                        lo = (cs[0], cs[1] - 1) if dirn == 0 else (cs[0] - 1, cs[1])
                        hi = (cs[0], cs[1] + 1) if dirn == 0 else (cs[0] + 1, cs[1])
                        qm, qp = tr(lo)[pop][i], tr(hi)[pop][i]
                        val += (-vt * dt / 2) * limit((ps - qm) / dx, (qp - ps) / dx)
                    return val

                # v_n = 0 exactly: the mean of the traces from both sides
                vals.append(one_sided(vn > 0) if vn != 0 else (one_sided(True) + one_sided(False)) / 2)
            out.append(vals)
        return out[0], out[1]

    def _update(self, cells, f, g, u, T, xf, yf, W4, W3, C4, C3, gfac):
        """Fluxes moved into each cell frame, DUGKS update, re-gauge, QE half."""
        mp, D = self.mp, self.D
        tau, dt, dx = self.tau, self.dt, self.dx
        a1 = (2 * tau - dt) / (2 * tau + dt)
        a2 = 2 * dt / (2 * tau + dt)
        new = {"f": {}, "g": {}, "u": {}, "T": {}}
        for c in cells:
            j, k = c
            uc, Tc = u[c], T[c]
            sT = mp.sqrt(Tc)
            Ff, Fg = [mp.mpf(0)] * 16, [mp.mpf(0)] * 9
            faces = [(xf[(j - 1, k)], 0, -1), (xf[(j, k)], 0, 1)]
            if D == 2:
                faces += [(yf[(j, k - 1)], 1, -1), (yf[(j, k)], 1, 1)]
            for (pf, pg, uF, TF), dirn, sgn in faces:
                for q, C, src, acc in ((4, C4, pf, Ff), (3, C3, pg, Fg)):
                    t = self.transform(q, src, uF, TF, uc, Tc)
                    for i, (cx, cy) in enumerate(C):
                        vn = sT * cx + uc[0] if dirn == 0 else sT * cy + uc[1]
                        acc[i] = acc[i] + sgn * vn * t[i]
            rho = sum(f[c])
            fn = [a1 * x + a2 * rho * w - dt / dx * Ff[i] for i, (x, w) in enumerate(zip(f[c], W4))]
            gn = [a1 * x + a2 * gfac(Tc) * rho * w - dt / dx * Fg[i] for i, (x, w) in enumerate(zip(g[c], W3))]
            rn, un, Tn = self.macro(fn, gn, uc, Tc)
            fn = self.transform(4, fn, uc, Tc, un, Tn)
            gn = self.transform(3, gn, uc, Tc, un, Tn)
            fn, gn = self.qe_half(fn, gn, Tn)
            new["f"][c], new["g"][c], new["u"][c], new["T"][c] = fn, gn, un, Tn
        return new

    # conversion helpers
    def from_arrays(self, f, g, ux, uy, T):
        mp = self.mp
        st = {"f": {}, "g": {}, "u": {}, "T": {}}
        for k in range(self.ny):
            for j in range(self.nx):
                c = (j, k)
                st["f"][c] = [mp.mpf(float(x)) for x in f[:, k, j]]
                st["g"][c] = [mp.mpf(float(x)) for x in g[:, k, j]]
                st["u"][c] = [mp.mpf(float(ux[k, j])), mp.mpf(float(uy[k, j]))]
                st["T"][c] = mp.mpf(float(T[k, j]))
        return st

    def to_arrays(self, st):
        Qf, Qg = (16, 9) if self.D == 2 else (4, 3)
        f = np.zeros((Qf, self.ny, self.nx)); g = np.zeros((Qg, self.ny, self.nx))
        ux = np.zeros((self.ny, self.nx)); uy = np.zeros((self.ny, self.nx)); T = np.zeros((self.ny, self.nx))
        for (j, k), v in st["f"].items():
            f[:, k, j] = [float(x) for x in v]
            g[:, k, j] = [float(x) for x in st["g"][(j, k)]]
            ux[k, j] = float(st["u"][(j, k)][0]); uy[k, j] = float(st["u"][(j, k)][1])
            T[k, j] = float(st["T"][(j, k)])
        return f, g, ux, uy, T
