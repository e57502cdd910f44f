"""One time step of the filtered SELBM, written step by step in the paper's order
(Sec. 2, summary list at the end of Sec. 2.4):

1. moments rho = sum f_bar, rho u = sum e f_bar                 (Eqs. pressure, momentum)
2. BGK collision with the higher-order force F**                  (collision equation, Sec. 2.1)
3. streaming d f_bar/dt = L(f_bar) by SSPRK3 with F* and the
   flux bounce-back boundary flux                                 (Eqs. full, entire; Sec. 2.2.2)
4. explicit modal filter on every f_alpha                         (Sec. 2.4)
5. moments for output

The state lives on unique (assembled) GLL nodes: f[Q, G].  The
continuous-Galerkin coupling is the assembly (direct stiffness summation) of
the element contributions, divided by the assembled lumped mass.

Readings of the paper taken here, where it is silent or garbled:
* L f = M^{-1}(R (n.j) - C f) + F*: the identity term printed in the
  operator definition is dropped (it would create mass).
* "3rd order SSP RK" is the Shu-Osher three-stage scheme.
* The geometric factor G_lk = rho rho rho J dr_l/dx_k (chain rule).
* No flux at interior element faces; assembly only (continuous Galerkin).
* The filter is applied once per step after the last stage, element by
  element; the copies of a shared node are reconciled by their
  mass-weighted average (they agree when every element has the same filter).
* F = rho g with rho from the step's moments, frozen through the stages;
  a per-node acceleration field (the pipe's perturbation force) enters the
  same way, with its time factor taken at the start of the step.
"""
import numpy as np

from . import geometry as geo
from . import gll
from .lattice import CS2, equilibrium, force_split, lattice


class OracleSELBM:
    """Plain FP64 filtered SELBM on unique GLL nodes."""

    def __init__(self, mesh, lattice_name, N, nu, cfl=0.5, dt=None, rho0=1.0,
                 filt=None, body_accel=None):
        self.mesh, self.N, self.dim = mesh, N, mesh.dim
        self.e, self.t, self.opp = lattice(lattice_name)
        self.Q = len(self.t)
        self.rho0 = rho0
        self.xi = gll.gll_nodes(N)
        self.w = gll.gll_weights(N, self.xi)
        self.D = gll.derivative_matrix(self.xi)
        node_form = hasattr(mesh, "xyz")               # GLL node coordinates + face connectivity
        self.X = geo.element_nodes_from_map(mesh, self.xi) if node_form else geo.element_nodes(mesh, self.xi)
        self.E, self.Np = self.X.shape[0], self.X.shape[1]
        self.dxdr, self.J, self.drdx, self.wJ = geo.metrics(self.X, self.D, N, self.dim, self.w)
        if np.any(self.J <= 0):
            raise ValueError("non-positive Jacobian")
        self.glo = geo.global_numbering_connectivity(mesh, N) if node_form else geo.global_numbering(self.X, mesh)
        self.G = int(self.glo.max()) + 1
        self.mass = np.zeros(self.G)
        np.add.at(self.mass, self.glo.ravel(), self.wJ.ravel())
        self.copies = np.bincount(self.glo.ravel(), minlength=self.G)
        _, first = np.unique(self.glo.ravel(), return_index=True)
        self.Xg = self.X.reshape(-1, self.dim)[first]          # coordinates of each unique node
        self.walls = geo.wall_faces(mesh, self.drdx, self.J, self.w, N)
        self.dt = dt if dt is not None else cfl * geo.min_node_spacing(self.X, N, self.dim)
        self.lam = nu / CS2                                      # nu = lambda cs^2 (Sec. 2.1)
        self.tau = self.lam / self.dt                            # tau = lambda / dt
        self.nu = nu
        f = filt or {"shape": 0, "gamma": 0.0, "kc": float(N), "p": 8.0}
        self.set_filter(f)
        g = np.zeros(self.dim) if body_accel is None else np.asarray(body_accel, float)[: self.dim]
        self.g = g
        self.fS = None                                           # extra per-node acceleration field
        self.time = 0.0
        self.scheme = 0                                # 0 Shu-Osher SSPRK3, 1 printed stages, 2 weighted

    def set_time_scheme(self, scheme):
        """0: the Shu-Osher SSPRK3 that the text names; 1: the four stages as printed in
        Sec. 2.2.2, with L applied to each stage combination as a whole; 2: the printed stages
        with L's source terms (F*, moving walls) weighted by the combination's weight sum, i.e.
        kept for the state arguments f0 and f0 - f1 + f2 and dropped for the differences
        f0 - f1 and f0 - f1 + f2 - f3."""
        self.scheme = int(scheme)

    def set_force_field(self, S, period, t_end):
        """Extra body acceleration A(t) S_g on unique nodes (Sec. 4, pipe: the perturbation
        force switched on for the first t_end of the run).  S [G, d]; A(t) = sin(2 pi t / period)
        for t < t_end and 0 after; period <= 0 keeps A = 1 while t < t_end.  The time is the
        time at the start of the step, and the force is frozen through the step."""
        self.fS = np.asarray(S, float)[:, : self.dim]
        self.f_period, self.f_tend = float(period), float(t_end)

    def amplitude(self, t):
        if self.fS is None or not t < self.f_tend:
            return 0.0
        return 1.0 if self.f_period <= 0 else float(np.sin(2.0 * np.pi * t / self.f_period))

    def accel(self):
        """Body acceleration at every unique node at the current time: g + A(t) S_g."""
        if self.fS is None:
            return self.g[None, :]
        return self.g[None, :] + self.amplitude(self.time) * self.fS

    # ------------------------------------------------------------------ setup
    def set_filter(self, f):
        self.filt = dict(f)
        sig = gll.filter_sigma(self.N, int(f["shape"]), float(f["gamma"]), float(f["kc"]), float(f.get("p", 8.0)))
        self.sigma = sig
        self.Fmat = gll.filter_matrix(self.N, self.xi, sig)
        self.filter_on = float(f["gamma"]) != 0.0 and float(f["kc"]) < self.N

    # --------------------------------------------------------------- helpers
    def to_local(self, fg):
        """Unique-node field [..., G] -> element-local copies [..., E, Np]."""
        return fg[..., self.glo]

    def moments(self, f):
        """rho = sum_alpha f_bar_alpha, u = (sum_alpha e_alpha f_bar_alpha) / rho (Eqs. pressure, momentum)."""
        rho = f.sum(axis=0)
        j = self.e.T.astype(float) @ f                    # [d, n]
        return rho, (j / rho).T                           # rho [n], u [n, d]

    def initial_state(self, rho, u):
        """f_bar at rest in equilibrium: f = f^eq, so f_bar = f^eq - dt/2 F** (Sec. 2.1)."""
        F = rho[:, None] * self.accel()
        _, Fss = force_split(self.e, self.t, u, F)
        return equilibrium(self.e, self.t, rho, u) - 0.5 * self.dt * Fss

    def initial_state_from(self, init):
        rho, u = init(self.Xg)
        return self.initial_state(rho, u[:, : self.dim])

    # -------------------------------------------------------------- collision
    def collide(self, f):
        """f* = f_bar - (f_bar - f_bar^eq)/(tau + 1/2) + dt F**, f_bar^eq = f^eq - dt/2 F** (Sec. 2.1).

        Returns (f*, F*) with F* the leading-order force for the streaming step."""
        rho, u = self.moments(f)
        F = rho[:, None] * self.accel()
        Fstar, Fss = force_split(self.e, self.t, u, F)
        feq_bar = equilibrium(self.e, self.t, rho, u) - 0.5 * self.dt * Fss
        fstar = f - (f - feq_bar) / (self.tau + 0.5) + self.dt * Fss
        return fstar, Fstar

    # ------------------------------------------------------------- streaming
    def element_contribution(self, f, wall_source=True):
        """Weighted element contribution c[Q, E, Np] of -C f + R (n.j) (Eqs. advection2, entire).

        Interior:  c = -wJ sum_l (sum_k e_k dr_l/dx_k) (D_l f)        (C = phi^T e G D* phi)
        Wall face: c += w_s J_s (n.e_alpha) [f_alpha - f_beta - 2 t_alpha rho0 (e_alpha.u_b)/cs2]
                   for n.e_alpha < 0 (flux bounce-back, Sec. 2.2.1).
        """
        fl = self.to_local(f)                                       # [Q, E, Np]
        grads = [geo.apply_axis(self.D, fl, l, self.N, self.dim) for l in range(self.dim)]
        c = np.zeros_like(fl)
        ef = self.e.astype(float)
        for a in range(self.Q):
            adv = np.zeros((self.E, self.Np))
            for l in range(self.dim):
                coef = (self.drdx[:, :, l, :] * ef[a][None, None, :]).sum(-1)   # sum_k e_k dr_l/dx_k
                adv += coef * grads[l][a]
            c[a] = -self.wJ * adv
        for (el, nodes, n, wsJs, wid) in self.walls:
            ub = self.mesh.wall_velocity[wid - 1][: self.dim]
            ne = n @ ef.T                                           # [nf, Q]
            for a in range(self.Q):
                b = self.opp[a]
                inc = ne[:, a] < 0.0
                jump = fl[a, el, nodes] - fl[b, el, nodes]
                if wall_source:
                    jump = jump - 2.0 * self.t[a] * self.rho0 * (ef[a] @ ub) / CS2
                c[a, el, nodes] += np.where(inc, wsJs * ne[:, a] * jump, 0.0)
        return c

    def rhs(self, f, Fstar, wall_source=True):
        """L(f) = M^{-1} assemble(c) + F* on unique nodes (continuous Galerkin)."""
        c = self.element_contribution(f, wall_source)
        R = np.zeros((self.Q, self.G))
        for a in range(self.Q):
            np.add.at(R[a], self.glo.ravel(), c[a].ravel())       # ascending copy order
        return R / self.mass[None, :] + Fstar

    def ssprk3(self, f0, Fstar):
        """Shu-Osher SSPRK3 (Sec. 2.2.2)."""
        dt = self.dt
        f1 = f0 + dt * self.rhs(f0, Fstar)
        f2 = 0.75 * f0 + 0.25 * (f1 + dt * self.rhs(f1, Fstar))
        return f0 / 3.0 + 2.0 / 3.0 * (f2 + dt * self.rhs(f2, Fstar))

    def rk_printed(self, f0, Fstar, weighted=False):
        """The four stages as printed (Sec. 2.2.2):
        f1 = f0 + dt/3 L f0,  f2 = f1 - 3dt/4 L(f0 - f1),  f3 = f2 + 2dt/3 L(f0 - f1 + f2),
        f = f3 - dt/4 L(f0 - f1 + f2 - f3).
        weighted: the arguments f0 - f1 and f0 - f1 + f2 - f3 (weights summing to zero) take
        L without its source terms (F*, wall velocity)."""
        dt = self.dt

        def Ld(g):
            return self.rhs(g, 0.0 * Fstar, wall_source=False) if weighted else self.rhs(g, Fstar)
        f1 = f0 + dt / 3.0 * self.rhs(f0, Fstar)
        f2 = f1 - 0.75 * dt * Ld(f0 - f1)
        f3 = f2 + 2.0 / 3.0 * dt * self.rhs(f0 - f1 + f2, Fstar)
        return f3 - 0.25 * dt * Ld(f0 - f1 + f2 - f3)

    def stream(self, f0, Fstar):
        if self.scheme == 0:
            return self.ssprk3(f0, Fstar)
        return self.rk_printed(f0, Fstar, weighted=self.scheme == 2)

    # ----------------------------------------------------------------- filter
    def assemble_average(self, fl):
        """Element copies [Q, E, Np] -> unique nodes: mass-weighted average sum_c wJ_c f_c / M.
        With the same filter in every element the copies agree and this returns their value;
        with element-dependent filters it keeps the total mass, since each element's filter
        keeps its own integral."""
        out = np.zeros((self.Q, self.G))
        for a in range(self.Q):
            np.add.at(out[a], self.glo.ravel(), (self.wJ * fl[a]).ravel())
        return out / self.mass[None, :]

    def apply_filter(self, f):
        """(F x F (x F)) f_alpha element by element (Sec. 2.4), then the copies of shared
        nodes are reconciled by their mass-weighted average."""
        if not self.filter_on:
            return f
        fl = self.to_local(f)
        for l in range(self.dim):
            fl = geo.apply_axis(self.Fmat, fl, l, self.N, self.dim)
        return self.assemble_average(fl)

    def apply_filter_elements(self, f, sigma_e):
        """Filter with a per-element transfer function sigma_e [E, N+1] (learned control);
        shared nodes take the mass-weighted average of their copies."""
        V = gll.modal_basis(self.N, self.xi)
        Vi = np.linalg.inv(V)
        fl = self.to_local(f).copy()
        rows, inv = np.unique(np.round(sigma_e, 15), axis=0, return_inverse=True)
        for r in range(len(rows)):
            es = np.nonzero(inv.ravel() == r)[0]
            F = V @ np.diag(sigma_e[es[0]]) @ Vi
            sub = fl[:, es]
            for l in range(self.dim):
                sub = geo.apply_axis(F, sub, l, self.N, self.dim)
            fl[:, es] = sub
        return self.assemble_average(fl)

    def learned_sigma(self, f, params, lo, hi):
        """Per-element transfer functions from the learned control (features of f, BF16
        weights, FP64 arithmetic); elements whose features leave [lo, hi] keep the fixed filter."""
        from . import learned as L
        rho, u = self.moments(f)
        x = L.features(rho[self.glo], u[self.glo], self.rho0, self.N, self.dim)
        gam, kc, inr = L.infer_filter(params, x, lo, hi, self.N)
        sig = np.array([gll.filter_sigma(self.N, 0, g, k) if ok else self.sigma
                        for g, k, ok in zip(gam, kc, inr)])
        return sig, x, inr

    def step_learned(self, f, params, lo, hi):
        """One step whose end-of-step filter is chosen per element by the learned control."""
        f0, Fstar = self.collide(f)
        f3 = self.stream(f0, Fstar)
        sig, _, _ = self.learned_sigma(f3, params, lo, hi)
        self.time += self.dt
        return self.apply_filter_elements(f3, sig)

    # ------------------------------------------------------------------- step
    def step(self, f):
        f0, Fstar = self.collide(f)
        f3 = self.stream(f0, Fstar)
        self.time += self.dt
        return self.apply_filter(f3)

    def run(self, f, nsteps):
        for _ in range(nsteps):
            f = self.step(f)
        return f

    # ------------------------------------------------------------ diagnostics
    def dissipation(self, f):
        """Viscous dissipation integral (Sec. 3.4, with the divergence term squared):
        eps = sum wJ [2 mu sum_i (d_i u_i)^2 - 2/3 mu (div u)^2 + mu sum_{i<j} (d_i u_j + d_j u_i)^2],
        mu = rho0 nu; gradients of the nodal velocity by D along each reference axis and the chain rule."""
        _, u = self.moments(f)
        ul = u[self.glo]                                             # [E, Np, d]
        d = self.dim
        dr = np.stack([np.stack([geo.apply_axis(self.D, ul[..., c], l, self.N, d) for c in range(d)], -1)
                       for l in range(d)], 2)                        # [E, Np, l, c] = du_c/dr_l
        g = np.einsum("eplk,eplc->epkc", self.drdx, dr)              # du_c/dx_k
        mu = self.rho0 * self.nu
        div = np.einsum("epkk->ep", g)
        diag = np.einsum("epkk,epkk->ep", g, g)
        off = np.zeros_like(div)
        for a in range(d):
            for b in range(a + 1, d):
                off += (g[:, :, a, b] + g[:, :, b, a]) ** 2
        dens = 2 * mu * diag - 2.0 / 3.0 * mu * div ** 2 + mu * off
        return float((self.wJ * dens).sum())

    def wall_stress(self, f, direction):
        """Wall shear stress along `direction` (Sec. 4, pipe flow: tau_w from the boundary nodes,
        tau_w = mu (sin theta du_z/dy + cos theta du_z/dx) on the pipe wall): the average over every
        wall face, weighted by w_s J_s, of -mu n . grad(u . d) at the face's GLL nodes, n the
        outward unit normal, mu = rho0 nu, gradients by D along each reference axis and the chain
        rule (as in `dissipation`)."""
        _, u = self.moments(f)
        d = np.asarray(direction, float)[: self.dim]
        d = d / np.linalg.norm(d)
        ud = (u @ d)[self.glo]                                                        # [E, Np]
        dr = np.stack([geo.apply_axis(self.D, ud, l, self.N, self.dim) for l in range(self.dim)], -1)
        grad = np.einsum("eplk,epl->epk", self.drdx, dr)                             # d(u.d)/dx_k
        mu = self.rho0 * self.nu
        num = den = 0.0
        for (el, nodes, n, wsJs, wid) in self.walls:
            dn = (n * grad[el, nodes]).sum(1)
            num += float((wsJs * (-mu * dn)).sum())
            den += float(wsJs.sum())
        return num / den if den > 0 else 0.0

    def radial_profile(self, f, origin, axis, radius, nbins):
        """Mean of u . axis over unique nodes binned by their distance r from the line through
        `origin` along `axis` (Sec. 4: space-averaged axial velocity): bin = min(floor(r nbins /
        radius), nbins - 1), weights = lumped mass M_g.  Returns (mean per bin, mass per bin)."""
        _, u = self.moments(f)
        a = np.asarray(axis, float)[: self.dim]
        a = a / np.linalg.norm(a)
        x = self.Xg - np.asarray(origin, float)[: self.dim]
        y = x - np.outer(x @ a, a)
        r = np.sqrt((y * y).sum(1))
        b = np.minimum(np.floor(r * nbins / radius).astype(int), nbins - 1)
        mass = np.bincount(b, weights=self.mass, minlength=nbins)
        su = np.bincount(b, weights=self.mass * (u @ a), minlength=nbins)
        mean = np.divide(su, mass, out=np.zeros(nbins), where=mass > 0)
        return mean, mass

    def stress(self, f):
        """Non-equilibrium second moment on unique nodes (Sec. 3.3: the stress recovered from the
        higher moments of the distribution), Pi_ij = tau / (tau + 1/2) sum_a e_ai e_aj (f_bar_a -
        f_bar_a^eq), with f_bar^eq = f^eq - dt/2 F** the collision's target at the node's (rho, u);
        the factor turns the non-equilibrium part of f_bar into that of f.  To leading order
        -Pi_ij = rho nu (d_i u_j + d_j u_i), the viscous stress.  Returns [G, d, d]."""
        rho, u = self.moments(f)
        F = rho[:, None] * self.accel()
        _, Fss = force_split(self.e, self.t, u, F)
        neq = f - (equilibrium(self.e, self.t, rho, u) - 0.5 * self.dt * Fss)
        ef = self.e.astype(float)
        return np.einsum("ai,aj,an->nij", ef, ef, neq) * (self.tau / (self.tau + 0.5))

    def integrals(self, f):
        """Quadrature integrals: mass sum M rho, momentum sum M rho u, KE = sum M rho0 |u|^2 / 2."""
        rho, u = self.moments(f)
        mass = float((self.mass * rho).sum())
        mom = (self.mass[:, None] * rho[:, None] * u).sum(0)
        ke = float(0.5 * self.rho0 * (self.mass * (u * u).sum(1)).sum())
        return mass, mom, ke
