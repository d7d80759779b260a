"""Strip solve: GMRES with the combination-technique preconditioner (Sect. 4.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``fgmres``: right-preconditioned flexible GMRES(m) with modified Gram-Schmidt
  and Givens rotations, in FP64; stops on the true relative residual
  ||b - A x|| / ||b||.
* ``ComponentSolver``: solves A_{l,l} du = r on one anisotropic full grid
  (Eq. 22) by GMRES, preconditioned by the inverse of
  (T_t + d C_t + G_t) (x) M^(1)_{l1} (x) M^(2)_{l2} (Sect. 4.3), each factor
  inverted exactly (2x2 inverse; sparse LU of the mass matrices).
* ``ct_precondition``: Algorithm 1's preconditioner step with 0-based levels:
  solves on the grids (l, L-l), l = 0..L and (l, L-1-l), l = 0..L-1 (residual
  restricted in dim 1 from grid (l+1, L-1-l)), then the combination
  du_l = dhat_l - (E^(1) (x) Id) dhat_(l-1, L-l).
* ``richardson``: Algorithm 1 itself (u <- u - P(A u - b)), stopped by the
  paper's test on the H^1(J x Omega) norm of the correction (or, as an
  option, on its Euclidean norm).
* ``StripSolver``: the implicit strip-by-strip scheme (Sect. 2): the right-hand
  side (U^-_{j-1}, w^+_{j-1}) = eta(t_{j-1}^+) (x) M_sg U^-_{j-1} (Eq. 5), with
  (u0, w^+) from load vectors for the first strip, plus the source part
  int_{I_j} (f, w + delta (d_t w + beta . grad w)) dt (``source_rhs``) and the
  inflow part -int_{I_j} <g, w>_{Gamma^-} dt (``inflow_rhs``), time integrals
  by adaptive quadrature; the end value U^-_j = sum_s eta_s(t_j) u_s.
* ``nodal_values``: the unique representation of a sparse-grid function: its
  values at the nodes of every component grid (prolongation from coarser
  levels, injection from finer ones).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from scipy import integrate

from .assembly import Factor, assemble_load, assemble_load_grad, gauss01
from .operator import SparseGridOperator, eta, eta_at, time_matrices


def fgmres(A, b, M=None, x0=None, tol=1e-10, restart=30, maxiter=1000):
    """Returns (x, iterations, relative true residual, history)."""
    M = M if M is not None else (lambda v: v)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, [0.0]
    r = b - A(x)
    beta = np.linalg.norm(r)
    hist = [beta / bnorm]
    it = 0
    while beta > tol * bnorm and it < maxiter:
        m = restart
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            z = M(V[j])
            Z.append(z)
            w = A(z)
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            it += 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or it >= maxiter:
                break
            nw = np.linalg.norm(w)
            if nw == 0.0:
                break
            V.append(w / nw)
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        for i in range(k):
            x = x + y[i] * Z[i]
        r = b - A(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
    return x, it, beta / bnorm, hist


class ComponentSolver:
    """The inverse of one component operator A_{l,l} (Algorithm 1): a sparse
    LU factorisation of the assembled block sum_k X_k (x) V_k (x) tau_k when it
    has at most ``direct_max`` unknowns, else GMRES to ``tol`` with the
    (T_t + d C_t + G_t) (x) M (x) M preconditioner."""

    def __init__(self, op: SparseGridOperator, tol=1e-12, restart=60, maxiter=5000, direct_max=20000):
        self.op = op
        self.tol, self.restart, self.maxiter = tol, restart, maxiter
        Mt, Tt, Ct, Gt = time_matrices(op.prob.dt, op.prob.r)
        self.Pt_inv = np.linalg.inv(Tt + op.prob.delta * Ct + Gt)
        self.direct_max = direct_max
        self._direct = (None, {})
        self._lu = {}
        self.iterations = []

    def _mass_lu(self, store, l):
        key = (id(store), l)
        if key not in self._lu:
            self._lu[key] = spla.splu(store.proj(Factor("vol"), l, l).tocsc())
        return self._lu[key]

    def precond(self, l1, l2, v):
        n1, n2 = self.op.grid_shape(l1, l2)
        R = self.op.R
        u = v.reshape(n1, n2, R)
        u = np.einsum("st,abt->abs", self.Pt_inv, u)
        lu1 = self._mass_lu(self.op.fx, l1)
        lu2 = self._mass_lu(self.op.fv, l2)
        u = lu1.solve(u.reshape(n1, n2 * R)).reshape(n1, n2, R)
        t = np.ascontiguousarray(u.transpose(1, 0, 2)).reshape(n2, n1 * R)
        u = lu2.solve(t).reshape(n2, n1, R).transpose(1, 0, 2)
        return np.ascontiguousarray(u).ravel()

    def block_matrix(self, l1, l2) -> sp.csc_matrix:
        """A_{l,l} in the layout u[k1, k2, s] (row-major), from the operator's
        current terms."""
        op = self.op
        A = None
        for tau, X, V in op.terms:
            K = sp.kron(op.fx.proj(X, l1, l1), sp.kron(op.fv.proj(V, l2, l2), sp.csr_matrix(tau)))
            A = K if A is None else A + K
        return A.tocsc()

    def solve(self, l1, l2, r):
        n1, n2 = self.op.grid_shape(l1, l2)
        R = self.op.R
        if n1 * n2 * R <= self.direct_max:
            # one factorisation per grid while the operator's term list is
            # the same object (the cache holds it, so its id is not reused)
            if self._direct[0] is not self.op.terms:
                self._direct = (self.op.terms, {})
            cache = self._direct[1]
            if (l1, l2) not in cache:
                cache[(l1, l2)] = spla.splu(self.block_matrix(l1, l2))
            x = cache[(l1, l2)].solve(r.ravel())
            self.iterations.append(1)
            return x.reshape(n1, n2, R)
        A = lambda x: self.op.apply_diag(l1, l2, x.reshape(n1, n2, R)).ravel()
        x, it, res, _ = fgmres(A, r.ravel(), lambda v: self.precond(l1, l2, v),
                               tol=self.tol, restart=self.restart, maxiter=self.maxiter)
        self.iterations.append(it)
        return x.reshape(n1, n2, R)


def ct_precondition(op: SparseGridOperator, comp: ComponentSolver, r: np.ndarray) -> np.ndarray:
    """Algorithm 1 (0-based levels): the preconditioned residual du = P(r)."""
    L = op.L
    up = [comp.solve(l, L - l, op.block(r, l)) for l in range(L + 1)]
    lo = []
    for l in range(L):
        r_hi = op.block(r, l + 1)                       # grid (l+1, L-1-l)
        E = op.hx.E[l]                                  # E_{l+1 <- l}
        r_lo = op.left(E.T.tocsr(), r_hi)               # restriction in dim 1
        lo.append(comp.solve(l, L - 1 - l, r_lo))
    out = np.zeros(op.size)
    for l in range(L + 1):
        du = up[l]
        if l >= 1:
            du = du - op.left(op.hx.E[l - 1], lo[l - 1])   # (l-1, L-l) -> (l, L-l)
        out[op.offsets[l]:op.offsets[l + 1]] = du.ravel()
    return out


def richardson(op, comp, b, tol=1e-10, maxiter=200, norm="h1"):
    """Algorithm 1: u <- u - P(A u - b) until the correction is small.

    norm="h1": the paper's stop, ||du||_{H^1(J x Omega)} < tol (the H^1 norm
    of the correction function over the strip, ``norms.h1_norm``);
    norm="l2": ||du||_2 < tol * ||b||_2 on the spanning-set coefficients."""
    from .norms import h1_norm
    u = np.zeros_like(b)
    bn = np.linalg.norm(b)
    for k in range(maxiter):
        du = ct_precondition(op, comp, op.apply(u) - b)
        u = u - du
        small = h1_norm(op, du) < tol if norm == "h1" else np.linalg.norm(du) < tol * bn
        if small:
            return u, k + 1
    return u, maxiter


class StripSolver:
    """Implicit time stepping over strips (Sect. 2) with FGMRES + CT."""

    def __init__(self, prob, tol=1e-10, inner_tol=1e-12, restart=30, maxiter=500):
        self.prob = prob
        self.op = SparseGridOperator(prob)
        self.comp = ComponentSolver(self.op, tol=inner_tol)
        self.tol, self.restart, self.maxiter = tol, restart, maxiter
        R = self.op.R
        self.e_start = eta_at(prob.r, 0.0)             # eta_s(t_{j-1}^+)
        self.e_end = eta_at(prob.r, 1.0)               # eta_s(t_j^-)
        self.outer_its = []

    def initial_mass_u0(self) -> np.ndarray:
        """(u0, phi_{l,k}) on every grid: sum of products of load vectors."""
        op = self.op
        out = np.zeros(op.size // op.R)
        off = 0
        for (l1, l2) in op.grids:
            n1, n2 = op.grid_shape(l1, l2)
            blk = np.zeros((n1, n2))
            for pr in self.prob.u0:
                fx = op.fx.embed(l1).T @ assemble_load(op.hx.levels[op.L], pr.fx)
                fv = op.fv.embed(l2).T @ assemble_load(op.hv.levels[op.L], pr.fv)
                blk += pr.coef * np.outer(fx, fv)
            out[off:off + n1 * n2] = blk.ravel()
            off += n1 * n2
        return out

    def mass_spatial(self, U: np.ndarray) -> np.ndarray:
        """M_sg U for a spatial sparse-grid vector (no time index)."""
        op = self.op
        u = np.zeros((U.size, op.R))
        u[:, 0] = U
        return op.apply_mass(u.ravel()).reshape(-1, op.R)[:, 0]

    def source_rhs(self, t0: float) -> np.ndarray:
        """int_I (f, w + delta (d_t w + beta . grad w)) dt for w = eta_s phi psi on
        the strip I = (t0, t0 + dt) (Sect. 2, b_j), f = sum_k c_k ft_k fx_k fv_k,
        beta_c = b_c(x) c_c(v):
          (f, w)            -> int ft eta_s      (fx, phi)(fv, psi)
          delta (f, d_t w)  -> delta int ft eta_s' (fx, phi)(fv, psi)
          delta (f, beta_c d_c w) -> delta int ft eta_s (fx b_c, D phi)(fv c_c, D psi)."""
        op, prob = self.op, self.prob
        R, d, dt, dl = op.R, prob.d, prob.dt, prob.delta
        out = np.zeros(op.size)
        if not prob.f:
            return out
        hx, hv = op.hx.levels[op.L], op.hv.levels[op.L]
        mul = lambda f, g: (None if f is None and g is None else
                            (lambda p: (f(p) if f is not None else 1.0) * (g(p) if g is not None else 1.0)))
        ev = lambda s, t: eta(s, np.array([(t - t0) / dt]), dt)[0][0]     # eta_s(t)
        ed = lambda s, t: eta(s, np.array([(t - t0) / dt]), dt)[1][0]     # d eta_s / dt

        terms = []   # (time weights [R], x load (finest), v load (finest), x axis or -1, v axis or -1)
        for src in prob.f:
            ft = (lambda t: 1.0) if src.ft is None else (lambda t, g=src.ft: float(np.asarray(g(np.array([t])))[0]))
            w_val = np.array([integrate.quad(lambda t, s=s: ft(t) * ev(s, t), t0, t0 + dt,
                                             epsabs=1e-15, epsrel=1e-13)[0] for s in range(R)])
            w_dt = np.array([integrate.quad(lambda t, s=s: ft(t) * ed(s, t), t0, t0 + dt,
                                            epsabs=1e-15, epsrel=1e-13)[0] for s in range(R)])
            terms.append((src.coef * (w_val + dl * w_dt), src.fx, src.fv, -1, -1))
            for c, b in enumerate(prob.beta):
                if b.coef == 0.0:
                    continue
                # a time factor of beta_c enters the integrand: the strip's
                # 3-point Gauss rule, like the operator's time couplings
                wb = w_val if getattr(b, "ft", None) is None else self._gauss_weights(t0, ft, b.ft)
                terms.append((src.coef * b.coef * dl * wb, mul(src.fx, b.fx), mul(src.fv, b.fv),
                              c if c < d else -1, c - d if c >= d else -1))
        off = 0
        for (l1, l2) in op.grids:
            n1, n2 = op.grid_shape(l1, l2)
            blk = np.zeros((n1, n2, R))
            for (wt, fx, fv, ax, av) in terms:
                Fx = assemble_load(hx, fx) if ax < 0 else assemble_load_grad(hx, fx, ax)
                Fv = assemble_load(hv, fv) if av < 0 else assemble_load_grad(hv, fv, av)
                blk += np.einsum("i,j,s->ijs", op.fx.embed(l1).T @ Fx, op.fv.embed(l2).T @ Fv, wt)
            out[off:off + blk.size] = blk.ravel()
            off += blk.size
        return out

    def _gauss_weights(self, t0: float, ft, bt, gate=None) -> np.ndarray:
        """[int_I ft(t) bt(t) [gate(t)] eta_s(t) dt]_s by the 3-point Gauss rule
        on the strip (t0, t0 + dt); gate(t) in {0, 1} selects the times where an
        inflow part is active."""
        R, dt = self.op.R, self.prob.dt
        tq, wq = gauss01(3)
        out = np.zeros(R)
        for q in range(3):
            t = t0 + tq[q] * dt
            g = ft(t) * float(np.asarray(bt(np.array([t])))[0])
            if gate is not None:
                g *= gate(t)
            out += wq[q] * dt * g * np.array([eta(s, tq[q:q + 1], dt)[0][0] for s in range(R)])
        return out

    def inflow_rhs(self, t0: float) -> np.ndarray:
        """-int_I <g, w>_{Gamma^-} dt for w = eta_s phi psi on the strip
        I = (t0, t0 + dt) (Sect. 2, b_j), g = sum_k c_k gt_k gx_k gv_k and
        <u, w>_{Gamma^-} = int_{Gamma^-} (beta . n) u w: per beta component
        p = b_p(x) c_p(v) the inflow part of the faces x_p = side (p < d) or
        v_{p-d} = side is split by the signs of the two factors exactly like
        the inflow term of the operator (Sect. 5.2); its x and v factors
        carry the extra weights gx and gv.  Load vectors follow from the
        factor matrices and the partition of unity: int w phi_i = sum_j
        int w phi_i phi_j."""
        op, prob = self.op, self.prob
        R, d, dt = op.R, prob.d, prob.dt
        out = np.zeros(op.size)
        if not prob.g:
            return out
        w = lambda f: (f,) if f is not None else ()
        fn = lambda f: f if f is not None else (lambda p: np.ones(p.shape[0]))
        ev = lambda s, t: eta(s, np.array([(t - t0) / dt]), dt)[0][0]
        terms = []   # (time weights [R], x factor, v factor)
        for src in prob.g:
            gt = (lambda t: 1.0) if src.ft is None else (lambda t, g=src.ft: float(np.asarray(g(np.array([t])))[0]))
            wt = -src.coef * np.array([integrate.quad(lambda t, s=s: gt(t) * ev(s, t), t0, t0 + dt,
                                                      epsabs=1e-15, epsrel=1e-13)[0] for s in range(R)])
            for p, b in enumerate(prob.beta):
                if b.coef == 0.0:
                    continue
                bt = getattr(b, "ft", None)
                # with a time factor tp of beta_p: both signs sc of coef tp(t)
                # give parts, each active where it holds, weighted by tp (the
                # strip's 3-point Gauss rule, like the operator's inflow term)
                for sc in ((+1, -1) if bt is not None else (None,)):
                  for side in (-1, +1):
                    for s1 in (+1, -1):
                        s2 = -side * s1
                        if sc is None:
                            wpart = wt
                            rx = ((fn(b.fx), b.coef, s1),)
                        else:
                            gate = (lambda t, sc=sc, bt=bt, c=b.coef:
                                    1.0 if sc * c * float(np.asarray(bt(np.array([t])))[0]) > 0 else 0.0)
                            wpart = -src.coef * self._gauss_weights(t0, gt, bt, gate)
                            # b.coef tp(t) fx(x) has sign s1 where fx has sign s1 sc
                            rx = ((fn(b.fx), sc, s1),)
                        rv = ((fn(b.fv), 1.0, s2),)
                        if p < d:
                            if prob.mesh_x.periodic[p]:
                                continue
                            X = Factor("face", side * b.coef, w(b.fx) + w(src.fx), restrict=rx, face=(p, side))
                            V = Factor("vol", 1.0, w(b.fv) + w(src.fv), restrict=rv)
                        else:
                            if prob.mesh_v.periodic[p - d]:
                                continue
                            X = Factor("vol", side * b.coef, w(b.fx) + w(src.fx), restrict=rx)
                            V = Factor("face", 1.0, w(b.fv) + w(src.fv), restrict=rv, face=(p - d, side))
                        terms.append((wpart, X, V))
        loads = [(wt, op.fx.fine(X) @ np.ones(op.fx.fine(X).shape[1]), op.fv.fine(V) @ np.ones(op.fv.fine(V).shape[1]))
                 for wt, X, V in terms]
        off = 0
        for (l1, l2) in op.grids:
            n1, n2 = op.grid_shape(l1, l2)
            blk = np.zeros((n1, n2, R))
            for wt, Fx, Fv in loads:
                blk += np.einsum("i,j,s->ijs", op.fx.embed(l1).T @ Fx, op.fv.embed(l2).T @ Fv, wt)
            out[off:off + blk.size] = blk.ravel()
            off += blk.size
        return out

    def rhs(self, MU: np.ndarray, t0: float = 0.0) -> np.ndarray:
        return np.outer(MU, self.e_start).ravel() + self.source_rhs(t0) + self.inflow_rhs(t0)

    def endpoint(self, u: np.ndarray) -> np.ndarray:
        return u.reshape(-1, self.op.R) @ self.e_end

    def solve_strip(self, b: np.ndarray, x0=None):
        op = self.op
        P = lambda v: ct_precondition(op, self.comp, v)
        x, it, res, hist = fgmres(op.apply, b, P, x0=x0, tol=self.tol,
                                  restart=self.restart, maxiter=self.maxiter)
        self.outer_its.append(it)
        return x, it, res

    def run(self, n_strips=None, solutions=None):
        """Returns the list of end values U^-_j (spatial sparse-grid vectors);
        appends every strip solution u_j to ``solutions`` when given."""
        n = self.prob.n_strips if n_strips is None else n_strips
        MU = self.initial_mass_u0()
        ends = []
        for j in range(n):
            self.op.set_time(j * self.prob.dt)
            u, it, res = self.solve_strip(self.rhs(MU, j * self.prob.dt))
            if solutions is not None:
                solutions.append(u)
            U = self.endpoint(u)
            ends.append(U)
            MU = self.mass_spatial(U)
        return ends


# ----------------------------------------------------------------------------
# unique representation and errors
# ----------------------------------------------------------------------------

def injection(hier, lc: int, lf: int) -> sp.csr_matrix:
    """Rows: level-lc vertices; picks the coinciding level-lf vertex (lf >= lc)."""
    cf = hier.levels[lf].coords
    cc = hier.levels[lc].coords
    idx = {tuple(x.tolist()): i for i, x in enumerate(cf)}
    cols = np.array([idx[tuple(x.tolist())] for x in cc])
    return sp.csr_matrix((np.ones(cc.shape[0]), (np.arange(cc.shape[0]), cols)),
                         shape=(cc.shape[0], cf.shape[0]))


def _transfer(hier, l_to: int, l_from: int) -> sp.csr_matrix:
    if l_from <= l_to:
        return hier.embed(l_to, l_from)
    return injection(hier, l_to, l_from)


def nodal_values(op: SparseGridOperator, U: np.ndarray, R: int = 1) -> np.ndarray:
    """Values of the sparse-grid function at the nodes of every component grid."""
    out = np.zeros(U.size)
    off = [0]
    for (a, b) in op.shape:
        off.append(off[-1] + a * b * R)
    for i, (l1, l2) in enumerate(op.grids):
        n1, n2 = op.shape[i]
        acc = np.zeros((n1, n2, R))
        for j, (m1, m2) in enumerate(op.grids):
            u = U[off[j]:off[j + 1]].reshape(op.shape[j] + (R,))
            acc += op.right(_transfer(op.hv, l2, m2), op.left(_transfer(op.hx, l1, m1), u))
        out[off[i]:off[i + 1]] = acc.ravel()
    return out


def full_grid_values(op: SparseGridOperator, U: np.ndarray) -> np.ndarray:
    """The sparse-grid function (spatial) on the finest full grid (L, L)."""
    L = op.L
    acc = np.zeros((op.hx.levels[L].n, op.hv.levels[L].n, 1))
    off = 0
    for i, (l1, l2) in enumerate(op.grids):
        n1, n2 = op.shape[i]
        u = U[off:off + n1 * n2].reshape(n1, n2, 1)
        off += n1 * n2
        acc += op.right(op.hv.embed(L, l2), op.left(op.hx.embed(L, l1), u))
    return acc[:, :, 0]


def coarse_values(op: SparseGridOperator, U: np.ndarray, R: int, lx: int, lv: int) -> np.ndarray:
    """Values at the nodes of the full grid (lx, lv) of a sparse-grid function
    (strip vector R = 2, spatial R = 1): injection from finer grids,
    prolongation from coarser ones; layout [kx][kv][s]."""
    nx, nv = op.hx.levels[lx].n, op.hv.levels[lv].n
    out = np.zeros((nx, nv, R))
    off = 0
    for (l1, l2) in op.grids:
        n1, n2 = op.grid_shape(l1, l2)
        u = U[off:off + n1 * n2 * R].reshape(n1, n2, R)
        off += n1 * n2 * R
        out += op.right(_transfer(op.hv, lv, l2), op.left(_transfer(op.hx, lx, l1), u))
    return out.ravel()
