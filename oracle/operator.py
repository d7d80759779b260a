"""The strip operator A^(delta) on the sparse grid (Sect. 4.1-4.2), blockwise.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Time basis (Sect. 4.1; the paper leaves the basis open): Legendre
  polynomials on the strip, eta_s(t) = P_s(2 (t - t_{j-1}) / dt - 1).
* Time matrices M^(t), T^(t), C^(t), G^(t) (Sect. 4.2, Eq. 10) from their
  definitions by Gauss quadrature in time (exact: the integrands are
  polynomials).
* The Kronecker block formula (Sect. 4.2) with time-constant coefficients
  (coefficients with a time factor: the quadrature sum over the strip's
  Gauss points, ``time_dependent_terms``):
      A = (T_t + d C_t) (x) M  +  d T_t (x) T^T  +  d T_t^T (x) (T + K)
          + M_t (x) (T + d C + K + d K~ - G)  +  G_t (x) M
  where the factor d on K~ is taken from the weak form of Sect. 2 (the printed
  block formula omits it; the brute-force test pins this reading).
* Spatial operators split into Kronecker factor pairs through the tensor
  product structure of beta and sigma (Sect. 4.2); the inflow term G is split
  by boundary side and by the sign of beta . n (Sect. 5.2).
* The sparse-grid vector is the concatenation over grids l = 0..L of the
  coefficient arrays u_(l, L-l)[k1, k2, s] (spanning set of Sect. 4.1).
* Blockwise apply [A u]_l = sum_l' A_{l,l'} u_l' with the ordering rule of
  Sect. 4.2: the dim-2 factor first when l1' + l2 <= l1 + l2', else the dim-1
  factor first; then the time factor.

Pinned by tests/test_oracle_operator.py: time matrices against closed forms,
the DG(1) amplification against the 2-stage Radau IIA stability function, the
block formula against brute-force assembly of the weak form, the energy
identity of the stability lemma, and blockwise apply against an assembled
dense matrix.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .assembly import Factor, FactorStore, gauss01
from .mesh import Hierarchy, P2Hierarchy


def ONE(p):
    return np.ones(p.shape[0])


# ----------------------------------------------------------------------------
# time matrices
# ----------------------------------------------------------------------------

def _leg(s: int, x: np.ndarray):
    c = np.zeros(s + 1)
    c[s] = 1.0
    P = np.polynomial.legendre.Legendre(c)
    return P(x), P.deriv()(x) if s > 0 else np.zeros_like(x)


def eta(s: int, tau: np.ndarray, dt: float):
    """eta_s and d eta_s / dt at reference times tau in [0, 1]."""
    v, dv = _leg(s, 2.0 * tau - 1.0)
    return v, dv * 2.0 / dt


def time_matrices(dt: float, r: int = 1):
    """M_t, T_t, C_t, G_t with entries [s, s'] (s: test, s': trial), Eq. 10."""
    tq, wq = gauss01(r + 2)
    R = r + 1
    ev = np.array([eta(s, tq, dt)[0] for s in range(R)])
    ed = np.array([eta(s, tq, dt)[1] for s in range(R)])
    w = wq * dt
    Mt = np.einsum("q,sq,tq->st", w, ev, ev)
    Tt = np.einsum("q,tq,sq->st", w, ed, ev)       # eta'_{s'} eta_s
    Ct = np.einsum("q,sq,tq->st", w, ed, ed)
    e0 = np.array([eta(s, np.array([0.0]), dt)[0][0] for s in range(R)])
    Gt = np.outer(e0, e0)
    return Mt, Tt, Ct, Gt


def eta_at(r: int, tau: float, dt: float = 1.0):
    return np.array([eta(s, np.array([tau]), dt)[0][0] for s in range(r + 1)])


# ----------------------------------------------------------------------------
# spatial operators as sums of Kronecker factor pairs
# ----------------------------------------------------------------------------

def _fn(f):
    return f if f is not None else ONE


def spatial_operators(prob):
    """Dict name -> list of (X factor on Omega_x, V factor on Omega_v)."""
    d = prob.d
    beta = prob.beta
    Dx = lambda p: p + 1 if p < d else 0
    Dv = lambda p: p - d + 1 if p >= d else 0
    w = lambda f: (f,) if f is not None else ()
    act = [p for p in range(2 * d) if beta[p].coef != 0.0]
    ops = {"M": [(Factor("vol"), Factor("vol"))]}
    ops["T"] = [(Factor("vol", beta[p].coef, w(beta[p].fx), 0, Dx(p)),
                 Factor("vol", 1.0, w(beta[p].fv), 0, Dv(p))) for p in act]
    ops["Tt"] = [(Factor("vol", beta[p].coef, w(beta[p].fx), Dx(p), 0),
                  Factor("vol", 1.0, w(beta[p].fv), Dv(p), 0)) for p in act]
    ops["C"] = [(Factor("vol", beta[p].coef * beta[q].coef, w(beta[p].fx) + w(beta[q].fx), Dx(q), Dx(p)),
                 Factor("vol", 1.0, w(beta[p].fv) + w(beta[q].fv), Dv(q), Dv(p)))
                for p in act for q in act]
    s = prob.sigma
    if s.coef != 0.0:
        ops["K"] = [(Factor("vol", s.coef, w(s.fx)), Factor("vol", 1.0, w(s.fv)))]
        ops["Kt"] = [(Factor("vol", s.coef * beta[q].coef, w(s.fx) + w(beta[q].fx), Dx(q), 0),
                      Factor("vol", 1.0, w(s.fv) + w(beta[q].fv), Dv(q), 0)) for q in act]
    else:
        ops["K"], ops["Kt"] = [], []
    G = []
    for p in act:
        b = beta[p]
        fx, fv = _fn(b.fx), _fn(b.fv)
        for side in (-1, +1):
            for s1 in (+1, -1):
                s2 = -side * s1          # side * s1 * s2 < 0: inflow
                rx = ((fx, b.coef, s1),)
                rv = ((fv, 1.0, s2),)
                if p < d:   # face of Omega_x
                    if prob.mesh_x.periodic[p]:
                        continue
                    X = Factor("face", side * b.coef, w(b.fx), restrict=rx, face=(p, side))
                    V = Factor("vol", 1.0, w(b.fv), restrict=rv)
                else:       # face of Omega_v
                    if prob.mesh_v.periodic[p - d]:
                        continue
                    X = Factor("vol", side * b.coef, w(b.fx), restrict=rx)
                    V = Factor("face", 1.0, w(b.fv), restrict=rv, face=(p - d, side))
                G.append((X, V))
    ops["G"] = G
    return ops


def kron_terms(prob, t0: float = 0.0, m: int = 3):
    """List of (tau (R x R), X, V): the block formula of Sect. 4.2 for the
    strip (t0, t0 + dt).  Time-constant coefficients: the exact time
    matrices.  Coefficients with a time factor (Product.ft): the paper's
    quadrature in time, m-point Gauss-Legendre on the strip, with the spatial
    operators frozen at every point tau_mu (``time_dependent_terms``)."""
    if is_time_dependent(prob):
        return time_dependent_terms(prob, t0, m)
    Mt, Tt, Ct, Gt = time_matrices(prob.dt, prob.r)
    dl = prob.delta
    ops = spatial_operators(prob)
    plan = [
        (Tt + dl * Ct, "M"), (Gt, "M"),
        (dl * Tt, "Tt"),
        (dl * Tt.T, "T"), (dl * Tt.T, "K"),
        (Mt, "T"), (dl * Mt, "C"), (Mt, "K"), (dl * Mt, "Kt"), (-Mt, "G"),
    ]
    out = []
    for tau, name in plan:
        for X, V in ops[name]:
            out.append((tau, X, V))
    return out


def is_time_dependent(prob) -> bool:
    return any(getattr(b, "ft", None) is not None for b in prob.beta) or getattr(prob.sigma, "ft", None) is not None


def _frozen(prob, t: float):
    """The problem with its coefficients frozen at time t: every time factor
    folded into the product's scalar coefficient."""
    import copy
    from dataclasses import replace

    def fz(pr):
        if getattr(pr, "ft", None) is None:
            return pr
        return replace(pr, coef=pr.coef * float(np.asarray(pr.ft(np.array([t])))[0]), ft=None)
    q = copy.copy(prob)
    q.beta = [fz(b) for b in prob.beta]
    q.sigma = fz(prob.sigma)
    return q


def time_dependent_terms(prob, t0: float, m: int = 3):
    """Sect. 4.2 with time-dependent beta, sigma: per Gauss point tau_mu of the
    strip (weight w_mu, sum w_mu = dt) the point matrices
        M_mu = [eta_s' eta_s], T_mu = [eta'_s' eta_s], C_mu = [eta'_s' eta'_s]
    at tau_mu and the spatial operators T, C, K, K~, G of the coefficients
    at tau_mu (the inflow boundary Gamma^-(tau_mu) included), summed as
        sum_mu w_mu [ (T_mu + d C_mu) (x) M + d T_mu (x) T_mu^T
                      + d T_mu^T (x) (T_mu + K_mu)
                      + M_mu (x) (T_mu + d C_mu + K_mu + d K~_mu - G_mu) ]
        + G^(t) (x) M,
    with the factor d on K~ as in the time-constant case."""
    R, dt, dl = prob.r + 1, prob.dt, prob.delta
    tq, wq = gauss01(m)
    _, _, _, Gt = time_matrices(dt, prob.r)
    out = []
    ops0 = spatial_operators(prob)
    out += [(Gt, X, V) for X, V in ops0["M"]]
    for q in range(m):
        ev = np.array([eta(s, tq[q:q + 1], dt)[0][0] for s in range(R)])
        ed = np.array([eta(s, tq[q:q + 1], dt)[1][0] for s in range(R)])
        w = wq[q] * dt
        Mm = w * np.outer(ev, ev)
        Tm = w * np.outer(ev, ed)          # [s, s'] = eta'_s' eta_s
        Cm = w * np.outer(ed, ed)
        ops = spatial_operators(_frozen(prob, t0 + tq[q] * dt))
        plan = [(Tm + dl * Cm, "M"), (dl * Tm, "Tt"), (dl * Tm.T, "T"), (dl * Tm.T, "K"),
                (Mm, "T"), (dl * Mm, "C"), (Mm, "K"), (dl * Mm, "Kt"), (-Mm, "G")]
        for tau, name in plan:
            for X, V in ops[name]:
                out.append((tau, X, V))
    return out


# ----------------------------------------------------------------------------
# the sparse grid and the blockwise apply
# ----------------------------------------------------------------------------

class SparseGridOperator:
    def __init__(self, prob):
        self.prob = prob
        self.L = prob.L
        self.R = prob.r + 1
        order = getattr(prob, "order", 1)
        if getattr(prob, "element", "P") == "Q":
            from .tensor import TensorHierarchy
            self.hx = TensorHierarchy(prob.mesh_x, prob.L, order)
            self.hv = TensorHierarchy(prob.mesh_v, prob.L, order)
        else:
            H = P2Hierarchy if order == 2 else Hierarchy
            self.hx = H(prob.mesh_x, prob.L)
            self.hv = H(prob.mesh_v, prob.L)
        self.fx = FactorStore(self.hx)
        self.fv = FactorStore(self.hv)
        self.terms = kron_terms(prob)
        self.t0 = 0.0
        self.grids = [(l, self.L - l) for l in range(self.L + 1)]
        self.shape = [(self.hx.levels[a].n, self.hv.levels[b].n) for a, b in self.grids]
        sizes = [a * b * self.R for a, b in self.shape]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)])
        self.size = int(self.offsets[-1])

    def set_time(self, t0: float):
        """The operator of the strip (t0, t0 + dt): only coefficients with a
        time factor make it depend on t0."""
        if is_time_dependent(self.prob) and t0 != self.t0:
            self.terms = kron_terms(self.prob, t0)
        self.t0 = t0

    # --- layout helpers
    def block(self, u: np.ndarray, i: int) -> np.ndarray:
        n1, n2 = self.shape[i]
        return u[self.offsets[i]:self.offsets[i + 1]].reshape(n1, n2, self.R)

    def grid_shape(self, l1: int, l2: int):
        return self.hx.levels[l1].n, self.hv.levels[l2].n

    # --- Kronecker factors
    @staticmethod
    def left(S: sp.spmatrix, u: np.ndarray) -> np.ndarray:
        """(S (x) Id) on the dim-1 index of u[k1, k2, s]."""
        a, b, R = u.shape
        return (S @ u.reshape(a, b * R)).reshape(S.shape[0], b, R)

    @staticmethod
    def right(S: sp.spmatrix, u: np.ndarray) -> np.ndarray:
        """(Id (x) S) on the dim-2 index of u[k1, k2, s]."""
        a, b, R = u.shape
        t = np.ascontiguousarray(u.transpose(1, 0, 2)).reshape(b, a * R)
        return (S @ t).reshape(S.shape[0], a, R).transpose(1, 0, 2)

    @staticmethod
    def time(tau: np.ndarray, u: np.ndarray) -> np.ndarray:
        return np.einsum("st,abt->abs", tau, u)

    def apply_block(self, terms, l, lp, u_lp) -> np.ndarray:
        """A_{l,l'} u_l' for target grid l = (l1, l2), source l' = (l1', l2')."""
        (l1, l2), (m1, m2) = l, lp
        out = np.zeros(self.grid_shape(l1, l2) + (u_lp.shape[2],))
        for tau, X, V in terms:
            S1 = self.fx.proj(X, l1, m1)
            S2 = self.fv.proj(V, l2, m2)
            if m1 + l2 <= l1 + m2:
                w = self.left(S1, self.right(S2, u_lp))
            else:
                w = self.right(S2, self.left(S1, u_lp))
            out += self.time(tau, w)
        return out

    def apply(self, u: np.ndarray, terms=None) -> np.ndarray:
        terms = self.terms if terms is None else terms
        y = np.zeros(self.size)
        for i, g in enumerate(self.grids):
            acc = np.zeros(self.shape[i] + (self.R,))
            for j, gp in enumerate(self.grids):
                acc += self.apply_block(terms, g, gp, self.block(u, j))
            y[self.offsets[i]:self.offsets[i + 1]] = acc.ravel()
        return y

    def apply_rows(self, us, rows, terms=None) -> np.ndarray:
        """Selected outputs of the blockwise apply, each from the definition
        (Sect. 4.2):
            [A u]_l[k1, k2, :] = sum_{l'} sum_t tau_t (X_{l1,l1'}[k1, :] U_l' V_{l2,l2'}[k2, :]^T)
        with only row k1 of X_{l1,l1'} and row k2 of V_{l2,l2'} formed, from
        the finest-level factor and the embeddings.  For sizes where the
        whole apply is out of reach.  us: list of coefficient vectors;
        rows: (grid i, k1, k2) triples.  Returns [len(us)][len(rows)][R]."""
        terms = self.terms if terms is None else terms
        out = np.zeros((len(us), len(rows), self.R))
        for n, (i, k1, k2) in enumerate(rows):
            l1, l2 = self.grids[i]
            xrow, vrow = {}, {}
            for _, X, V in terms:
                if X not in xrow:
                    xrow[X] = self.fx.test_row(X, l1, k1)
                if V not in vrow:
                    vrow[V] = self.fv.test_row(V, l2, k2)
            for j, (m1, m2) in enumerate(self.grids):
                xr = {X: self.fx.proj_row(r, m1) for X, r in xrow.items()}
                vr = {V: self.fv.proj_row(r, m2) for V, r in vrow.items()}
                blocks = [self.block(u, j) for u in us]
                for tau, X, V in terms:
                    x, v = xr[X], vr[V]
                    if x.nnz == 0 or v.nnz == 0:
                        continue
                    for q, U in enumerate(blocks):
                        sub = U[np.ix_(x.indices, v.indices)]          # (nx, nv, R)
                        w = np.einsum("a,abt,b->t", x.data, sub, v.data)
                        out[q, n] += tau @ w
        return out

    def apply_diag(self, l1: int, l2: int, u: np.ndarray, terms=None) -> np.ndarray:
        """A_{l,l} on one anisotropic full grid (used by the component solves)."""
        terms = self.terms if terms is None else terms
        return self.apply_block(terms, (l1, l2), (l1, l2), u)

    # --- mass
    def mass_terms(self):
        return [(np.eye(self.R), Factor("vol"), Factor("vol"))]

    def apply_mass(self, u: np.ndarray) -> np.ndarray:
        """Sparse-grid mass matrix (Id_t (x) M_sg) applied to u."""
        return self.apply(u, self.mass_terms())

    # --- dense assembly for tiny cases
    def dense(self, terms=None) -> np.ndarray:
        terms = self.terms if terms is None else terms
        A = np.zeros((self.size, self.size))
        for j, gp in enumerate(self.grids):
            n1, n2 = self.shape[j]
            for c in range(n1 * n2 * self.R):
                e = np.zeros(n1 * n2 * self.R)
                e[c] = 1.0
                col = np.zeros(self.size)
                for i, g in enumerate(self.grids):
                    col[self.offsets[i]:self.offsets[i + 1]] = self.apply_block(
                        terms, g, gp, e.reshape(n1, n2, self.R)).ravel()
                A[:, self.offsets[j] + c] = col
        return A
