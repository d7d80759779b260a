"""Literal full-grid assembly of the strip weak form (Sect. 2, Eq. 5) for tiny levels.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

No tensor-product splitting is used here: the 2d-dimensional integrals of
    a(v, w) = int_I ( d_t v + beta . grad v + sigma v,  w + delta (d_t w + beta . grad w) )
              - <v, w>_{Gamma^-}  dt  +  (v(t_{j-1}^+), w(t_{j-1}^+))
are evaluated directly by product quadrature over pairs of cells (x-cell,
v-cell) and time points, with beta and sigma evaluated as full functions of
(x, v) and the inflow boundary Gamma^- selected pointwise by beta . n < 0.
The space is the full grid V^(1)_Lx (x) V^(2)_Lv (x) P^r(I); dofs are ordered
(i, j, s) with s fastest, like the sparse-grid blocks.

``energy_terms`` evaluates the right-hand side of the energy identity in the
proof of the stability lemma (Sect. 3, case sigma = 0, one strip) by the same
kind of direct quadrature.
"""
from __future__ import annotations

import numpy as np

from .assembly import gauss01, simplex_rule
from .mesh import Hierarchy
from .operator import eta


def _cell_data(lev, q):
    """Quadrature points, weights, basis values and gradients per cell."""
    cc = lev.cell_coords
    nc, d1, d = cc.shape
    v0 = cc[:, 0, :]
    J = np.transpose(cc[:, 1:, :] - v0[:, None, :], (0, 2, 1))
    det = np.abs(np.linalg.det(J))
    Jinv = np.linalg.inv(J)
    rp, rw = simplex_rule(d, q)
    pts = v0[:, None, :] + np.einsum("cij,qj->cqi", J, rp)
    lam = np.concatenate([1.0 - rp.sum(axis=1, keepdims=True), rp], axis=1)
    gref = np.vstack([-np.ones((1, d)), np.eye(d)])
    grad = np.einsum("cji,kj->cki", Jinv, gref)          # (nc, d+1, d)
    w = rw[None, :] * det[:, None]
    return pts, w, lam, grad


def _face_data(lev, q):
    fc = lev.bface_coords
    nf, dv, d = fc.shape
    rp, rw = simplex_rule(dv - 1, q)
    f0 = fc[:, 0, :]
    Jf = np.transpose(fc[:, 1:, :] - f0[:, None, :], (0, 2, 1))
    meas = np.ones(nf) if dv == 1 else np.sqrt(np.abs(np.linalg.det(np.einsum("fki,fkj->fij", Jf, Jf))))
    pts = f0[:, None, :] + np.einsum("fij,qj->fqi", Jf, rp)
    lam = np.concatenate([1.0 - rp.sum(axis=1, keepdims=True), rp], axis=1)
    return pts, rw[None, :] * meas[:, None], lam


def _tf(pr, t):
    """The time factor of a coefficient product at time t (1 without one)."""
    ft = getattr(pr, "ft", None)
    return 1.0 if ft is None else float(np.asarray(ft(np.array([t])))[0])


def _beta(prob, X, V, t=0.0):
    """beta_p(t, x, v) on all point pairs: (2d, nx, nv)."""
    out = []
    for b in prob.beta:
        fx = b.fx(X) if b.fx is not None else np.ones(X.shape[0])
        fv = b.fv(V) if b.fv is not None else np.ones(V.shape[0])
        out.append(b.coef * _tf(b, t) * np.outer(fx, fv))
    return np.array(out)


def _sigma(prob, X, V, t=0.0):
    s = prob.sigma
    fx = s.fx(X) if s.fx is not None else np.ones(X.shape[0])
    fv = s.fv(V) if s.fv is not None else np.ones(V.shape[0])
    return s.coef * _tf(s, t) * np.outer(fx, fv)


def full_matrix(prob, Lx: int, Lv: int, q: int = 4, t0: float = 0.0) -> np.ndarray:
    """The strip (t0, t0 + dt); beta and sigma evaluated at every time
    quadrature point (3-point Gauss-Legendre for r = 1), pointwise in
    (t, x, v), Gamma^- included."""
    d, R, dt, dl = prob.d, prob.r + 1, prob.dt, prob.delta
    hx, hv = Hierarchy(prob.mesh_x, Lx), Hierarchy(prob.mesh_v, Lv)
    lx, lv = hx.levels[Lx], hv.levels[Lv]
    n1, n2 = lx.n, lv.n
    N = n1 * n2 * R
    A = np.zeros((N, N))
    tq, tw = gauss01(R + 1)
    et = np.array([eta(s, tq, dt)[0] for s in range(R)])   # (R, nt)
    ed = np.array([eta(s, tq, dt)[1] for s in range(R)])
    tw = tw * dt
    px, wx, lamx, gx = _cell_data(lx, q)
    pv, wv, lamv, gv = _cell_data(lv, q)
    ncx, ncv = px.shape[0], pv.shape[0]
    d1 = d + 1

    def dofs(cx, cv):
        i = lx.cells[cx][:, None, None]
        j = lv.cells[cv][None, :, None]
        s = np.arange(R)[None, None, :]
        return ((i * n2 + j) * R + s).ravel()

    tabs = t0 + tq * dt                                  # absolute time points
    for cx in range(ncx):
        for cv in range(ncv):
            B = np.array([_beta(prob, px[cx], pv[cv], t) for t in tabs])    # (nt, 2d, qx, qv)
            S = np.array([_sigma(prob, px[cx], pv[cv], t) for t in tabs])   # (nt, qx, qv)
            W = np.outer(wx[cx], wv[cv])               # (qx, qv)
            # basis product values phi = lamx[qx,a] lamv[qv,b]; shape (qx,qv,a,b)
            phi = np.einsum("xa,vb->xvab", lamx, lamv)
            # beta . grad of the spatial basis functions at every time point: (nt, qx, qv, a, b)
            bg = np.einsum("tpxv,ap->txva", B[:, :d], gx[cx])[..., None] * lamv[None, None, :, None, :]
            bg = bg + lamx[None, :, None, :, None] * np.einsum("tpxv,bp->txvb", B[:, d:], gv[cv])[:, :, :, None, :]
            # time: L(Phi') = eta' phi + eta (bg + sigma phi);  W(Phi) = eta phi + dl (eta' phi + eta bg)
            Lop = (np.einsum("st,xvab->txvsab", ed, phi)
                   + np.einsum("st,txvab->txvsab", et, bg + S[..., None, None] * phi))
            Wop = (np.einsum("st,xvab->txvsab", et, phi)
                   + dl * (np.einsum("st,xvab->txvsab", ed, phi) + np.einsum("st,txvab->txvsab", et, bg)))
            wts = tw[:, None, None] * W[None]
            # sum over the quadrature points (t, x, v) of wts * Wop[s, a, b] * Lop[S, A, B]: a
            # matrix product over the points, rows test (s, a, b), columns trial (S, A, B)
            npt = wts.size
            Wm = Wop.reshape(npt, R * d1 * d1) * wts.reshape(npt, 1)
            loc = Wm.T @ Lop.reshape(npt, R * d1 * d1)
            # reorder to test (a, b, s) x trial (A, B, S), the dof order
            loc = loc.reshape(R, d1, d1, R, d1, d1).transpose(1, 2, 0, 4, 5, 3).reshape(d1 * d1 * R, d1 * d1 * R)
            idx = dofs(cx, cv)
            A[np.ix_(idx, idx)] += loc

    # initial term (v^+, w^+) at t_{j-1}
    e0 = np.array([eta(s, np.array([0.0]), dt)[0][0] for s in range(R)])
    for cx in range(ncx):
        for cv in range(ncv):
            W = np.outer(wx[cx], wv[cv])
            phi = np.einsum("xa,vb->xvab", lamx, lamv)
            m = np.einsum("xv,xvab,xvAB->abAB", W, phi, phi)
            loc = np.einsum("abAB,s,S->absABS", m, e0, e0).reshape(d1 * d1 * R, d1 * d1 * R)
            idx = dofs(cx, cv)
            A[np.ix_(idx, idx)] += loc

    # inflow boundary: - int_I int_{Gamma^-} (beta . n) v w
    for side_of, lev_b, lev_o, pts_o, w_o, lam_o, is_x in (
            ("x", lx, lv, pv, wv, lamv, True), ("v", lv, lx, px, wx, lamx, False)):
        if lev_b.bfaces.shape[0] == 0:
            continue
        pf, wf, lamf = _face_data(lev_b, q)
        for f in range(lev_b.bfaces.shape[0]):
            ax, sd = lev_b.bface_axis[f], lev_b.bface_side[f]
            for co in range(lev_o.cells.shape[0]):
                if is_x:
                    B = np.array([_beta(prob, pf[f], pts_o[co], t) for t in tabs])   # (nt, 2d, qf, qo)
                    bn = sd * B[:, ax]
                    phi = np.einsum("fa,ob->foab", lamf, lam_o)
                    W = np.outer(wf[f], w_o[co])
                    di = lev_b.bfaces[f][:, None, None]
                    dj = lev_o.cells[co][None, :, None]
                else:
                    B = np.array([_beta(prob, pts_o[co], pf[f], t) for t in tabs])   # (nt, 2d, qo, qf)
                    bn = sd * np.transpose(B[:, d + ax], (0, 2, 1))                  # (nt, qf, qo)
                    phi = np.einsum("fb,oa->foab", lamf, lam_o)
                    W = np.outer(wf[f], w_o[co])
                    di = lev_o.cells[co][:, None, None]
                    dj = lev_b.bfaces[f][None, :, None]
                inflow = (bn < 0.0).astype(float)                       # Gamma^- at every time point
                g = W[None] * bn * inflow                               # (nt, qf, qo)
                m = np.einsum("tfo,foab,foAB->tabAB", g, phi, phi)
                loc = -np.einsum("tabAB,t,st,St->absABS", m, tw, et, et)
                a_n, b_n = m.shape[1], m.shape[2]
                loc = loc.reshape(a_n * b_n * R, a_n * b_n * R)
                idx = ((di * n2 + dj) * R + np.arange(R)[None, None, :]).ravel()
                A[np.ix_(idx, idx)] += loc
    return A


def energy_terms(prob, Lx: int, Lv: int, u: np.ndarray, q: int = 4) -> float:
    """RHS of the sigma = 0 energy identity for one strip (Sect. 3):
    int_I 1/2 |v|^2_{dOmega} + delta ||d_t v + d_beta v||^2 dt
    + 1/2 ||v(t_{j-1}^+)||^2 + 1/2 ||v(t_j^-)||^2, by direct quadrature."""
    d, R, dt, dl = prob.d, prob.r + 1, prob.dt, prob.delta
    hx, hv = Hierarchy(prob.mesh_x, Lx), Hierarchy(prob.mesh_v, Lv)
    lx, lv = hx.levels[Lx], hv.levels[Lv]
    n1, n2 = lx.n, lv.n
    U = u.reshape(n1, n2, R)
    tq, tw = gauss01(R + 1)
    et = np.array([eta(s, tq, dt)[0] for s in range(R)])
    ed = np.array([eta(s, tq, dt)[1] for s in range(R)])
    tw = tw * dt
    e0 = np.array([eta(s, np.array([0.0]), dt)[0][0] for s in range(R)])
    e1 = np.array([eta(s, np.array([1.0]), dt)[0][0] for s in range(R)])
    px, wx, lamx, gx = _cell_data(lx, q)
    pv, wv, lamv, gv = _cell_data(lv, q)
    total = 0.0
    for cx in range(px.shape[0]):
        for cv in range(pv.shape[0]):
            Uc = U[np.ix_(lx.cells[cx], lv.cells[cv])]                # (a, b, s)
            B = _beta(prob, px[cx], pv[cv])
            W = np.outer(wx[cx], wv[cv])
            val = np.einsum("xa,vb,abs->xvs", lamx, lamv, Uc)         # spatial value per time coef
            dxv = np.einsum("pxv,ap,vb,abs->xvs", B[:d], gx[cx], lamv, Uc, optimize=True)
            dvv = np.einsum("pxv,bp,xa,abs->xvs", B[d:], gv[cv], lamx, Uc, optimize=True)
            bgrad = dxv + dvv
            # d_t v + d_beta v at time points
            res = np.einsum("st,xvs->txv", ed, val) + np.einsum("st,xvs->txv", et, bgrad)
            total += dl * np.einsum("t,xv,txv->", tw, W, res ** 2)
            v0 = np.einsum("s,xvs->xv", e0, val)
            v1 = np.einsum("s,xvs->xv", e1, val)
            total += 0.5 * np.einsum("xv,xv->", W, v0 ** 2) + 0.5 * np.einsum("xv,xv->", W, v1 ** 2)
    for lev_b, lev_o, pts_o, w_o, lam_o, is_x in ((lx, lv, pv, wv, lamv, True), (lv, lx, px, wx, lamx, False)):
        if lev_b.bfaces.shape[0] == 0:
            continue
        pf, wf, lamf = _face_data(lev_b, q)
        for f in range(lev_b.bfaces.shape[0]):
            ax, sd = lev_b.bface_axis[f], lev_b.bface_side[f]
            for co in range(lev_o.cells.shape[0]):
                if is_x:
                    B = _beta(prob, pf[f], pts_o[co])
                    bn = sd * B[ax]
                    Uc = U[np.ix_(lev_b.bfaces[f], lev_o.cells[co])]
                    val = np.einsum("fa,ob,abs->fos", lamf, lam_o, Uc)
                else:
                    B = _beta(prob, pts_o[co], pf[f])
                    bn = sd * B[d + ax].T
                    Uc = U[np.ix_(lev_o.cells[co], lev_b.bfaces[f])]
                    val = np.einsum("fb,oa,abs->fos", lamf, lam_o, Uc)
                W = np.outer(wf[f], w_o[co])
                vt = np.einsum("st,fos->tfo", et, val)
                total += 0.5 * np.einsum("t,fo,fo,tfo->", tw, W, np.abs(bn), vt ** 2)
    return total
