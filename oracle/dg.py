"""Oracle DG right-hand side, time stepping and diagnostics.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

PDE (Section 2): (1/kappa) p_t + div u = 0,  rho u_t + grad p = 0, kappa = rho c^2,
piecewise constant per element.  Strong DG form, eq. (1):

  int (1/kappa) p_t phi = -int (div u) phi + oint 1/2 (tau_p [p] - n.[u]) phi
  int rho u_t . psi     = -int grad p . psi + oint 1/2 (tau_u [u].n - [p]) psi.n

with [p] = p+ - p-, tau_p = 1/{rho c}, tau_u = {rho c} (upwind) or 0
(central), {rho c} the average of both sides (the boundary ghost carries the
interior value).  Boundary ghosts (Section 2 and the rigid-wall variant):
Dirichlet p+ = -p-, u+ = u-;  rigid p+ = p-, u+ = u- - 2 (n.u-) n.
The volume terms carry the minus sign of eq. (1) (the discrete equations of
Section 2.1 print them without it).

Two independent evaluations of the same semi-discretisation:

* `rhs_brute` (Section 2.1, plain definition): per element the full Np x Np
  mass, weak-derivative and face-mass matrices by quadrature of the generic
  vertex map (Jacobian matrix, determinant and inverse at every point), then
  M^{-1}(...).  Small meshes only.
* `rhs` (Section 4.2, method form): Lemma 3.1 geometric factors, the
  Kronecker identities
      D_x = (r_x D_r + s_x D_s) (x) I + L^tri (x) diag(t_x J) D_t, ...,
      D_z = L^tri (x) t_z J D_t,
      tri-face lift  J_f L^tri (x) (M^1D)^{-1} e,
      quad-face lift (M^tri)^{-1} M~_edge (x) I,
  with L^tri = (M^tri)^{-1} M^tri_hat and M^tri = sum_a J_a M_a (J is linear
  in r, s), applied slice by slice; tets use the affine reference operators.

Both share only the face-node fluxes.  Field layout: q[4][total_nodes]
(p, ux, uy, uz), canonical node order (see oracle.mesh).
"""
from __future__ import annotations

import numpy as np

from . import reference as R
from .mesh import Connectivity, WEDGE, TET

BC_DIRICHLET = "dirichlet"
BC_RIGID = "rigid"


class Solver:
    def __init__(self, VX, EToV, etype, N: int, c2=None, rho=None,
                 bc: str = BC_RIGID, flux: str = "upwind", lumped: bool = False):
        self.conn = C = Connectivity(VX, EToV, etype, N)
        self.N = N
        self.K = C.K
        self.bc = bc
        self.flux = flux
        self.lumped = lumped
        c2 = np.ones(self.K) if c2 is None else np.asarray(c2, dtype=np.float64)
        rho = np.ones(self.K) if rho is None else np.asarray(rho, dtype=np.float64)
        self.c2, self.rho = c2, rho
        self.kappa = rho * c2
        self.rhoc = rho * np.sqrt(c2)
        self.W, self.T = C.W, C.T
        self.sources = []   # (element, g = kappa M^{-1} l(x_s), f0, t0, amp)
        self._wedge_geometry()
        self._tet_geometry()
        self._face_tables()

    # ------------------------------------------------------------------
    # geometry (Lemma 3.1 for wedges, affine for tets)
    # ------------------------------------------------------------------
    def _wedge_geometry(self):
        C = self.conn
        w = C.wedges
        self.Kw = len(w)
        if self.Kw == 0:
            return
        V = C.VX[C.EToV[w, :6]]                       # (Kw, 6, 3)
        x = V[:, :3, 0]
        y = V[:, :3, 1]
        z = V[:, :, 2]
        xr, xs = (x[:, 1] - x[:, 0]) / 2, (x[:, 2] - x[:, 0]) / 2
        yr, ys = (y[:, 1] - y[:, 0]) / 2, (y[:, 2] - y[:, 0]) / 2
        A = xr * ys - xs * yr
        h = z[:, 3:6] - z[:, 0:3]                     # column heights
        g = {}
        g["A"] = A
        g["Ja"] = A[:, None] * h / 2                  # J at the three columns
        g["rx"], g["ry"] = ys / A, -xs / A
        g["sx"], g["sy"] = -yr / A, xr / A
        t = self.W.line.x
        zeta = lambda a: ((1 - t)[None, :] / 2) * z[:, a, None] + ((1 + t)[None, :] / 2) * z[:, a + 3, None]
        zr = (zeta(1) - zeta(0)) / 2                  # (Kw, Nq)
        zs = (zeta(2) - zeta(0)) / 2
        g["txJ"] = yr[:, None] * zs - zr * ys[:, None]
        g["tyJ"] = zr * xs[:, None] - xr[:, None] * zs
        # faces: normals and Jacobians (constant on every face except the
        # quad J_f, which is linear along the edge)
        P = V
        cb = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
        ct = np.cross(P[:, 4] - P[:, 3], P[:, 5] - P[:, 3])
        nb = np.linalg.norm(cb, axis=1)
        nt = np.linalg.norm(ct, axis=1)
        g["n_bot"] = -cb / nb[:, None]
        g["n_top"] = ct / nt[:, None]
        g["Jf_bot"] = nb / 4
        g["Jf_top"] = nt / 4
        nq = np.zeros((self.Kw, 3, 3))
        Le = np.zeros((self.Kw, 3))
        for e, (a, b) in enumerate(self.W.tri.edge_vertices):
            dx = x[:, b] - x[:, a]
            dy = y[:, b] - y[:, a]
            Le[:, e] = np.hypot(dx, dy)
            nq[:, e, 0] = dy / Le[:, e]
            nq[:, e, 1] = -dx / Le[:, e]
        g["n_quad"] = nq
        g["Le"] = g_le = Le
        g["h"] = h
        vol = (2.0 / 3.0) * A * h.sum(axis=1)
        areas = [nb / 2, nt / 2] + [g_le[:, e] * (h[:, a] + h[:, b]) / 2
                                     for e, (a, b) in enumerate(self.W.tri.edge_vertices)]
        g["vol"] = vol
        g["area"] = np.stack(areas, axis=1)
        self.wg = g

    def _tet_geometry(self):
        C = self.conn
        tt = C.tets
        self.Kt = len(tt)
        if self.Kt == 0:
            return
        V = C.VX[C.EToV[tt, :4]]                      # (Kt, 4, 3)
        G = np.stack([V[:, 1] - V[:, 0], V[:, 2] - V[:, 0], V[:, 3] - V[:, 0]], axis=2) / 2  # dx_d/dr_m
        J = np.linalg.det(G)
        Ginv = np.linalg.inv(G)                       # dr_m/dx_d
        g = {"J": J, "Ginv": Ginv}
        n = np.zeros((self.Kt, 4, 3))
        Jf = np.zeros((self.Kt, 4))
        cen = V.mean(axis=1)
        for f, fv in enumerate(R.Tet.FACE_VERTS):
            c = np.cross(V[:, fv[1]] - V[:, fv[0]], V[:, fv[2]] - V[:, fv[0]])
            nn = np.linalg.norm(c, axis=1)
            c = c / nn[:, None]
            sgn = np.sign(np.einsum("kd,kd->k", c, V[:, fv[0]] - cen))
            n[:, f] = c * sgn[:, None]
            Jf[:, f] = nn / 4
        g["n"] = n
        g["Jf"] = Jf
        g["vol"] = J * 4.0 / 3.0
        g["area"] = 2 * Jf
        self.tg = g

    # ------------------------------------------------------------------
    # face tables (vectorised gather indices)
    # ------------------------------------------------------------------
    def _face_tables(self):
        C = self.conn
        self.ftab = {}
        for (typ, elems, nf) in ((WEDGE, C.wedges, 5), (TET, C.tets, 4)):
            for f in range(nf):
                if len(elems) == 0:
                    continue
                gM = np.stack([C.vmapM[(k, f)] for k in elems])
                gP = np.stack([C.vmapP[(k, f)] for k in elems])
                nbr = C.EToE[elems, f]
                self.ftab[(typ, f)] = (gM, gP, nbr)

    def _normal(self, typ, f):
        if typ == WEDGE:
            if f == 0:
                return self.wg["n_bot"]
            if f == 1:
                return self.wg["n_top"]
            return self.wg["n_quad"][:, f - 2]
        return self.tg["n"][:, f]

    def face_flux(self, q, typ, f, normal):
        """Penalty fluxes F_p, F_u at the face nodes of face f of every
        element of type `typ` (eq. (1)); normal: (Ke, 3) outward unit normal."""
        gM, gP, nbr = self.ftab[(typ, f)]
        elems = self.conn.wedges if typ == WEDGE else self.conn.tets
        bnd = nbr < 0
        n = normal[:, None, :]                        # (Ke, 1, 3)
        pM = q[0, gM]
        uM = np.stack([q[1, gM], q[2, gM], q[3, gM]], axis=2)
        pP = q[0, gP].copy()
        uP = np.stack([q[1, gP], q[2, gP], q[3, gP]], axis=2)
        unM = np.sum(uM * n, axis=2)
        if np.any(bnd):
            if self.bc == BC_DIRICHLET:
                pP[bnd] = -pM[bnd]
                uP[bnd] = uM[bnd]
            else:
                pP[bnd] = pM[bnd]
                uP[bnd] = uM[bnd] - 2 * unM[bnd][:, :, None] * n[bnd]
        unP = np.sum(uP * n, axis=2)
        zM = self.rhoc[elems]
        zP = np.where(bnd, zM, self.rhoc[np.where(bnd, elems, nbr)])
        zavg = 0.5 * (zM + zP)
        if self.flux == "upwind":
            tau_p, tau_u = 1.0 / zavg, zavg
        else:
            tau_p, tau_u = np.zeros_like(zavg), np.zeros_like(zavg)
        dp = pP - pM
        dun = unP - unM
        Fp = 0.5 * (tau_p[:, None] * dp - dun)
        Fu = 0.5 * (tau_u[:, None] * dun - dp)
        return Fp, Fu

    # ------------------------------------------------------------------
    # point sources (pressure equation; not part of the paper)
    # ------------------------------------------------------------------
    def reference_coords(self, k: int, x) -> np.ndarray:
        """Invert the vertex map of element k at physical point x by Newton
        iteration on the generic map (no Lemma 3.1 shortcut)."""
        C = self.conn
        wedge = C.etype[k] == WEDGE
        vf = R.wedge_vertex_functions if wedge else R.tet_vertex_functions
        verts = C.VX[C.EToV[k, :6 if wedge else 4]]
        X = np.array([[-1.0 / 3, -1.0 / 3, 0.0]]) if wedge else np.array([[-0.5, -0.5, -0.5]])
        for _ in range(50):
            v, gv = vf(X)
            F = v[0] @ verts - np.asarray(x, dtype=np.float64)
            G = np.einsum("vm,vd->dm", gv[0], verts)
            dX = np.linalg.solve(G, F)
            X = X - dX
            if np.max(np.abs(dX)) < 1e-15:
                break
        return X[0]

    def _inside(self, k: int, X, tol: float = 1e-12) -> bool:
        r, s, t = X
        if self.conn.etype[k] == WEDGE:
            return r >= -1 - tol and s >= -1 - tol and r + s <= tol and abs(t) <= 1 + tol
        return r >= -1 - tol and s >= -1 - tol and t >= -1 - tol and r + s + t <= -1 + tol

    def add_source(self, x, y, z, f0: float, t0: float, amp: float):
        """rhs_p += amp R(t) kappa_k M_k^{-1} l(x_s) in the lowest-id element
        containing (x, y, z); R is the Ricker wavelet (1 - 2a) e^{-a},
        a = (pi f0 (t - t0))^2."""
        for k in range(self.K):
            X = self.reference_coords(k, (x, y, z))
            if not self._inside(k, X):
                continue
            ref = self.W if self.conn.etype[k] == WEDGE else self.T
            ell = ref.eval(X[None, :])[0]
            M, _, _ = self.element_matrices(k)
            g = self.kappa[k] * np.linalg.solve(M, ell)
            self.sources.append((k, g, f0, t0, amp))
            return k
        raise ValueError("source point outside the mesh")

    @staticmethod
    def ricker(f0: float, tau: float) -> float:
        a = (np.pi * f0 * tau) ** 2
        return (1.0 - 2.0 * a) * np.exp(-a)

    # ------------------------------------------------------------------
    # method form (Section 4.2)
    # ------------------------------------------------------------------
    def rhs(self, q: np.ndarray, t: float = 0.0) -> np.ndarray:
        q = np.asarray(q, dtype=np.float64)
        out = np.zeros_like(q)
        if self.Kw:
            self._rhs_wedge(q, out)
        if self.Kt:
            self._rhs_tet(q, out)
        self._add_sources(out, t)
        return out

    def _add_sources(self, out, t):
        C = self.conn
        for (k, g, f0, t0, amp) in self.sources:
            out[0, C.offset[k]:C.offset[k + 1]] += amp * self.ricker(f0, t - t0) * g

    def wedge_tri_mass(self):
        """M^{tri,k} = sum_a J_a M_a  (Kw, Nt, Nt)."""
        Ma = np.stack(self.W.tri.Ma)                 # (3, Nt, Nt)
        return np.einsum("ka,aij->kij", self.wg["Ja"], Ma)

    def _rhs_wedge(self, q, out):
        W, g = self.W, self.wg
        tri, line = W.tri, W.line
        Nt, Nq = W.Nt, W.Nq
        C = self.conn
        idx = C.offset[C.wedges][:, None] + np.arange(W.Np)[None, :]
        Q = q[:, idx].reshape(4, self.Kw, Nq, Nt)          # [field, k, j, i]
        p, ux, uy, uz = Q
        rx, ry, sx, sy, A = (g[k][:, None, None] for k in ("rx", "ry", "sx", "sy", "A"))
        tri_apply = lambda M, f: np.einsum("il,kjl->kji", M, f)
        line_apply = lambda M, f: np.einsum("jm,kmi->kji", M, f)
        # strong r/s parts (per slice)
        pr, ps = tri_apply(tri.Dr, p), tri_apply(tri.Ds, p)
        Vp = -(tri_apply(tri.Dr, rx * ux + ry * uy) + tri_apply(tri.Ds, sx * ux + sy * uy))
        Vu = [-(rx * pr + sx * ps), -(ry * pr + sy * ps), np.zeros_like(p)]
        # t parts, to be hit by L^tri
        txJ = g["txJ"][:, :, None]
        tyJ = g["tyJ"][:, :, None]
        pt = line_apply(line.D, p)
        Tp = -(txJ * line_apply(line.D, ux) + tyJ * line_apply(line.D, uy) + A * line_apply(line.D, uz))
        Tu = [-txJ * pt, -tyJ * pt, -A * pt]
        # face fluxes
        Fb = self.face_flux(q, WEDGE, 0, g["n_bot"])
        Ft = self.face_flux(q, WEDGE, 1, g["n_top"])
        if self.lumped:
            e0 = np.zeros(Nq)
            eN = np.zeros(Nq)
            e0[0] = 1.0 / line.w[0]
            eN[-1] = 1.0 / line.w[-1]
        else:
            e0, eN = line.ell0, line.ellN
        Jb = g["Jf_bot"][:, None, None]
        Jt = g["Jf_top"][:, None, None]
        tri_face = lambda Fb_, Ft_, cb, ct: (Jb * cb * e0[None, :, None] * Fb_[:, None, :]
                                             + Jt * ct * eN[None, :, None] * Ft_[:, None, :])
        Gp = Tp + tri_face(Fb[0], Ft[0], 1.0, 1.0)
        Gu = [Tu[c] + tri_face(Fb[1], Ft[1], g["n_bot"][:, c, None, None], g["n_top"][:, c, None, None])
              for c in range(3)]
        Wp = tri_apply(tri.M, Gp)
        Wu = [tri_apply(tri.M, Gu[c]) for c in range(3)]
        # quad faces: M~_e = (L_e/2)(h_a/2 Ma + h_b/2 Mb) along the edge, identity in t
        for e, (a, b) in enumerate(tri.edge_vertices):
            Fp, Fu = self.face_flux(q, WEDGE, 2 + e, g["n_quad"][:, e])
            Fp = Fp.reshape(self.Kw, Nq, Nq)           # [k, j, m]
            Fu = Fu.reshape(self.Kw, Nq, Nq)
            Mt = (g["Le"][:, e, None, None] / 2) * (g["h"][:, a, None, None] / 2 * line.Ma[None]
                                                     + g["h"][:, b, None, None] / 2 * line.Mb[None])
            Gp_e = np.einsum("kmn,kjn->kjm", Mt, Fp)
            Gu_e = np.einsum("kmn,kjn->kjm", Mt, Fu)
            en = tri.edges[e]
            for m in range(Nq):
                Wp[:, :, en[m]] += Gp_e[:, :, m]
                for c in range(2):
                    Wu[c][:, :, en[m]] += g["n_quad"][:, e, c, None] * Gu_e[:, :, m]
        # exact inverse of the Jacobian-weighted mass: (M^tri)^{-1} per slice
        Mk = self.wedge_tri_mass()
        Minv = np.linalg.inv(Mk)
        solve = lambda Wf: np.einsum("kil,kjl->kji", Minv, Wf)
        kap = self.kappa[C.wedges][:, None, None]
        irho = 1.0 / self.rho[C.wedges][:, None, None]
        rp = kap * (Vp + solve(Wp))
        ru = [irho * (Vu[c] + solve(Wu[c])) for c in range(3)]
        R_ = np.stack([rp] + ru).reshape(4, self.Kw, W.Np)
        out[:, idx] = R_

    def _rhs_tet(self, q, out):
        T, g = self.T, self.tg
        C = self.conn
        idx = C.offset[C.tets][:, None] + np.arange(T.Np)[None, :]
        Q = q[:, idx]                                       # (4, Kt, Np)
        Gi = g["Ginv"]                                      # (Kt, m, d)
        Dref = np.stack([T.Dr, T.Ds, T.Dt])                 # (3, Np, Np)
        dref = lambda f: np.einsum("mij,kj->kmi", Dref, f)  # (Kt, m, Np)
        grad = lambda f: np.einsum("kmd,kmi->kdi", Gi, dref(f))
        gp = grad(Q[0])
        div = sum(grad(Q[1 + c])[:, c] for c in range(3))
        rp = -div
        ru = [-gp[:, c] for c in range(3)]
        Minv = np.linalg.inv(T.M)
        for f in range(4):
            Fp, Fu = self.face_flux(q, TET, f, g["n"][:, f])
            lift = Minv[:, T.faces[f]] @ self.W.tri.M       # (Np, Nfp)
            s = (g["Jf"][:, f] / g["J"])[:, None]
            rp = rp + s * (Fp @ lift.T)
            for c in range(3):
                ru[c] = ru[c] + s * g["n"][:, f, c, None] * (Fu @ lift.T)
        kap = self.kappa[C.tets][:, None]
        irho = 1.0 / self.rho[C.tets][:, None]
        out[0][idx] = kap * rp
        for c in range(3):
            out[1 + c][idx] = irho * ru[c]

    # ------------------------------------------------------------------
    # brute-force form (Section 2.1)
    # ------------------------------------------------------------------
    def element_matrices(self, k: int):
        """Full-quadrature M, S_x, S_y, S_z and per-face (face nodes, M_f[:, face nodes],
        unit normal) for element k, from the generic vertex map."""
        C = self.conn
        N = self.N
        if C.etype[k] == WEDGE:
            ref = self.W
            Xq, wq = R.wedge_quadrature(N + 3)
            vf = R.wedge_vertex_functions
            verts = C.VX[C.EToV[k, :6]]
        else:
            ref = self.T
            Xq, wq = R.tet_quadrature(N + 3)
            vf = R.tet_vertex_functions
            verts = C.VX[C.EToV[k, :4]]
        _, gv = vf(Xq)
        G = np.einsum("qvm,vd->qdm", gv, verts)              # dx_d/dr_m
        J = np.linalg.det(G)
        Gi = np.linalg.inv(G)                                # dr_m/dx_d
        L = ref.eval(Xq)
        dL = np.stack(ref.grad(Xq))                          # (3, q, Np) in r,s,t
        dLx = np.einsum("qmd,mqj->dqj", Gi, dL)
        wJ = wq * J
        M = L.T @ (wJ[:, None] * L)
        S = [L.T @ (wJ[:, None] * dLx[d]) for d in range(3)]
        cen = verts.mean(axis=0)
        faces = []
        for f in range(C.nfaces(k)):
            Xf, wf, tu, tv = self._ref_face_quadrature(C.etype[k], f, N + 3)
            _, gvf = vf(Xf)
            Gf = np.einsum("qvm,vd->qdm", gvf, verts)
            T1 = np.einsum("qdm,m->qd", Gf, tu)
            T2 = np.einsum("qdm,m->qd", Gf, tv)
            cr = np.cross(T1, T2)
            dA = np.linalg.norm(cr, axis=1)
            nrm = cr[0] / dA[0]
            xf = np.einsum("qv,vd->qd", vf(Xf)[0], verts)
            if np.dot(nrm, xf[0] - cen) < 0:
                nrm = -nrm
            Lf = ref.eval(Xf)
            fn = C.face_nodes(k, f)
            Mf = Lf.T @ ((wf * dA)[:, None] * Lf[:, fn])
            faces.append((fn, Mf, nrm))
        return M, S, faces

    @staticmethod
    def _ref_face_quadrature(etype, f, q):
        """Quadrature on reference face f: points X (in element reference
        coordinates), weights, and the two reference tangent vectors."""
        if etype == WEDGE:
            if f in (0, 1):
                Xt, wt = R.tri_quadrature(q)
                tz = -1.0 if f == 0 else 1.0
                X = np.column_stack([Xt, np.full(len(wt), tz)])
                return X, wt, np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
            tv = np.array([[-1.0, -1.0], [1.0, -1.0], [-1.0, 1.0]])
            a, b = ((0, 1), (1, 2), (2, 0))[f - 2]
            x1, w1 = R.gauss(q)
            S_, Tt = np.meshgrid(x1, x1, indexing="ij")
            WS, WT = np.meshgrid(w1, w1, indexing="ij")
            sg, tg = S_.ravel(), Tt.ravel()
            rs = tv[a][None, :] + (tv[b] - tv[a])[None, :] * ((1 + sg) / 2)[:, None]
            X = np.column_stack([rs, tg])
            d = (tv[b] - tv[a]) / 2
            return X, (WS * WT).ravel(), np.array([d[0], d[1], 0.0]), np.array([0, 0, 1.0])
        # tet faces parametrised over the bi-unit triangle by their vertices
        tv = np.array([[-1.0, -1, -1], [1.0, -1, -1], [-1.0, 1, -1], [-1.0, -1, 1]])
        fv = R.Tet.FACE_VERTS[f]
        Xt, wt = R.tri_quadrature(q)
        l1 = -(Xt[:, 0] + Xt[:, 1]) / 2
        l2 = (1 + Xt[:, 0]) / 2
        l3 = (1 + Xt[:, 1]) / 2
        X = l1[:, None] * tv[fv[0]] + l2[:, None] * tv[fv[1]] + l3[:, None] * tv[fv[2]]
        tu = (tv[fv[1]] - tv[fv[0]]) / 2
        tw = (tv[fv[2]] - tv[fv[0]]) / 2
        return X, wt, tu, tw

    def brute_setup(self):
        if getattr(self, "_brute", None) is None:
            self._brute = [self.element_matrices(k) for k in range(self.K)]
        return self._brute

    def rhs_brute(self, q: np.ndarray, t: float = 0.0) -> np.ndarray:
        C = self.conn
        mats = self.brute_setup()
        q = np.asarray(q, dtype=np.float64)
        out = np.zeros_like(q)
        for k in range(self.K):
            M, S, faces = mats[k]
            sl = slice(C.offset[k], C.offset[k + 1])
            p, ux, uy, uz = q[0, sl], q[1, sl], q[2, sl], q[3, sl]
            bp = -(S[0] @ ux + S[1] @ uy + S[2] @ uz)
            bu = [-(S[c] @ p) for c in range(3)]
            for f, (fn, Mf, nrm) in enumerate(faces):
                Fp, Fu = self._single_face_flux(q, k, f, nrm)
                bp = bp + Mf @ Fp
                for c in range(3):
                    bu[c] = bu[c] + nrm[c] * (Mf @ Fu)
            out[0, sl] = self.kappa[k] * np.linalg.solve(M, bp)
            for c in range(3):
                out[1 + c, sl] = np.linalg.solve(M, bu[c]) / self.rho[k]
        self._add_sources(out, t)
        return out

    def _single_face_flux(self, q, k, f, nrm):
        C = self.conn
        gM = C.vmapM[(k, f)]
        gP = C.vmapP[(k, f)]
        k2 = C.EToE[k, f]
        pM = q[0, gM]
        uM = q[1:4, gM]
        unM = nrm @ uM
        if k2 < 0:
            if self.bc == BC_DIRICHLET:
                pP, uP = -pM, uM
            else:
                pP, uP = pM, uM - 2 * np.outer(nrm, unM)
            zP = self.rhoc[k]
        else:
            pP, uP = q[0, gP], q[1:4, gP]
            zP = self.rhoc[k2]
        unP = nrm @ uP
        zavg = 0.5 * (self.rhoc[k] + zP)
        tau_p, tau_u = (1.0 / zavg, zavg) if self.flux == "upwind" else (0.0, 0.0)
        dp = pP - pM
        dun = unP - unM
        return 0.5 * (tau_p * dp - dun), 0.5 * (tau_u * dun - dp)

    # ------------------------------------------------------------------
    # energy, mass, dense operator
    # ------------------------------------------------------------------
    def element_mass_method(self):
        """Per-element mass matrices from the Kronecker form (Section 4.2)."""
        C = self.conn
        out = {}
        if self.Kw:
            Mt = self.wedge_tri_mass()
            M1 = np.diag(self.W.line.w) if self.lumped else self.W.line.M
            for n, k in enumerate(C.wedges):
                out[k] = np.kron(M1, Mt[n])                  # slice-major node order
        for n, k in enumerate(C.tets):
            out[k] = self.tg["J"][n] * self.T.M
        return out

    def energy(self, q: np.ndarray) -> float:
        """E = 1/2 sum_k int (p^2/kappa + rho |u|^2) with the scheme's mass
        matrices (Section 4.1)."""
        C = self.conn
        q = np.asarray(q, dtype=np.float64)
        E = 0.0
        Ms = self.element_mass_method()
        for k in range(self.K):
            sl = slice(C.offset[k], C.offset[k + 1])
            M = Ms[k]
            E += q[0, sl] @ M @ q[0, sl] / self.kappa[k]
            E += self.rho[k] * sum(q[c, sl] @ M @ q[c, sl] for c in (1, 2, 3))
        return 0.5 * E

    def energy_weights(self):
        """Block-diagonal energy matrix W with E = 1/2 q^T W q (flattened q)."""
        C = self.conn
        n = C.total_nodes
        Wm = np.zeros((4 * n, 4 * n))
        Ms = self.element_mass_method()
        for k in range(self.K):
            sl = np.arange(C.offset[k], C.offset[k + 1])
            for f in range(4):
                s = 1.0 / self.kappa[k] if f == 0 else self.rho[k]
                ii = f * n + sl
                Wm[np.ix_(ii, ii)] = s * Ms[k]
        return Wm

    def dense_A(self, brute: bool = False) -> np.ndarray:
        n = self.conn.total_nodes
        A = np.zeros((4 * n, 4 * n))
        f = self.rhs_brute if brute else self.rhs
        e = np.zeros((4, n))
        for col in range(4 * n):
            e.flat[col] = 1.0
            A[:, col] = f(e).ravel()
            e.flat[col] = 0.0
        return A

    def face_dissipation(self, q: np.ndarray) -> float:
        """-1/2 sum_interior int (tau_p [p]^2 + tau_u [u_n]^2)
        -1/4 sum_boundary int (same with the ghost jumps): the exact value of
        dE/dt for the semi-discrete scheme (Section 4.1, eq. (2))."""
        C = self.conn
        mats = self.brute_setup()
        total = 0.0
        for k in range(self.K):
            _, _, faces = mats[k]
            for f, (fn, Mf, nrm) in enumerate(faces):
                k2 = C.EToE[k, f]
                gM, gP = C.vmapM[(k, f)], C.vmapP[(k, f)]
                pM, uM = q[0, gM], q[1:4, gM]
                unM = nrm @ uM
                if k2 < 0:
                    if self.bc == BC_DIRICHLET:
                        jp, jun = -2 * pM, np.zeros_like(pM)
                    else:
                        jp, jun = np.zeros_like(pM), -2 * unM
                    zavg = self.rhoc[k]
                    wgt = 0.25
                else:
                    if k2 < k:
                        continue
                    jp = q[0, gP] - pM
                    jun = nrm @ q[1:4, gP] - unM
                    zavg = 0.5 * (self.rhoc[k] + self.rhoc[k2])
                    wgt = 0.5
                tau_p, tau_u = (1.0 / zavg, zavg) if self.flux == "upwind" else (0.0, 0.0)
                Mff = Mf[fn, :]                               # face mass on face nodes
                total -= wgt * (tau_p * jp @ Mff @ jp + tau_u * jun @ Mff @ jun)
        return total

    # ------------------------------------------------------------------
    # time stepping and errors
    # ------------------------------------------------------------------
    def step(self, q: np.ndarray, dt: float, nsteps: int, rhs=None, t0: float = 0.0) -> np.ndarray:
        """LSRK45 (Carpenter-Kennedy 2N-storage), nsteps steps of size dt from
        time t0 (stage times t + c_s dt reach the sources)."""
        return lsrk45(self.rhs if rhs is None else rhs, q, dt, nsteps, t0)

    def stable_dt(self, cfl: float) -> float:
        """dt = CFL * min_k 1 / (c_k (N+1)^2 max_f(area_f / vol_k))."""
        ratios = np.zeros(self.K)
        C = self.conn
        if self.Kw:
            ratios[C.wedges] = self.wg["area"].max(axis=1) / self.wg["vol"]
        if self.Kt:
            ratios[C.tets] = self.tg["area"].max(axis=1) / self.tg["vol"]
        c = np.sqrt(self.c2)
        return float(cfl * np.min(1.0 / (c * (self.N + 1) ** 2 * ratios)))

    def l2_error(self, q: np.ndarray, exact, t: float):
        """Per-field L2 errors against exact(xyz[3][n], t) -> [4][n], by
        quadrature exact for degree 2N+4 on each element."""
        C = self.conn
        N = self.N
        err = np.zeros(4)
        for typ, elems in ((WEDGE, C.wedges), (TET, C.tets)):
            if len(elems) == 0:
                continue
            if typ == WEDGE:
                ref, (Xq, wq), vf, nv = self.W, R.wedge_quadrature(N + 3), R.wedge_vertex_functions, 6
            else:
                ref, (Xq, wq), vf, nv = self.T, R.tet_quadrature(N + 4), R.tet_vertex_functions, 4
            L = ref.eval(Xq)
            v, gv = vf(Xq)
            for k in elems:
                verts = C.VX[C.EToV[k, :nv]]
                xq = (v @ verts).T
                J = np.linalg.det(np.einsum("qvm,vd->qdm", gv, verts))
                qh = q[:, C.offset[k]:C.offset[k + 1]] @ L.T
                d = qh - exact(xq, t)
                err += (d * d) @ (wq * J)
        return np.sqrt(err)


def lsrk45(f, q, dt: float, nsteps: int, t0: float = 0.0):
    """Five-stage fourth-order 2N-storage Runge-Kutta (Carpenter & Kennedy
    1994): per stage res <- a_s res + dt f(q), q <- q + b_s res.  `f` takes
    q, or (q, t) when it accepts two arguments (stage time t + c_s dt)."""
    import inspect
    two = len(inspect.signature(f).parameters) >= 2
    q = np.array(q, copy=True)
    res = np.zeros_like(q)
    t = t0
    for _ in range(nsteps):
        for s in range(5):
            fq = f(q, t + R.LSRK45_C[s] * dt) if two else f(q)
            res = R.LSRK45_A[s] * res + dt * fq
            q = q + R.LSRK45_B[s] * res
        t += dt
    return q
