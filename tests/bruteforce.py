"""Independent brute-force restatement of the mEVP subcycle for tiny meshes.

Written from the mathematics, not from the oracle: numpy's Legendre module
for the quadrature (a 10x10 rule for every linear stage, so its results only
agree with the oracle if the oracle's NGP rule is exact as claimed) and for a
differently normalised DG basis (shifted Legendre P_i(2xi-1) P_j(2eta-1),
i + j <= degree), power-series Lagrange polynomials for Q2, global
vectorised assembly, complex arithmetic for the velocity update.  DG fields
are compared through their values at sample points, which do not depend on
the basis.

The stress update evaluates the nonlinear rheology at the method's own
NGP x NGP Gauss points (the paper's quadrature-based update), so that stage
uses numpy's leggauss(NGP).
"""
import numpy as np
from numpy.polynomial import legendre as Lg
from numpy.polynomial import polynomial as Pl

DEG = {3: 1, 6: 2, 8: 2}
NGP = {3: 2, 6: 3, 8: 3}


def gauss01(n):
    x, w = Lg.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _lagrange():
    nodes = [0.0, 0.5, 1.0]
    out = []
    for a in range(3):
        c = Pl.polyfromroots([nodes[b] for b in range(3) if b != a])
        out.append(c / Pl.polyval(nodes[a], c))
    return out


LAG = _lagrange()
DLAG = [Pl.polyder(c) for c in LAG]


def q2(xi, eta):
    """Values and reference gradients, shape (..., 9); j = a + 3b."""
    lx = [Pl.polyval(xi, c) for c in LAG]
    ly = [Pl.polyval(eta, c) for c in LAG]
    dx = [Pl.polyval(xi, c) for c in DLAG]
    dy = [Pl.polyval(eta, c) for c in DLAG]
    phi = np.stack([lx[a] * ly[b] for b in range(3) for a in range(3)], -1)
    gx = np.stack([dx[a] * ly[b] for b in range(3) for a in range(3)], -1)
    gy = np.stack([lx[a] * dy[b] for b in range(3) for a in range(3)], -1)
    return phi, gx, gy


def dg_bf(n_s, xi, eta):
    """Brute-force DG basis: shifted Legendre products of total degree <= k;
    the 8-dof space is Q2 without the biquadratic product (degree <= 2 in
    each variable, total degree <= 3)."""
    if n_s == 8:
        pairs = [(i, j) for i in range(3) for j in range(3) if i + j <= 3]
    else:
        k = {1: 0, 3: 1, 6: 2}[n_s]
        pairs = [(i, j) for i in range(k + 1) for j in range(k + 1 - i)]
    cols = []
    for i, j in pairs:
        ei = np.zeros(i + 1); ei[i] = 1.0
        ej = np.zeros(j + 1); ej[j] = 1.0
        cols.append(Lg.legval(2 * xi - 1, ei) * Lg.legval(2 * eta - 1, ej))
    return np.stack(cols, -1)


def dg_documented(n_s, xi, eta):
    """The library's documented coefficient convention (xh = xi-1/2, eh = eta-1/2):
    {1, xh, eh, xh^2-1/12, xh eh, eh^2-1/12, (xh^2-1/12) eh, xh (eh^2-1/12)}[:n_s]."""
    xh, eh = xi - 0.5, eta - 0.5
    allb = [np.ones_like(xh), xh, eh, xh * xh - 1 / 12, xh * eh, eh * eh - 1 / 12,
            (xh * xh - 1 / 12) * eh, xh * (eh * eh - 1 / 12)]
    return np.stack(allb[:n_s], -1)


class Mesh:
    def __init__(self, nx, ny, xy, n_s):
        """xy: the vertices [(nx+1)(ny+1)][2] (bilinear element maps), or the
        CG2 node positions [(2nx+1)(2ny+1)][2] (isoparametric Q2 maps; the
        "exact" rule is then the method's own, since curved elements make the
        integrands rational)."""
        self.nx, self.ny, self.n_s = nx, ny, n_s
        self.ne = nx * ny
        self.nw, self.nh = 2 * nx + 1, 2 * ny + 1
        self.nn = self.nw * self.nh
        kx, ky = np.meshgrid(np.arange(nx), np.arange(ny))
        kx, ky = kx.ravel(), ky.ravel()
        self.nodes = np.stack([(2 * ky + b) * self.nw + 2 * kx + a
                               for b in range(3) for a in range(3)], -1)  # (ne, 9)
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        self.iso = xy.shape[0] == self.nn
        if self.iso:
            self.XN = xy[self.nodes]  # (ne, 9, 2)
        else:
            xy = xy.reshape(ny + 1, nx + 1, 2)
            self.X00, self.X10 = xy[ky, kx], xy[ky, kx + 1]
            self.X01, self.X11 = xy[ky + 1, kx], xy[ky + 1, kx + 1]
        self.rule_exact = self._rule(*self._tensor(gauss01(NGP[n_s] if self.iso else 10)))
        self.rule_method = self._rule(*self._tensor(gauss01(NGP[n_s])))
        sp = np.array([0.1, 0.35, 0.6, 0.9])
        XI, ET = np.meshgrid(sp, sp)
        self.sample = (XI.ravel(), ET.ravel())

    @staticmethod
    def _tensor(rule):
        x, w = rule
        XI, ET = np.meshgrid(x, x)
        W = np.outer(w, w)
        return XI.ravel(), ET.ravel(), W.ravel()

    def _map(self, xi, eta):
        """Jacobian entries (ne, nq) of the bilinear or isoparametric map."""
        if self.iso:
            _, gxi, geta = q2(xi, eta)  # (nq, 9)
            dxi = np.einsum("qj,kjc->kqc", gxi, self.XN)
            deta = np.einsum("qj,kjc->kqc", geta, self.XN)
            return dxi[..., 0], deta[..., 0], dxi[..., 1], deta[..., 1]
        X00, X10, X01, X11 = (v[:, None, :] for v in (self.X00, self.X10, self.X01, self.X11))
        e = eta[None, :, None]
        x = xi[None, :, None]
        dxi = (X10 - X00) * (1 - e) + (X11 - X01) * e
        deta = (X01 - X00) * (1 - x) + (X11 - X10) * x
        return dxi[..., 0], deta[..., 0], dxi[..., 1], deta[..., 1]

    def _rule(self, xi, eta, w):
        J00, J01, J10, J11 = self._map(xi, eta)
        det = J00 * J11 - J01 * J10
        phi, gxi, geta = q2(xi, eta)
        # physical gradients (ne, nq, 9)
        dx = (J11[..., None] * gxi[None] - J10[..., None] * geta[None]) / det[..., None]
        dy = (-J01[..., None] * gxi[None] + J00[..., None] * geta[None]) / det[..., None]
        psi = dg_bf(self.n_s, xi, eta)  # (nq, nb)
        wdet = w[None] * det  # (ne, nq)
        M = np.einsum("kq,qs,qt->kst", wdet, psi, psi)
        return dict(xi=xi, eta=eta, wdet=wdet, phi=phi, dx=dx, dy=dy, psi=psi,
                    Minv=np.linalg.inv(M))

    # --- DG conversions ---------------------------------------------------
    def values(self, coef_bf):
        """(3, ne, nb) brute-force coefficients -> values (3, ne, nsample)."""
        psi = dg_bf(self.n_s, *self.sample)
        return np.einsum("cks,qs->ckq", coef_bf, psi)

    def values_documented(self, S):
        """(3, n_s, ne) coefficients in the documented basis -> values (3, ne, nsample)."""
        psi = dg_documented(self.n_s, *self.sample)
        return np.einsum("csk,qs->ckq", S, psi)

    def from_documented(self, S):
        psi_bf = dg_bf(self.n_s, *self.sample)
        vals = self.values_documented(S)
        sol = np.linalg.lstsq(psi_bf, vals.reshape(-1, vals.shape[-1]).T, rcond=None)[0]
        return sol.T.reshape(3, self.ne, -1)

    # --- stages ------------------------------------------------------------
    def strain(self, vel):
        r = self.rule_exact
        u = vel[0][self.nodes]  # (ne, 9)
        v = vel[1][self.nodes]
        ux = np.einsum("kqj,kj->kq", r["dx"], u)
        uy = np.einsum("kqj,kj->kq", r["dy"], u)
        vx = np.einsum("kqj,kj->kq", r["dx"], v)
        vy = np.einsum("kqj,kj->kq", r["dy"], v)
        eps = np.stack([ux, 0.5 * (uy + vx), vy])  # (3, ne, nq)
        rhs = np.einsum("kq,qs,ckq->cks", r["wdet"], r["psi"], eps)
        return np.einsum("kst,ckt->cks", r["Minv"], rhs)

    def ice_at(self, F, rule):
        """Values (ne, nq) at a rule's points of a DG ice field given as
        documented coefficients (n_a, ne); n_a = 1 is the constant."""
        F = np.asarray(F, dtype=np.float64)
        return np.einsum("tk,qt->kq", F, dg_documented(F.shape[0], rule["xi"], rule["eta"]))

    def stress(self, Ebf, H, A, Sbf, p, Pstar_K=None):
        r = self.rule_method
        e = np.einsum("cks,qs->ckq", Ebf, r["psi"])  # (3, ne, nq)
        e11, e12, e22 = e
        # clamps at the Gauss points, after evaluating the (DG) ice fields
        h = np.maximum(0.0, self.ice_at(H, r))
        a = np.clip(self.ice_at(A, r), 0.0, 1.0)
        Ps = p["Pstar"] if Pstar_K is None else np.asarray(Pstar_K, dtype=np.float64)[:, None]
        P = Ps * h * np.exp(-p["C"] * (1.0 - a))
        # Hibler's viscous-plastic law: zeta = P/(2 Delta), eta = zeta/e^2,
        # sigma = 2 eta eps + (zeta - eta) tr(eps) I - P/2 I
        ecc = p["e"]
        delta = np.sqrt(p["DeltaMin"] ** 2 + (e11 ** 2 + e22 ** 2) * (1 + ecc ** -2)
                        + 4 * ecc ** -2 * e12 ** 2 + 2 * (1 - ecc ** -2) * e11 * e22)
        zeta = P / (2 * delta)
        eta = zeta / ecc ** 2
        tr = e11 + e22
        s = np.stack([2 * eta * e11 + (zeta - eta) * tr - P / 2, 2 * eta * e12,
                      2 * eta * e22 + (zeta - eta) * tr - P / 2])
        rhs = np.einsum("kq,qs,ckq->cks", r["wdet"], r["psi"], s)
        proj = np.einsum("kst,ckt->cks", r["Minv"], rhs)
        return (1 - 1 / p["alpha"]) * Sbf + proj / p["alpha"]

    def divergence(self, Sbf):
        r = self.rule_exact
        sig = np.einsum("cks,qs->ckq", Sbf, r["psi"])
        fx = -np.einsum("kq,kq,kqj->kj", r["wdet"], sig[0], r["dx"]) \
             - np.einsum("kq,kq,kqj->kj", r["wdet"], sig[1], r["dy"])
        fy = -np.einsum("kq,kq,kqj->kj", r["wdet"], sig[1], r["dx"]) \
             - np.einsum("kq,kq,kqj->kj", r["wdet"], sig[2], r["dy"])
        F = np.zeros((2, self.nn))
        np.add.at(F[0], self.nodes, fx)
        np.add.at(F[1], self.nodes, fy)
        return F

    def lumped(self, H, rho, rule="exact"):
        """m_j = rho sum_K int_K max(0, H) phi_j, l_j = sum_K int_K phi_j with
        the 10x10 rule ("exact", exact for positive polynomial H) or the
        method's own NGP x NGP rule ("method")."""
        r = self.rule_exact if rule == "exact" else self.rule_method
        h = np.maximum(0.0, self.ice_at(H, r))  # (ne, nq)
        m = np.zeros(self.nn)
        l = np.zeros(self.nn)
        np.add.at(l, self.nodes, np.einsum("kq,qj->kj", r["wdet"], r["phi"]))
        np.add.at(m, self.nodes, rho * np.einsum("kq,kq,qj->kj", r["wdet"], h, r["phi"]))
        return m, l

    def boundary(self):
        ix = np.arange(self.nn) % self.nw
        iy = np.arange(self.nn) // self.nw
        return (ix == 0) | (iy == 0) | (ix == self.nw - 1) | (iy == self.nh - 1)

    def velocity(self, F, vprev, vn, tau, m, l, p, vo=None):
        """Complex form with the ocean velocity z_o (0 when vo is None):
        (m(1+beta)/dt + c + i m f) v = (m/dt)(beta v^{p-1} + v^n) + F + l tau + c z_o,
        c = l Cw rho_w |z_o - v^{p-1}|."""
        z = vprev[0] + 1j * vprev[1]
        zn = vn[0] + 1j * vn[1]
        zo = 0.0 if vo is None else vo[0] + 1j * vo[1]
        c = l * p["Cw"] * p["rho_water"] * np.abs(zo - z)
        lhs = m * (1 + p["beta"]) / p["dt"] + c + 1j * m * p["coriolis_f"]
        rhs = (m / p["dt"] * (p["beta"] * z + zn) + (F[0] + 1j * F[1]) + l * (tau[0] + 1j * tau[1])
               + c * zo)
        out = np.where(lhs != 0, rhs / np.where(lhs != 0, lhs, 1), 0)
        out[self.boundary()] = 0
        return np.stack([out.real, out.imag])

    def subcycles(self, vel0, S0_documented, H, A, tau, p, n_sub, vn=None, vo=None,
                  Pstar_K=None):
        """H, A: documented DG coefficients (n_a, ne).  The lumped mass of DG0
        ice takes the 10x10 rule; of DG1/DG2 ice the method's own rule (the
        reading that integrates the clamped ice field with the stress rule)."""
        vel = np.array(vel0, dtype=np.float64)
        vn = vel.copy() if vn is None else np.asarray(vn)
        S = self.from_documented(S0_documented)
        H = np.asarray(H, dtype=np.float64)
        m, l = self.lumped(H, p["rho_ice"], "exact" if H.shape[0] == 1 else "method")
        E = None
        for _ in range(n_sub):
            E = self.strain(vel)
            S = self.stress(E, H, A, S, p, Pstar_K)
            F = self.divergence(S)
            vel = self.velocity(F, vel, vn, tau, m, l, p, vo)
        return vel, S, E


# --------------------------------------------------------------------------
# Advection (transport of H, A with the CG2 velocity), written independently
# of the oracle: physical gradients through J^-T, physical outward normals of
# the counter-clockwise element boundary (v.n ds = v_x dy - v_y dx), the
# shifted-Legendre DG basis, and 10-point rules everywhere.
# --------------------------------------------------------------------------
def _q2_at(xi, eta):
    phi, _, _ = q2(np.atleast_1d(xi), np.atleast_1d(eta))
    return phi


class Advection:
    def __init__(self, nx, ny, xy, n_a, nq=None):
        """xy: vertices (bilinear maps; default rule 10 points) or CG2 node
        positions (isoparametric maps; default rule the method's own, 3 or 4
        points, since curved elements make the integrands rational)."""
        self.nx, self.ny, self.n_a = nx, ny, n_a
        self.ne = nx * ny
        self.nw = 2 * nx + 1
        self.nn = self.nw * (2 * ny + 1)
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        self.iso = xy.shape[0] == self.nn
        if nq is None:
            nq = ({1: 3, 3: 3, 6: 4}[n_a]) if self.iso else 10
        if self.iso:
            self.nxy = xy
        else:
            self.xy = xy.reshape(ny + 1, nx + 1, 2)
        self.x1, self.w1 = gauss01(nq)
        XI, ET = np.meshgrid(self.x1, self.x1)
        self.vxi, self.veta, self.vw = XI.ravel(), ET.ravel(), np.outer(self.w1, self.w1).ravel()

    def corners(self, K):
        kx, ky = K % self.nx, K // self.nx
        v = self.xy
        return v[ky, kx], v[ky, kx + 1], v[ky + 1, kx], v[ky + 1, kx + 1]

    def elem_nodes(self, K):
        kx, ky = K % self.nx, K // self.nx
        idx = [(2 * ky + b) * self.nw + 2 * kx + a for b in range(3) for a in range(3)]
        return self.nxy[idx]  # (9, 2)

    def xmap(self, K, xi, eta):
        if self.iso:
            phi, _, _ = q2(np.atleast_1d(xi), np.atleast_1d(eta))
            return phi @ self.elem_nodes(K)
        x00, x10, x01, x11 = self.corners(K)
        xi, eta = np.asarray(xi)[..., None], np.asarray(eta)[..., None]
        return (x00 * (1 - xi) * (1 - eta) + x10 * xi * (1 - eta) + x01 * (1 - xi) * eta
                + x11 * xi * eta)

    def jac(self, K, xi, eta):
        if self.iso:
            _, gxi, geta = q2(np.atleast_1d(xi), np.atleast_1d(eta))
            X = self.elem_nodes(K)
            return gxi @ X, geta @ X  # columns d x/d xi, d x/d eta
        x00, x10, x01, x11 = self.corners(K)
        xi, eta = np.asarray(xi)[..., None], np.asarray(eta)[..., None]
        dxi = (x10 - x00) * (1 - eta) + (x11 - x01) * eta
        deta = (x01 - x00) * (1 - xi) + (x11 - x10) * xi
        return dxi, deta  # columns of J: d x/d xi, d x/d eta

    def vel_at(self, vel, K, xi, eta):
        kx, ky = K % self.nx, K // self.nx
        nodes = np.array([(2 * ky + b) * self.nw + 2 * kx + a for b in range(3) for a in range(3)])
        phi = _q2_at(xi, eta)  # (nq, 9)
        return phi @ vel[0][nodes], phi @ vel[1][nodes]

    def basis(self, xi, eta):
        return dg_bf(self.n_a, np.asarray(xi), np.asarray(eta))

    def dbasis(self, xi, eta, h=0.5):
        # derivatives of the basis by central differences, exact for the
        # degree <= 2 (per variable) polynomials of the advection space
        xi, eta = np.asarray(xi), np.asarray(eta)
        dx = (self.basis(xi + h, eta) - self.basis(xi - h, eta)) / (2 * h)
        de = (self.basis(xi, eta + h) - self.basis(xi, eta - h)) / (2 * h)
        return dx, de

    def to_bf(self, F_doc):
        """(n_a, N_e) documented coefficients -> (N_e, n_a) brute-force coefficients."""
        xs = np.array([0.1, 0.35, 0.6, 0.9])
        XI, ET = np.meshgrid(xs, xs)
        pd = dg_documented(self.n_a, XI.ravel(), ET.ravel())
        pb = self.basis(XI.ravel(), ET.ravel())
        vals = pd @ F_doc  # (ns, N_e)
        return np.linalg.lstsq(pb, vals, rcond=None)[0].T

    def to_doc(self, F_bf):
        xs = np.array([0.1, 0.35, 0.6, 0.9])
        XI, ET = np.meshgrid(xs, xs)
        pd = dg_documented(self.n_a, XI.ravel(), ET.ravel())
        pb = self.basis(XI.ravel(), ET.ravel())
        vals = pb @ F_bf.T
        return np.linalg.lstsq(pd, vals, rcond=None)[0]

    def operator(self, vel, F_doc):
        """M^-1 R(F) in documented coefficients, (n_a, N_e)."""
        F = self.to_bf(F_doc)
        out = np.zeros_like(F)
        for K in range(self.ne):
            kx, ky = K % self.nx, K // self.nx
            xi, eta, w = self.vxi, self.veta, self.vw
            jx, je = self.jac(K, xi, eta)
            det = jx[:, 0] * je[:, 1] - je[:, 0] * jx[:, 1]
            vx, vy = self.vel_at(vel, K, xi, eta)
            psi = self.basis(xi, eta)
            dpx, dpe = self.dbasis(xi, eta)
            # physical gradient: grad = J^-T (d/dxi, d/deta)
            gx = (je[:, 1, None] * dpx - jx[:, 1, None] * dpe) / det[:, None]
            gy = (-je[:, 0, None] * dpx + jx[:, 0, None] * dpe) / det[:, None]
            h = psi @ F[K]
            R = ((w * det * h)[:, None] * (vx[:, None] * gx + vy[:, None] * gy)).sum(0)
            M = np.einsum("q,qi,qj->ij", w * det, psi, psi)
            # counter-clockwise boundary: S (x00->x10), E (x10->x11), N (x11->x01), W (x01->x00)
            t = self.x1
            edges = [(t, 0 * t, lambda s: (s, 1.0), ky > 0, K - self.nx),                 # south
                     (1 + 0 * t, t, lambda s: (0.0, s), kx < self.nx - 1, K + 1),       # east
                     (1 - t, 1 + 0 * t, lambda s: (s, 0.0), ky < self.ny - 1, K + self.nx),  # north
                     (0 * t, 1 - t, lambda s: (1.0, s), kx > 0, K - 1)]                 # west
            for exi, eeta, nbmap, has_nb, nb in edges:
                # tangent of the counter-clockwise traversal by the chain rule
                jx, je = self.jac(K, exi, eeta)
                dxi_dt = (exi[-1] - exi[0]) / (t[-1] - t[0])
                deta_dt = (eeta[-1] - eeta[0]) / (t[-1] - t[0])
                tx = jx[:, 0] * dxi_dt + je[:, 0] * deta_dt
                ty = jx[:, 1] * dxi_dt + je[:, 1] * deta_dt
                vx, vy = self.vel_at(vel, K, exi, eeta)
                flux = vx * ty - vy * tx  # v.n ds/dt
                own = self.basis(exi, eeta) @ F[K]
                if has_nb:
                    s = eeta if exi[0] == exi[-1] else exi
                    nxi, neta = nbmap(s)
                    nxi = np.broadcast_to(nxi, s.shape)
                    neta = np.broadcast_to(neta, s.shape)
                    other = self.basis(nxi, neta) @ F[nb]
                else:
                    other = own
                hat = np.where(flux >= 0, own, other)
                R -= ((self.w1 * flux * hat)[:, None] * self.basis(exi, eeta)).sum(0)
            out[K] = np.linalg.solve(M, R)
        return self.to_doc(out)

    def integral(self, F_doc):
        """sum_K int_K F dx."""
        F = self.to_bf(F_doc)
        tot = 0.0
        for K in range(self.ne):
            jx, je = self.jac(K, self.vxi, self.veta)
            det = jx[:, 0] * je[:, 1] - je[:, 0] * jx[:, 1]
            tot += (self.vw * det * (self.basis(self.vxi, self.veta) @ F[K])).sum()
        return tot
