"""Stokes single- and double-layer operators on SH drop surfaces (oracle; test infrastructure only).

Eq. main_eq (the boundary integral equation), Thm 1 and Sec. 2.2 (singular quadrature with the
target rotated to the pole), Sec. 2.1 (regular rule), Sec. 2.3 (region split, upsampling,
near-singular interpolation), Sec. 1.2 (Galerkin projection).

Kernels (Eq. main_eq), with xh = x0 - x and r = |xh|:
    G(xh) f = f/r + (xh.f) xh/r^3                      (Stokeslet)
    u.T(xh).n = -6 (u.xh)(xh.n) xh / r^5                (stresslet contracted with u and n)
Normalisation used for the two operators returned by `Drops.apply_single/apply_double`:
    S[f](x0) = -(1/4pi) sum_j int_{gamma_j} f.G dS,
    D[u](x0) = (1/4pi) sum_j (lambda_j - 1) PV int_{gamma_j} u.T.n dS,
so the system of Eq. main_eq reads (lambda_i + 1) u - D[u] = 2 u_inf + S[f].  The coefficient of
the double layer is the source drop's lambda_j (the printed lambda_i inside the sum over j is read
as lambda_j; the two agree when all ratios are equal).

Readings of the text:
  * singular weights (Thm 1): w_j^s = (pi/(p_q+1)) w_j^G sum_{n<=p_q} 2 sin(theta_j/2) P_n(cos theta_j),
    applied to K(x0 - x') rho' W'/sin(theta_j) -- the 1/sin(theta) appears once (the printed w_j
    already holds one, and the rule divides by sin(theta) again);
  * the target rotation uses z-y-z Euler angles (alpha, beta, gamma) = (phi_b, theta_a, 0);
  * the rotated geometry x', n', W' is the exact geometry of the rotated parametrisation, computed
    from the rotated coefficients of x and their analytic derivatives;
  * the region of a (target, source drop) pair uses the distance from the target to the nearest
    point of the source drop's upsampled grid, h_j = R_j pi/(p_j+1) with R_j the mean radius,
    Omega_0: d > A h_j, Omega_1: h_j < d <= A h_j, Omega_2: d <= h_j, A = 5;
  * the upsampled grid of factor U has degree U(p+1)-1.
"""
from __future__ import annotations

import numpy as np

from . import geometry, sh, wigner


# ----------------------------------------------------------------------------------------------
# kernels
# ----------------------------------------------------------------------------------------------

def stokeslet(xh: np.ndarray, f: np.ndarray) -> np.ndarray:
    """G(xh) f for arrays [3][...]."""
    r2 = np.sum(xh * xh, axis=0)
    r = np.sqrt(r2)
    xf = np.sum(xh * f, axis=0)
    return f / r + xh * (xf / (r2 * r))


def stresslet(xh: np.ndarray, u: np.ndarray, n: np.ndarray) -> np.ndarray:
    """u.T(xh).n = -6 (u.xh)(xh.n) xh / r^5 for arrays [3][...]."""
    r2 = np.sum(xh * xh, axis=0)
    r5 = r2 * r2 * np.sqrt(r2)
    return -6.0 * xh * (np.sum(u * xh, axis=0) * np.sum(xh * n, axis=0) / r5)


# ----------------------------------------------------------------------------------------------
# singular self quadrature (Thm 1, Sec. 2.2)
# ----------------------------------------------------------------------------------------------

def legendre_p(nmax: int, t: np.ndarray) -> np.ndarray:
    """Unnormalised Legendre polynomials P_0..P_nmax at t (Bonnet recursion), [n][len(t)]."""
    P = np.zeros((nmax + 1, len(t)))
    P[0] = 1.0
    if nmax >= 1:
        P[1] = t
    for n in range(1, nmax):
        P[n + 1] = ((2 * n + 1) * t * P[n] - n * P[n - 1]) / (n + 1)
    return P


def singular_weights(pq: int) -> np.ndarray:
    """w_j^s of Thm 1 with the regular weight pi/(p_q+1) w_j^G (the 1/sin(theta) kept in the integrand)."""
    t, w, theta, phi = sh.gauss_grid(pq)
    P = legendre_p(pq, t)
    return (np.pi / (pq + 1)) * w * np.sum(2.0 * np.sin(theta / 2.0) * P, axis=0)


def rotate_batch(coefs: np.ndarray, p: int, alphas: np.ndarray, beta: float) -> np.ndarray:
    """Complex rotated coefficients [field][b][n][m>=0] of f_field(R_z(alpha_b) R_y(beta) s)."""
    nf = coefs.shape[0]
    nb = len(alphas)
    c = np.stack([sh.to_complex(coefs[i], p) for i in range(nf)])  # [f][n][m]
    out = np.zeros((nf, nb, p + 1, p + 1), dtype=np.complex128)
    for n in range(p + 1):
        ms = np.arange(-n, n + 1)
        g = np.zeros((nf, nb, 2 * n + 1), dtype=np.complex128)
        for m in range(0, n + 1):
            ph = np.exp(1j * m * alphas)  # [b]
            g[:, :, n + m] = c[:, n, m][:, None] * ph[None, :]
            if m > 0:
                g[:, :, n - m] = ((-1) ** m) * np.conj(c[:, n, m])[:, None] * np.conj(ph)[None, :]
        dd = wigner.small_d(n, beta).T  # rows m', cols m
        res = np.einsum("qm,fbm->fbq", dd, g)
        out[:, :, n, :n + 1] = res[:, :, n:]
        del ms
    return out


def synth_complex(c: np.ndarray, p: int, table: np.ndarray, phi: np.ndarray, dphi: int = 0) -> np.ndarray:
    """Values on a grid from complex coefficients c[...][n][m>=0] and a theta table [n][m][j]."""
    h = np.einsum("...nm,nmj->...mj", c, table)  # [...][m][j]
    m = np.arange(p + 1)
    if dphi:
        h = h * ((1j * m) ** dphi)[:, None]
    fac = np.where(m == 0, 1.0, 2.0)
    e = np.exp(1j * np.outer(m, phi)) * fac[:, None]  # [m][k]
    return np.einsum("...mj,mk->...jk", h, e).real


class SelfQuadrature:
    """The singular rule of Thm 1 applied at every grid target of one drop (Sec. 2.2).

    For the target (theta_a, phi_b) of the degree-p grid the coefficients of x and of the density
    are rotated so that the target sits at the pole, synthesised with their derivatives on the
    degree-p_q grid, and summed with w_j^s.
    """

    def __init__(self, xcoef: np.ndarray, p: int, pq: int, cache: bool = True):
        self.xcoef = np.asarray(xcoef, dtype=np.float64).reshape(3, sh.ncoef(p))
        self.p, self.pq = p, pq
        _, _, self.theta, self.phi = sh.gauss_grid(p)
        self.tq, _, self.thq, self.phq = sh.gauss_grid(pq)
        self.ws = singular_weights(pq)
        P, dP, _ = sh.legendre_dtheta(p, self.thq)
        self.Pq, self.dPq = P, dP
        self.cache = cache
        self._geo = {}
        self.x0 = geometry.surface_fields(self.xcoef, p, p)["f"]  # targets [3][a][b]

    def rotated_geometry(self, a: int):
        """x', n' and w^s J' (J' = W'/sin theta_j) for every target of latitude a: arrays [b][3][j][k]."""
        if a in self._geo:
            return self._geo[a]
        c = rotate_batch(self.xcoef, self.p, self.phi, self.theta[a])  # [3][b][n][m]
        x = synth_complex(c, self.p, self.Pq, self.phq)
        xt = synth_complex(c, self.p, self.dPq, self.phq)
        xp = synth_complex(c, self.p, self.Pq, self.phq, dphi=1)
        x, xt, xp = (np.moveaxis(v, 0, 1) for v in (x, xt, xp))  # [b][3][j][k]
        cr = np.cross(xt, xp, axis=1)
        W = np.sqrt(np.sum(cr * cr, axis=1))  # [b][j][k]
        n = cr / W[:, None]
        wJ = self.ws[None, :, None] * W / np.sin(self.thq)[None, :, None]
        out = (x, n, wJ)
        if self.cache:
            self._geo[a] = out
        return out

    def apply(self, dens: np.ndarray, kind: str, lats=None) -> np.ndarray:
        """Raw rule Q at every target: sum_jk w_j^s K(x0 - x'_jk) rho'_jk J'_jk, returns [3][a][b].

        kind 'S': K = Stokeslet acting on rho; kind 'D': stresslet contracted with rho and n'.
        """
        dens = np.asarray(dens, dtype=np.float64).reshape(3, sh.ncoef(self.p))
        out = np.zeros((3, self.p + 1, 2 * self.p + 2))
        for a in (range(self.p + 1) if lats is None else lats):
            x, n, wJ = self.rotated_geometry(a)
            c = rotate_batch(dens, self.p, self.phi, self.theta[a])
            rho = np.moveaxis(synth_complex(c, self.p, self.Pq, self.phq), 0, 1)  # [b][3][j][k]
            x0 = self.x0[:, a, :].T  # [b][3]
            xh = x0[:, :, None, None] - x
            xh, rho_, n_ = (np.moveaxis(v, 1, 0) for v in (xh, rho, n))  # [3][b][j][k]
            if kind == "S":
                K = stokeslet(xh, rho_)
            else:
                K = stresslet(xh, rho_, n_)
            out[:, a, :] = np.sum(K * wJ[None], axis=(2, 3))
        return out


def rotated_points(theta_a: float, phi_b: float, pq: int):
    """Parameter points R s(theta_j, phi_k) of the rotated grid, R = R_z(phi_b) R_y(theta_a)."""
    _, _, th, ph = sh.gauss_grid(pq)
    T, Ph = np.meshgrid(th, ph, indexing="ij")
    s = np.stack([np.sin(T) * np.cos(Ph), np.sin(T) * np.sin(Ph), np.cos(T)])
    v = np.einsum("ab,bjk->ajk", wigner.rotation_matrix(phi_b, theta_a, 0.0), s)
    return np.arccos(np.clip(v[2], -1.0, 1.0)), np.arctan2(v[1], v[0])


# ----------------------------------------------------------------------------------------------
# regular rule, regions and the multi-drop operator (Sec. 2.1, 2.3)
# ----------------------------------------------------------------------------------------------

class DropGrid:
    """Source data of one drop on the Gauss grid of degree P >= p: x, n, regular weight * J."""

    def __init__(self, xcoef: np.ndarray, p: int, P: int):
        self.p, self.P = p, P
        t, w, theta, phi = sh.gauss_grid(P)
        g = geometry.forms(geometry.surface_fields(xcoef, p, P))
        self.x = g["x"].reshape(3, -1)
        self.n = g["n"].reshape(3, -1)
        self.wJ = ((np.pi / (P + 1)) * w[:, None] * geometry.area_density(g["W"], theta)).reshape(-1)

    def density(self, coef: np.ndarray) -> np.ndarray:
        coef = np.asarray(coef).reshape(3, sh.ncoef(self.p))
        return np.stack([sh.synthesize(coef[c], self.p, self.P).reshape(-1) for c in range(3)])


def regular_sum(targets: np.ndarray, src: DropGrid, rho: np.ndarray, kind: str, chunk: int = 256) -> np.ndarray:
    """Regular rule of Sec. 2.1 at arbitrary targets [3][nt]: sum_s K(x0 - x_s) rho_s w_s J_s."""
    nt = targets.shape[1]
    out = np.zeros((3, nt))
    for s in range(0, nt, chunk):
        x0 = targets[:, s:s + chunk]
        xh = x0[:, :, None] - src.x[:, None, :]
        if kind == "S":
            K = stokeslet(xh, rho[:, None, :])
        else:
            K = stresslet(xh, rho[:, None, :], src.n[:, None, :])
        out[:, s:s + chunk] = np.sum(K * src.wJ[None, None, :], axis=2)
    return out


class Drops:
    """N drops: geometry, region lists and the two layer operators in coefficient space."""

    A_TILDE = 5.0

    def __init__(self, xcoef_list, p_list, pq_list, lam, up: int = 4, cache: bool = True):
        self.N = len(p_list)
        self.p = list(p_list)
        self.pq = list(pq_list)
        self.up = up
        self.lam = np.asarray(lam, dtype=np.float64)
        self.xcoef = [np.asarray(x, dtype=np.float64).reshape(3, sh.ncoef(p)) for x, p in zip(xcoef_list, p_list)]
        self.selfq = [SelfQuadrature(x, p, q, cache=cache) for x, p, q in zip(self.xcoef, self.p, self.pq)]
        self.R = [geometry.mean_radius(x, p) for x, p in zip(self.xcoef, self.p)]
        self.h = [R * np.pi / (p + 1) for R, p in zip(self.R, self.p)]
        self.std = [DropGrid(x, p, p) for x, p in zip(self.xcoef, self.p)]
        self.ups = [DropGrid(x, p, up * (p + 1) - 1) for x, p in zip(self.xcoef, self.p)] if self.N > 1 else []
        self.targets = [self.std[i].x for i in range(self.N)]
        self.region = {}
        for i in range(self.N):
            for j in range(self.N):
                if i != j:
                    self.region[(i, j)] = self.classify(self.targets[i], j)

    def classify(self, pts: np.ndarray, j: int) -> np.ndarray:
        """0, 1 or 2 for Omega_0/1/2 of each point [3][n] with respect to source drop j."""
        d = np.full(pts.shape[1], np.inf)
        for s in range(0, pts.shape[1], 256):
            diff = pts[:, s:s + 256, None] - self.ups[j].x[:, None, :]
            d[s:s + 256] = np.sqrt(np.min(np.sum(diff * diff, axis=0), axis=1))
        reg = np.zeros(pts.shape[1], dtype=np.int64)
        reg[d <= self.A_TILDE * self.h[j]] = 1
        reg[d <= self.h[j]] = 2
        return reg

    def _layer_values(self, dens_list, kind: str, weights) -> list:
        """Grid values at every drop's targets of sum_j weights[j] * (raw integral over drop j)."""
        from . import near
        out = []
        self_raw = [self.selfq[j].apply(dens_list[j], kind) for j in range(self.N)]
        std_rho = [self.std[j].density(dens_list[j]) for j in range(self.N)]
        up_rho = [self.ups[j].density(dens_list[j]) for j in range(self.N)] if self.N > 1 else []
        for i in range(self.N):
            p = self.p[i]
            v = weights[i] * self_raw[i].reshape(3, -1)
            for j in range(self.N):
                if j == i or weights[j] == 0.0:
                    continue
                reg = self.region[(i, j)]
                for r, src, rho in ((0, self.std[j], std_rho[j]), (1, self.ups[j], up_rho[j])):
                    sel = np.nonzero(reg == r)[0]
                    if len(sel):
                        v[:, sel] += weights[j] * regular_sum(self.targets[i][:, sel], src, rho, kind)
                sel = np.nonzero(reg == 2)[0]
                if len(sel):
                    v[:, sel] += weights[j] * near.near_values(self, i, j, sel, dens_list[j], kind, self_raw[j])
            out.append(v.reshape(3, p + 1, 2 * p + 2))
        return out

    def project(self, vals: list) -> list:
        """Galerkin projection (Sec. 1.2): grid values -> degree-p coefficients per drop."""
        return [np.stack([sh.analyze(v[c], self.p[i], self.p[i]) for c in range(3)]) for i, v in enumerate(vals)]

    def apply_single(self, f_list, raw: bool = False) -> list:
        """-(1/4pi) sum_j int f_j.G as coefficients (raw: (1/8pi) int f.G, the standard S)."""
        w = [1.0 / (8.0 * np.pi) if raw else -1.0 / (4.0 * np.pi)] * self.N
        return self.project(self._layer_values(f_list, "S", w))

    def apply_double(self, u_list, raw: bool = False) -> list:
        """(1/4pi) sum_j (lambda_j - 1) PV int u_j.T.n as coefficients (raw: (1/4pi) PV int u.T.n)."""
        w = [1.0 / (4.0 * np.pi) if raw else (self.lam[j] - 1.0) / (4.0 * np.pi) for j in range(self.N)]
        return self.project(self._layer_values(u_list, "D", w))

    def apply_single_grid(self, f_list, raw: bool = False) -> list:
        w = [1.0 / (8.0 * np.pi) if raw else -1.0 / (4.0 * np.pi)] * self.N
        return self._layer_values(f_list, "S", w)

    def apply_double_grid(self, u_list, raw: bool = False) -> list:
        w = [1.0 / (4.0 * np.pi) if raw else (self.lam[j] - 1.0) / (4.0 * np.pi) for j in range(self.N)]
        return self._layer_values(u_list, "D", w)

    # ---- the system of Eq. main_eq in coefficient space ----
    def split(self, vec: np.ndarray) -> list:
        out, o = [], 0
        for p in self.p:
            k = 3 * sh.ncoef(p)
            out.append(vec[o:o + k].reshape(3, sh.ncoef(p)))
            o += k
        return out

    @staticmethod
    def join(lst) -> np.ndarray:
        return np.concatenate([np.asarray(v).reshape(-1) for v in lst])

    def system_matvec(self, u: np.ndarray) -> np.ndarray:
        """(lambda_i + 1) u_i - D[u]_i."""
        ul = self.split(u)
        d = self.apply_double(ul)
        return self.join([(self.lam[i] + 1.0) * ul[i] - d[i] for i in range(self.N)])

    def rhs(self, f_list, shear: float) -> np.ndarray:
        """2 u_inf + S[f] with u_inf = (shear z, 0, 0), projected."""
        s = self.apply_single(f_list)
        out = []
        for i in range(self.N):
            p = self.p[i]
            z = self.std[i].x[2].reshape(p + 1, 2 * p + 2)
            uinf = np.zeros((3, sh.ncoef(p)))
            uinf[0] = sh.analyze(shear * z, p, p)
            out.append(2.0 * uinf + s[i])
        return self.join(out)
