"""Exact (symbolic) point data for the oracle pins: analytic metrics and scalar fields,
their derivatives by sympy, and a small numpy 4D-geometry toolkit used as an independent
brute-force reference (4D Christoffels -> Riemann -> stress tensor in coordinates).
"""
import math

import numpy as np

try:
    import sympy as sp
except ImportError:  # pragma: no cover - sympy is optional; these tests are CPU-only
    sp = None

SYM_PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
F_CHI, F_H, F_K, F_A, F_TH, F_GAM, F_LAPSE, F_SHIFT, F_B, F_PHI, F_PI = 0, 1, 7, 8, 14, 15, 18, 19, 22, 25, 26
NEED_D2 = [F_CHI] + list(range(F_H, F_H + 6)) + [F_LAPSE] + list(range(F_SHIFT, F_SHIFT + 3)) + [F_PHI]


def symbols():
    return sp.symbols("t x y z", real=True)


def evaluate(exprs, syms, pt):
    """Evaluates a list of sympy expressions at one point (double precision)."""
    return np.array(sp.lambdify(syms, [sp.sympify(e) for e in exprs], modules="math")(*pt), dtype=np.float64)


def conformal_point(fields, pt, xyz):
    """fields: list of 27 sympy expressions in (x, y, z). Returns v[27], d1[27,3], d2[27,6]
    evaluated at pt (exact derivatives, double-precision evaluation). pt may also be a list
    of points, in which case a list of triples is returned."""
    exprs = []
    for f, e in enumerate(fields):
        e = sp.sympify(e)
        firsts = [sp.diff(e, s) for s in xyz]
        exprs.append(e)
        exprs.extend(firsts)
        if f in NEED_D2 or f == F_PI:
            exprs.extend(sp.diff(firsts[a], xyz[b]) for a, b in SYM_PAIRS)
        else:
            exprs.extend([sp.Integer(0)] * 6)
    fn = sp.lambdify(xyz, exprs, modules="math")
    single = not isinstance(pt[0], (tuple, list, np.ndarray))
    res = []
    for q in ([pt] if single else list(pt)):
        vals = np.array(fn(*q), dtype=np.float64).reshape(27, 10)
        res.append((vals[:, 0].copy(), vals[:, 1:4].copy(), vals[:, 4:10].copy()))
    return res[0] if single else res


def christoffel_first(g, X):
    n = len(X)
    return [[[sp.Rational(1, 2) * (sp.diff(g[l, j], X[i]) + sp.diff(g[l, i], X[j]) - sp.diff(g[i, j], X[l]))
              for j in range(n)] for i in range(n)] for l in range(n)]


def kerr_schild_fields(M=1.0):
    """Schwarzschild in Kerr-Schild (ingoing Eddington-Finkelstein) coordinates with its own
    stationary lapse and shift, written in the 27 conformal CCZ4 variables with Theta = 0,
    Gamma-hat = Gamma-tilde (Z = 0), B = 0, phi = Pi = 0. Returns (fields, (x, y, z))."""
    t, x, y, z = symbols()
    X = (x, y, z)
    r = sp.sqrt(x * x + y * y + z * z)
    H = M / r
    l = [x / r, y / r, z / r]
    g = sp.Matrix(3, 3, lambda i, j: (1 if i == j else 0) + 2 * H * l[i] * l[j])
    gi = sp.Matrix(3, 3, lambda i, j: (1 if i == j else 0) - 2 * H * l[i] * l[j] / (1 + 2 * H))
    beta_l = [2 * H * l[i] for i in range(3)]
    beta_u = [2 * H * l[i] / (1 + 2 * H) for i in range(3)]
    alpha = 1 / sp.sqrt(1 + 2 * H)
    G1 = christoffel_first(g, X)
    Dbeta = [[sp.diff(beta_l[j], X[i]) - sum(G1[m][i][j] * beta_u[m] for m in range(3)) for j in range(3)]
             for i in range(3)]
    K = sp.Matrix(3, 3, lambda i, j: (Dbeta[i][j] + Dbeta[j][i]) / (2 * alpha))
    Ktr = sum(gi[i, j] * K[i, j] for i in range(3) for j in range(3))
    chi = (1 + 2 * H) ** sp.Rational(-1, 3)
    h = chi * g
    A = chi * (K - g * Ktr / 3)
    hi = gi / chi
    Gt1 = christoffel_first(h, X)
    Gam = [sum(hi[j, k] * sum(hi[i, l] * Gt1[l][j][k] for l in range(3)) for j in range(3) for k in range(3))
           for i in range(3)]
    fields = [chi] + [h[i, j] for i, j in SYM_PAIRS] + [Ktr] + [A[i, j] for i, j in SYM_PAIRS] + [0] \
             + Gam + [alpha] + beta_u + [0, 0, 0] + [0, 0]
    return fields, X


def tt_plane_wave_point(direction, amp_a, amp_b, k, X0):
    """A transverse-traceless gravitational plane wave along x on flat space at t = 0:
    gamma = delta + h, h_yy = -h_zz = a(u), h_yz = b(u), u = t - x (outgoing for x > 0) or
    u = t + x (ingoing), a = amp_a sin(k u), b = amp_b sin(k u + 0.3); unit lapse, zero shift,
    K_ij = -d_t gamma_ij / 2, in the 27 conformal variables (Theta = 0, Gamma-hat from h)."""
    t, x, y, z = symbols()
    X = (x, y, z)
    u = t - direction * x
    a = amp_a * sp.sin(k * u)
    b = amp_b * sp.sin(k * u + sp.Rational(3, 10))
    g4 = sp.Matrix([[1, 0, 0], [0, 1 + a, b], [0, b, 1 - a]])
    Kt = -sp.Rational(1, 2) * sp.diff(g4, t)
    g = g4.subs(t, 0)
    K = Kt.subs(t, 0)
    gi = g.inv()
    chi = g.det() ** sp.Rational(-1, 3)
    Ktr = sum(gi[i, j] * K[i, j] for i in range(3) for j in range(3))
    h = chi * g
    A = chi * (K - g * Ktr / 3)
    hi = gi / chi
    Gt1 = christoffel_first(h, X)
    Gam = [sum(hi[j, kk] * sum(hi[i, l] * Gt1[l][j][kk] for l in range(3)) for j in range(3) for kk in range(3))
           for i in range(3)]
    fields = [chi] + [h[i, j] for i, j in SYM_PAIRS] + [Ktr] + [A[i, j] for i, j in SYM_PAIRS] + [0] \
        + Gam + [1, 0, 0, 0, 0, 0, 0, 0, 0]
    ddot = lambda e: float(sp.diff(e, t, 2).subs({t: 0, x: X0}))
    return conformal_point(fields, (X0, 0.0, 0.0), X), ddot(a), ddot(b)


def isotropic_schwarzschild_fields(M=1.0, lapse="precollapsed", phi_amp=0.0):
    """Schwarzschild puncture data (time-symmetric slice, isotropic radius) with a chosen lapse."""
    t, x, y, z = symbols()
    X = (x, y, z)
    r = sp.sqrt(x * x + y * y + z * z)
    psi = 1 + M / (2 * r)
    chi = psi ** -4
    if lapse == "precollapsed":
        alpha = psi ** -2
    elif lapse == "static":
        alpha = (1 - M / (2 * r)) / (1 + M / (2 * r))
    else:
        alpha = sp.Integer(1)
    phi = phi_amp * sp.exp(-(r - 2) ** 2)
    fields = [chi, 1, 0, 0, 1, 0, 1, 0] + [0] * 6 + [0] + [0, 0, 0] + [alpha] + [0] * 3 + [0] * 3 + [phi, 0]
    return [sp.sympify(f) for f in fields], X


def areal_radius_isotropic(r, M=1.0):
    return r * (1 + M / (2 * r)) ** 2


# ---------------------------------------------------------------------------------------
# Generic analytic spacetime (lapse, shift, spatial metric, scalar) for the 4D checks
# ---------------------------------------------------------------------------------------
ROT = None


def rotation():
    """A fixed generic rotation (all entries non-zero), so that R^T diag(d) R has six
    non-trivial components but a cheap symbolic inverse."""
    a, b, c = 0.4, -0.7, 1.1
    Rz = sp.Matrix([[sp.cos(a), -sp.sin(a), 0], [sp.sin(a), sp.cos(a), 0], [0, 0, 1]])
    Ry = sp.Matrix([[sp.cos(b), 0, sp.sin(b)], [0, 1, 0], [-sp.sin(b), 0, sp.cos(b)]])
    Rx = sp.Matrix([[1, 0, 0], [0, sp.cos(c), -sp.sin(c)], [0, sp.sin(c), sp.cos(c)]])
    return sp.N(Rz * Ry * Rx, 20)


def rotated_diag(d):
    """Returns (M, M^-1) for M = R^T diag(d) R."""
    R = rotation()
    M = sp.Matrix(3, 3, lambda i, j: sum(R[a, i] * R[a, j] * d[a] for a in range(3)))
    Mi = sp.Matrix(3, 3, lambda i, j: sum(R[a, i] * R[a, j] / d[a] for a in range(3)))
    return M, Mi


def generic_spacetime():
    t, x, y, z = symbols()
    alpha = 1 + sp.Rational(1, 5) * sp.sin(0.7 * x + 0.3 * y - 0.5 * z + 0.4 * t)
    beta_u = [sp.Rational(1, 10) * sp.cos(0.5 * y + 0.2 * t + 0.3 * z),
              0.15 * sp.sin(0.4 * z - 0.3 * x + 0.25 * t),
              0.1 * sp.sin(x + t) * sp.cos(0.3 * y)]
    d = [1 + 0.20 * sp.sin(0.3 * x + 0.2 * t - 0.4 * z), 1 + 0.15 * sp.cos(0.6 * z + 0.2 * x - 0.35 * t + 0.5 * y),
         1 + 0.18 * sp.sin(0.5 * y + 0.3 * z + 0.45 * t)]
    g, gi = rotated_diag(d)
    phi = 0.3 * sp.sin(0.6 * x + 0.2 * t - 0.1 * y) * sp.cos(0.4 * y + 0.2 * z) + 0.2 * z * t + 0.1 * x
    return (t, x, y, z), alpha, beta_u, g, phi


def four_metric(alpha, beta_u, g):
    beta_l = [sum(g[i, j] * beta_u[j] for j in range(3)) for i in range(3)]
    g4 = sp.zeros(4, 4)
    g4[0, 0] = -alpha ** 2 + sum(beta_l[i] * beta_u[i] for i in range(3))
    for i in range(3):
        g4[0, i + 1] = g4[i + 1, 0] = beta_l[i]
        for j in range(3):
            g4[i + 1, j + 1] = g[i, j]
    return g4


def lambdify_metric_derivs(g4, phi, T):
    """Returns a function pt -> (g, dg[r][m][n], ddg[r][s][m][n], dphi[m], ddphi[m][n])."""
    comps = []
    for m in range(4):
        for n in range(4):
            comps.append(g4[m, n])
    firsts = [[sp.diff(c, v) for v in T] for c in comps]
    seconds = [[[sp.diff(f1, v) for v in T] for f1 in row] for row in firsts]
    pf = [sp.diff(phi, v) for v in T]
    pff = [[sp.diff(a, v) for v in T] for a in pf]
    flat = comps + [f for row in firsts for f in row] + [s for row in seconds for r2 in row for s in r2] + pf \
           + [a for row in pff for a in row]
    fn = sp.lambdify(T, flat, modules="math")

    def at(pt):
        vals = np.array(fn(*pt), dtype=np.float64)
        o = 0
        g = vals[o:o + 16].reshape(4, 4); o += 16
        dg = vals[o:o + 64].reshape(4, 4, 4); o += 64            # [comp m*4+n][r]
        dg = np.transpose(dg.reshape(4, 4, 4), (2, 0, 1))         # -> dg[r][m][n]
        ddg = vals[o:o + 256].reshape(4, 4, 4, 4); o += 256       # [m][n][r][s]
        ddg = np.transpose(ddg, (2, 3, 0, 1))                     # -> ddg[r][s][m][n]
        dphi = vals[o:o + 4]; o += 4
        ddphi = vals[o:o + 16].reshape(4, 4)
        return g, dg, ddg, dphi, ddphi
    return at


def geometry4(g, dg, ddg):
    """Christoffels, Riemann (all lower), Ricci, scalar from metric data (coordinate basis,
    any dimension): dg[r][m][n] = d_r g_mn, ddg[r][s][m][n] = d_r d_s g_mn."""
    n = g.shape[0]
    gi = np.linalg.inv(g)
    # Gamma_lij = 1/2(d_i g_lj + d_j g_li - d_l g_ij)
    G1 = np.zeros((n, n, n))
    for l in range(n):
        for i in range(n):
            for j in range(n):
                G1[l, i, j] = 0.5 * (dg[i, l, j] + dg[j, l, i] - dg[l, i, j])
    Gam = np.einsum("kl,lij->kij", gi, G1)
    dgi = -np.einsum("ka,mab,bl->mkl", gi, dg, gi)
    dG1 = np.zeros((n, n, n, n))  # dG1[m][l][i][j]
    for m in range(n):
        for l in range(n):
            for i in range(n):
                for j in range(n):
                    dG1[m, l, i, j] = 0.5 * (ddg[m, i, l, j] + ddg[m, j, l, i] - ddg[m, l, i, j])
    dGam = np.einsum("mkl,lij->mkij", dgi, G1) + np.einsum("kl,mlij->mkij", gi, dG1)
    # R^r_{s m n} = d_m Gam^r_{n s} - d_n Gam^r_{m s} + Gam^r_{m l} Gam^l_{n s} - Gam^r_{n l} Gam^l_{m s}
    Rud = (np.einsum("mrns->rsmn", dGam) - np.einsum("nrms->rsmn", dGam)
           + np.einsum("rml,lns->rsmn", Gam, Gam) - np.einsum("rnl,lms->rsmn", Gam, Gam))
    Rdn = np.einsum("ra,asmn->rsmn", g, Rud)
    Ric = np.einsum("rsrn->sn", Rud)
    Rs = np.einsum("sn,sn->", gi, Ric)
    return gi, Gam, Rdn, Ric, Rs


def beta_derivatives(phi, lam, beta_kind, kappa=1.0):
    """beta'(phi), beta''(phi) by symbolic differentiation of the coupling function."""
    f = sp.Symbol("f", real=True)
    beta = {0: lam * f, 1: lam * f ** 2 / 2,
            2: lam / (2 * kappa) * (1 - sp.exp(-kappa * f ** 2))}[beta_kind]
    b1 = sp.diff(beta, f)
    b2 = sp.diff(b1, f)
    return float(b1.subs(f, phi)), float(b2.subs(f, phi))


def stress_and_scalar(g, gi, Gam, Rdn, Ric, Rs, dphi, ddphi, phi, lam, g2, beta_kind, kappa=1.0, g3=0.0,
                      parts=False):
    """8 pi T_mn and the scalar-equation residual E for the action
    (1/16 pi) int [R + X + g2 X^2 + g3 X box(phi) + beta(phi) L_GB]
    (4dST, plus the cubic Horndeski term G3 = g3 X). With parts=True the cubic term's share of
    8 pi T is returned as well."""
    b1, b2 = beta_derivatives(phi, lam, beta_kind, kappa)
    Hphi = ddphi - np.einsum("lmn,l->mn", Gam, dphi)
    Phi = b1 * Hphi + b2 * np.outer(dphi, dphi)
    Phiu = gi @ Phi @ gi
    X = -0.5 * dphi @ gi @ dphi
    Ru = np.einsum("ai,bj,ck,dl,ijkl->abcd", gi, gi, gi, gi, Rdn)
    Ricu = gi @ Ric @ gi
    LGB = np.einsum("abcd,abcd->", Rdn, Ru) - 4 * np.einsum("ab,ab->", Ric, Ricu) + Rs * Rs
    P = (Rdn - np.einsum("ac,bd->abcd", g, Ric) + np.einsum("ad,bc->abcd", g, Ric)
         + np.einsum("bc,ad->abcd", g, Ric) - np.einsum("bd,ac->abcd", g, Ric)
         + 0.5 * Rs * (np.einsum("ac,bd->abcd", g, g) - np.einsum("ad,bc->abcd", g, g)))
    T8gb = -4 * np.einsum("acbd,cd->ab", P, Phiu)
    T8 = 0.5 * (1 + 2 * g2 * X) * np.outer(dphi, dphi) + 0.5 * g * (X + g2 * X * X) + T8gb
    dphu = gi @ dphi
    box = np.einsum("ab,ab->", gi, Hphi)
    E = (1 + 2 * g2 * X) * box - 2 * g2 * dphu @ Hphi @ dphu + b1 * LGB
    # cubic term g3 X box(phi): with nabla_a X = -nabla^c phi nabla_a nabla_c phi,
    #   8 pi T3_ab = g3 [1/2 box(phi) d_a phi d_b phi + nabla_(a X nabla_b) phi - 1/2 g_ab nabla X . nabla phi]
    #   E3 = g3 [box(phi)^2 - nabla_a nabla_b phi nabla^a nabla^b phi - R_ab nabla^a phi nabla^b phi]
    dX = -Hphi @ dphu
    T8c = g3 * (0.5 * box * np.outer(dphi, dphi) + 0.5 * (np.outer(dX, dphi) + np.outer(dphi, dX))
                - 0.5 * g * (dX @ dphu))
    Hu = gi @ Hphi @ gi
    E = E + g3 * (box * box - np.einsum("ab,ab->", Hphi, Hu) - dphu @ Ric @ dphu)
    T8 = T8 + T8c
    if parts:
        return T8, E, LGB, T8gb, T8c
    return T8, E, LGB, T8gb


def phys_pack_generic(alpha, beta_u, g, phi, T, pt):
    """120-double physical 3+1 pack (see orc_phys_sources) plus u = d_t K_ij and w = d_t Pi,
    all from exact derivatives of the analytic spacetime at pt."""
    t, x, y, z = T
    X = (x, y, z)
    beta_l = [sum(g[i, j] * beta_u[j] for j in range(3)) for i in range(3)]
    G1 = christoffel_first(g, X)
    Dbeta = [[sp.diff(beta_l[j], X[i]) - sum(G1[l][i][j] * beta_u[l] for l in range(3)) for j in range(3)]
             for i in range(3)]
    K = sp.Matrix(3, 3, lambda i, j: -(sp.diff(g[i, j], t) - Dbeta[i][j] - Dbeta[j][i]) / (2 * alpha))
    Pi = (sp.diff(phi, t) - sum(beta_u[k] * sp.diff(phi, X[k]) for k in range(3))) / alpha

    ex = []
    ex += [g[i, j] for i, j in SYM_PAIRS]
    for k in range(3):
        ex += [sp.diff(g[i, j], X[k]) for i, j in SYM_PAIRS]
    for a, b in SYM_PAIRS:
        ex += [sp.diff(g[i, j], X[a], X[b]) for i, j in SYM_PAIRS]
    ex += [K[i, j] for i, j in SYM_PAIRS]
    for k in range(3):
        ex += [sp.diff(K[i, j], X[k]) for i, j in SYM_PAIRS]
    ex += [alpha] + [sp.diff(alpha, X[k]) for k in range(3)]
    ex += [sp.diff(alpha, X[a], X[b]) for a, b in SYM_PAIRS]
    ex += [beta_u[k] for k in range(3)]
    for j in range(3):
        ex += [sp.diff(beta_u[i], X[j]) for i in range(3)]
    ex += [phi] + [sp.diff(phi, X[k]) for k in range(3)]
    ex += [sp.diff(phi, X[a], X[b]) for a, b in SYM_PAIRS]
    ex += [Pi] + [sp.diff(Pi, X[k]) for k in range(3)]
    ex += [sp.diff(K[i, j], t) for i, j in SYM_PAIRS]
    ex += [sp.diff(Pi, t)]
    vals = np.array(sp.lambdify(T, ex, modules="math")(*pt), dtype=np.float64)
    return vals[:120].copy(), vals[120:126].copy(), float(vals[126])


# ---------------------------------------------------------------------------------------
# Covariant modified damped Z4 (the equation the CCZ4 system is the 3+1 projection of)
# ---------------------------------------------------------------------------------------
def z4_spacetime():
    """A generic spacetime (lapse, shift, rotated-diagonal spatial metric, scalar) and a generic
    Z4 covector Z_a, all analytic in (t, x, y, z). The spatial metric is R^T diag(d) R, so its
    inverse and determinant are closed forms."""
    t, x, y, z = symbols()
    alpha = 1 + sp.Rational(1, 5) * sp.sin(0.7 * x + 0.3 * y - 0.5 * z + 0.4 * t)
    beta_u = [sp.Rational(1, 10) * sp.cos(0.5 * y + 0.2 * t + 0.3 * z),
              0.15 * sp.sin(0.4 * z - 0.3 * x + 0.25 * t),
              0.1 * sp.sin(x + t) * sp.cos(0.3 * y)]
    d = [1 + 0.20 * sp.sin(0.3 * x + 0.2 * t - 0.4 * z), 1 + 0.15 * sp.cos(0.6 * z + 0.2 * x - 0.35 * t + 0.5 * y),
         1 + 0.18 * sp.sin(0.5 * y + 0.3 * z + 0.45 * t)]
    g, g_inv = rotated_diag(d)
    phi = 0.3 * sp.sin(0.6 * x + 0.2 * t - 0.1 * y) * sp.cos(0.4 * y + 0.2 * z) + 0.2 * z * t + 0.1 * x
    Z = [0.05 * sp.sin(0.3 * x - 0.2 * y + 0.5 * t) + 0.02, 0.04 * sp.cos(0.4 * y + 0.3 * z - 0.2 * t),
         -0.03 * sp.sin(0.6 * z + 0.1 * x + 0.3 * t), 0.05 * sp.cos(0.2 * x + 0.5 * y - 0.4 * z + 0.1 * t)]
    return (t, x, y, z), alpha, beta_u, d, g, g_inv, phi, Z


def z4_point_data(pt):
    """Everything the covariant check needs at the spacetime point pt = (t, x, y, z):
    the 27 conformal fields with their spatial derivatives (oracle input), their exact time
    derivatives, and the 4-metric, scalar and Z data with derivatives. The conformal fields
    follow the CCZ4 definitions: chi = det(gamma)^(-1/3), h = chi gamma, K_ij from the metric's
    time derivative, A = chi (K_ij - gamma_ij K/3), Theta = -n^a Z_a, and Gamma-hat^i =
    Gamma-tilde^i + 2 h^ij Z_j (Z_j the spatial components of Z_a)."""
    T, alpha, beta_u, d, g, g_inv, phi, Z = z4_spacetime()
    t, x, y, z = T
    X = (x, y, z)
    chi = (d[0] * d[1] * d[2]) ** sp.Rational(-1, 3)
    h = chi * g
    hi = g_inv / chi
    beta_l = [sum(g[i, j] * beta_u[j] for j in range(3)) for i in range(3)]
    G1 = christoffel_first(g, X)
    Dbeta = [[sp.diff(beta_l[j], X[i]) - sum(G1[l][i][j] * beta_u[l] for l in range(3)) for j in range(3)]
             for i in range(3)]
    K = sp.Matrix(3, 3, lambda i, j: -(sp.diff(g[i, j], t) - Dbeta[i][j] - Dbeta[j][i]) / (2 * alpha))
    Ktr = sum(g_inv[i, j] * K[i, j] for i in range(3) for j in range(3))
    A = chi * (K - g * Ktr / 3)
    # det h = 1, so Gamma-tilde^i = h^jk Gt^i_jk = -d_j h^ij
    Gamt = [-sum(sp.diff(hi[i, j], X[j]) for j in range(3)) for i in range(3)]
    Ghat = [Gamt[i] + 2 * sum(hi[i, j] * Z[1 + j] for j in range(3)) for i in range(3)]
    Theta = -(Z[0] - sum(beta_u[i] * Z[1 + i] for i in range(3))) / alpha
    Pi = (sp.diff(phi, t) - sum(beta_u[k] * sp.diff(phi, X[k]) for k in range(3))) / alpha
    F = [chi] + [h[i, j] for i, j in SYM_PAIRS] + [Ktr] + [A[i, j] for i, j in SYM_PAIRS] + [Theta] \
        + Ghat + [alpha] + list(beta_u) + [sp.Float(0.01), sp.Float(-0.02), sp.Float(0.03)] + [phi, Pi]
    F0 = [sp.sympify(f).subs(t, pt[0]) for f in F]
    v, d1, d2 = conformal_point(F0, pt[1:], X)
    dt = np.array(sp.lambdify(T, [sp.diff(sp.sympify(f), t) for f in F], modules="math")(*pt), dtype=np.float64)
    g4 = four_metric(alpha, beta_u, g)
    g4v, dg, ddg, dphi, ddphi = lambdify_metric_derivs(g4, phi, T)(pt)
    zv = np.array(sp.lambdify(T, Z + [sp.diff(Za, s) for Za in Z for s in T], modules="math")(*pt), dtype=np.float64)
    return dict(v=v, d1=d1, d2=d2, dt=dt, g4=g4v, dg=dg, ddg=ddg, dphi=dphi, ddphi=ddphi,
                phi=float(v[F_PHI]), Z=zv[:4], dZ=zv[4:].reshape(4, 4).T.copy())


def z4_residual(D, unk, b, k1, k2, lam, g2, kind, variant="covariant", g3=0.0):
    """Residual of the covariant modified damped Z4 equations with the 4dST stress tensor,
        G^mn + 2 Phat_a^{b mn} nabla_b Z^a - kappa1 [n^m Z^n + n^n Z^m + kappa2 (n.Z) g^mn] - 8 pi T^mn = 0,
        Phat_a^{b mn} = delta_a^(m gh^n)b - 1/2 delta_a^b gh^mn,   gh^mn = g^mn - b n^m n^n,
    and of the scalar equation (the cubic term g3 X box(phi) included), at the data of
    z4_point_data modified by the unknowns
    unk = (d_t^2 gamma_ij (6, added), d_t Z_a (4, added), d_t^2 phi (1, added)). Every
    component is affine in unk. `variant` plants a change in the equation for the
    discrimination checks: "b_half" (b/2 in gh), "k2_moved" ((1 + kappa2) instead of kappa2
    in the damping), "gh_first_only" (g instead of gh in the trace term of Phat), "g3_half" (half
    the cubic term's stress tensor)."""
    g = D["g4"]
    ddg = D["ddg"].copy()
    for m, (i, j) in enumerate(SYM_PAIRS):
        ddg[0, 0, i + 1, j + 1] += unk[m]
        if i != j:
            ddg[0, 0, j + 1, i + 1] += unk[m]
    dZ = D["dZ"].copy()
    dZ[0, :] += unk[6:10]
    ddphi = D["ddphi"].copy()
    ddphi[0, 0] += unk[10]
    gi, Gam, Rdn, Ric, Rs = geometry4(g, D["dg"], ddg)
    Z = D["Z"]
    nabZu = (dZ - np.einsum("cba,c->ba", Gam, Z)) @ gi   # [b, m] = nabla_b Z^m
    divZ = np.trace(nabZu)
    al = 1.0 / np.sqrt(-gi[0, 0])
    n_up = gi @ np.array([-al, 0.0, 0.0, 0.0])
    bb = 0.5 * b if variant == "b_half" else b
    gh = gi - bb * np.outer(n_up, n_up)
    gh_tr = gi if variant == "gh_first_only" else gh
    Zpart = np.einsum("nb,bm->mn", gh, nabZu) + np.einsum("mb,bn->mn", gh, nabZu) - gh_tr * divZ
    Zu = gi @ Z
    nZ = n_up @ Z
    c2 = 1.0 + k2 if variant == "k2_moved" else k2
    damp = -k1 * (np.outer(n_up, Zu) + np.outer(Zu, n_up) + c2 * nZ * gi)
    T8, E, _, _, T8c = stress_and_scalar(g, gi, Gam, Rdn, Ric, Rs, D["dphi"], ddphi, D["phi"], lam, g2, kind,
                                         g3=g3, parts=True)
    if variant == "g3_half":
        T8 = T8 - 0.5 * T8c
    Emn = gi @ (Ric - 0.5 * g * Rs) @ gi + Zpart + damp - gi @ T8 @ gi
    return np.array([Emn[i, j] for i in range(4) for j in range(i, 4)] + [E])


def z4_unknowns(D, **kw):
    """Solves the 11 covariant equations for the unknowns. They are affine in the unknowns (the
    cubic term's box(phi)^2 - nabla nabla phi . nabla nabla phi loses its (d_t^2 phi)^2 part), so
    12 evaluations give the solution exactly; the residual there is checked."""
    f0 = z4_residual(D, np.zeros(11), **kw)
    J = np.empty((11, 11))
    for c in range(11):
        e = np.zeros(11)
        e[c] = 1.0
        J[:, c] = z4_residual(D, e, **kw) - f0
    unk = np.linalg.solve(J, -f0)
    res = z4_residual(D, unk, **kw)
    assert np.max(np.abs(res)) <= 1e-10 * max(1.0, np.max(np.abs(f0))), res
    return unk


def z4_time_derivatives(D, **kw):
    """The exact time derivatives of the 27 conformal fields at the point that the solution of
    the 11 covariant equations gives."""
    unk = z4_unknowns(D, **kw)
    # the unknowns shift the time derivatives of K_ij, Theta, Z_j and Pi at the point
    out = D["dt"].copy()
    gam = D["g4"][1:, 1:]
    gam_i = np.linalg.inv(gam)
    al = 1.0 / np.sqrt(-np.linalg.inv(D["g4"])[0, 0])
    chi = np.linalg.det(gam) ** (-1.0 / 3.0)
    P = np.zeros((3, 3))
    for m, (i, j) in enumerate(SYM_PAIRS):
        P[i, j] = P[j, i] = unk[m]
    dKij = -P / (2.0 * al)              # K_ij = -(d_t gamma_ij - ...)/(2 alpha)
    dK = np.einsum("ij,ij->", gam_i, dKij)
    dA = chi * (dKij - gam * dK / 3.0)
    out[F_K] += dK
    for m, (i, j) in enumerate(SYM_PAIRS):
        out[F_A + m] += dA[i, j]
    beta_u = gam_i @ D["g4"][0, 1:]
    out[F_TH] += -(unk[6] - beta_u @ unk[7:10]) / al
    out[F_GAM:F_GAM + 3] += 2.0 * (gam_i / chi) @ unk[7:10]
    out[F_PI] += unk[10] / al
    return out
