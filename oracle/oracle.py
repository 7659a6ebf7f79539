"""ORACLE — test infrastructure only (plain, slow, FP64).

Python side of the oracle: a ctypes wrapper around bem_oracle.c and the closed
forms used to pin it. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import this module. Nothing here is shared
with the GPU path; inputs (meshes, densities) come in as plain arrays.

Contents (each cites the passage it follows):
  geometry, kernels, local regions, corrected weights, rows / dense matrix of
    A = c I + beta_D Dbar + beta_H Hbar            -- Sec. 2.2, Eq. kcorrection, Eq. bm
  bm_rhs: b = u_inc + alpha du_inc/dn            -- Eq. bm with q = 0, Sec. 5.3
  spherical Bessel functions by recurrence, Mie series of the rigid sphere
    (Hankel functions of the first kind, matching G = e^{ikr}/(4 pi r))   -- Sec. 5.3
  eigenvalues of the layer operators on a sphere (addition theorem)       -- Eq. operator
  gmres: restarted GMRES with modified Gram-Schmidt                       -- Sec. 2.2 (Eq. Axb)
  tree(): octree + near/interaction lists + wedges under integer rules    -- Sec. 3.1.1
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        from . import build as _b
        path = _b.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        i64p = C.POINTER(C.c_int64)
        i32p = C.POINTER(C.c_int32)
        u64p = C.POINTER(C.c_uint64)
        L.orc_set_quadrature.argtypes = [C.c_int, C.c_int, C.c_double, C.c_int, C.c_int]
        L.orc_set_debug.argtypes = [C.c_int]
        L.orc_gauss_legendre01.argtypes = [C.c_int, dp, dp]
        L.orc_nystrom_rule.argtypes = [dp, dp]
        L.orc_kernel_eval.argtypes = [C.c_int64, dp, dp, dp, dp, C.c_double, dp]
        L.orc_phi_matrix.argtypes = [dp, dp]
        L.orc_moments.argtypes = [dp, i32p, C.c_int64, C.c_int, dp, dp, C.c_double, dp]
        L.orc_geometry.argtypes = [dp, C.c_int64, i32p, C.c_int64, dp, dp, dp]
        L.orc_local_region.argtypes = [dp, C.c_int64, i32p, C.c_int64, i64p, C.c_int64, C.c_int64, i64p, i32p]
        L.orc_correction_weights.argtypes = [dp, C.c_int64, i32p, C.c_int64, C.c_double, i64p, C.c_int64,
                                             C.c_int64, i64p, i32p, dp, dp]
        L.orc_matvec_rows.argtypes = [dp, C.c_int64, i32p, C.c_int64, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_double, dp, i64p, C.c_int64, dp]
        L.orc_dense_matrix.argtypes = [dp, C.c_int64, i32p, C.c_int64, C.c_double, C.c_double, C.c_double,
                                       C.c_double, C.c_double, C.c_double, dp]
        L.orc_particle_rows.argtypes = [dp, dp, C.c_int64, C.c_double, C.c_double, C.c_double, dp, i64p, C.c_int64,
                                        dp]
        L.orc_particle_field.argtypes = [dp, dp, C.c_int64, C.c_double, C.c_double, C.c_double, dp, dp, C.c_int64,
                                         dp]
        L.orc_rows4.argtypes = [dp, C.c_int64, i32p, C.c_int64, C.c_double, C.c_double, C.c_double, dp, dp, i64p,
                                C.c_int64, dp]
        L.orc_wedge_of.argtypes = [C.c_int, C.c_int32, C.c_int32, C.c_int32]
        L.orc_wedge_of.restype = C.c_int32
        L.orc_tree_build.argtypes = [dp, C.c_int64, C.c_int, C.c_double]
        L.orc_tree_build.restype = C.c_void_p
        L.orc_tree_sizes.argtypes = [C.c_void_p, i64p]
        L.orc_tree_export.argtypes = [C.c_void_p, dp, i64p, u64p, i32p, i64p, i32p, i64p, i64p, i32p]
        L.orc_tree_free.argtypes = [C.c_void_p]
        L.orc_num_threads.restype = C.c_int
        _LIB = L
    return _LIB


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def _mesh_args(nodes, elems):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    return nodes, elems


def set_quadrature(ntheta=24, nrho=20, eta=3.0, nsub=10, maxdepth=14):
    lib().orc_set_quadrature(ntheta, nrho, eta, nsub, maxdepth)


def set_debug(flags: int = 0):
    """Plant a mistake in the oracle (tests only): bit0 drop F_-1, bit1 drop gamma, bit2 flip normals."""
    lib().orc_set_debug(flags)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def gauss_legendre01(n):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().orc_gauss_legendre01(n, _p(x), _p(w)):
        raise ValueError(n)
    return x, w


def nystrom_rule():
    xi = np.zeros((6, 2))
    w = np.zeros(6)
    lib().orc_nystrom_rule(_p(xi), _p(w))
    return xi, w


def phi_matrix():
    a = np.zeros((6, 6))
    b = np.zeros((6, 6))
    lib().orc_phi_matrix(_p(a), _p(b))
    return a, b


def kernels(x, nx, y, ny, k):
    """G, dG/dn_y, dG/dn_x, d2G/dn_x dn_y at point pairs (r = x - y); returns (m, 4) complex."""
    x, nx, y, ny = (np.ascontiguousarray(np.atleast_2d(a), dtype=np.float64) for a in (x, nx, y, ny))
    m = x.shape[0]
    out = np.zeros((m, 8))
    lib().orc_kernel_eval(m, _p(x), _p(nx), _p(y), _p(ny), float(k), _p(out))
    return out.view(np.complex128).reshape(m, 4)


def geometry(nodes, elems):
    """Nystrom points x (N,3), paper normals n (N,3) pointing into the body, weights w (N,)."""
    nodes, elems = _mesh_args(nodes, elems)
    N = 6 * elems.shape[0]
    xs = np.zeros((N, 3))
    ns = np.zeros((N, 3))
    ws = np.zeros(N)
    lib().orc_geometry(_p(nodes), nodes.shape[0], _p(elems, C.c_int32), elems.shape[0], _p(xs), _p(ns), _p(ws))
    return xs, ns, ws


def moments(nodes, elems, e, k, self_g=-1, x=None, nx=None):
    """(ID, IH): moments of element e against basis xi1^p xi2^q (p+q<=2) for dG/dn_y and d2G/dn_x dn_y."""
    nodes, elems = _mesh_args(nodes, elems)
    x = np.zeros(3) if x is None else np.ascontiguousarray(x, dtype=np.float64)
    nx = np.zeros(3) if nx is None else np.ascontiguousarray(nx, dtype=np.float64)
    out = np.zeros(24)
    lib().orc_moments(_p(nodes), _p(elems, C.c_int32), int(e), int(self_g), _p(x), _p(nx), float(k), _p(out))
    o = out.view(np.complex128)
    return o[:6].copy(), o[6:].copy()


def local_region(nodes, elems, rows, cap=512):
    nodes, elems = _mesh_args(nodes, elems)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cnt = np.zeros(len(rows), dtype=np.int64)
    lst = np.zeros((len(rows), cap), dtype=np.int32)
    rc = lib().orc_local_region(_p(nodes), nodes.shape[0], _p(elems, C.c_int32), elems.shape[0],
                                _p(rows, C.c_int64), len(rows), cap, _p(cnt, C.c_int64), _p(lst, C.c_int32))
    if rc:
        raise RuntimeError(f"orc_local_region failed ({rc})")
    return [lst[r, :cnt[r]].copy() for r in range(len(rows))]


def correction_weights(nodes, elems, k, rows, cap=512):
    """Per row: (elements of D_i, wD (n,6), wH (n,6)) corrected weights for dG/dn_y and d2G/dn_x dn_y."""
    nodes, elems = _mesh_args(nodes, elems)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    R = len(rows)
    cnt = np.zeros(R, dtype=np.int64)
    lst = np.zeros((R, cap), dtype=np.int32)
    wD = np.zeros((R, cap, 6, 2))
    wH = np.zeros((R, cap, 6, 2))
    rc = lib().orc_correction_weights(_p(nodes), nodes.shape[0], _p(elems, C.c_int32), elems.shape[0], float(k),
                                      _p(rows, C.c_int64), R, cap, _p(cnt, C.c_int64), _p(lst, C.c_int32),
                                      _p(wD), _p(wH))
    if rc:
        raise RuntimeError(f"orc_correction_weights failed ({rc})")
    out = []
    for r in range(R):
        n = int(cnt[r])
        a = wD[r, :n].copy().view(np.complex128)[..., 0]
        b = wH[r, :n].copy().view(np.complex128)[..., 0]
        out.append((lst[r, :n].copy(), a, b))
    return out


def particle_rows(x, n, k, q, rows, alpha=None):
    """Direct sum p_i = sum_{j != i} [G + alpha dG/dn_y](x_i, x_j; n_j) q_j at the given rows (Eq. sum)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.complex128)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    a = complex(1j / k) if alpha is None else complex(alpha)
    out = np.zeros(len(rows), dtype=np.complex128)
    lib().orc_particle_rows(_p(x), _p(n), x.shape[0], float(k), a.real, a.imag, _p(q.view(np.float64)),
                            _p(rows, C.c_int64), len(rows), _p(out.view(np.float64)))
    return out


def particle_field(x, n, k, q, targets, alpha=None):
    """p(t) = sum_j [G + alpha dG/dn_y](t, x_j; n_j) q_j at target points t (not sources)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.complex128)
    t = np.ascontiguousarray(np.atleast_2d(targets), dtype=np.float64)
    a = complex(1j / k) if alpha is None else complex(alpha)
    out = np.zeros(t.shape[0], dtype=np.complex128)
    lib().orc_particle_field(_p(x), _p(n), x.shape[0], float(k), a.real, a.imag, _p(q.view(np.float64)), _p(t),
                             t.shape[0], _p(out.view(np.float64)))
    return out


def matvec_rows(nodes, elems, k, x, rows, c=0.5, beta_d=1.0, beta_h=None):
    """Rows of (c I + beta_D Dbar + beta_H Hbar) x; default is the rigid-scatter Burton-Miller
    operator with alpha = i/k (Eq. bm with q = 0)."""
    nodes, elems = _mesh_args(nodes, elems)
    if beta_h is None:
        beta_h = 1j / k
    x = np.ascontiguousarray(x, dtype=np.complex128)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.zeros(len(rows), dtype=np.complex128)
    bd, bh = complex(beta_d), complex(beta_h)
    rc = lib().orc_matvec_rows(_p(nodes), nodes.shape[0], _p(elems, C.c_int32), elems.shape[0], float(k),
                               float(c), bd.real, bd.imag, bh.real, bh.imag, _p(x.view(np.float64)),
                               _p(rows, C.c_int64), len(rows), _p(y.view(np.float64)))
    if rc:
        raise RuntimeError(f"orc_matvec_rows failed ({rc})")
    return y


def rows4(nodes, elems, k, x, rows, c=0.0, b_s=0.0, b_d=0.0, b_m=0.0, b_h=0.0):
    """Rows of (c I + b_s Sbar + b_d Dbar + b_m Mbar + b_h Hbar) x, every operator with its own locally
    corrected weights (Eq. local correction)."""
    nodes, elems = _mesh_args(nodes, elems)
    x = np.ascontiguousarray(x, dtype=np.complex128)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    b = np.array([b_s, b_d, b_m, b_h], dtype=np.complex128)
    y = np.zeros(len(rows), dtype=np.complex128)
    cc = complex(c)
    rc = lib().orc_rows4(_p(nodes), nodes.shape[0], _p(elems, C.c_int32), elems.shape[0], float(k), cc.real, cc.imag,
                         _p(b.view(np.float64)), _p(x.view(np.float64)), _p(rows, C.c_int64), len(rows),
                         _p(y.view(np.float64)))
    if rc:
        raise RuntimeError(f"orc_rows4 failed ({rc})")
    return y


def radiation_rhs_rows(nodes, elems, k, q, rows, alpha=None):
    """Rows of the radiation right-hand side of Eq. bm (no incident wave): (Sbar + alpha Mbar - alpha/2 I) q."""
    a = 1j / k if alpha is None else complex(alpha)
    return rows4(nodes, elems, k, q, rows, c=-0.5 * a, b_s=1.0, b_m=a)


def pulsating_sphere(k, a):
    """Surface potential of a sphere of radius a pulsating with q = du/dn = 1, n into the body (Sec. 5.2: the
    paper prints u = 1/(1 - ik) for the unit sphere): u = a / (1 - i k a)."""
    return a / (1.0 - 1j * k * a)


def robin_rows(nodes, elems, k, x, rows, gamma, alpha=None):
    """Rows of the Burton-Miller operator under Robin data a u + b q = g (Eq. bm, Sec. 2.2, q = (g - a u)/b
    eliminated): (A + gamma B) x with gamma = a/b, A = 1/2 I + Dbar + alpha Hbar, B = Sbar + alpha Mbar - alpha/2 I."""
    a = 1j / k if alpha is None else complex(alpha)
    g = complex(gamma)
    return rows4(nodes, elems, k, x, rows, c=0.5 - 0.5 * a * g, b_s=g, b_d=1.0, b_m=g * a, b_h=a)


def robin_sphere(k, a, ac, bc, g):
    """Surface potential of the radiating monopole u = C e^{ikr}/r outside a sphere of radius a that meets the
    Robin condition ac u + bc du/dn = g with constant g (n into the body, so du/dn = -du/dr = u (1/a - ik)):
    u = g / (ac + bc (1/a - ik)). With ac = 0, bc = 1 (q = g = 1) it is the pulsating sphere of Sec. 5.2."""
    return complex(g) / (complex(ac) + complex(bc) * (1.0 / a - 1j * k))


def dense_matrix(nodes, elems, k, c=0.5, beta_d=1.0, beta_h=None):
    nodes, elems = _mesh_args(nodes, elems)
    if beta_h is None:
        beta_h = 1j / k
    N = 6 * elems.shape[0]
    A = np.zeros((N, N), dtype=np.complex128)
    bd, bh = complex(beta_d), complex(beta_h)
    rc = lib().orc_dense_matrix(_p(nodes), nodes.shape[0], _p(elems, C.c_int32), elems.shape[0], float(k),
                                float(c), bd.real, bd.imag, bh.real, bh.imag, _p(A.view(np.float64)))
    if rc:
        raise RuntimeError(f"orc_dense_matrix failed ({rc})")
    return A


def bm_rhs(xs, ns, k, direction, alpha=None):
    """b = u_inc + alpha du_inc/dn_x with u_inc = exp(i k d.x) (Eq. bm, q = 0; Sec. 5.3)."""
    if alpha is None:
        alpha = 1j / k
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    u = np.exp(1j * k * (xs @ d))
    dudn = 1j * k * (ns @ d) * u
    return u + alpha * dudn


# ------------------------------------------------------------------------------------------------
# Closed forms
# ------------------------------------------------------------------------------------------------
def sph_jn(nmax, z):
    """Spherical Bessel j_0..j_nmax at real z > 0 by downward (Miller) recurrence normalised with j_0."""
    z = float(z)
    start = int(max(nmax, z) + 30 + 2 * math.sqrt(max(nmax, z)))
    f = np.zeros(start + 2)
    f[start + 1] = 0.0
    f[start] = 1e-300
    for n in range(start, 0, -1):
        f[n - 1] = (2 * n + 1) / z * f[n] - f[n + 1]
        if abs(f[n - 1]) > 1e250:
            f[n - 1:] *= 1e-250
    j0 = math.sin(z) / z
    return f[: nmax + 1] * (j0 / f[0])


def sph_yn(nmax, z):
    """Spherical Bessel y_0..y_nmax at real z > 0 by upward recurrence (stable for the dominant solution)."""
    z = float(z)
    y = np.zeros(nmax + 1)
    y[0] = -math.cos(z) / z
    if nmax >= 1:
        y[1] = -math.cos(z) / (z * z) - math.sin(z) / z
    for n in range(1, nmax):
        y[n + 1] = (2 * n + 1) / z * y[n] - y[n - 1]
    return y


def sph_derivative(f, z):
    """f_n' = f_{n-1} - (n+1)/z f_n (n >= 1), f_0' = -f_1, for any spherical Bessel family."""
    n = np.arange(len(f) - 1)
    d = np.zeros(len(f) - 1, dtype=f.dtype)
    d[0] = -f[1]
    d[1:] = f[:-2] - (n[1:] + 1) / z * f[1:-1]
    return d


def sph_all(nmax, z):
    """(j, j', h, h') for n = 0..nmax with h = h^(1) = j + i y."""
    j = sph_jn(nmax + 1, z)
    y = sph_yn(nmax + 1, z)
    h = j + 1j * y
    return j[: nmax + 1], sph_derivative(j, z), h[: nmax + 1], sph_derivative(h, z)


def legendre(nmax, x):
    x = np.asarray(x, dtype=np.float64)
    P = np.zeros((nmax + 1,) + x.shape)
    P[0] = 1.0
    if nmax >= 1:
        P[1] = x
    for n in range(1, nmax):
        P[n + 1] = ((2 * n + 1) * x * P[n] - n * P[n - 1]) / (n + 1)
    return P


def mie_nmax(z):
    return int(z + 10 * z ** (1.0 / 3.0) + 10)


def mie_total_surface(theta, k, a):
    """Total field on a rigid sphere for u_inc = exp(i k d.x): with h_n = h_n^(1) and the Wronskian
    j_n h_n' - j_n' h_n = i/z^2, u(theta) = (i/z^2) sum_n (2n+1) i^n P_n(cos theta) / h_n'(z), z = k a.
    (The paper's series, Sec. 5.3, written with the first-kind Hankel function of G = e^{ikr}/(4 pi r).)"""
    z = k * a
    nmax = mie_nmax(z)
    _, _, _, dh = sph_all(nmax, z)
    P = legendre(nmax, np.cos(theta))
    n = np.arange(nmax + 1)
    coef = (2 * n + 1) * (1j ** n) / dh
    return (1j / z ** 2) * np.tensordot(coef, P, axes=(0, 0))


def sphere_eigenvalues(nmax, k, a, alpha=None):
    """Eigenvalues on a sphere of radius a for zonal harmonics P_n, with the paper's normal (into the body):
       S: i k a^2 j_n h_n;  D (Cauchy principal value): -(i z^2 j_n h_n' + 1/2);  H (finite part): i k z^2 j_n' h_n';
       rigid-scatter Burton-Miller operator 1/2 + D + alpha H."""
    if alpha is None:
        alpha = 1j / k
    z = k * a
    j, dj, h, dh = sph_all(nmax, z)
    S = 1j * k * a * a * j * h
    D = -(1j * z * z * j * dh + 0.5)
    H = 1j * k * z * z * dj * dh
    return dict(S=S, D=D, H=H, A=0.5 + D + alpha * H)


def gmres(matvec, b, tol=1e-6, restart=50, maxiter=1000, x0=None):
    """Restarted GMRES(m) with modified Gram-Schmidt Arnoldi and Givens rotations, FP64.
    Stops when ||b - A x|| / ||b|| <= tol (the recurrence estimate, confirmed by a true residual)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bn = np.linalg.norm(b)
    if bn == 0:
        return x, 0, 0.0
    it = 0
    hist = []
    while it < maxiter:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta / bn <= tol:
            return x, it, beta / bn
        m = restart
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Hm = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            w = matvec(V[j])
            it += 1
            for i in range(j + 1):
                Hm[i, j] = np.vdot(V[i], w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] != 0:
                V[j + 1] = w / Hm[j + 1, j]
            # rotations G_i = [[conj(c), conj(s)], [-s, c]] annihilate the subdiagonal
            for i in range(j):
                t = np.conj(cs[i]) * Hm[i, j] + np.conj(sn[i]) * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            a_, b_ = Hm[j, j], Hm[j + 1, j]
            den = math.sqrt(abs(a_) ** 2 + abs(b_) ** 2)
            cs[j] = a_ / den if den else 1.0
            sn[j] = b_ / den if den else 0.0
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bn)
            if abs(g[j + 1]) / bn <= tol or it >= maxiter:
                break
        y = np.linalg.solve(np.triu(Hm[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y
    r = b - matvec(x)
    return x, it, np.linalg.norm(r) / bn


# ------------------------------------------------------------------------------------------------
# Octree + lists
# ------------------------------------------------------------------------------------------------
def tree(points, leaf_max, k):
    """Octree and lists under the integer rules of Sec. 3.1.1 (see bem_oracle.c). Returns a dict."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    L = lib()
    h = L.orc_tree_build(_p(pts), pts.shape[0], int(leaf_max), float(k))
    try:
        s = np.zeros(4, dtype=np.int64)
        L.orc_tree_sizes(h, _p(s, C.c_int64))
        nbox, nlev, ndir, nm = (int(v) for v in s)
        N = pts.shape[0]
        geom = np.zeros(4)
        perm = np.zeros(N, dtype=np.int64)
        keys = np.zeros(N, dtype=np.uint64)
        bi32 = np.zeros((nbox, 6), dtype=np.int32)
        bi64 = np.zeros((nbox, 4), dtype=np.int64)
        lev = np.zeros((nlev, 3), dtype=np.int32)
        direct = np.zeros((ndir, 2), dtype=np.int64)
        m64 = np.zeros((nm, 2), dtype=np.int64)
        m32 = np.zeros((nm, 6), dtype=np.int32)
        L.orc_tree_export(h, _p(geom), _p(perm, C.c_int64), _p(keys, C.c_uint64), _p(bi32, C.c_int32),
                          _p(bi64, C.c_int64), _p(lev, C.c_int32), _p(direct, C.c_int64), _p(m64, C.c_int64),
                          _p(m32, C.c_int32))
    finally:
        L.orc_tree_free(h)
    return dict(corner=geom[:3], side=geom[3], perm=perm, keys=keys,
                level=bi32[:, 0], ix=bi32[:, 1], iy=bi32[:, 2], iz=bi32[:, 3], nchild=bi32[:, 4],
                leaf=bi32[:, 5], parent=bi64[:, 0], child_begin=bi64[:, 1], pbeg=bi64[:, 2], pend=bi64[:, 3],
                lev_hf=lev[:, 0], lev_T=lev[:, 1], lev_n=lev[:, 2], direct=direct,
                m2l_tgt=m64[:, 0], m2l_src=m64[:, 1], m2l_level=m32[:, 0], m2l_off=m32[:, 1:4],
                m2l_wout=m32[:, 4], m2l_win=m32[:, 5])


def wedge_of(n, d):
    return int(lib().orc_wedge_of(int(n), int(d[0]), int(d[1]), int(d[2])))


# ------------------------------------------------------------------------------------------------
# Learned leaf-block preconditioner: the network, written out plainly in FP64 (the GPU trains it in FP32)
# ------------------------------------------------------------------------------------------------
def net_layout(H):
    W1 = 0
    b1 = W1 + 6 * H
    W2 = b1 + H
    b2 = W2 + H * H
    W3 = b2 + H
    b3 = W3 + 4 * H
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3, n=b3 + 4)


def net_unpack(w, H):
    L = net_layout(H)
    w = np.asarray(w, dtype=np.float64)
    return (w[L["W1"]:L["b1"]].reshape(H, 6), w[L["b1"]:L["W2"]], w[L["W2"]:L["b2"]].reshape(H, H),
            w[L["b2"]:L["W3"]], w[L["W3"]:L["b3"]].reshape(4, H), w[L["b3"]:L["n"]])


def leaf_features(r, y, segments):
    """Per point: u = r/s_L, v = y/s_L and mean_L(v), s_L = leaf mean of r (RMS of r when the mean is below
    1e-3 RMS). segments: list of index arrays (one per leaf). Returns (features (N,6), s per point)."""
    N = len(r)
    f = np.zeros((N, 6))
    s_pt = np.ones(N, dtype=np.complex128)
    for idx in segments:
        rr, yy = r[idx], y[idx]
        mr = rr.mean()
        rms = np.sqrt(np.mean(np.abs(rr) ** 2))
        s = mr if (abs(mr) > 1e-3 * rms and abs(mr) > 0) else complex(rms if rms > 0 else 1.0)
        u, v = rr / s, yy / s
        mv = v.mean()
        f[idx, 0], f[idx, 1], f[idx, 2], f[idx, 3] = u.real, u.imag, v.real, v.imag
        f[idx, 4], f[idx, 5] = mv.real, mv.imag
        s_pt[idx] = s
    return f, s_pt


def net_loss_grad(w, H, r, y, e, segments):
    """Loss |z - e|^2 / |e|^2 with z_i = (o0 + i o1) r_i + (o2 + i o3) y_i, o = net(features_i), and its gradient
    with respect to the parameters (plain backpropagation). Points outside every segment do not contribute."""
    W1, b1, W2, b2, W3, b3 = net_unpack(w, H)
    f, _ = leaf_features(r, y, segments)
    mask = np.zeros(len(r), dtype=bool)
    for idx in segments:
        mask[idx] = True
    a1 = f @ W1.T + b1
    h1 = np.tanh(a1)
    a2 = h1 @ W2.T + b2
    h2 = np.tanh(a2)
    o = h2 @ W3.T + b3
    z = (o[:, 0] + 1j * o[:, 1]) * r + (o[:, 2] + 1j * o[:, 3]) * y
    E = np.sum(np.abs(e) ** 2)
    d = (z - e) * mask
    loss = np.sum(np.abs(d) ** 2) / E
    gz = 2.0 * d / E  # dL/dRe z + i dL/dIm z
    go = np.stack([np.real(np.conj(gz) * r), np.real(np.conj(gz) * 1j * r), np.real(np.conj(gz) * y),
                   np.real(np.conj(gz) * 1j * y)], axis=1)
    gW3 = go.T @ h2
    gb3 = go.sum(0)
    dh2 = (go @ W3) * (1 - h2 ** 2)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (1 - h1 ** 2)
    gW1 = dh1.T @ f
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
