"""Pins of the oracle's AO integrals against closed forms, quadrature,
finite differences and identities (nothing here re-uses the oracle's own
formulas)."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2606_04316_gb300 import synth


def rand_centres(rng, n=4, s=1.5):
    return [rng.uniform(-s, s, 3) for _ in range(n)]


# ------------------------------------------------------------------ Boys

@pytest.mark.parametrize("T", [0.0, 1e-8, 0.3, 2.0, 11.0, 30.0, 44.9, 45.1, 80.0, 400.0])
def test_boys_against_quadrature(oracle, T):
    import mpmath
    mpmath.mp.dps = 30
    F = oracle.boys(T, 12)
    for m in range(13):
        ref = float(mpmath.quad(lambda t: t ** (2 * m) * mpmath.exp(-T * t * t), [0, 0.25, 0.5, 1]))
        assert abs(F[m] - ref) <= 1e-13 * ref


def test_boys_zero_and_erf(oracle):
    F = oracle.boys(0.0, 20)
    assert np.allclose(F, 1.0 / (2 * np.arange(21) + 1), rtol=1e-15, atol=0)
    for T in (0.5, 7.0, 60.0):
        assert abs(oracle.boys(T, 0)[0] - 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))) < 1e-15


def test_boys_minus1_derivative(oracle):
    # F_{-1}' = -F_0 and F_{-1}(0) = -1
    assert abs(oracle.boys_minus1(0.0) + 1.0) < 1e-15
    for T in (0.2, 3.0, 20.0, 70.0):
        h = 1e-4 * max(1.0, T)
        d = (oracle.boys_minus1(T + h) - oracle.boys_minus1(T - h)) / (2 * h)
        assert abs(d + oracle.boys(T, 0)[0]) < 1e-7


# ------------------------------------------------------- (ss|ss) closed forms

def ss_prefactor(A, a, B, b, C, c, D, d):
    p, q = a + b, c + d
    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
    K = math.exp(-a * b / p * np.sum((A - B) ** 2)) * math.exp(-c * d / q * np.sum((C - D) ** 2))
    return p, q, P, Q, K


def test_ssss_coulomb_closed_form(oracle):
    rng = np.random.default_rng(1)
    for _ in range(20):
        A, B, C, D = rand_centres(rng)
        a, b, c, d = rng.uniform(0.1, 10, 4)
        p, q, P, Q, K = ss_prefactor(A, a, B, b, C, c, D, d)
        rho = p * q / (p + q)
        R = np.linalg.norm(P - Q)
        # <1/r> of two Gaussian charges: erf(sqrt(rho) R) / R
        smeared = math.erf(math.sqrt(rho) * R) / R if R > 0 else 2 * math.sqrt(rho / math.pi)
        ref = (math.pi / p) ** 1.5 * (math.pi / q) ** 1.5 * K * smeared
        v = oracle.prim_block(0, A, a, 0, B, b, 0, C, c, 0, D, d, 0)[0, 0, 0, 0]
        assert abs(v - ref) <= 1e-13 * abs(ref)


def smeared_distance_quad(R, rho):
    """E|R + u| for u ~ N(0, 1/(2 rho) I_3) by radial quadrature of the
    non-central chi density."""
    if R == 0:
        return 2.0 / math.sqrt(math.pi * rho)
    f = lambda r: r * (r / R) * math.sqrt(rho / math.pi) * (
        math.exp(-rho * (r - R) ** 2) - math.exp(-rho * (r + R) ** 2))
    v, _ = integrate.quad(f, 0, R + 40 / math.sqrt(rho), epsabs=0, epsrel=1e-13, limit=400, points=[max(R - 8 / math.sqrt(rho), 0) + 1e-9, R, R + 8 / math.sqrt(rho)])
    return v


def test_ssss_r12_kernel_against_radial_quadrature(oracle):
    rng = np.random.default_rng(2)
    for _ in range(12):
        A, B, C, D = rand_centres(rng)
        a, b, c, d = rng.uniform(0.1, 6, 4)
        p, q, P, Q, K = ss_prefactor(A, a, B, b, C, c, D, d)
        rho = p * q / (p + q)
        ref = (math.pi / p) ** 1.5 * (math.pi / q) ** 1.5 * K * smeared_distance_quad(np.linalg.norm(P - Q), rho)
        v = oracle.prim_block(1, A, a, 0, B, b, 0, C, c, 0, D, d, 0)[0, 0, 0, 0]
        assert abs(v - ref) <= 1e-11 * abs(ref)


# --------------------------------------------- higher l by centre derivatives

def fd_centre(f, X, k, h=2e-3):
    """4th-order accurate central difference of f(X) along axis k (Richardson)."""
    def d(hh):
        e = np.zeros(3); e[k] = hh
        return (f(X + e) - f(X - e)) / (2 * hh)
    return (4 * d(h / 2) - d(h)) / 3


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 0, 0), (2, 1, 1, 0), (1, 2, 0, 1), (2, 2, 2, 1), (3, 0, 1, 2)])
def test_raise_by_centre_derivative(oracle, kernel, ls):
    """d/dA_k g_a = 2 alpha g_{a+1_k} - a_k g_{a-1_k}: raise the first index by
    finite differences of lower-order blocks."""
    rng = np.random.default_rng(10 + sum(ls) + 7 * kernel)
    A, B, C, D = rand_centres(rng, s=1.0)
    a, b, c, d = rng.uniform(0.3, 2.5, 4)
    la, lb, lc, ld = ls
    hi = oracle.prim_block(kernel, A, a, la + 1, B, b, lb, C, c, lc, D, d, ld)
    lo = oracle.prim_block(kernel, A, a, la, B, b, lb, C, c, lc, D, d, ld)
    lom = oracle.prim_block(kernel, A, a, la - 1, B, b, lb, C, c, lc, D, d, ld) if la > 0 else None
    cart_hi = {t: i for i, t in enumerate(oracle.cart_list(la + 1))}
    cart_lm = {t: i for i, t in enumerate(oracle.cart_list(la - 1))} if la > 0 else {}
    for ia, t in enumerate(oracle.cart_list(la)):
        for k in range(3):
            deriv = fd_centre(lambda X: oracle.prim_block(kernel, X, a, la, B, b, lb, C, c, lc, D, d, ld)[ia], A, k)
            tp = list(t); tp[k] += 1
            pred = 2 * a * hi[cart_hi[tuple(tp)]]
            if t[k] > 0:
                tm = list(t); tm[k] -= 1
                pred = pred - t[k] * lom[cart_lm[tuple(tm)]]
            scale = np.abs(pred).max() + 1e-3
            assert np.abs(deriv - pred).max() <= 2e-7 * scale


@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 0, 1, 0), (1, 1, 0, 1), (2, 0, 1, 1)])
def test_bra_ket_permutation_symmetry(oracle, ls):
    rng = np.random.default_rng(3 + sum(ls))
    A, B, C, D = rand_centres(rng)
    a, b, c, d = rng.uniform(0.2, 4, 4)
    la, lb, lc, ld = ls
    for kernel in (0, 1):
        x = oracle.prim_block(kernel, A, a, la, B, b, lb, C, c, lc, D, d, ld)
        y = oracle.prim_block(kernel, B, b, lb, A, a, la, C, c, lc, D, d, ld)
        z = oracle.prim_block(kernel, C, c, lc, D, d, ld, A, a, la, B, b, lb)
        s = np.abs(x).max()
        assert np.allclose(x, y.transpose(1, 0, 2, 3), atol=1e-13 * s, rtol=0)
        assert np.allclose(x, z.transpose(2, 3, 0, 1), atol=1e-13 * s, rtol=0)


# ------------------------------------------------------------------ gauge

@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 0, 0, 1), (1, 1, 1, 0), (2, 1, 0, 1)])
def test_gauge_translational_invariance(oracle, ls):
    """(d_A+d_B)_I (d_A+d_B)_J (ab|r|cd) == -(d_A+d_B)_I (d_C+d_D)_J (ab|r|cd)."""
    rng = np.random.default_rng(20 + sum(ls))
    A, B, C, D = rand_centres(rng)
    a, b, c, d = rng.uniform(0.3, 3, 4)
    f1 = oracle.prim_ddr(1, A, a, ls[0], B, b, ls[1], C, c, ls[2], D, d, ls[3])
    f2 = oracle.prim_ddr(2, A, a, ls[0], B, b, ls[1], C, c, ls[2], D, d, ls[3])
    assert np.abs(f1 - f2).max() <= 1e-12 * np.abs(f1).max()


@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 0, 1, 0), (1, 1, 0, 1), (2, 1, 1, 0)])
def test_gauge_trace_identity(oracle, ls):
    """sum_I r_I r_I / r^3 = 1/r: the laplacian of the r12-kernel integral is
    twice the Coulomb integral."""
    rng = np.random.default_rng(30 + sum(ls))
    A, B, C, D = rand_centres(rng)
    a, b, c, d = rng.uniform(0.3, 3, 4)
    ddr = oracle.prim_ddr(1, A, a, ls[0], B, b, ls[1], C, c, ls[2], D, d, ls[3])
    coul = oracle.prim_block(0, A, a, ls[0], B, b, ls[1], C, c, ls[2], D, d, ls[3])
    lap = ddr[0] + ddr[3] + ddr[5]
    assert np.abs(lap - 2 * coul).max() <= 1e-12 * np.abs(coul).max()


def test_gauge_large_distance_limit(oracle):
    """Two s charge clouds far apart.  The smeared distance is exactly
    R + 1/(2 rho R) up to exp(-rho R^2), so the kernel r_I r_J / r^3 (not
    harmonic) gives R_I R_J / R^3 - (3 R_I R_J / R^5 - delta_IJ / R^3) / (2 rho)."""
    A = np.zeros(3); C = np.array([9.0, 5.0, -7.0])
    a = b = c = d = 30.0
    basis = synth.Basis(np.array([A, C]), np.array([0, 1], np.int32), np.array([0, 0], np.int32),
                        np.array([1, 1], np.int32), np.array([a, c]), np.array([1.0, 1.0]))
    ob = oracle.OracleBasis(basis)
    K = ob.shell_block(2, 0, 0, 1, 1)[:, 0, 0, 0, 0]
    coul = ob.shell_block(0, 0, 0, 1, 1)[0, 0, 0, 0]
    R = C - A
    r = np.linalg.norm(R)
    # charges of normalised s^2 densities are 1; Coulomb -> 1/R
    assert abs(coul - 1 / r) < 1e-10
    rho = (2 * a) * (2 * c) / (2 * a + 2 * c)
    for ij, (I, J) in enumerate(oracle.IJ6):
        ref = R[I] * R[J] / r ** 3 - (3 * R[I] * R[J] / r ** 5 - (I == J) / r ** 3) / (2 * rho)
        assert abs(K[ij] - ref) < 1e-12


def test_gauge_trace_on_basis_blocks(oracle):
    p = synth.chain_problem(2, 1, seed=7, shells=(0, 1))
    ob = oracle.OracleBasis(p.basis)
    n = ob.nsh
    for sa, sb, sc, sd in [(0, n + 2, 1, n + 3), (1, n + 3, 2, n), (3, n, 1, n + 1)]:
        K = ob.shell_block(2, sa, sb, sc, sd)
        C = ob.shell_block(0, sa, sb, sc, sd)
        assert np.abs(C).max() > 1e-4
        assert np.abs(K[0] + K[3] + K[5] - C).max() <= 1e-12 * max(np.abs(C).max(), np.abs(K).max())


# ---------------------------------------------------- basis construction

def test_normalisation_and_overlaps_against_quadrature(oracle):
    """Every large-component function is normalised; overlaps of derivative
    functions equal a direct Gauss-Hermite quadrature of the analytic
    derivatives of the raw contracted Gaussians."""
    p = synth.chain_problem(2, 1, seed=11, shells=(0, 1, 2))
    ob = oracle.OracleBasis(p.basis)
    for s in range(ob.nsh):
        assert np.allclose(np.diag(ob.overlap_block(s, s)), 1.0, atol=1e-13, rtol=0)
    # moderate exponents so that one Gauss-Hermite product grid resolves all
    bs = synth.Basis(np.array([[0.0, 0.1, -0.2], [1.1, -0.3, 0.4]]), np.array([0, 0, 1, 1, 1, 1], np.int32),
                     np.array([0, 2, 0, 1, 2, 1], np.int32), np.array([2, 2, 2, 2, 2, 1], np.int32),
                     np.array([1.9, 0.9, 2.2, 1.0, 1.7, 0.8, 2.4, 1.1, 1.5, 0.95, 1.3]),
                     np.array([0.5, 0.7, 0.6, 0.4, 0.9, 0.3, 0.8, 0.6, 0.5, 0.7, 1.0]))
    ob = oracle.OracleBasis(bs)
    for s in range(ob.nsh):
        assert np.allclose(np.diag(ob.overlap_block(s, s)), 1.0, atol=1e-13, rtol=0)
    # quadrature: product grid, Gauss-Hermite with weight exp(-x^2) around centre 0
    xg, wg = np.polynomial.hermite.hermgauss(60)
    off = np.concatenate([[0], np.cumsum(bs.shell_nprim)])
    def func_values(s, deriv_K, comp, pts):
        l = int(bs.shell_l[s]); A = bs.xyz[bs.shell_center[s]]
        ex = bs.exps[off[s]:off[s + 1]]; co = bs.coefs[off[s]:off[s + 1]]
        t = oracle.cart_list(l)[comp]
        X = pts - A
        r2 = (X ** 2).sum(-1)
        val = np.zeros(len(pts))
        for e, cc in zip(ex, co):
            g = np.exp(-e * r2)
            poly = np.prod([X[:, k] ** t[k] for k in range(3)], axis=0)
            if deriv_K is None:
                val += cc * poly * g
            else:
                k = deriv_K
                dpoly = t[k] * np.prod([X[:, m] ** (t[m] - (m == k)) for m in range(3)], axis=0) if t[k] else 0
                val += cc * (dpoly - 2 * e * X[:, k] * poly) * g
        return val
    # overlap of two raw functions on shells 1 and 4 (p and d, different centres)
    s1, s2 = 1, 5
    mid = 0.5 * (bs.xyz[bs.shell_center[s1]] + bs.xyz[bs.shell_center[s2]])
    scale = 0.6
    g = xg * scale
    P = np.stack(np.meshgrid(g, g, g, indexing='ij'), -1).reshape(-1, 3) + mid
    W = (np.einsum('i,j,k->ijk', wg, wg, wg).reshape(-1)) * scale ** 3 * np.exp(((P - mid) ** 2).sum(-1) / scale ** 2)
    S_or = ob.overlap_block(ob.nsh + s1, ob.nsh + s2)     # derivative functions
    N1 = 1 / np.sqrt([np.sum(W * func_values(s1, None, c, P) ** 2) for c in range(oracle.ncart(int(bs.shell_l[s1])))])
    N2 = 1 / np.sqrt([np.sum(W * func_values(s2, None, c, P) ** 2) for c in range(oracle.ncart(int(bs.shell_l[s2])))])
    for m1 in range(S_or.shape[0]):
        for m2 in range(S_or.shape[1]):
            f1 = func_values(s1, m1 % 3, m1 // 3, P) * N1[m1 // 3]
            f2 = func_values(s2, m2 % 3, m2 // 3, P) * N2[m2 // 3]
            ref = np.sum(W * f1 * f2)
            assert abs(S_or[m1, m2] - ref) < 1e-9 * max(1, abs(ref))


def test_derivative_functions_are_minus_centre_derivatives(oracle):
    """(d_K chi_mu ...| ...) = -d/dA_K (chi_mu ...|...) when chi_mu alone sits
    on centre A: pins the small-component (derivative) basis."""
    rng = np.random.default_rng(5)
    xyz = rng.uniform(-1, 1, (4, 3))
    def basis_at(x0):
        x = xyz.copy(); x[0] = x0
        return synth.Basis(x, np.array([0, 1, 2, 3], np.int32), np.array([1, 0, 1, 0], np.int32),
                           np.array([2, 2, 1, 2], np.int32),
                           np.array([1.3, 0.4, 0.9, 2.0, 0.3, 0.7, 1.5]),
                           np.array([0.6, 0.8, 0.5, 0.9, 1.0, 0.4, 0.7]))
    ob = oracle.OracleBasis(basis_at(xyz[0]))
    n = ob.nsh
    blkS = ob.shell_block(0, n + 0, 1, 2, 3)            # derivative shell of shell 0
    for K in range(3):
        def f(X):
            o = oracle.OracleBasis(basis_at(X))
            return o.shell_block(0, 0, 1, 2, 3)
        d = fd_centre(f, xyz[0], K)
        for mu in range(3):
            assert np.abs(blkS[3 * mu + K] + d[mu]).max() <= 2e-7 * (np.abs(d).max() + 1e-3)
