"""Plain, slow FP64 CPU oracle for the quaternion Dirac-Coulomb-Breit AO->MO
integral transformation (paper Secs. 2.1-2.5).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path: AO integrals come from ``qdt_oracle.c`` (Obara-Saika), and
everything else here is numpy written from the paper's equations.

Conventions (the paper leaves them to its references; readings listed in the
design notes):
  * quaternion q = q0 + q1 i + q2 j + q3 k of row a, Kramers pair k gives the
    two-spinor coefficients C[a, alpha, 2k] = q0 + i q1, C[a, beta, 2k] =
    q2 + i q3; the Kramers partner 2k+1 is C[a, alpha, 2k+1] = -conj(C[a, beta,
    2k]), C[a, beta, 2k+1] = conj(C[a, alpha, 2k]);
  * Mulliken order (pq|rs) = int int psi_p^+ psi_q (1/r12) psi_r^+ psi_s
    (Eq. AOtoMO);
  * Coulomb (Eq. DCInt):  sum_{X,Y in L,S} D^{X,pq}_{ab} (ab|cd) D^{Y,rs}_{cd},
    D^{pq}_{ab} = sum_tau conj(C[a,tau,p]) C[b,tau,q]   (Eq. Den);
  * Gaunt (Eq. GauntInt): sum_J over L-S and S-L pairs of D^{J,pq} (ab|cd)
    D^{J,rs}, D^{J,pq}_{ab} = sum conj(C[a,tau,p]) sigma_J[tau,tau'] C[b,tau',q];
  * gauge (Eq. gaugeInt): sum_{I,J} D^{I,pq}_{ab} (ab|r_I r_J / r^3|cd) D^{J,rs}_{cd};
  * Breit = -1/2 Gaunt - 1/2 gauge (from Eq. breit); blocks are returned
    unsigned and separately.
  * Screening (Eq. SchwarzDen): a shell quartet (AB, CD) is kept iff
    Q_AB * (Q_CD * Dmax_CD) >= tau, Q = max sqrt((ab|ab)) over the shell pair,
    Dmax = max |real part| of the symmetrised quaternion density over the
    pair's functions and all active Kramers-pair columns.
  * Packed output: for canonical Kramers pairs PQ (P<=Q), RS (R<=S), PQ<=RS,
    16 reals O[PQ,i][RS,j] = sum Dq[ab,PQ,i] G[ab,cd] Dq[cd,RS,j], with the 4
    real parts i of the symmetrised densities A = D^{PQ}, B = D^{P'Q}
    (P' = Kramers partner): (Re A, Im A, Re B, Im B).
  * Kramers-unrestricted input (the paper's runs, Sec. 3): every spinor p has
    its own coefficients C[a, tau, p], given per row as 4 reals (Re alpha,
    Im alpha, Re beta, Im beta); the densities are those of spinor pairs p <= q
    (D^{qp} = conj D^{pq} after symmetrisation), and the packed output holds 4
    reals O[pq,i][rs,j] (i, j = Re, Im) per canonical pair of pairs pq <= rs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()

SIGMA = np.array([[[0, 1], [1, 0]],
                  [[0, -1j], [1j, 0]],
                  [[1, 0], [0, -1]]], dtype=np.complex128)
IJ6 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def lib_path():
    return os.path.join(_HERE, "_build", "libqdt_oracle.so")


def build(force=False):
    """Compile the C part of the oracle with gcc (seconds)."""
    out = lib_path()
    src = os.path.join(_HERE, "qdt_oracle.c")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                           "-D_DEFAULT_SOURCE", src, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lp = ctypes.POINTER(ctypes.c_long)
            L.or_boys.argtypes = [ctypes.c_double, ctypes.c_int, dp]
            L.or_boys_minus1.argtypes = [ctypes.c_double]
            L.or_boys_minus1.restype = ctypes.c_double
            L.or_prim_block.argtypes = [ctypes.c_int] + [dp, ctypes.c_double, ctypes.c_int] * 4 + [dp]
            L.or_prim_ddr.argtypes = [ctypes.c_int] + [dp, ctypes.c_double, ctypes.c_int] * 4 + [dp]
            L.or_basis_create.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, ip, ip, dp, dp]
            L.or_basis_create.restype = ctypes.c_void_p
            L.or_basis_free.argtypes = [ctypes.c_void_p]
            L.or_basis_sizes.argtypes = [ctypes.c_void_p, ip]
            L.or_shell_block.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, dp]
            L.or_npairs.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.or_npairs.restype = ctypes.c_long
            L.or_pair_rows.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_long, lp, dp]
            L.or_pair_matrix.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, dp]
            L.or_pair_diag.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
            L.or_shell_pair_rows.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_void_p, lp, dp]
            L.or_shell_pair_rows.restype = ctypes.c_long
            L.or_set_threads.argtypes = [ctypes.c_int]
            L.or_set_threads.restype = None
            L.or_overlap_block.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, dp]
            _LIB = L
    return _LIB


def set_threads(n):
    """Host threads of the C integral loops (OpenMP)."""
    lib().or_set_threads(int(n))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# --------------------------------------------------------------- primitives

def boys(T, mmax):
    F = np.zeros(mmax + 1)
    lib().or_boys(float(T), int(mmax), _dp(F))
    return F


def boys_minus1(T):
    return lib().or_boys_minus1(float(T))


def ncart(l):
    return (l + 1) * (l + 2) // 2


def cart_list(l):
    """Cartesian exponent triples of order l in the library's order."""
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


def prim_block(kernel, A, a, la, B, b, lb, C, c, lc, D, d, ld):
    """Primitive Cartesian block, unnormalised Gaussians; kernel 0 = 1/r12, 1 = r12."""
    out = np.zeros((ncart(la), ncart(lb), ncart(lc), ncart(ld)))
    keep = [np.ascontiguousarray(v, dtype=np.float64) for v in (A, B, C, D)]
    args = []
    for X, e, l in zip(keep, (a, b, c, d), (la, lb, lc, ld)):
        args += [_dp(X), float(e), int(l)]
    lib().or_prim_block(int(kernel), *args, _dp(out))
    return out


def prim_ddr(form, A, a, la, B, b, lb, C, c, lc, D, d, ld):
    """(ab| d_I d_J r12 |cd) primitive blocks [6][...], form 1 or 2."""
    out = np.zeros((6, ncart(la), ncart(lb), ncart(lc), ncart(ld)))
    keep = [np.ascontiguousarray(v, dtype=np.float64) for v in (A, B, C, D)]
    args = []
    for X, e, l in zip(keep, (a, b, c, d), (la, lb, lc, ld)):
        args += [_dp(X), float(e), int(l)]
    lib().or_prim_ddr(int(form), *args, _dp(out))
    return out


# ------------------------------------------------------------------- basis

class OracleBasis:
    """Large-component shells and their derivative (small-component) shells."""

    def __init__(self, basis):
        self.basis = basis
        self._keep = [np.ascontiguousarray(basis.xyz, dtype=np.float64),
                      np.ascontiguousarray(basis.shell_center, dtype=np.int32),
                      np.ascontiguousarray(basis.shell_l, dtype=np.int32),
                      np.ascontiguousarray(basis.shell_nprim, dtype=np.int32),
                      np.ascontiguousarray(basis.exps, dtype=np.float64),
                      np.ascontiguousarray(basis.coefs, dtype=np.float64)]
        k = self._keep
        self.h = lib().or_basis_create(int(k[0].shape[0]), _dp(k[0]), int(k[1].shape[0]), _ip(k[1]),
                                       _ip(k[2]), _ip(k[3]), _dp(k[4]), _dp(k[5]))
        sz = np.zeros(3, np.int32)
        lib().or_basis_sizes(self.h, _ip(sz))
        self.nL, self.nS, self.nsh = int(sz[0]), int(sz[1]), int(sz[2])
        nc = [ncart(int(l)) for l in basis.shell_l]
        self.Loff = np.concatenate([[0], np.cumsum(nc)]).astype(np.int64)
        # shell of every L function and every S function
        self.shell_of_L = np.repeat(np.arange(self.nsh), nc)
        self.shell_of_S = np.repeat(self.shell_of_L, 3)
        # d/dr_K chi_i and d/dr_i chi_K of one p shell are the same function
        # (delta_iK g - 2 a x_i x_K g): canonical S index of every S function
        canon = np.arange(self.nS)
        for s_ in range(self.nsh):
            if int(basis.shell_l[s_]) == 1:
                mu0 = int(self.Loff[s_])
                for i in range(3):
                    for K in range(3):
                        canon[3 * (mu0 + i) + K] = 3 * (mu0 + min(i, K)) + max(i, K)
        self.s_canonical = canon
        self._pairs = {}

    def __del__(self):
        try:
            lib().or_basis_free(self.h)
        except Exception:
            pass

    # function pairs ------------------------------------------------------
    def pairs(self, cls):
        """(a, b, shell_pair_id) arrays of the class-``cls`` function pairs.
        cls 0: LL pairs a<=b then SS pairs a<=b (S functions offset by nL in
        the combined index used by ``a``/``b``); cls 1: L-S pairs a*nS+b."""
        if cls in self._pairs:
            return self._pairs[cls]
        nL, nS, n = self.nL, self.nS, self.nsh
        if cls == 0:
            iL, jL = np.triu_indices(nL)
            iS, jS = np.triu_indices(nS)
            sa = np.concatenate([self.shell_of_L[iL], n + self.shell_of_S[iS]])
            sb = np.concatenate([self.shell_of_L[jL], n + self.shell_of_S[jS]])
            a = np.concatenate([iL, nL + iS])
            b = np.concatenate([jL, nL + jS])
            # shell pair ids: LL (A<=B) then SS (A<=B), row-major
            lo, hi = np.minimum(sa % n, sb % n), np.maximum(sa % n, sb % n)
            spid = lo * n - lo * (lo - 1) // 2 + (hi - lo) + np.where(sa >= n, n * (n + 1) // 2, 0)
        else:
            a = np.repeat(np.arange(nL), nS)
            b = np.tile(np.arange(nS), nL)
            spid = self.shell_of_L[a] * n + self.shell_of_S[b]
            b = b + nL
        r = (a.astype(np.int64), b.astype(np.int64), spid.astype(np.int64))
        self._pairs[cls] = r
        return r

    def npairs(self, cls):
        return int(lib().or_npairs(self.h, cls))

    def n_shell_pairs(self, cls):
        n = self.nsh
        return n * (n + 1) if cls == 0 else n * n

    def pair_matrix(self, cls, kernel):
        """cls 0 kernel 0: G_C [M,M]; cls 1 kernel 0: G_G [M,M];
        cls 1 kernel 2: gauge [6,M,M] (IJ = xx,xy,xz,yy,yz,zz)."""
        M = self.npairs(cls)
        shape = (6, M, M) if kernel == 2 else (M, M)
        out = np.zeros(shape)
        lib().or_pair_matrix(self.h, cls, kernel, _dp(out))
        return out

    def pair_rows(self, cls, kernel, rows):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        M = self.npairs(cls)
        out = np.zeros((rows.shape[0], 6, M) if kernel == 2 else (rows.shape[0], M))
        lib().or_pair_rows(self.h, cls, kernel, int(rows.shape[0]),
                           rows.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(out))
        return out

    def shell_pair_rows(self, cls, kernel, p, keep):
        """Rows of the pair matrix for the function pairs of shell pair ``p``
        (the ``pairs(cls)`` shell-pair id), computed only against the ket shell
        pairs with keep[q] true (the others stay zero).  Returns (row pair
        indices [n], values [n, M] or [n, 6, M] for kernel 2)."""
        M = self.npairs(cls)
        keep = np.ascontiguousarray(keep, dtype=np.uint8)
        n = self.n_shell_pairs(cls)
        if keep.shape != (n,):
            raise ValueError("keep must have one entry per shell pair")
        sa, sb = self._shell_pair_shells(cls, int(p))
        nmax = self._nfunc(sa) * self._nfunc(sb)
        ncomp = 6 if kernel == 2 else 1
        rows = np.zeros(nmax, np.int64)
        out = np.zeros((nmax, ncomp, M))
        nr = lib().or_shell_pair_rows(self.h, int(cls), int(kernel), int(p), keep.ctypes.data_as(ctypes.c_void_p),
                                      rows.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(out))
        rows, out = rows[:nr], out[:nr]
        return rows, (out if kernel == 2 else out[:, 0, :])

    def _shell_pair_shells(self, cls, p):
        """Oracle shells (index >= nsh: derivative shell) of shell pair p:
        class 0 = LL pairs A <= B (row-major) then SS pairs A <= B; class 1 =
        (A, derivative shell of B), p = A nsh + B."""
        n = self.nsh
        if cls == 1:
            return p // n, n + p % n
        off = 0
        if p >= n * (n + 1) // 2:
            p -= n * (n + 1) // 2
            off = n
        a = 0
        while p >= n - a:
            p -= n - a
            a += 1
        return a + off, a + p + off

    def pair_diag(self, cls):
        out = np.zeros(self.npairs(cls))
        lib().or_pair_diag(self.h, cls, _dp(out))
        return out

    def shell_block(self, mode, sa, sb, sc, sd):
        nf = [self._nfunc(s) for s in (sa, sb, sc, sd)]
        out = np.zeros(((6,) if mode >= 2 else ()) + tuple(nf))
        lib().or_shell_block(self.h, int(mode), int(sa), int(sb), int(sc), int(sd), _dp(out))
        return out

    def overlap_block(self, sa, sb):
        out = np.zeros((self._nfunc(sa), self._nfunc(sb)))
        lib().or_overlap_block(self.h, int(sa), int(sb), _dp(out))
        return out

    def _nfunc(self, s):
        l = int(self.basis.shell_l[s % self.nsh])
        return ncart(l) * (3 if s >= self.nsh else 1)


# ------------------------------------------------------------ coefficients

def spinor_coefficients(Cq, k_begin=0, k_end=None):
    """Quaternion coefficients [nrows, nK, 4] -> complex two-spinor coefficients
    [nrows, 2 (alpha, beta), 2 nKa] with spinor 2k = Kramers pair k and 2k+1 its
    partner."""
    if k_end is None:
        k_end = Cq.shape[1]
    q = Cq[:, k_begin:k_end, :]
    ca = q[..., 0] + 1j * q[..., 1]
    cb = q[..., 2] + 1j * q[..., 3]
    n = 2 * q.shape[1]
    C = np.zeros((q.shape[0], 2, n), dtype=np.complex128)
    C[:, 0, 0::2] = ca
    C[:, 1, 0::2] = cb
    C[:, 0, 1::2] = -np.conj(cb)
    C[:, 1, 1::2] = np.conj(ca)
    return C


def rkb_to_derivative(CS4, c_light, spinors=False):
    """Restricted kinetic balance (Eq. RKB): chi^S_mu = (1/2c) sigma.p chi^L_mu
    with p = -i grad, so sum_mu chi^S_mu c^S_mu = sum_{mu,K} d_K chi_mu
    Ct[(mu,K)] with Ct[(mu,K)] = (-i/2c) sigma_K c^S_mu.  Small-component
    coefficients [nL, n, 4] -> derivative-basis coefficients [3 nL, n, 4]
    (rows 3 mu + K).  spinors=False: quaternion columns (the Kramers partner
    maps to the partner of the image, so the unbarred member carries it);
    spinors=True: per-spinor (Re a, Im a, Re b, Im b)."""
    if spinors:
        C = np.stack([CS4[..., 0] + 1j * CS4[..., 1], CS4[..., 2] + 1j * CS4[..., 3]], axis=1)
    else:
        C = spinor_coefficients(CS4)[:, :, 0::2]                   # the unbarred spinors
    nL, n = C.shape[0], C.shape[2]
    Ct = np.einsum('Kuv,mvp->mKup', SIGMA, C) * (-1j / (2.0 * c_light))
    Ct = Ct.reshape(3 * nL, 2, n)
    a, b = Ct[:, 0], Ct[:, 1]
    return np.ascontiguousarray(np.stack([a.real, a.imag, b.real, b.imag], axis=-1))


def kramers_pairs(nKa):
    """Canonical Kramers-pair list (P<=Q), row-major."""
    return [(P, Q) for P in range(nKa) for Q in range(P, nKa)]


def spinor_coefficients_ku(C4, s_begin=0, s_end=None):
    """Kramers-unrestricted coefficients [nrows, n, 4] (Re alpha, Im alpha,
    Re beta, Im beta per spinor) -> complex two-spinor coefficients
    [nrows, 2 (alpha, beta), s_end - s_begin]."""
    if s_end is None:
        s_end = C4.shape[1]
    q = C4[:, s_begin:s_end, :]
    C = np.zeros((q.shape[0], 2, q.shape[1]), dtype=np.complex128)
    C[:, 0, :] = q[..., 0] + 1j * q[..., 1]
    C[:, 1, :] = q[..., 2] + 1j * q[..., 3]
    return C


def spinor_pairs(n):
    """Canonical spinor-pair list (p<=q), row-major."""
    return [(p, q) for p in range(n) for q in range(p, n)]


# ----------------------------------------------------------------- densities

def quaternion_density_coulomb(ob, CL, CS):
    """Symmetrised real quaternion density Dq[pair, rs*4 + part] over the
    class-0 pairs (LL then SS), parts (Re A, Im A, Re B, Im B) with
    A = D^{R S}, B = D^{R' S} (Eqs. Den, QuaternionScatter)."""
    a, b, _ = ob.pairs(0)
    C = np.concatenate([CL, CS], axis=0)          # [nL+nS, 2, n]
    nKa = C.shape[2] // 2
    prs = kramers_pairs(nKa)
    R = np.array([p for p, _ in prs]); S = np.array([q for _, q in prs])
    out = np.zeros((a.shape[0], len(prs), 4))
    for which, rsp in ((0, 2 * R), (1, 2 * R + 1)):
        # D^{x y}_{ab} = sum_tau conj(C[a,tau,x]) C[b,tau,y]
        Dab = np.einsum('ptk,ptk->pk', np.conj(C[a][:, :, rsp]), C[b][:, :, 2 * S])
        Dba = np.einsum('ptk,ptk->pk', np.conj(C[b][:, :, rsp]), C[a][:, :, 2 * S])
        sym = np.where((a == b)[:, None], Dab, Dab + Dba)
        out[:, :, 2 * which] = sym.real
        out[:, :, 2 * which + 1] = sym.imag
    return out.reshape(a.shape[0], -1)


def quaternion_density_gaunt(ob, CL, CS):
    """Folded L-S alpha-density Dg[pair, J, rs*4 + part] over the class-1 pairs
    (a in L, b in S): D^{J}_{ab} + D^{J}_{ba} with sigma_J between the spin
    components (Eq. GauntInt)."""
    a, b, _ = ob.pairs(1)
    bS = b - ob.nL
    nKa = CL.shape[2] // 2
    prs = kramers_pairs(nKa)
    R = np.array([p for p, _ in prs]); S = np.array([q for _, q in prs])
    out = np.zeros((a.shape[0], 3, len(prs), 4))
    for J in range(3):
        sg = SIGMA[J]
        for which, rsp in ((0, 2 * R), (1, 2 * R + 1)):
            # L first: conj(CL[a]) sigma CS[b];  S first: conj(CS[b]) sigma CL[a]
            d1 = np.einsum('ptk,tu,puk->pk', np.conj(CL[a][:, :, rsp]), sg, CS[bS][:, :, 2 * S])
            d2 = np.einsum('ptk,tu,puk->pk', np.conj(CS[bS][:, :, rsp]), sg, CL[a][:, :, 2 * S])
            out[:, J, :, 2 * which] = (d1 + d2).real
            out[:, J, :, 2 * which + 1] = (d1 + d2).imag
    return out.reshape(a.shape[0], 3, -1)


def ku_density_coulomb(ob, CL, CS):
    """Symmetrised spinor-pair density D[pair, pq*2 + part] over the class-0
    pairs, parts (Re, Im) of D^{pq}_{ab} + D^{pq}_{ba} (a != b), p <= q (Eq. Den)."""
    a, b, _ = ob.pairs(0)
    C = np.concatenate([CL, CS], axis=0)
    prs = spinor_pairs(C.shape[2])
    P = np.array([p for p, _ in prs]); Q = np.array([q for _, q in prs])
    Dab = np.einsum('ptk,ptk->pk', np.conj(C[a][:, :, P]), C[b][:, :, Q])
    Dba = np.einsum('ptk,ptk->pk', np.conj(C[b][:, :, P]), C[a][:, :, Q])
    sym = np.where((a == b)[:, None], Dab, Dab + Dba)
    out = np.stack([sym.real, sym.imag], axis=-1)
    return out.reshape(a.shape[0], -1)


def ku_density_gaunt(ob, CL, CS):
    """Folded L-S alpha-density of spinor pairs D[pair, J, pq*2 + part] over
    the class-1 pairs (a in L, b in S), sigma_J between the spin components
    (Eq. GauntInt)."""
    a, b, _ = ob.pairs(1)
    bS = b - ob.nL
    prs = spinor_pairs(CL.shape[2])
    P = np.array([p for p, _ in prs]); Q = np.array([q for _, q in prs])
    out = np.zeros((a.shape[0], 3, len(prs), 2))
    for J in range(3):
        sg = SIGMA[J]
        d1 = np.einsum('ptk,tu,puk->pk', np.conj(CL[a][:, :, P]), sg, CS[bS][:, :, Q])
        d2 = np.einsum('ptk,tu,puk->pk', np.conj(CS[bS][:, :, P]), sg, CL[a][:, :, Q])
        out[:, J, :, 0] = (d1 + d2).real
        out[:, J, :, 1] = (d1 + d2).imag
    return out.reshape(a.shape[0], 3, -1)


# ---------------------------------------------------------------- screening

def schwarz_q(ob, cls):
    """Q per shell pair of a class: max over its function pairs of sqrt((ab|ab))
    (Coulomb diagonal; the gauge block uses the Coulomb Q of its L-S pairs)."""
    diag = ob.pair_diag(cls)
    _, _, sp = ob.pairs(cls)
    Q = np.zeros(ob.n_shell_pairs(cls))
    np.maximum.at(Q, sp, np.sqrt(np.abs(diag)))
    return Q


def density_max(ob, cls, Dq):
    """Dmax per shell pair: max |entry| of the density over the pair's distinct
    functions.  Rows of identical derivative functions (d_K chi_i = d_i chi_K of
    a p shell) are summed first, so the density is that of the actual basis
    functions (Eq. SchwarzDen)."""
    a, b, sp = ob.pairs(cls)
    nL = ob.nL
    X = Dq.reshape(Dq.shape[0], -1)
    ca = np.where(a >= nL, nL + ob.s_canonical[np.clip(a - nL, 0, None)], a)
    cb = np.where(b >= nL, nL + ob.s_canonical[np.clip(b - nL, 0, None)], b)
    if cls == 0:
        lo, hi = np.minimum(ca, cb), np.maximum(ca, cb)
    else:
        lo, hi = ca, cb
    nF = nL + ob.nS
    key = lo.astype(np.int64) * nF + hi
    uk, inv = np.unique(key, return_inverse=True)
    merged = np.zeros((uk.shape[0], X.shape[1]))
    np.add.at(merged, inv, X)
    kmax = np.abs(merged).max(axis=1) if X.size else np.zeros(uk.shape[0])
    Dm = np.zeros(ob.n_shell_pairs(cls))
    np.maximum.at(Dm, sp, kmax[inv])
    return Dm


def coefficient_bound_max(ob, CL4, CS4):
    """Screening bound of the O(N^5) quarter route (Sec. 2.2), which forms no
    density: per Coulomb-class shell pair, 2 m_A m_B with m_F the largest
    two-spinor norm |C_{fk}| over the shell's functions f and the given columns
    (CL4 [nL, n, 4], CS4 [nS, n, 4]: Re a, Im a, Re b, Im b per column, Kramers
    pairs or spinors alike).  By Cauchy-Schwarz it bounds every entry of the
    symmetrised density of the pair (Eq. Den), partner columns included.  Rows
    of identical derivative functions are summed first, as in density_max."""
    nL = ob.nL
    merged = np.zeros((ob.nS,) + CS4.shape[1:])
    np.add.at(merged, ob.s_canonical, CS4)
    C = np.concatenate([CL4, merged], axis=0)
    sq = C[..., 0] ** 2 + C[..., 1] ** 2 + C[..., 2] ** 2 + C[..., 3] ** 2
    m2 = sq.max(axis=1) if sq.shape[1] else np.zeros(sq.shape[0])
    a, b, sp = ob.pairs(0)
    ca = np.where(a >= nL, nL + ob.s_canonical[np.clip(a - nL, 0, None)], a)
    cb = np.where(b >= nL, nL + ob.s_canonical[np.clip(b - nL, 0, None)], b)
    ma = np.zeros(ob.n_shell_pairs(0))
    mb = np.zeros(ob.n_shell_pairs(0))
    np.maximum.at(ma, sp, m2[ca])
    np.maximum.at(mb, sp, m2[cb])
    return 2.0 * np.sqrt(ma) * np.sqrt(mb)


def screen_mask(Q, Dmax, tau):
    """keep[AB, CD] = Q_AB * (Q_CD * Dmax_CD) >= tau (Eq. SchwarzDen)."""
    w = Q * Dmax
    return (Q[:, None] * w[None, :]) >= tau


# ----------------------------------------------------------------- transform

def _expand_full(ob, cls, G):
    """Pair matrix over packed/class pairs -> 4-index tensor over the combined
    function list F = L (0..nL-1) then S (nL..nL+nS-1)."""
    nF = ob.nL + ob.nS
    a, b, _ = ob.pairs(cls)
    if G.ndim == 2:
        T = np.zeros((nF, nF, nF, nF))
        T[a[:, None], b[:, None], a[None, :], b[None, :]] = G
        T[b[:, None], a[:, None], a[None, :], b[None, :]] = G
        T[a[:, None], b[:, None], b[None, :], a[None, :]] = G
        T[b[:, None], a[:, None], b[None, :], a[None, :]] = G
        return T
    raise ValueError


def apply_screen(ob, cls, G, mask):
    _, _, sp = ob.pairs(cls)
    keep = mask[sp[:, None], sp[None, :]]
    if G.ndim == 3:
        return G * keep[None]
    return G * keep


class Transform:
    """Everything the oracle knows about one transformation request."""

    def __init__(self, problem, k_begin=0, k_end=None, tau=None, bound="density"):
        self.p = problem
        self.ob = OracleBasis(problem.basis)
        self.bound = bound       # Coulomb screening weight: "density" or "coefficients"
        self.k_begin = k_begin
        self.k_end = problem.nK if k_end is None else k_end
        self.nKa = self.k_end - self.k_begin
        self.tau = problem.tau if tau is None else tau
        self.CL = spinor_coefficients(problem.CL, self.k_begin, self.k_end)
        self.CS = spinor_coefficients(problem.CS, self.k_begin, self.k_end)
        self._cache = {}

    # integrals
    def G(self, block):
        if block not in self._cache:
            if block == "coulomb":
                self._cache[block] = self.ob.pair_matrix(0, 0)
            elif block == "gaunt":
                self._cache[block] = self.ob.pair_matrix(1, 0)
            elif block == "gauge":
                self._cache[block] = self.ob.pair_matrix(1, 2)
        return self._cache[block]

    def density(self, block):
        key = "D" + ("C" if block == "coulomb" else "G")
        if key not in self._cache:
            if block == "coulomb":
                self._cache[key] = quaternion_density_coulomb(self.ob, self.CL, self.CS)
            else:
                self._cache[key] = quaternion_density_gaunt(self.ob, self.CL, self.CS)
        return self._cache[key]

    def mask(self, block):
        cls = 0 if block == "coulomb" else 1
        key = "mask%d" % cls
        if key not in self._cache:
            Q = schwarz_q(self.ob, cls)
            if cls == 0 and self.bound == "coefficients":
                ks = slice(self.k_begin, self.k_end)
                Dm = coefficient_bound_max(self.ob, self.p.CL[:, ks], self.p.CS[:, ks])
            else:
                Dm = density_max(self.ob, cls, self.density(block))
            self._cache[key] = screen_mask(Q, Dm, self.tau)
            self._cache["Q%d" % cls] = Q
            self._cache["Dmax%d" % cls] = Dm
        return self._cache[key]

    def screened_fraction(self, block):
        m = self.mask(block)
        return 1.0 - m.mean()

    def G_screened(self, block):
        cls = 0 if block == "coulomb" else 1
        return apply_screen(self.ob, cls, self.G(block), self.mask(block))

    # packed quaternion route: O = Dq^T G Dq --------------------------------
    def packed_full(self, block, screened=True):
        """O[(PQ,i), (RS,j)] for all canonical PQ, RS (symmetric matrix)."""
        G = self.G_screened(block) if screened else self.G(block)
        D = self.density(block)
        if block == "coulomb":
            return D.T @ (G @ D)
        if block == "gaunt":
            M = D.shape[0]
            out = 0
            for J in range(3):
                out = out + D[:, J, :].T @ (G @ D[:, J, :])
            return out
        # gauge: sum_IJ D^I^T K_IJ D^J
        out = 0
        for ij, (I, J) in enumerate(IJ6):
            K = G[ij]
            t = D[:, I, :].T @ (K @ D[:, J, :])
            out = out + t if I == J else out + t + t.T
        return out

    def packed(self, block, screened=True):
        return pack_canonical(self.packed_full(block, screened), self.nKa)

    # the same, streamed by bra shell pairs (large systems) ----------------
    def V_rows_streamed(self, block, bra_pairs=None):
        """First half V = G_screened D (Eq. firsthalf) one bra shell pair at a
        time, without the whole pair matrix: yields (rows, V[rows]) for every
        bra shell pair AB of ``bra_pairs`` (all if None), from the integral
        rows of AB's function pairs against the ket shell pairs the screening
        keeps for AB (Eq. SchwarzDen).  For a fixed AB the rule
        Q_AB (Q_CD Dmax_CD) >= tau keeps exactly the kets whose weight
        w_CD = Q_CD Dmax_CD is at least tau / Q_AB, a leading run of the kets
        in w order, so the contraction runs over the density rows of that run
        (asserted below).  V[rows] is [n, ncol] (Coulomb), [n, 3, ncol]
        (Gaunt, one slice per J) or [n, 3, ncol] (gauge: V^I = sum_J K_IJ D^J)."""
        cls = 0 if block == "coulomb" else 1
        mask = self.mask(block)
        key = "order%d" % cls
        if key not in self._cache:
            Q, Dm = self._cache["Q%d" % cls], self._cache["Dmax%d" % cls]
            _, _, sp = self.ob.pairs(cls)
            order = np.argsort(-(Q * Dm)[sp], kind="stable")     # function-pair columns, w descending
            self._cache[key] = (order, self.density(block)[order])
        order, Dw = self._cache[key]
        _, _, sp = self.ob.pairs(cls)
        kernel = 2 if block == "gauge" else 0
        todo = range(self.ob.n_shell_pairs(cls)) if bra_pairs is None else bra_pairs
        for p in todo:
            keep = mask[p]
            kept = keep[sp[order]]
            n = int(kept.sum())
            assert kept[:n].all(), "screening kept set is not a leading run in w order"
            if n == 0:
                continue
            rows, G = self.ob.shell_pair_rows(cls, kernel, p, keep)
            if block == "coulomb":
                yield rows, G[:, order[:n]] @ Dw[:n]
            elif block == "gaunt":
                Gk = G[:, order[:n]]
                yield rows, np.stack([Gk @ Dw[:n, J] for J in range(3)], axis=1)
            else:
                Vr = np.zeros((rows.shape[0], 3, Dw.shape[-1]))
                for ij, (I, J) in enumerate(IJ6):
                    Kk = G[:, ij][:, order[:n]]
                    Vr[:, I] += Kk @ Dw[:n, J]
                    if I != J:
                        Vr[:, J] += Kk @ Dw[:n, I]
                yield rows, Vr

    def V_streamed(self, block, progress=None):
        """The whole V of V_rows_streamed, [M, ncol] or [M, 3, ncol]."""
        V = np.zeros(self.density(block).shape)
        n = self.ob.n_shell_pairs(0 if block == "coulomb" else 1)
        for i, (rows, Vr) in enumerate(self.V_rows_streamed(block)):
            V[rows] = Vr
            if progress and i % 200 == 0:
                progress(i, n)
        return V

    def second_half_rows(self, block, rows, Vr):
        """The contribution D[rows]^T V[rows] of some bra rows to O = D^T V
        (Eq. secondhalf; O is the sum over all bra rows)."""
        D = self.density(block)
        if block == "coulomb":
            return D[rows].T @ Vr
        return sum(D[rows, J, :].T @ Vr[:, J, :] for J in range(3))

    def packed_full_streamed(self, block, progress=None):
        """O = D^T V with V from V_streamed: the same matrix as packed_full
        (to rounding), within memory O(M ncol)."""
        V = self.V_streamed(block, progress=progress)
        D = self.density(block)
        if block == "coulomb":
            return D.T @ V
        return sum(D[:, J, :].T @ V[:, J, :] for J in range(3))

    def packed_streamed(self, block, progress=None):
        return pack_canonical(self.packed_full_streamed(block, progress), self.nKa)

    # MO-driven route (Sec. 3.3) ----------------------------------------------
    def _n_parts(self):
        return self.nKa, 4

    def mask_columns(self, block, c0, c1):
        """Screening mask from the density maximum over the columns [c0, c1)
        only (every J component of an L-S density)."""
        cls = 0 if block == "coulomb" else 1
        Q = schwarz_q(self.ob, cls)
        Dm = density_max(self.ob, cls, self.density(block)[..., c0:c1])
        return screen_mask(Q, Dm, self.tau)

    def packed_full_mo(self, block, nb):
        """O of the MO-driven route: the outer MO index r runs in blocks of nb;
        the density columns (r, s >= r, part) of a block are contracted with
        the integrals that the block's own density maximum keeps."""
        n, parts = self._n_parts()
        cls = 0 if block == "coulomb" else 1
        D = self.density(block)
        ncol = D.shape[-1]
        out = np.zeros((ncol, ncol))
        for r0 in range(0, n, nb):
            r1 = min(n, r0 + nb)
            c0 = parts * pair_index(r0, r0, n)
            c1 = parts * pair_index(r1, r1, n) if r1 < n else ncol
            G = apply_screen(self.ob, cls, self.G(block), self.mask_columns(block, c0, c1))
            if block == "coulomb":
                out[:, c0:c1] = D.T @ (G @ D[:, c0:c1])
            elif block == "gaunt":
                for J in range(3):
                    out[:, c0:c1] += D[:, J, :].T @ (G @ D[:, J, c0:c1])
            else:
                for ij, (I, J) in enumerate(IJ6):
                    K = G[ij]
                    out[:, c0:c1] += D[:, I, :].T @ (K @ D[:, J, c0:c1])
                    if I != J:
                        out[:, c0:c1] += D[:, J, :].T @ (K.T @ D[:, I, c0:c1])
        return out

    def packed_mo(self, block, nb):
        return pack_canonical(self.packed_full_mo(block, nb), self.nKa)

    # plain definition: full complex (pq|rs) ---------------------------------
    def full(self, block, screened=True):
        """(pq|rs) over all 2 nKa spinors by the literal sum over ordered AO
        pairs: sum D^{pq}_{ab} (ab|K|cd) D^{rs}_{cd}."""
        G = self.G_screened(block) if screened else self.G(block)
        C = np.concatenate([self.CL, self.CS], axis=0)      # [nF, 2, n]
        nL = self.ob.nL
        if block == "coulomb":
            T = _expand_full(self.ob, 0, G)
            # quarter transforms with the spin sum inside each density
            t1 = np.einsum('abcd,dts->abcts', T, C)
            t2 = np.einsum('ctr,abcts->abrs', np.conj(C), t1)
            t3 = np.einsum('btq,abrs->atqrs', C, t2)
            return np.einsum('atp,atqrs->pqrs', np.conj(C), t3)
        # L-S blocks: build the alpha densities over ordered pairs (a,b)
        n = C.shape[2]
        nF = C.shape[0]
        isL = np.arange(nF) < nL
        mixed = isL[:, None] != isL[None, :]
        DJ = np.einsum('atp,Jtu,bus->Jabps', np.conj(C), SIGMA, C) * mixed[None, :, :, None, None]
        a, b, _ = self.ob.pairs(1)
        if block == "gaunt":
            T = np.zeros((nF, nF, nF, nF))
            for (x, y) in ((a, b), (b, a)):
                for (u, v) in ((a, b), (b, a)):
                    T[x[:, None], y[:, None], u[None, :], v[None, :]] = G
            return np.einsum('Jabpq,abcd,Jcdrs->pqrs', DJ, T, DJ, optimize=True)
        out = np.zeros((n, n, n, n), dtype=np.complex128)
        for ij, (I, J) in enumerate(IJ6):
            T = np.zeros((nF, nF, nF, nF))
            for (x, y) in ((a, b), (b, a)):
                for (u, v) in ((a, b), (b, a)):
                    T[x[:, None], y[:, None], u[None, :], v[None, :]] = G[ij]
            t = np.einsum('abpq,abcd,cdrs->pqrs', DJ[I], T, DJ[J], optimize=True)
            out += t
            if I != J:
                out += np.einsum('abpq,abcd,cdrs->pqrs', DJ[J], T, DJ[I], optimize=True)
        return out


class TransformKU(Transform):
    """The same transformation for Kramers-unrestricted input: problem.CL/CS
    hold per-spinor coefficients [nrows, n, 4]; [s_begin, s_end) selects the
    active spinors.  G, screening rule and the literal definition full() are
    the Kramers-restricted ones; the densities are those of spinor pairs."""

    def __init__(self, problem, s_begin=0, s_end=None, tau=None, bound="density"):
        self.p = problem
        self.ob = OracleBasis(problem.basis)
        self.bound = bound
        self.k_begin = s_begin
        self.k_end = problem.CL.shape[1] if s_end is None else s_end
        self.n = self.k_end - self.k_begin
        self.tau = problem.tau if tau is None else tau
        self.CL = spinor_coefficients_ku(problem.CL, self.k_begin, self.k_end)
        self.CS = spinor_coefficients_ku(problem.CS, self.k_begin, self.k_end)
        self._cache = {}

    def density(self, block):
        key = "D" + ("C" if block == "coulomb" else "G")
        if key not in self._cache:
            if block == "coulomb":
                self._cache[key] = ku_density_coulomb(self.ob, self.CL, self.CS)
            else:
                self._cache[key] = ku_density_gaunt(self.ob, self.CL, self.CS)
        return self._cache[key]

    def packed(self, block, screened=True):
        return pack_canonical_ku(self.packed_full(block, screened), self.n)

    def _n_parts(self):
        return self.n, 2

    def packed_mo(self, block, nb):
        return pack_canonical_ku(self.packed_full_mo(block, nb), self.n)


# -------------------------------------------------------------- packing

def pair_index(P, Q, n):
    return P * n - P * (P - 1) // 2 + (Q - P)


def pack_canonical(Ofull, nKa):
    """Symmetric O[(PQ,i),(RS,j)] -> packed [nP(nP+1)/2, 16] over PQ <= RS."""
    nP = nKa * (nKa + 1) // 2
    O = Ofull.reshape(nP, 4, nP, 4)
    iu, ju = np.triu_indices(nP)
    return O[iu, :, ju, :].reshape(-1, 16).copy()


def _density_map(x, y, block):
    """Symmetrised spinor density of spinor pair (x, y) as (X, Y, which, sign,
    conj): D^{xy} = sign * [conj](Z), Z = A^{XY} (which 0) or B^{XY} (which 1),
    X <= Y Kramers pairs."""
    X, bx, Y, by = x // 2, x % 2, y // 2, y % 2
    swap = X > Y
    if swap:   # sym D^{xy} = conj(sym D^{yx})
        X, bx, Y, by = Y, by, X, bx
    gaunt = block != "coulomb"
    if (bx, by) == (0, 0):
        which, sign, cj = 0, 1.0, False
    elif (bx, by) == (1, 0):
        which, sign, cj = 1, 1.0, False
    elif (bx, by) == (0, 1):
        which, sign, cj = 1, (1.0 if gaunt else -1.0), True
    else:
        which, sign, cj = 0, (-1.0 if gaunt else 1.0), True
    if swap:
        cj = not cj
    return X, Y, which, sign, cj


def unpack(packed, nKa, block):
    """Packed canonical array -> full complex (pq|rs) over 2 nKa spinors."""
    nP = nKa * (nKa + 1) // 2
    O = np.zeros((nP, 4, nP, 4))
    iu, ju = np.triu_indices(nP)
    blk = packed.reshape(-1, 4, 4)
    O[iu, :, ju, :] = blk
    O[ju, :, iu, :] = blk.transpose(0, 2, 1)
    n = 2 * nKa
    out = np.zeros((n, n, n, n), dtype=np.complex128)
    maps = [[_density_map(x, y, block) for y in range(n)] for x in range(n)]
    for p in range(n):
        for q in range(n):
            X1, Y1, w1, s1, c1 = maps[p][q]
            i1 = pair_index(X1, Y1, nKa)
            for r in range(n):
                for s in range(n):
                    X2, Y2, w2, s2, c2 = maps[r][s]
                    i2 = pair_index(X2, Y2, nKa)
                    o = O[i1, :, i2, :]
                    re1, im1, re2, im2 = 2 * w1, 2 * w1 + 1, 2 * w2, 2 * w2 + 1
                    t1 = -1.0 if c1 else 1.0
                    t2 = -1.0 if c2 else 1.0
                    val = (o[re1, re2] - t1 * t2 * o[im1, im2]) + 1j * (t2 * o[re1, im2] + t1 * o[im1, re2])
                    out[p, q, r, s] = s1 * s2 * val
    return out


def pack_canonical_ku(Ofull, n):
    """Symmetric O[(pq,i),(rs,j)] over spinor pairs -> packed [nP(nP+1)/2, 4]
    over pq <= rs, nP = n(n+1)/2, entries (RR, RI, IR, II)."""
    nP = n * (n + 1) // 2
    O = Ofull.reshape(nP, 2, nP, 2)
    iu, ju = np.triu_indices(nP)
    return O[iu, :, ju, :].reshape(-1, 4).copy()


def unpack_ku(packed, n):
    """Packed Kramers-unrestricted array -> full complex (pq|rs) over n spinors:
    D^{pq} = Dr + i c Di with the pair (min, max) and c = -1 when p > q."""
    nP = n * (n + 1) // 2
    O = np.zeros((nP, 2, nP, 2))
    iu, ju = np.triu_indices(nP)
    blk = packed.reshape(-1, 2, 2)
    O[iu, :, ju, :] = blk
    O[ju, :, iu, :] = blk.transpose(0, 2, 1)
    out = np.zeros((n, n, n, n), dtype=np.complex128)
    for p in range(n):
        for q in range(n):
            i1 = pair_index(min(p, q), max(p, q), n)
            c1 = -1.0 if p > q else 1.0
            for r in range(n):
                for s_ in range(n):
                    i2 = pair_index(min(r, s_), max(r, s_), n)
                    c2 = -1.0 if r > s_ else 1.0
                    o = O[i1, :, i2, :]
                    out[p, q, r, s_] = (o[0, 0] - c1 * c2 * o[1, 1]) + 1j * (c2 * o[0, 1] + c1 * o[1, 0])
    return out
