"""Seeded synthetic inputs for the quaternion AO->MO transformation.

This module holds the input recipe only: geometries, raw Gaussian exponents and
contraction coefficients, and orthonormal quaternion MO coefficients.  It
contains none of the transformation's arithmetic (no normalisation of basis
functions, no integrals, no densities), so both the CUDA path and the CPU
oracle can draw identical inputs from it.

Recipe (stands in for the Dyall-basis Hg/Pu chains and the Au6 cluster of the
paper's Sec. 3, which are not available):
  * chains: centres on the x axis, spacing 1.4 bohr, every Cartesian coordinate
    jittered by U(-0.2, 0.2) bohr;
  * clusters: jittered simple-cubic grids with the same spacing and jitter;
  * shells: Cartesian s/p/d, ``nprim`` primitives each, exponents log-uniform
    in [lo, hi], raw contraction coefficients U(0.2, 1);
  * MO coefficients: quaternions q = q0 + q1 i + q2 j + q3 k over the
    nL large-component rows and the nS = 3 nL small-component (derivative
    basis) rows, every real part N(0, 1), orthonormalised by modified
    Gram-Schmidt on the Kramers-paired complex two-spinor columns, then the
    small-component rows scaled by 1/(2 * 137.036).
"""
from __future__ import annotations

import dataclasses
import numpy as np

C_LIGHT_GEN = 137.036       # speed of light used by the generator's S-row scaling
SEED_BASE = 20260000


@dataclasses.dataclass
class Basis:
    """Contracted Cartesian shells (large-component basis)."""
    xyz: np.ndarray            # [n_centers, 3] bohr
    shell_center: np.ndarray   # [n_shells] int32
    shell_l: np.ndarray        # [n_shells] int32
    shell_nprim: np.ndarray    # [n_shells] int32
    exps: np.ndarray           # [sum nprim] float64
    coefs: np.ndarray          # [sum nprim] float64 raw contraction coefficients

    @property
    def n_shells(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def nL(self) -> int:
        return int(sum((l + 1) * (l + 2) // 2 for l in self.shell_l))

    @property
    def nS(self) -> int:
        return 3 * self.nL


@dataclasses.dataclass
class Problem:
    name: str
    basis: Basis
    CL: np.ndarray             # [nL, nK, 4] quaternion coefficients
    CS: np.ndarray             # [nS, nK, 4]
    blocks: tuple              # subset of ("coulomb", "gaunt", "gauge")
    tau: float                 # Schwarz threshold
    kramers: bool = True       # False: CL/CS are per-spinor [nrows, n, 4] (Kramers-unrestricted)
    rkb: bool = False          # True: CS holds nL restricted-kinetic-balance rows c^S [nL, n, 4]

    @property
    def nK(self) -> int:
        return int(self.CL.shape[1])


def chain_xyz(rng, n, spacing=1.4, jitter=0.2):
    xyz = np.zeros((n, 3))
    xyz[:, 0] = spacing * np.arange(n)
    xyz += rng.uniform(-jitter, jitter, size=(n, 3))
    return xyz


def cluster_xyz(rng, dims, spacing=1.4, jitter=0.2):
    g = np.array([(i, j, k) for i in range(dims[0]) for j in range(dims[1])
                  for k in range(dims[2])], dtype=np.float64)
    return spacing * g + rng.uniform(-jitter, jitter, size=g.shape)


def make_basis(rng, xyz, shells_per_center, nprim, lo, hi):
    """shells_per_center(i) -> list of l values placed on centre i."""
    sc, sl, sn, ex, co = [], [], [], [], []
    for i in range(xyz.shape[0]):
        for l in shells_per_center(i):
            sc.append(i); sl.append(l); sn.append(nprim)
            e = np.exp(rng.uniform(np.log(lo), np.log(hi), size=nprim))
            ex.extend(np.sort(e)[::-1])
            co.extend(rng.uniform(0.2, 1.0, size=nprim))
    return Basis(np.ascontiguousarray(xyz, dtype=np.float64),
                 np.array(sc, np.int32), np.array(sl, np.int32),
                 np.array(sn, np.int32), np.array(ex, np.float64),
                 np.array(co, np.float64))


def quaternion_mos(rng, nrows, nK):
    """nK orthonormal Kramers-paired quaternion columns over ``nrows`` rows.

    Column k as a complex two-spinor: alpha = q0 + i q1, beta = q2 + i q3; its
    Kramers partner is (-conj(beta), conj(alpha)).  Gram-Schmidt against both
    members of every earlier pair keeps the quaternion structure.
    """
    if nK > 2 * nrows:
        raise ValueError("more Kramers pairs than the space holds")
    q = rng.standard_normal((nrows, nK, 4))
    cols = []
    for k in range(nK):
        v = np.concatenate([q[:, k, 0] + 1j * q[:, k, 1], q[:, k, 2] + 1j * q[:, k, 3]])
        for _ in range(2):
            for u in cols:
                v = v - u * np.vdot(u, v)
        v = v / np.linalg.norm(v)
        a, b = v[:nrows], v[nrows:]
        cols.append(v)
        cols.append(np.concatenate([-np.conj(b), np.conj(a)]))
    out = np.empty((nrows, nK, 4))
    for k in range(nK):
        v = cols[2 * k]
        out[:, k, 0] = v[:nrows].real; out[:, k, 1] = v[:nrows].imag
        out[:, k, 2] = v[nrows:].real; out[:, k, 3] = v[nrows:].imag
    return out


def coefficients(rng, nL, nK):
    Q = quaternion_mos(rng, 4 * nL, nK)
    CL = np.ascontiguousarray(Q[:nL])
    CS = np.ascontiguousarray(Q[nL:] / (2.0 * C_LIGHT_GEN))
    return CL, CS


def ku_coefficients(rng, nL, n):
    """Kramers-unrestricted coefficients: n orthonormal complex two-spinor
    columns over the nL large and 3 nL derivative rows (QR of a seeded complex
    Gaussian matrix), the S rows scaled by 1/(2c); per row and spinor the 4
    reals (Re alpha, Im alpha, Re beta, Im beta)."""
    rows = 4 * nL
    Z = rng.standard_normal((2 * rows, n)) + 1j * rng.standard_normal((2 * rows, n))
    Qm, _ = np.linalg.qr(Z)
    C = Qm.reshape(rows, 2, n)
    C4 = np.stack([C[:, 0].real, C[:, 0].imag, C[:, 1].real, C[:, 1].imag], axis=-1)   # [rows, n, 4]
    CL = np.ascontiguousarray(C4[:nL])
    CS = np.ascontiguousarray(C4[nL:] / (2.0 * C_LIGHT_GEN))
    return CL, CS


def ku_chain_problem(n_centers, n_spinors, *, seed, shells=(0, 1), nprim=3, lo=0.1, hi=10.0,
                     blocks=("coulomb",), tau=1e-12, name="ku-chain"):
    """The chain recipe with Kramers-unrestricted coefficients."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = chain_xyz(rng, n_centers)
    basis = make_basis(rng, xyz, lambda i: shells, nprim, lo, hi)
    CL, CS = ku_coefficients(rng, basis.nL, n_spinors)
    return Problem(name, basis, CL, CS, tuple(blocks), float(tau), kramers=False)


def rkb_chain_problem(n_centers, n, *, seed, shells=(0, 1), nprim=3, lo=0.1, hi=10.0,
                      blocks=("coulomb",), tau=1e-12, kramers=True, name="rkb-chain"):
    """The chain recipe with restricted-kinetic-balance small components: CS
    has nL rows (c^S of the large-component functions, not yet scaled by
    1/2c).  Coefficient scale as in the derivative-basis recipe: columns
    orthonormal over 4 nL rows, of which the first nL give c^L and the next
    nL give c^S."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = chain_xyz(rng, n_centers)
    basis = make_basis(rng, xyz, lambda i: shells, nprim, lo, hi)
    nL = basis.nL
    if kramers:
        Q = quaternion_mos(rng, 4 * nL, n)
    else:
        Z = rng.standard_normal((8 * nL, n)) + 1j * rng.standard_normal((8 * nL, n))
        C = np.linalg.qr(Z)[0].reshape(4 * nL, 2, n)
        Q = np.stack([C[:, 0].real, C[:, 0].imag, C[:, 1].real, C[:, 1].imag], axis=-1)
    CL, CS = np.ascontiguousarray(Q[:nL]), np.ascontiguousarray(Q[nL:2 * nL])
    return Problem(name, basis, CL, CS, tuple(blocks), float(tau), kramers=kramers, rkb=True)


def chain_problem(n_centers, nK, *, seed, shells=(0, 1), nprim=3, lo=0.1, hi=10.0,
                  blocks=("coulomb",), tau=1e-12, name="chain"):
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = chain_xyz(rng, n_centers)
    basis = make_basis(rng, xyz, lambda i: shells, nprim, lo, hi)
    CL, CS = coefficients(rng, basis.nL, nK)
    return Problem(name, basis, CL, CS, tuple(blocks), float(tau))


def cluster_problem(dims, nK, *, seed, shells_fn=None, nprim=3, lo=0.1, hi=10.0,
                    blocks=("coulomb", "gaunt", "gauge"), tau=1e-12, name="cluster"):
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = cluster_xyz(rng, dims)
    basis = make_basis(rng, xyz, shells_fn or (lambda i: (0, 1)), nprim, lo, hi)
    CL, CS = coefficients(rng, basis.nL, nK)
    return Problem(name, basis, CL, CS, tuple(blocks), float(tau))


def tiny_dc(seed=SEED_BASE + 0):
    """6 centres on a line, 2 uncontracted s per centre, nL=12, nS=36, 8 Kramers
    pairs, Dirac-Coulomb, Schwarz threshold 0."""
    return chain_problem(6, 8, seed=seed, shells=(0, 0), nprim=1, blocks=("coulomb",),
                         tau=0.0, name="tiny-dc-6s")


def medium_dc(seed=SEED_BASE + 1, n_centers=40, nK=40):
    """40-centre chain, contracted s+p (3 primitives), nL=160, nS=480, 40 Kramers
    pairs, Dirac-Coulomb, Schwarz threshold 1e-12."""
    return chain_problem(n_centers, nK, seed=seed, shells=(0, 1), nprim=3,
                         blocks=("coulomb",), tau=1e-12, name=f"chain{n_centers}-sp-dc")


def dcb_cluster(seed=SEED_BASE + 2, dims=(4, 4, 4), nK=64):
    """4x4x4 jittered cubic cluster, s+p, nL=256, nS=768, 64 Kramers pairs,
    Coulomb + Gaunt + gauge, Schwarz threshold 1e-12."""
    return cluster_problem(dims, nK, seed=seed, blocks=("coulomb", "gaunt", "gauge"),
                           tau=1e-12, name="cluster%dx%dx%d-sp-dcb" % tuple(dims))


def large_dcb(seed=SEED_BASE + 4, dims=(8, 5, 4), nK=100):
    """160-centre cluster; s on every centre, p on every 2nd, d on every 4th
    (nL=640, nS=1920); exponents log-uniform in [0.05, 30]; 100 Kramers pairs."""
    def shells(i):
        s = [0]
        if i % 2 == 0:
            s.append(1)
        if i % 4 == 0:
            s.append(2)
        return s
    return cluster_problem(dims, nK, seed=seed, shells_fn=shells, lo=0.05, hi=30.0,
                           name="cluster160-spd-dcb")


def serving_requests(n=256, seed=SEED_BASE + 3, nl_range=(24, 200), nk_range=(8, 48)):
    """Seeded request stream: chain or cluster, nL ~ U[24,200] (s+p), nK ~
    U[8,48], half Dirac-Coulomb and half Dirac-Coulomb-Breit, tau = 1e-11."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for i in range(n):
        ncent = max(1, int(rng.integers(nl_range[0], nl_range[1] + 1)) // 4)
        nK = int(rng.integers(nk_range[0], nk_range[1] + 1))
        nK = min(nK, 2 * 4 * ncent * 4)
        dcb = bool(rng.integers(0, 2))
        blocks = ("coulomb", "gaunt", "gauge") if dcb else ("coulomb",)
        if rng.integers(0, 2):
            p = chain_problem(ncent, nK, seed=seed + 1000 * (i + 1), blocks=blocks, tau=1e-11,
                              name=f"req{i}-chain{ncent}")
        else:
            side = max(1, round(ncent ** (1 / 3)))
            dims = (side, side, max(1, ncent // (side * side)))
            p = cluster_problem(dims, nK, seed=seed + 1000 * (i + 1), blocks=blocks, tau=1e-11,
                                name=f"req{i}-cluster")
        reqs.append(p)
    return reqs
