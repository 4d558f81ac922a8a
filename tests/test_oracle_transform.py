"""Pins of the oracle's AO->MO transformation: a literal four-component brute
force, symmetries, identity coefficients, energy traces, the
nonrelativistic limit and the screening rule."""
import numpy as np
import pytest

from paper_2606_04316_gb300 import synth

BLOCKS = ("coulomb", "gaunt", "gauge")


def tiny(nK=2, seed=3, shells=(0, 0), ncent=2, nprim=1):
    return synth.chain_problem(ncent, nK, seed=seed, shells=shells, nprim=nprim,
                               blocks=BLOCKS, tau=0.0, name="tiny")


def four_spinors(tr):
    """psi_p[f, c], c = (L alpha, L beta, S alpha, S beta)."""
    nL = tr.ob.nL
    n = tr.CL.shape[2]
    nF = nL + tr.ob.nS
    psi = np.zeros((n, nF, 4), dtype=complex)
    psi[:, :nL, 0] = tr.CL[:, 0, :].T
    psi[:, :nL, 1] = tr.CL[:, 1, :].T
    psi[:, nL:, 2] = tr.CS[:, 0, :].T
    psi[:, nL:, 3] = tr.CS[:, 1, :].T
    return psi


def alpha_matrices():
    s = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    out = []
    for J in range(3):
        a = np.zeros((4, 4), dtype=complex)
        a[0:2, 2:4] = s[J]
        a[2:4, 0:2] = s[J]
        out.append(a)
    return out


def brute_force(tr, block, T4C, T4g):
    """(pq|rs) = sum over AO quadruples and four-spinor components of
    psi_p^+ M psi_q (ab|K|cd) psi_r^+ M' psi_s (Eqs. Coulomb, breit, DCInt,
    GauntInt, gaugeInt), one (p,q,r,s) at a time."""
    psi = four_spinors(tr)
    n = psi.shape[0]
    al = alpha_matrices()
    IJ6 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    out = np.zeros((n,) * 4, dtype=complex)
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for s in range(n):
                    if block == "coulomb":
                        r1 = np.einsum('ai,bi->ab', np.conj(psi[p]), psi[q])
                        r2 = np.einsum('ci,di->cd', np.conj(psi[r]), psi[s])
                        out[p, q, r, s] = np.einsum('ab,abcd,cd->', r1, T4C, r2)
                    elif block == "gaunt":
                        v = 0
                        for J in range(3):
                            r1 = np.einsum('ai,ij,bj->ab', np.conj(psi[p]), al[J], psi[q])
                            r2 = np.einsum('ci,ij,dj->cd', np.conj(psi[r]), al[J], psi[s])
                            v += np.einsum('ab,abcd,cd->', r1, T4C, r2)
                        out[p, q, r, s] = v
                    else:
                        v = 0
                        for I in range(3):
                            for J in range(3):
                                ij = IJ6.index((min(I, J), max(I, J)))
                                r1 = np.einsum('ai,ij,bj->ab', np.conj(psi[p]), al[I], psi[q])
                                r2 = np.einsum('ci,ij,dj->cd', np.conj(psi[r]), al[J], psi[s])
                                v += np.einsum('ab,abcd,cd->', r1, T4g[ij], r2)
                        out[p, q, r, s] = v
    return out


@pytest.fixture(scope="module")
def tiny_tr(oracle):
    tr = oracle.Transform(tiny())
    ob = tr.ob
    nF = ob.nL + ob.nS
    # Coulomb tensor over all pairs, including L-S pairs (class 1)
    T4C = np.zeros((nF,) * 4)
    for cls in (0, 1):
        a, b, _ = ob.pairs(cls)
        G = ob.pair_matrix(cls, 0)
        for (x, y) in ((a, b), (b, a)):
            for (u, v) in ((a, b), (b, a)):
                T4C[x[:, None], y[:, None], u[None, :], v[None, :]] = G
    # cross-class Coulomb (LL|LS) etc. is never needed: the four-spinor
    # component structure makes those products vanish.
    a, b, _ = ob.pairs(1)
    Gg = ob.pair_matrix(1, 2)
    T4g = np.zeros((6,) + (nF,) * 4)
    for ij in range(6):
        for (x, y) in ((a, b), (b, a)):
            for (u, v) in ((a, b), (b, a)):
                T4g[ij][x[:, None], y[:, None], u[None, :], v[None, :]] = Gg[ij]
    return tr, T4C, T4g


@pytest.mark.parametrize("block", BLOCKS)
def test_brute_force_four_component(tiny_tr, block):
    tr, T4C, T4g = tiny_tr
    bf = brute_force(tr, block, T4C, T4g)
    full = tr.full(block)
    scale = np.abs(bf).max()
    assert scale > 1e-6
    assert np.abs(full - bf).max() <= 1e-13 * scale


@pytest.mark.parametrize("block", BLOCKS)
def test_packed_unpacks_to_definition(oracle, tiny_tr, block):
    tr, _, _ = tiny_tr
    full = tr.full(block)
    un = oracle.unpack(tr.packed(block), tr.nKa, block)
    assert np.abs(un - full).max() <= 1e-13 * np.abs(full).max()


@pytest.fixture(scope="module")
def cfg0(oracle):
    p = synth.tiny_dc()
    return oracle.Transform(p)


def test_packed_unpacks_to_definition_tiny_config(oracle, cfg0):
    full = cfg0.full("coulomb")
    un = oracle.unpack(cfg0.packed("coulomb"), cfg0.nKa, "coulomb")
    assert np.abs(un - full).max() <= 1e-13 * np.abs(full).max()


@pytest.mark.parametrize("block", BLOCKS)
def test_symmetries(oracle, block):
    tr = oracle.Transform(tiny(nK=3, shells=(0, 1), nprim=2, seed=9))
    x = tr.full(block)
    n = x.shape[0]
    s = np.abs(x).max()
    # bra-ket exchange and hermiticity of each density
    assert np.abs(x - x.transpose(2, 3, 0, 1)).max() <= 1e-13 * s
    assert np.abs(x - np.conj(x.transpose(1, 0, 3, 2))).max() <= 1e-13 * s
    # Kramers: psi_{bar p} = eta_p K psi_p with K^2 = -1 (eta = +1 for even p,
    # -1 for odd p); (Kp Kq| = +-(q p| and (p Kq| = -+(q Kp|, the lower sign
    # for the time-odd alpha densities.
    bar = np.arange(n) ^ 1
    eta = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    E = (eta[:, None] * eta[None, :])[:, :, None, None]
    sign = 1.0 if block == "coulomb" else -1.0
    assert np.abs(x[bar][:, bar] - sign * E * x.transpose(1, 0, 2, 3)).max() <= 1e-13 * s
    z = x[:, bar].transpose(1, 0, 2, 3)
    assert np.abs(x[:, bar] + sign * E * z).max() <= 1e-13 * s


def test_real_coefficients_give_eightfold_symmetry(oracle):
    p = tiny(nK=3, shells=(0, 1), nprim=2, seed=4)
    p.CS[:] = 0.0
    p.CL[..., 1:] = 0.0                        # real alpha-only spinors
    tr = oracle.Transform(p)
    x = tr.full("coulomb")
    u = x[0::2, 0::2, 0::2, 0::2]              # unbarred spinors
    assert np.abs(u.imag).max() < 1e-14
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.abs(u - u.transpose(perm)).max() < 1e-13 * np.abs(u).max()


def test_nonrelativistic_limit_is_einsum(oracle):
    """C^S = 0, real alpha coefficients: the unbarred block is the plain real
    four-index transform of the LL integrals (Eq. AOtoMO)."""
    p = tiny(nK=3, shells=(0, 1), nprim=2, seed=4)
    p.CS[:] = 0.0
    p.CL[..., 1:] = 0.0
    tr = oracle.Transform(p)
    ob = tr.ob
    a, b, _ = ob.pairs(0)
    nLLp = ob.nL * (ob.nL + 1) // 2
    G = ob.pair_matrix(0, 0)[:nLLp, :nLLp]
    nL = ob.nL
    T = np.zeros((nL,) * 4)
    aa, bb = a[:nLLp], b[:nLLp]
    for (x, y) in ((aa, bb), (bb, aa)):
        for (u, v) in ((aa, bb), (bb, aa)):
            T[x[:, None], y[:, None], u[None, :], v[None, :]] = G
    c = p.CL[:, :, 0]
    ref = np.einsum('ap,bq,abcd,cr,ds->pqrs', c, c, T, c, c)
    x = tr.full("coulomb")[0::2, 0::2, 0::2, 0::2]
    assert np.abs(x - ref).max() < 1e-13 * np.abs(ref).max()
    # barred (beta) block equals the same numbers
    y = tr.full("coulomb")[1::2, 1::2, 1::2, 1::2]
    assert np.abs(y - ref).max() < 1e-13 * np.abs(ref).max()


def test_identity_coefficients_return_ao_integrals(oracle):
    """Kramers pair k = pure alpha/beta on one basis function gives back the
    scalar AO integrals (Coulomb over LL/SS, Coulomb over LS for Gaunt z)."""
    base = tiny(nK=1, shells=(0, 1), nprim=2, seed=12)
    ob = oracle.OracleBasis(base.basis)
    nL, nS = ob.nL, ob.nS
    fL = [0, 3]            # two large functions
    fS = [1, 7]            # two small functions
    nK = 4
    CL = np.zeros((nL, nK, 4)); CS = np.zeros((nS, nK, 4))
    CL[fL[0], 0, 0] = 1; CL[fL[1], 1, 0] = 1; CS[fS[0], 2, 0] = 1; CS[fS[1], 3, 0] = 1
    p = synth.Problem("identity", base.basis, CL, CS, BLOCKS, 0.0)
    tr = oracle.Transform(p)
    C = tr.full("coulomb")
    G = tr.ob.pair_matrix(0, 0)
    a, b, _ = tr.ob.pairs(0)
    lut = {(int(x), int(y)): i for i, (x, y) in enumerate(zip(a, b))}
    fn = [fL[0], fL[1], nL + fS[0], nL + fS[1]]           # combined indices
    def pidx(x, y):
        return lut[(min(x, y), max(x, y))]
    for k in range(4):
        for l in range(4):
            for m in range(4):
                for n in range(4):
                    x, y, u, v = fn[k], fn[l], fn[m], fn[n]
                    same1 = (x < nL) == (y < nL)
                    same2 = (u < nL) == (v < nL)
                    ref = G[pidx(x, y), pidx(u, v)] if (same1 and same2) else 0.0
                    assert abs(C[2 * k, 2 * l, 2 * m, 2 * n] - ref) < 1e-14
                    assert abs(C[2 * k + 1, 2 * l + 1, 2 * m, 2 * n] - ref) < 1e-14
                    assert abs(C[2 * k, 2 * l + 1, 2 * m, 2 * n]) < 1e-14
    # Gaunt: alpha-alpha element of sigma_z is 1 -> (L S | L S) Coulomb integrals
    Gt = tr.full("gaunt")
    GG = tr.ob.pair_matrix(1, 0)
    ls = lambda x, y: x * nS + (y - nL)
    ref = GG[ls(fn[0], fn[2]), ls(fn[1], fn[3])]
    assert abs(Gt[0, 4, 2, 6] - ref) < 1e-14


def test_energy_traces_ao_vs_mo(oracle):
    """Coulomb and exchange energies of an occupied subset agree between the
    MO integrals and the AO density contraction."""
    p = tiny(nK=3, shells=(0, 1), nprim=2, seed=21)
    tr = oracle.Transform(p)
    x = tr.full("coulomb")
    occ = [0, 1, 3, 4]
    EJ_mo = 0.5 * sum(x[i, i, j, j] for i in occ for j in occ)
    EK_mo = 0.5 * sum(x[i, j, j, i] for i in occ for j in occ)
    ob = tr.ob
    nF = ob.nL + ob.nS
    C = np.concatenate([tr.CL, tr.CS], axis=0)
    # spin-orbital density P[a tau, b tau'] = sum_i conj(C[a,tau,i]) C[b,tau',i]
    P = np.einsum('ati,bui->atbu', np.conj(C[:, :, occ]), C[:, :, occ])
    a, b, _ = ob.pairs(0)
    G = ob.pair_matrix(0, 0)
    T = np.zeros((nF,) * 4)
    for (xx, yy) in ((a, b), (b, a)):
        for (u, v) in ((a, b), (b, a)):
            T[xx[:, None], yy[:, None], u[None, :], v[None, :]] = G
    Ps = np.einsum('atbt->ab', P)
    EJ_ao = 0.5 * np.einsum('ab,abcd,cd->', Ps, T, Ps)
    # exchange: sum_ij (ij|ji) = sum P[a t, d u] (ab|cd) P[c u, b t]
    EK_ao = 0.5 * np.einsum('atdu,abcd,cubt->', P, T, P)
    assert abs(EJ_mo - EJ_ao) < 1e-12 * abs(EJ_ao)
    assert abs(EK_mo - EK_ao) < 1e-12 * abs(EK_ao)
    assert abs(EJ_mo.imag) < 1e-14 and abs(EK_mo.imag) < 1e-14


# ------------------------------------------------------------------ screening

def test_threshold_zero_keeps_everything(oracle):
    p = synth.chain_problem(3, 2, seed=31, shells=(0, 1), blocks=BLOCKS, tau=0.0)
    tr = oracle.Transform(p)
    for block in BLOCKS:
        assert tr.mask(block).all()
        assert np.array_equal(tr.packed(block, screened=True), tr.packed(block, screened=False))


def test_screening_error_within_bound(oracle):
    p = synth.chain_problem(6, 3, seed=32, shells=(0, 1), blocks=("coulomb",), tau=1e-6)
    tr = oracle.Transform(p)
    m = tr.mask("coulomb")
    assert 0 < m.mean() < 1
    diff = np.abs(tr.packed_full("coulomb", True) - tr.packed_full("coulomb", False)).max()
    # each dropped quartet contributes at most n_ab n_cd tau |Dq_bra|max to one element
    D = tr.density("coulomb")
    _, _, sp = tr.ob.pairs(0)
    Q, Dm = tr._cache["Q0"], tr._cache["Dmax0"]
    nfp = np.bincount(sp, minlength=len(Q))
    bound = 0.0
    Dbra = np.zeros(len(Q)); np.maximum.at(Dbra, sp, np.abs(D).max(axis=1))
    dropped = ~m
    bound = np.sum((nfp[:, None] * nfp[None, :] * Dbra[:, None] * Q[:, None] * Q[None, :] * Dm[None, :])[dropped])
    assert diff <= bound


def test_screened_fraction_grows_with_chain_and_ssss_most(oracle):
    """Tab. screening_pu trend: the screened share rises with chain length and
    the SSSS class is screened more than the whole Dirac-Coulomb set."""
    fr, fr_ssss = [], []
    for n in (6, 8, 12, 16):
        p = synth.chain_problem(n, 4, seed=40, shells=(0, 1), blocks=("coulomb",), tau=1e-12)
        tr = oracle.Transform(p)
        m = tr.mask("coulomb")
        fr.append(1 - m.mean())
        ns = tr.ob.nsh * (tr.ob.nsh + 1) // 2
        fr_ssss.append(1 - m[ns:, ns:].mean())
    assert all(b > a for a, b in zip(fr, fr[1:]))
    assert all(s > f for s, f in zip(fr_ssss, fr))


def test_noise_floor_of_a_second_summation_order(oracle):
    """The oracle's fixed order (D^T (G D)) against a second order ((D^T G) D):
    the FP64 noise floor sits far below the 1e-12 parity bar."""
    p = synth.chain_problem(4, 3, seed=655, shells=(0, 1), nprim=2, blocks=BLOCKS, tau=0.0)
    tr = oracle.Transform(p)
    for b in BLOCKS:
        O1 = tr.packed_full(b, screened=False)
        G, D = tr.G(b), tr.density(b)
        if b == "coulomb":
            O2 = (D.T @ G) @ D
        elif b == "gaunt":
            O2 = sum((D[:, J, :].T @ G) @ D[:, J, :] for J in range(3))
        else:
            O2 = 0
            for ij, (I, J) in enumerate(oracle.IJ6):
                t = (D[:, I, :].T @ G[ij]) @ D[:, J, :]
                O2 = O2 + (t if I == J else t + t.T)
        assert np.abs(O1 - O2).max() <= 1e-14 * max(1.0, np.abs(O1).max())
