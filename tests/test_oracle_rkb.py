"""Pins of the oracle's restricted-kinetic-balance mapping (Eq. RKB): small
component (1/2c) sigma.p chi^L c^S written in the derivative basis."""
import numpy as np

from paper_2606_04316_gb300 import synth

C_LIGHT = 137.035999084


def ss_overlap(ob):
    """Overlaps of the derivative functions d_K chi_mu (rows 3 mu + K)."""
    n = ob.nsh
    rows = []
    for sa in range(n, 2 * n):
        rows.append(np.concatenate([ob.overlap_block(sa, sb) for sb in range(n, 2 * n)], axis=1))
    return np.concatenate(rows, axis=0)


def test_rkb_small_component_norm_is_kinetic(oracle):
    """<psi^S_p|psi^S_q> = (1/4c^2) sum c^S_mu^+ c^S_nu <grad chi_mu . grad chi_nu>: the
    spin-orbit part i eps_KLM <d_K chi_mu|d_L chi_nu> sigma_M vanishes because the
    overlap of two derivatives is symmetric in K, L (integration by parts)."""
    p = synth.chain_problem(2, 2, seed=611, shells=(0, 1), nprim=2)
    ob = oracle.OracleBasis(p.basis)
    cs = p.CL                                       # any quaternion coefficients as c^S
    Ct = oracle.spinor_coefficients(oracle.rkb_to_derivative(cs, C_LIGHT))   # [3 nL, 2, n]
    S = ss_overlap(ob)
    lhs = np.einsum('atp,ab,btq->pq', np.conj(Ct), S, Ct)
    c = oracle.spinor_coefficients(cs)                                        # [nL, 2, n]
    nL = c.shape[0]
    Tk = np.einsum('mKnK->mn', S.reshape(nL, 3, nL, 3))                       # <grad chi_mu . grad chi_nu>
    rhs = np.einsum('mtp,mn,ntq->pq', np.conj(c), Tk, c) / (4.0 * C_LIGHT ** 2)
    assert np.abs(rhs).max() > 1e-8
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()


def test_rkb_mapping_keeps_kramers_pairs(oracle):
    """sigma.p commutes with time reversal: the Kramers partner of a mapped spinor is the
    mapped partner, so the quaternion form carries the whole mapping."""
    p = synth.chain_problem(2, 3, seed=612, shells=(0, 1), nprim=1)
    cs = p.CL
    C = oracle.spinor_coefficients(cs)
    full = (np.einsum('Kuv,mvp->mKup', oracle.SIGMA, C) * (-1j / (2.0 * C_LIGHT))).reshape(-1, 2, C.shape[2])
    via_q = oracle.spinor_coefficients(oracle.rkb_to_derivative(cs, C_LIGHT))
    assert np.abs(full - via_q).max() <= 1e-16 + 1e-14 * np.abs(full).max()


def test_rkb_sigma_components(oracle):
    """Single alpha spinor on one function: d_x carries -i beta-less sigma_x -> beta = -i/2c,
    d_z -> alpha = -i/2c (sigma_z), d_y -> beta = +1/2c (sigma_y (1, 0) = (0, i))."""
    q = np.zeros((1, 1, 4))
    q[0, 0, 0] = 1.0                                 # alpha = 1, beta = 0
    out = oracle.rkb_to_derivative(q, C_LIGHT)       # rows K = x, y, z
    h = 1.0 / (2.0 * C_LIGHT)
    ax, bx = out[0, 0, 0] + 1j * out[0, 0, 1], out[0, 0, 2] + 1j * out[0, 0, 3]
    ay, by = out[1, 0, 0] + 1j * out[1, 0, 1], out[1, 0, 2] + 1j * out[1, 0, 3]
    az, bz = out[2, 0, 0] + 1j * out[2, 0, 1], out[2, 0, 2] + 1j * out[2, 0, 3]
    assert abs(ax) < 1e-18 and abs(bx - (-1j * h)) < 1e-18
    assert abs(ay) < 1e-18 and abs(by - h) < 1e-18
    assert abs(az - (-1j * h)) < 1e-18 and abs(bz) < 1e-18


def test_rkb_spinor_form_matches_quaternion_form(oracle):
    """Per-spinor input of the unbarred members maps to the unbarred members of
    the quaternion image; the barred members (Kramers partners) map to the
    partners of the image (time reversal commutes with sigma.p)."""
    p = synth.rkb_chain_problem(2, 3, seed=613, shells=(0, 1), nprim=1)
    C = oracle.spinor_coefficients(p.CS)                                    # [nL, 2, 2 nK]
    four = lambda Z: np.stack([Z[:, 0].real, Z[:, 0].imag, Z[:, 1].real, Z[:, 1].imag], axis=-1)
    qimg = oracle.spinor_coefficients(oracle.rkb_to_derivative(p.CS, C_LIGHT))
    s_even = oracle.rkb_to_derivative(four(C[:, :, 0::2]), C_LIGHT, spinors=True)
    s_odd = oracle.rkb_to_derivative(four(C[:, :, 1::2]), C_LIGHT, spinors=True)
    z = lambda f: np.stack([f[..., 0] + 1j * f[..., 1], f[..., 2] + 1j * f[..., 3]], axis=1)
    assert np.abs(z(s_even) - qimg[:, :, 0::2]).max() <= 1e-16
    assert np.abs(z(s_odd) - qimg[:, :, 1::2]).max() <= 1e-16


def test_rkb_reproduces_the_quaternion_first_half(oracle):
    """Eq. firsthalf, small-component ket term, for one spinor pair (r, t): with
    D_s = sum_tau c*_k c_l and D_M = c*_k sigma_M c_l (quaternion density of the
    RKB coefficients c^S, Eq. QuaternionScatter read with sigma_M between the
    spinors), V_s(mu nu) = (1/2c^2) sum [D_s (mu nu|grad k . grad l) +
    i sum_M D_M (mu nu|(grad k x grad l)_M)].  The same quantity through the
    derivative-function expansion: the bra spin trace (V_aa + V_bb) of
    sum_cd (mu nu|cd) D_cd with the expanded coefficients."""
    p = synth.rkb_chain_problem(2, 2, seed=614, shells=(0, 1), nprim=1, kramers=False)
    ob = oracle.OracleBasis(p.basis)
    nL = ob.nL
    T = oracle._expand_full(ob, 0, ob.pair_matrix(0, 0))            # (ab|cd) over F = L, S
    S = lambda k, K: nL + 3 * k + K
    cS = np.stack([p.CS[..., 0] + 1j * p.CS[..., 1], p.CS[..., 2] + 1j * p.CS[..., 3]], axis=1)   # [nL, 2, n]
    r, t = 0, 1
    # route A: expansion over the derivative functions, then the plain density sum
    Ct4 = oracle.rkb_to_derivative(p.CS, C_LIGHT, spinors=True)
    Ct = np.stack([Ct4[..., 0] + 1j * Ct4[..., 1], Ct4[..., 2] + 1j * Ct4[..., 3]], axis=1)     # [3 nL, 2, n]
    Dd = np.einsum('ct,dt->cd', np.conj(Ct[:, :, r]), Ct[:, :, t])
    VA = 2.0 * np.einsum('mncd,cd->mn', T[:nL, :nL, nL:, nL:], Dd)
    # route B: the quaternion formula from scalar integrals of dot and cross products
    Ds = np.einsum('kt,lt->kl', np.conj(cS[:, :, r]), cS[:, :, t])
    DM = np.einsum('kt,Mtu,lu->Mkl', np.conj(cS[:, :, r]), oracle.SIGMA, cS[:, :, t])
    idx = np.array([[S(k, K) for K in range(3)] for k in range(nL)])                      # [nL, 3]
    Tb = T[:nL, :nL][:, :, idx[:, :, None, None], idx[None, None, :, :]]                  # [m, n, k, K, l, L]
    dot = np.einsum('mnkKlK->mnkl', Tb)
    eps = np.zeros((3, 3, 3))
    for (a, b, c) in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        eps[a, b, c], eps[b, a, c] = 1.0, -1.0
    cross = np.einsum('KLM,mnkKlL->Mmnkl', eps, Tb)
    VB = (np.einsum('kl,mnkl->mn', Ds, dot) + 1j * np.einsum('Mkl,Mmnkl->mn', DM, cross)) / (2.0 * C_LIGHT ** 2)
    assert np.abs(VB).max() > 0 and np.abs(np.einsum('Mkl,Mmnkl->mn', DM, cross)).max() > 1e-6 * np.abs(VB).max() * C_LIGHT ** 2
    assert np.abs(VA - VB).max() <= 1e-13 * np.abs(VB).max()
