"""Pins of the oracle's Kramers-unrestricted path (general complex two-spinor
coefficients, spinor-pair densities, 4 reals per canonical pair of pairs):
the literal four-component brute force, packed -> unpacked equals the
definition, Kramers-structured input reproduces the Kramers-restricted
result, and the symmetries of (pq|rs)."""
import numpy as np
import pytest

from paper_2606_04316_gb300 import synth
from test_oracle_transform import brute_force

BLOCKS = ("coulomb", "gaunt", "gauge")


def tiny_ku(n=3, seed=41, shells=(0, 0), ncent=2, nprim=1, tau=0.0):
    return synth.ku_chain_problem(ncent, n, seed=seed, shells=shells, nprim=nprim, blocks=BLOCKS, tau=tau,
                                  name="tiny-ku")


def ao_tensors(ob):
    nF = ob.nL + ob.nS
    T4C = np.zeros((nF,) * 4)
    for cls in (0, 1):
        a, b, _ = ob.pairs(cls)
        G = ob.pair_matrix(cls, 0)
        for (x, y) in ((a, b), (b, a)):
            for (u, v) in ((a, b), (b, a)):
                T4C[x[:, None], y[:, None], u[None, :], v[None, :]] = G
    a, b, _ = ob.pairs(1)
    Gg = ob.pair_matrix(1, 2)
    T4g = np.zeros((6,) + (nF,) * 4)
    for ij in range(6):
        for (x, y) in ((a, b), (b, a)):
            for (u, v) in ((a, b), (b, a)):
                T4g[ij][x[:, None], y[:, None], u[None, :], v[None, :]] = Gg[ij]
    return T4C, T4g


@pytest.fixture(scope="module")
def ku_tr(oracle):
    tr = oracle.TransformKU(tiny_ku())
    return (tr,) + ao_tensors(tr.ob)


@pytest.mark.parametrize("block", BLOCKS)
def test_ku_brute_force_four_component(ku_tr, block):
    tr, T4C, T4g = ku_tr
    bf = brute_force(tr, block, T4C, T4g)
    full = tr.full(block)
    scale = np.abs(bf).max()
    assert scale > 1e-8          # small-component blocks carry (1/2c)^2
    assert np.abs(full - bf).max() <= 1e-13 * scale


@pytest.mark.parametrize("block", BLOCKS)
def test_ku_packed_unpacks_to_definition(oracle, block):
    p = tiny_ku(n=3, seed=42, shells=(0, 1), nprim=2)
    tr = oracle.TransformKU(p)
    got = oracle.unpack_ku(tr.packed(block), tr.n)
    ref = tr.full(block)
    assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("block", BLOCKS)
def test_ku_with_kramers_coefficients_matches_kr(oracle, block):
    """Spinor 2k and its Kramers partner 2k+1 given as independent KU
    spinors: the KU path must reproduce the Kramers-restricted integrals."""
    pk = synth.chain_problem(2, 2, seed=43, shells=(0, 1), nprim=1, blocks=BLOCKS, tau=0.0)
    kr = oracle.Transform(pk)
    def c4(Cq):
        C = oracle.spinor_coefficients(Cq)                      # [rows, 2, 2 nK] complex
        return np.stack([C[:, 0].real, C[:, 0].imag, C[:, 1].real, C[:, 1].imag], axis=-1)
    pu = synth.Problem("ku-of-kr", pk.basis, c4(pk.CL), c4(pk.CS), pk.blocks, 0.0, kramers=False)
    ku = oracle.TransformKU(pu)
    a = oracle.unpack_ku(ku.packed(block), ku.n)
    b = oracle.unpack(kr.packed(block), kr.nKa, block)
    assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max())


def test_ku_symmetries(oracle):
    p = tiny_ku(n=4, seed=44, shells=(0, 1), nprim=1)
    tr = oracle.TransformKU(p)
    for block in BLOCKS:
        f = tr.full(block)
        tol = 1e-13 * max(1.0, np.abs(f).max())
        assert np.abs(f - f.transpose(2, 3, 0, 1)).max() <= tol                # (pq|rs) = (rs|pq)
        assert np.abs(f - np.conj(f.transpose(1, 0, 3, 2))).max() <= tol       # (pq|rs) = conj (qp|sr)


def test_ku_threshold_zero_keeps_everything(oracle):
    tr = oracle.TransformKU(tiny_ku(n=3, seed=45, shells=(0, 1), nprim=2, tau=0.0))
    for block in BLOCKS:
        assert tr.mask(block).all()
