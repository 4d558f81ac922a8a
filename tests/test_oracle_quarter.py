"""Pins of the oracle's screening bound for the O(N^5) quarter route (Sec. 2.2):
it bounds the density maximum of every shell pair, is attained when all
coefficient rows point the same way, and keeps a superset of the quartets that
the density route keeps."""
import numpy as np

from paper_2606_04316_gb300 import synth


def test_coefficient_bound_covers_density_max(oracle):
    for kramers, p in ((True, synth.chain_problem(4, 3, seed=631, shells=(0, 1), nprim=2)),
                       (False, synth.ku_chain_problem(4, 5, seed=632, shells=(0, 1), nprim=2))):
        tr = oracle.Transform(p) if kramers else oracle.TransformKU(p)
        dm = oracle.density_max(tr.ob, 0, tr.density("coulomb"))
        cb = oracle.coefficient_bound_max(tr.ob, p.CL, p.CS)
        assert dm.shape == cb.shape and dm.max() > 0
        assert np.all(dm <= cb * (1 + 1e-14))
        assert np.all(cb <= 8 * dm.max() / dm.min())    # same scale, not a vacuous bound


def test_coefficient_bound_attained_for_parallel_rows(oracle):
    """s functions only, one Kramers pair, every row a positive multiple of
    (alpha = 1, beta = 0): D^{RR}_{ab} + D^{RR}_{ba} = 2 s_a s_b and the barred
    density vanishes, so the bound equals the density maximum of every pair of
    two different shells (a diagonal pair also holds the unsymmetrised D_aa)."""
    p = synth.chain_problem(3, 1, seed=633, shells=(0,), nprim=1)
    rng = np.random.default_rng(5)
    CL = np.zeros_like(p.CL)
    CS = np.zeros_like(p.CS)
    CL[:, 0, 0] = rng.uniform(0.5, 2.0, CL.shape[0])
    CS[:, 0, 0] = rng.uniform(0.5, 2.0, CS.shape[0]) * 1e-2
    q = p.__class__(p.name, p.basis, CL, CS, p.blocks, p.tau)
    tr = oracle.Transform(q)
    dm = oracle.density_max(tr.ob, 0, tr.density("coulomb"))
    cb = oracle.coefficient_bound_max(tr.ob, CL, CS)
    a, b, sp = tr.ob.pairs(0)
    nL = tr.ob.nL
    shell = lambda f: np.where(f < nL, tr.ob.shell_of_L[np.minimum(f, nL - 1)],
                               tr.ob.nsh + tr.ob.shell_of_S[np.maximum(f - nL, 0)])
    diag = np.zeros(cb.shape, bool)
    np.logical_or.at(diag, sp, shell(a) == shell(b))
    assert (~diag).sum() > 0
    assert np.allclose(dm[~diag], cb[~diag], rtol=1e-14, atol=0)
    assert np.all(dm[diag] <= cb[diag])


def test_quarter_screening_keeps_a_superset(oracle):
    p = synth.chain_problem(8, 4, seed=634, shells=(0, 1), nprim=2, tau=1e-9)
    dens = oracle.Transform(p).mask("coulomb")
    coef = oracle.Transform(p, bound="coefficients").mask("coulomb")
    assert dens.mean() < 1.0
    assert np.all(coef | ~dens)                       # every density-kept quartet is kept
    assert coef.sum() >= dens.sum()
