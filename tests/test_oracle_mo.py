"""Pins of the oracle's MO-driven route (Sec. 3.3): unscreened it is the
AO-driven transform for every block size; one block is the AO-driven screened
transform; screened per block, its error stays within the dropped quartets'
bounds, and a block's own density maximum never exceeds the whole one."""
import numpy as np

from paper_2606_04316_gb300 import synth

BLOCKS = ("coulomb", "gaunt", "gauge")


def test_mo_unscreened_equals_ao_for_every_block_size(oracle):
    p = synth.chain_problem(3, 4, seed=651, shells=(0, 1), nprim=2, tau=0.0)
    tr = oracle.Transform(p)
    for b in BLOCKS:
        ref = tr.packed(b)
        for nb in (1, 2, 3, 4):
            assert np.abs(tr.packed_mo(b, nb) - ref).max() <= 1e-13 * np.abs(ref).max()
    pk = synth.ku_chain_problem(3, 5, seed=652, shells=(0, 1), nprim=2, tau=0.0)
    tk = oracle.TransformKU(pk)
    for b in BLOCKS:
        ref = tk.packed(b)
        assert np.abs(tk.packed_mo(b, 2) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_mo_one_block_is_ao_screened(oracle):
    p = synth.chain_problem(8, 3, seed=653, shells=(0, 1), nprim=2, tau=1e-9)
    tr = oracle.Transform(p)
    for b in BLOCKS:
        assert tr.mask(b).mean() < 1.0
        ref = tr.packed(b)
        # the same products; the gauge sum adds the transposed (I, J) terms in another order
        assert np.abs(tr.packed_mo(b, 3) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_mo_screening_error_within_dropped_bounds(oracle):
    """Per block, every dropped quartet contributes at most
    nfp_AB nfp_CD Q_AB Q_CD Dmax_CD(block) to a first-half element, times the
    largest bra density over all columns in the second half."""
    p = synth.chain_problem(8, 4, seed=654, shells=(0, 1), nprim=2, tau=1e-8)
    tr = oracle.Transform(p)
    ob = tr.ob
    _, _, sp = ob.pairs(0)
    nfp = np.bincount(sp)
    Q = oracle.schwarz_q(ob, 0)
    D = tr.density("coulomb")
    n, parts = 4, 4
    full = tr.packed_full("coulomb", screened=False)
    mo = tr.packed_full_mo("coulomb", 1)
    dmax_all = oracle.density_max(ob, 0, D)
    dropped = 0
    for r0 in range(n):
        c0 = parts * oracle.pair_index(r0, r0, n)
        c1 = parts * oracle.pair_index(r0 + 1, r0 + 1, n) if r0 + 1 < n else D.shape[-1]
        dm = oracle.density_max(ob, 0, D[..., c0:c1])
        assert np.all(dm <= dmax_all)
        mask = tr.mask_columns("coulomb", c0, c1)
        bound_v = ((~mask) * (Q[:, None] * Q[None, :] * dm[None, :]) * nfp[None, :]).sum(axis=1)
        bound = float((nfp * dmax_all * bound_v).sum())
        err = np.abs(mo[:, c0:c1] - full[:, c0:c1]).max()
        assert err <= bound
        dropped += int((~mask).sum())
    assert dropped > 0
