"""Pins of the oracle's pair assembly: the pair matrices (or_pair_matrix,
or_pair_rows, or_pair_diag, or_shell_pair_rows) put each shell-block integral
at the function-pair index of the documented order, for LL, SS (derivative),
LL-SS and LS pairs of s, p and d shells.

The shell blocks themselves are pinned elsewhere (closed forms, quadrature,
finite differences in the centres: tests/test_oracle_integrals.py), including
the order of the functions inside a shell (Cartesian order of cart_list) and
inside a derivative shell (3 mu + K).  Here the function-pair index of every
sampled entry is built by hand from that order:
  class 0: LL pairs a <= b, index a nL - a(a-1)/2 + (b - a); then SS pairs of
           derivative functions s = 3 mu + K, offset nL(nL+1)/2;
  class 1: (a in L, s in S), index a nS + s.
A misplaced pair index, a wrong SS or LS offset or a transposed block fails
one of these checks."""
import numpy as np
import pytest

from paper_2606_04316_gb300 import synth


@pytest.fixture(scope="module")
def spd(oracle):
    # two centres with one s, one p and one d shell each: nL = 20, nS = 60
    p = synth.chain_problem(2, 1, seed=41, shells=(0, 1, 2), nprim=1, blocks=("coulomb", "gaunt", "gauge"))
    return oracle.OracleBasis(p.basis)


def ncart(l):
    return (l + 1) * (l + 2) // 2


def loff(ob):
    nc = [ncart(int(l)) for l in ob.basis.shell_l]
    return np.concatenate([[0], np.cumsum(nc)]).astype(int)


def tri(a, b, n):
    return a * n - a * (a - 1) // 2 + (b - a)


_FUNCS = {}


def funcs(ob, s):
    """Global function indices of oracle shell s (s >= nsh: derivative shell),
    in the shell's own order: L functions Loff + i, derivative functions
    3 (Loff + i) + K for component index 3 i + K."""
    key = (id(ob), s)
    if key not in _FUNCS:
        n = ob.nsh
        lo = loff(ob)
        if s < n:
            _FUNCS[key] = list(range(lo[s], lo[s + 1]))
        else:
            _FUNCS[key] = [3 * mu + K for mu in range(lo[s - n], lo[s - n + 1]) for K in range(3)]
    return _FUNCS[key]


def row_c0(ob, sa, sb, fa, fb):
    """Class-0 pair index of (function fa of shell sa, fb of sb) or None if the
    pair is not stored (a > b)."""
    n, nL, nS = ob.nsh, ob.nL, ob.nS
    a, b = funcs(ob, sa)[fa], funcs(ob, sb)[fb]
    if a > b:
        return None
    if sa < n:
        assert sb < n
        return tri(a, b, nL)
    return nL * (nL + 1) // 2 + tri(a, b, nS)


def row_c1(ob, sa, sb, fa, fb):
    return funcs(ob, sa)[fa] * ob.nS + funcs(ob, sb)[fb]


def same(v, direct, mirrored):
    """A pair matrix computes each shell quartet once and stores it at (ab, cd)
    and (cd, ab): an entry is exactly the block value of (ab|cd) or of the
    mirrored (cd|ab) (equal up to rounding, by the permutation symmetry pinned
    in test_oracle_integrals.py), whichever quartet the loop visited."""
    return v == direct or v == mirrored


def shell_pairs_c0(ob):
    n = ob.nsh
    return [(a + off, b + off) for off in (0, n) for a in range(n) for b in range(a, n)]


def test_class0_coulomb_pair_matrix_entries(oracle, spd):
    ob = spd
    G = ob.pair_matrix(0, 0)
    M = ob.npairs(0)
    assert M == ob.nL * (ob.nL + 1) // 2 + ob.nS * (ob.nS + 1) // 2
    sps = shell_pairs_c0(ob)
    rng = np.random.default_rng(3)
    n = ob.nsh
    # every combination of (LL or SS) x (LL or SS) shell pairs, several samples each
    kinds = {(x, y): [] for x in (0, 1) for y in (0, 1)}
    for i, (sa, sb) in enumerate(sps):
        for j, (sc, sd) in enumerate(sps):
            kinds[(sa >= n, sc >= n)].append((sa, sb, sc, sd))
    checked = 0
    for key, lst in kinds.items():
        for t in rng.choice(len(lst), size=min(25, len(lst)), replace=False):
            sa, sb, sc, sd = lst[t]
            blk = ob.shell_block(0, sa, sb, sc, sd)
            mir = ob.shell_block(0, sc, sd, sa, sb)
            for fa in range(blk.shape[0]):
                for fb in range(blk.shape[1]):
                    r = row_c0(ob, sa, sb, fa, fb)
                    if r is None:
                        continue
                    for fc in range(blk.shape[2]):
                        for fd in range(blk.shape[3]):
                            c = row_c0(ob, sc, sd, fc, fd)
                            if c is None:
                                continue
                            assert same(G[r, c], blk[fa, fb, fc, fd], mir[fc, fd, fa, fb])
                            checked += 1
    assert checked > 2000
    # every stored pair has exactly one row: the hand-built indices cover 0..M-1
    seen = set()
    for sa, sb in sps:
        for fa in range(len(funcs(ob, sa))):
            for fb in range(len(funcs(ob, sb))):
                r = row_c0(ob, sa, sb, fa, fb)
                if r is not None:
                    assert r not in seen
                    seen.add(r)
    assert seen == set(range(M))


def test_class1_gaunt_and_gauge_pair_matrix_entries(oracle, spd):
    ob = spd
    n = ob.nsh
    GG = ob.pair_matrix(1, 0)
    GK = ob.pair_matrix(1, 2)
    assert GG.shape == (ob.nL * ob.nS,) * 2 and GK.shape == (6,) + GG.shape
    sps = [(a, n + b) for a in range(n) for b in range(n)]
    rng = np.random.default_rng(4)
    checked = 0
    for t in rng.choice(len(sps) ** 2, size=40, replace=False):
        (sa, sb), (sc, sd) = sps[t // len(sps)], sps[t % len(sps)]
        bC = ob.shell_block(0, sa, sb, sc, sd)
        bK = ob.shell_block(2, sa, sb, sc, sd)
        mC = ob.shell_block(0, sc, sd, sa, sb)
        mK = ob.shell_block(2, sc, sd, sa, sb)
        for fa in range(bC.shape[0]):
            for fb in range(bC.shape[1]):
                r = row_c1(ob, sa, sb, fa, fb)
                for fc in range(bC.shape[2]):
                    for fd in range(bC.shape[3]):
                        c = row_c1(ob, sc, sd, fc, fd)
                        assert same(GG[r, c], bC[fa, fb, fc, fd], mC[fc, fd, fa, fb])
                        for k in range(6):
                            assert same(GK[k, r, c], bK[k, fa, fb, fc, fd], mK[k, fc, fd, fa, fb])
                        checked += 1
    assert checked > 1000
    rows = sorted(row_c1(ob, sa, sb, fa, fb) for sa, sb in sps
                  for fa in range(len(funcs(ob, sa))) for fb in range(len(funcs(ob, sb))))
    assert rows == list(range(ob.nL * ob.nS))


def test_pair_diag_and_rows_match_the_blocks(oracle, spd):
    ob = spd
    n = ob.nsh
    d0 = ob.pair_diag(0)
    d1 = ob.pair_diag(1)
    for sa, sb in shell_pairs_c0(ob):
        blk = ob.shell_block(0, sa, sb, sa, sb)
        for fa in range(blk.shape[0]):
            for fb in range(blk.shape[1]):
                r = row_c0(ob, sa, sb, fa, fb)
                if r is not None:
                    assert d0[r] == blk[fa, fb, fa, fb]
    for sa in range(n):
        for sb in range(n, 2 * n):
            blk = ob.shell_block(0, sa, sb, sa, sb)
            for fa in range(blk.shape[0]):
                for fb in range(blk.shape[1]):
                    assert d1[row_c1(ob, sa, sb, fa, fb)] == blk[fa, fb, fa, fb]
    # pair_rows returns the rows of the pair matrix (each quartet computed in
    # the bra->ket orientation, so equal to the mirrored entries to rounding)
    G0 = ob.pair_matrix(0, 0)
    rows = np.array([0, 5, ob.nL * (ob.nL + 1) // 2 + 7, ob.npairs(0) - 1])
    R0 = ob.pair_rows(0, 0, rows)
    assert np.abs(R0 - G0[rows]).max() <= 1e-13 * np.abs(G0).max()
    GK = ob.pair_matrix(1, 2)
    rows = np.array([3, 100, ob.npairs(1) - 1])
    RK = ob.pair_rows(1, 2, rows)
    # the gauge kernel delta_IJ/r - d_I d_J r cancels: with f-like derivative
    # shells the two orientations differ by ~1e-12 relative (a misplaced entry
    # would differ by O(1))
    assert np.abs(RK - GK[:, rows, :].transpose(1, 0, 2)).max() <= 1e-11 * np.abs(GK).max()


def test_shell_pair_rows_are_masked_rows_of_the_pair_matrix(oracle, spd):
    """or_shell_pair_rows: the rows of one bra shell pair, zero outside the kept
    ket shell pairs, equal to the pair matrix's rows inside them."""
    ob = spd
    rng = np.random.default_rng(6)
    for cls, kernel in ((0, 0), (1, 0), (1, 2)):
        _, _, sp = ob.pairs(cls)
        nsp = ob.n_shell_pairs(cls)
        for p in rng.choice(nsp, size=5, replace=False):
            keep = rng.random(nsp) < 0.5
            rows, R = ob.shell_pair_rows(cls, kernel, int(p), keep)
            # the rows are exactly the stored function pairs of shell pair p
            assert sorted(rows.tolist()) == sorted(np.nonzero(sp == p)[0].tolist())
            colkeep = keep[sp]
            ref = ob.pair_rows(cls, kernel, rows)     # same orientation: bit-equal where kept
            if kernel == 2:
                assert np.array_equal(R[:, :, colkeep], ref[:, :, colkeep])
                assert not R[:, :, ~colkeep].any()
            else:
                assert np.array_equal(R[:, colkeep], ref[:, colkeep])
                assert not R[:, ~colkeep].any()


@pytest.mark.parametrize("blocks", [("coulomb",), ("coulomb", "gaunt", "gauge")])
def test_streamed_transform_equals_dense_form(oracle, blocks):
    """The row-streamed transform (bra shell pair by bra shell pair, screened
    kets only) equals the dense O = D^T (G_screened D) to rounding: the two sum
    the same products in a different order, so they agree to ~1e-16 relative,
    not bit for bit."""
    for tau in (0.0, 1e-9):
        p = synth.chain_problem(3, 3, seed=7, shells=(0, 1), nprim=2, blocks=blocks, tau=tau)
        tr = oracle.Transform(p)
        for b in blocks:
            a = tr.packed(b)
            c = tr.packed_streamed(b)
            # the gauge block's values (~1e-7 here) result from cancelling terms
            # ~1e3 times larger, so its reordering noise is ~1e-20 absolute
            assert np.abs(a - c).max() <= 1e-14 * np.abs(a).max() + 1e-18
    p = synth.chain_problem(4, 2, seed=9, shells=(0, 1, 2), nprim=1, blocks=("coulomb",), tau=1e-8)
    tr = oracle.Transform(p)
    a, c = tr.packed("coulomb"), tr.packed_streamed("coulomb")
    assert np.abs(a - c).max() <= 1e-14 * np.abs(a).max()
