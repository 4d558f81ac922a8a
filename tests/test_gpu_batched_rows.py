"""The row-batched path of a transformation: when a class's integral rows do
not fit one batch, they run in batches of bra rows (large systems take this
path).  Bra-ket symmetry holds across batches: a block whose mirror is kept
too is computed once and its transpose contracted into the later rows.
QDT_W_BUDGET forces the path on a small input, QDT_BATCH_SYM=0 turns the
symmetry off; both forms, all three blocks, against the oracle and against
the one-batch result."""
import os

import numpy as np
import pytest

from paper_2606_04316_gb300 import synth

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-12
TOL_SPLIT = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def run(p, blocks, precision, budget=None, sym=True):
    from paper_2606_04316_gb300 import qdt
    old = os.environ.get("QDT_W_BUDGET")
    old_sym = os.environ.get("QDT_BATCH_SYM")
    if budget is not None:
        os.environ["QDT_W_BUDGET"] = str(budget)
    if not sym:
        os.environ["QDT_BATCH_SYM"] = "0"
    try:
        ctx = qdt.Context(0)
        ctx.set_basis(p.basis)
        ctx.set_coefficients(p.CL, p.CS)
        out = np.zeros(ctx.packed_size(blocks, 0, p.nK) // 8)
        st = ctx.transform(blocks, 0, p.nK, p.tau, precision, out)
        ctx.close()
    finally:
        if old is None:
            os.environ.pop("QDT_W_BUDGET", None)
        else:
            os.environ["QDT_W_BUDGET"] = old
        if old_sym is None:
            os.environ.pop("QDT_BATCH_SYM", None)
        else:
            os.environ["QDT_BATCH_SYM"] = old_sym
    return out.reshape(len(blocks), -1), st


_REF = {}


def cases():
    blocks = ("coulomb", "gaunt", "gauge")
    # 4 centres of a jittered cluster, s+p with 2 primitives: class 0 has 1312
    # function-pair rows (W about 14 MB), the L-S class 768 (gauge W about 42 MB);
    # a 2 MB budget cuts them into many batches with ragged last ones.  tau
    # 1e-10 drops quartets, some of them in one direction only
    yield "cluster", synth.cluster_problem((2, 2, 1), 3, seed=611, nprim=2, blocks=blocks, tau=1e-10), 2 << 20
    # a chain screens harder and less symmetrically: many blocks kept one way
    # only, whose ket pairs lie in earlier batches
    yield "chain", synth.chain_problem(8, 3, seed=612, shells=(0, 1), nprim=2, blocks=blocks, tau=1e-9), 1 << 20


@pytest.mark.parametrize("case", ["cluster", "chain"])
@pytest.mark.parametrize("sym", [True, False])
@pytest.mark.parametrize("precision", [0, 1])
def test_forced_row_batches_match_oracle_and_one_batch(oracle, torch_cuda, precision, sym, case):
    blocks = ["coulomb", "gaunt", "gauge"]
    p, budget = {name: (pp, b) for name, pp, b in cases()}[case]
    got, st = run(p, blocks, precision, budget=budget, sym=sym)
    one, st1 = run(p, blocks, precision)
    if case not in _REF:                      # the oracle once per case
        tr = oracle.Transform(p)
        _REF[case] = [tr.packed(b).reshape(-1) for b in blocks]
    tol = TOL_FP64 if precision == 0 else TOL_SPLIT
    for i, b in enumerate(blocks):
        ref = _REF[case][i]
        assert np.abs(got[i] - ref).max() <= tol, b
        assert np.abs(got[i] - one[i]).max() <= tol, b
    # the same quartets are kept either way; with bra-ket symmetry every block
    # is computed once, as in one batch, without it the batches compute more
    assert st["quartets_kept"] == st1["quartets_kept"]
    if sym:
        assert st["flops_eri"] == st1["flops_eri"]
    else:
        assert st["flops_eri"] > st1["flops_eri"]
