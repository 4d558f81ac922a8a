"""Batched transformations (qdt_transform_batch): the kept integral tiles of
several requests fused into one persistent launch over a shared tile queue,
optionally captured into a CUDA graph and replayed.  Every item must equal
its own qdt_transform (both forms) and, on a small case, the oracle."""
import numpy as np
import pytest

from paper_2606_04316_gb300 import synth

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def problems(tau=1e-11):
    """Four requests of different size, shell mix, blocks and precision."""
    return [
        (synth.chain_problem(4, 3, seed=701, shells=(0, 1), nprim=2, blocks=("coulomb",), tau=tau), 0),
        (synth.cluster_problem((2, 2, 1), 3, seed=702, nprim=2, blocks=("coulomb", "gaunt", "gauge"), tau=tau), 1),
        (synth.chain_problem(5, 4, seed=703, shells=(0,), nprim=3, blocks=("coulomb", "gaunt"), tau=tau), 0),
        (synth.chain_problem(3, 2, seed=704, shells=(0, 1), nprim=1, blocks=("gauge",), tau=tau), 1),
    ]


def make_ctx(qdt, p):
    ctx = qdt.Context(0)
    ctx.set_basis(p.basis)
    ctx.set_coefficients(p.CL, p.CS)
    return ctx


def out_for(torch, ctx, p):
    n = ctx.packed_size(list(p.blocks), 0, p.nK) // 8
    return torch.zeros(n, dtype=torch.float64, device="cuda")


def alone(torch, qdt, p, prec):
    ctx = make_ctx(qdt, p)
    out = out_for(torch, ctx, p)
    st = ctx.transform(list(p.blocks), 0, p.nK, p.tau, prec, out)
    return out.cpu().numpy(), st


def test_batch_matches_alone_and_oracle(oracle, torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    probs = problems()
    ctxs = [make_ctx(qdt, p) for p, _ in probs]
    outs = [out_for(torch, c, p) for c, (p, _) in zip(ctxs, probs)]
    jobs = [(c, list(p.blocks), 0, p.nK, p.tau, prec, o) for c, (p, prec), o in zip(ctxs, probs, outs)]
    status, stats = qdt.transform_batch(jobs)
    assert status == [0] * len(jobs)
    for (p, prec), o, st in zip(probs, outs, stats):
        ref, st1 = alone(torch, qdt, p, prec)
        assert np.abs(o.cpu().numpy() - ref).max() <= TOL_FP64
        assert st["quartets_kept"] == st1["quartets_kept"]
        assert st["kernel_launches"] > 0
    # the first request against the oracle
    p = probs[0][0]
    ref = oracle.Transform(p).packed("coulomb").reshape(-1)
    assert np.abs(outs[0].cpu().numpy() - ref).max() <= TOL_FP64


def test_batch_host_output(torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    probs = problems()[:2]
    ctxs = [make_ctx(qdt, p) for p, _ in probs]
    outs = [np.zeros(c.packed_size(list(p.blocks), 0, p.nK) // 8) for c, (p, _) in zip(ctxs, probs)]
    jobs = [(c, list(p.blocks), 0, p.nK, p.tau, prec, o) for c, (p, prec), o in zip(ctxs, probs, outs)]
    qdt.transform_batch(jobs)
    for (p, prec), o in zip(probs, outs):
        ref, _ = alone(torch, qdt, p, prec)
        assert np.abs(o - ref).max() <= TOL_FP64


def test_batch_graph_capture_and_replay(torch_cuda, monkeypatch):
    """tau = 0 keeps the screening outcome fixed when the coefficients change,
    and a zero FP32 budget keeps every integral in compensated pairs (the
    FP32 set follows the densities), so the same batch signature recurs: the
    graph is captured, replayed, and a replay after new coefficients gives the
    new results."""
    monkeypatch.setenv("QDT_F32_BUDGET", "0")
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    probs = problems(tau=0.0)
    ctxs = [make_ctx(qdt, p) for p, _ in probs]
    outs = [out_for(torch, c, p) for c, (p, _) in zip(ctxs, probs)]
    jobs = [(c, list(p.blocks), 0, p.nK, p.tau, prec, o) for c, (p, prec), o in zip(ctxs, probs, outs)]
    first = None
    counts = []
    for _ in range(6):
        for o in outs:
            o.zero_()
        qdt.transform_batch(jobs, graph=True)
        counts.append(ctxs[0].graph_counts())
        got = [o.cpu().numpy() for o in outs]
        if first is None:
            first = got
        else:
            for a, b in zip(first, got):
                assert np.array_equal(a, b)
    caps, reps = ctxs[0].graph_counts()
    # every round (Coulomb class; Gaunt/gauge class) owns one graph: the first
    # runs size the buffers, the signature is seen twice, then captured once
    # and replayed
    assert caps == 2 and reps >= 2, counts
    for (p, prec), a in zip(probs, first):
        ref, _ = alone(torch, qdt, p, prec)
        assert np.abs(a - ref).max() <= TOL_FP64
    # new coefficients of the same shape: a replay must read them
    rng = np.random.Generator(np.random.PCG64(705))
    newp = []
    for c, (p, prec) in zip(ctxs, probs):
        CL, CS = synth.coefficients(rng, p.basis.nL, p.nK)
        c.set_coefficients(CL, CS)
        newp.append((synth.Problem(p.name, p.basis, CL, CS, p.blocks, p.tau), prec))
    for o in outs:
        o.zero_()
    qdt.transform_batch(jobs, graph=True)
    caps2, reps2 = ctxs[0].graph_counts()
    assert reps2 == reps + 2 and caps2 == caps, (counts, caps2, reps2)
    for (p, prec), o in zip(newp, outs):
        ref, _ = alone(torch, qdt, p, prec)
        assert np.abs(o.cpu().numpy() - ref).max() <= TOL_FP64


def test_batch_item_errors(torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    (p0, prec0), (p1, prec1) = problems()[:2]
    c0, c1 = make_ctx(qdt, p0), make_ctx(qdt, p1)
    o0, o1 = out_for(torch, c0, p0), out_for(torch, c1, p1)
    jobs = [(c0, list(p0.blocks), 0, p0.nK, p0.tau, prec0, o0),
            (c1, list(p1.blocks), 0, p1.nK + 1, p1.tau, prec1, o1)]     # bad Kramers range
    status, _ = qdt.transform_batch(jobs, raise_on_error=False)
    assert status == [0, -1]
    ref, _ = alone(torch, qdt, p0, prec0)
    assert np.abs(o0.cpu().numpy() - ref).max() <= TOL_FP64
    with pytest.raises(qdt.QdtError):
        qdt.transform_batch(jobs)
    # the same context twice is refused for the second item
    status, _ = qdt.transform_batch([jobs[0], jobs[0]], raise_on_error=False)
    assert status == [0, -1]
