"""The O(N^5) two-quarter first half of the Coulomb block (qdt_set_route
'quarter', Sec. 2.2) on the GPU: against the oracle unscreened and with its
coefficient-norm screening, against the density route, over row chunks, and
the routes' boundaries (Gaunt/gauge unaffected, batches refused)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2606_04316_gb300 import synth

pytestmark = pytest.mark.gpu
TOL_FP64, TOL_SPLIT = 1e-12, 1e-10
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make_ctx(qdt, p, route):
    ctx = qdt.Context(0)
    ctx.set_basis(p.basis)
    if p.kramers:
        ctx.set_coefficients(p.CL, p.CS)
    else:
        ctx.set_spinor_coefficients(p.CL, p.CS)
    ctx.set_route(route)
    return ctx


def run(torch, ctx, blocks, k0, k1, tau, prec):
    out = torch.zeros(ctx.packed_size(list(blocks), k0, k1) // 8, dtype=torch.float64, device="cuda")
    st = ctx.transform(list(blocks), k0, k1, tau, prec, out)
    return out, st


@pytest.mark.parametrize("kramers", [True, False])
@pytest.mark.parametrize("prec,tol", [(0, TOL_FP64), (1, TOL_SPLIT)])
def test_quarter_unscreened_against_oracle(oracle, torch_cuda, kramers, prec, tol):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    if kramers:
        p = synth.chain_problem(4, 3, seed=641, shells=(0, 1), nprim=2, tau=0.0)
        tr = oracle.Transform(p)
    else:
        p = synth.ku_chain_problem(4, 5, seed=642, shells=(0, 1), nprim=2, tau=0.0)
        tr = oracle.TransformKU(p)
    ctx = make_ctx(qdt, p, "quarter")
    out, st = run(torch, ctx, ["coulomb"], 0, p.CL.shape[1], 0.0, prec)
    ref = tr.packed("coulomb").reshape(-1)
    assert st["quartets_kept"][0] == st["quartets_total"][0]
    assert np.abs(out.cpu().numpy() - ref).max() <= tol


@pytest.mark.parametrize("kramers", [True, False])
def test_quarter_screened_against_oracle(oracle, torch_cuda, kramers):
    """Screened on 2 max|C_c| max|C_d| per ket pair: the kept quartets are the
    oracle's for that bound (a superset of the density route's), and the values
    match the oracle's screened transform."""
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    if kramers:
        p = synth.chain_problem(8, 4, seed=643, shells=(0, 1), nprim=2, tau=1e-9)
        trq, trd = oracle.Transform(p, bound="coefficients"), oracle.Transform(p)
    else:
        p = synth.ku_chain_problem(8, 6, seed=644, shells=(0, 1), nprim=2, tau=1e-9)
        trq, trd = oracle.TransformKU(p, bound="coefficients"), oracle.TransformKU(p)
    n = p.CL.shape[1]
    q = make_ctx(qdt, p, "quarter")
    d = make_ctx(qdt, p, "density")
    oq, sq = run(torch, q, ["coulomb"], 0, n, p.tau, 0)
    od, sd = run(torch, d, ["coulomb"], 0, n, p.tau, 0)
    mq, md = trq.mask("coulomb"), trd.mask("coulomb")
    assert md.mean() < 1.0
    assert sq["quartets_kept"][0] == int(mq.sum())
    assert sd["quartets_kept"][0] == int(md.sum())
    assert sq["quartets_kept"][0] >= sd["quartets_kept"][0]
    assert np.abs(oq.cpu().numpy() - trq.packed("coulomb").reshape(-1)).max() <= TOL_FP64


def test_quarter_matches_density_route_and_range(torch_cuda):
    """tau = 0 keeps everything on both routes, so they agree to rounding; an
    active range inside the coefficients picks the same columns."""
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    p = synth.chain_problem(6, 5, seed=645, shells=(0, 1), nprim=2, tau=0.0)
    q = make_ctx(qdt, p, "quarter")
    d = make_ctx(qdt, p, "density")
    for prec, tol in ((0, TOL_FP64), (1, TOL_SPLIT)):
        oq, _ = run(torch, q, ["coulomb"], 1, 4, 0.0, prec)
        od, _ = run(torch, d, ["coulomb"], 1, 4, 0.0, prec)
        assert (oq - od).abs().max().item() <= tol


def test_quarter_row_chunks_in_subprocess(torch_cuda):
    """Row chunks of 7 (ragged against every block) give the same result as
    one chunk: FP64 bit for bit."""
    code = r'''
import sys, numpy as np, torch
sys.path.insert(0, %r)
from paper_2606_04316_gb300 import qdt, synth
p = synth.chain_problem(5, 3, seed=646, shells=(0, 1), nprim=2, tau=1e-10)
ctx = qdt.Context(0); ctx.set_basis(p.basis); ctx.set_coefficients(p.CL, p.CS); ctx.set_route("quarter")
for prec in (0, 1):
    out = torch.zeros(ctx.packed_size(["coulomb"], 0, 3) // 8, dtype=torch.float64, device="cuda")
    ctx.transform(["coulomb"], 0, 3, p.tau, prec, out)
    np.save(sys.argv[1] + "_%%d.npy" %% prec, out.cpu().numpy())
''' % os.path.dirname(HERE)
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        outs = {}
        for tag, env in (("one", {}), ("chunked", {"QDT_QUARTER_CHUNK_ROWS": "7"})):
            e = dict(os.environ, **env)
            subprocess.run([sys.executable, "-c", code, os.path.join(td, tag)], check=True, env=e, timeout=600)
            outs[tag] = [np.load(os.path.join(td, "%s_%d.npy" % (tag, k))) for k in (0, 1)]
        assert np.array_equal(outs["one"][0], outs["chunked"][0])
        assert np.abs(outs["one"][1] - outs["chunked"][1]).max() <= 1e-12


def test_route_leaves_gaunt_gauge_and_refuses_batches(torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    p = synth.chain_problem(3, 2, seed=647, shells=(0, 1), nprim=2, tau=1e-11)
    q = make_ctx(qdt, p, "quarter")
    d = make_ctx(qdt, p, "density")
    oq, _ = run(torch, q, ["gaunt", "gauge"], 0, 2, p.tau, 0)
    od, _ = run(torch, d, ["gaunt", "gauge"], 0, 2, p.tau, 0)
    assert torch.equal(oq, od)
    out = torch.zeros_like(oq)
    with pytest.raises(qdt.QdtError):
        qdt.transform_batch([(q, ["gaunt", "gauge"], 0, 2, p.tau, 0, out)])
    assert q.L.qdt_set_route(q.h, 7, 0) == -1
    assert q.L.qdt_set_route(q.h, 2, 0) == -1
