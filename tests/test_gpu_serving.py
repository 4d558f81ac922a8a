"""Serving with continuous batching: every result is the same alone and in
the mix; admission by footprint; failing requests do not disturb the others."""
import numpy as np
import pytest

from paper_2606_04316_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def requests():
    out = []
    out.append((synth.chain_problem(3, 3, seed=401, shells=(0, 1), nprim=2, blocks=("coulomb",), tau=1e-11), ["coulomb"]))
    out.append((synth.chain_problem(5, 4, seed=402, shells=(0, 1), nprim=2, blocks=("coulomb", "gaunt", "gauge"), tau=1e-11),
                ["coulomb", "gaunt", "gauge"]))
    out.append((synth.cluster_problem((2, 2, 1), 3, seed=403, nprim=2, tau=1e-11), ["coulomb", "gaunt", "gauge"]))
    out.append((synth.chain_problem(4, 5, seed=404, shells=(0,), nprim=3, blocks=("coulomb",), tau=1e-11), ["coulomb"]))
    # same basis as the first request, different coefficients: slot reuse of the basis
    p0 = out[0][0]
    rng = np.random.default_rng(9)
    p5 = synth.Problem("same-basis", p0.basis, p0.CL + 0.01 * rng.standard_normal(p0.CL.shape),
                       p0.CS, p0.blocks, p0.tau)
    out.append((p5, ["coulomb"]))
    out.append((synth.chain_problem(6, 6, seed=406, shells=(0, 1), nprim=3, blocks=("coulomb",), tau=1e-11), ["coulomb"]))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_alone_equals_in_the_mix(torch_cuda, precision):
    from paper_2606_04316_gb300 import qdt
    reqs = requests()
    alone = []
    ctx = qdt.Context(0)
    for p, blocks in reqs:
        ctx.set_basis(p.basis)
        ctx.set_coefficients(p.CL, p.CS)
        o = np.zeros(ctx.packed_size(blocks, 0, p.nK) // 8)
        ctx.transform(blocks, 0, p.nK, p.tau, precision, o)
        alone.append(o)
    ctx.close()
    srv = qdt.Server(0, n_slots=3)
    handles, outs = [], []
    for p, blocks in reqs:
        o = np.zeros_like(alone[len(outs)])
        r, keep = srv.make_request(p, blocks, 0, p.nK, p.tau, precision, o)
        handles.append(srv.submit(r, keep))
        outs.append(o)
    lat = []
    for h in handles:
        l, st = srv.wait(h, timeout=300)
        lat.append(l)
    srv.close()
    for a, b in zip(alone, outs):
        assert np.array_equal(a, b)
    assert all(x > 0 for x in lat)


def test_admission_and_failures(torch_cuda):
    from paper_2606_04316_gb300 import qdt
    p, blocks = requests()[0]
    srv = qdt.Server(0, n_slots=2, pool_bytes=1 << 30)
    o = np.zeros(qdt.Context(0).packed_size(blocks, 0, p.nK) // 8)
    r, keep = srv.make_request(p, blocks, 0, p.nK, p.tau, 0, o)
    assert 0 < srv.footprint(r) <= (1 << 30)
    # a request larger than the whole pool is refused at submission
    big = synth.chain_problem(40, 40, seed=1, shells=(0, 1), blocks=("coulomb",))
    ob = np.zeros(8)
    rb, kb = srv.make_request(big, ["coulomb"], 0, 40, 1e-12, 0, ob)
    with pytest.raises(qdt.QdtError) as e:
        srv.submit(rb, kb)
    assert e.value.code == -7
    # malformed request: rejected on submission
    rbad, kbad = srv.make_request(p, blocks, 0, p.nK + 5, p.tau, 0, o)
    with pytest.raises(qdt.QdtError):
        srv.submit(rbad, kbad)
    # a request that fails inside a worker (shell order 5) reports its error;
    # the next one still runs
    badp = synth.chain_problem(2, 2, seed=3, shells=(0,), nprim=1, blocks=("coulomb",), tau=0.0)
    badp.basis.shell_l[:] = 5
    o2 = np.zeros(1000)
    r2, k2 = srv.make_request(badp, ["coulomb"], 0, 2, 0.0, 0, o2)
    h2 = srv.submit(r2, k2)
    h1 = srv.submit(r, keep)
    with pytest.raises(qdt.QdtError) as e2:
        srv.wait(h2, timeout=120)
    assert e2.value.code == -1
    srv.wait(h1, timeout=120)
    assert np.abs(o).max() > 0
    srv.close()
