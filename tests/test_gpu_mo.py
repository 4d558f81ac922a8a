"""The MO-driven route (qdt_set_route 'mo', Sec. 3.3) on the GPU: every block
against the oracle's MO-driven transform (per-block screening), the kept
quartets summed over the blocks, and equality with the AO-driven route when
nothing is screened."""
import numpy as np
import pytest

from paper_2606_04316_gb300 import synth

pytestmark = pytest.mark.gpu
TOL_FP64, TOL_SPLIT = 1e-12, 1e-10
BLOCKS = ("coulomb", "gaunt", "gauge")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make_ctx(qdt, p, route, nb=0):
    ctx = qdt.Context(0)
    ctx.set_basis(p.basis)
    if p.kramers:
        ctx.set_coefficients(p.CL, p.CS)
    else:
        ctx.set_spinor_coefficients(p.CL, p.CS)
    ctx.set_route(route, nb)
    return ctx


def run(torch, ctx, blocks, k0, k1, tau, prec):
    out = torch.zeros(ctx.packed_size(list(blocks), k0, k1) // 8, dtype=torch.float64, device="cuda")
    st = ctx.transform(list(blocks), k0, k1, tau, prec, out)
    return out, st


def kept_mo(oracle, tr, block, nb, n, parts):
    tot = 0
    D = tr.density(block)
    for r0 in range(0, n, nb):
        r1 = min(n, r0 + nb)
        c0 = parts * oracle.pair_index(r0, r0, n)
        c1 = parts * oracle.pair_index(r1, r1, n) if r1 < n else D.shape[-1]
        tot += int(tr.mask_columns(block, c0, c1).sum())
    return tot


@pytest.mark.parametrize("kramers,nb", [(True, 1), (True, 2), (False, 3)])
@pytest.mark.parametrize("prec,tol", [(0, TOL_FP64), (1, TOL_SPLIT)])
def test_mo_against_oracle(oracle, torch_cuda, kramers, nb, prec, tol):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    if kramers:
        p = synth.chain_problem(8, 4, seed=661, shells=(0, 1), nprim=2, blocks=BLOCKS, tau=1e-9)
        tr, n, parts = oracle.Transform(p), 4, 4
    else:
        p = synth.ku_chain_problem(8, 7, seed=662, shells=(0, 1), nprim=2, blocks=BLOCKS, tau=1e-9)
        tr, n, parts = oracle.TransformKU(p), 7, 2
    ctx = make_ctx(qdt, p, "mo", nb)
    out, st = run(torch, ctx, BLOCKS, 0, n, p.tau, prec)
    got = out.cpu().numpy().reshape(len(BLOCKS), -1)
    for i, b in enumerate(BLOCKS):
        ref = tr.packed_mo(b, nb).reshape(-1)
        assert np.abs(got[i] - ref).max() <= tol
    assert st["quartets_kept"][0] == kept_mo(oracle, tr, "coulomb", nb, n, parts)
    assert st["quartets_kept"][1] == kept_mo(oracle, tr, "gaunt", nb, n, parts)


def test_mo_unscreened_equals_ao_route(torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    p = synth.chain_problem(5, 5, seed=663, shells=(0, 1), nprim=2, blocks=BLOCKS, tau=0.0)
    mo = make_ctx(qdt, p, "mo", 2)
    ao = make_ctx(qdt, p, "density")
    for prec, tol in ((0, TOL_FP64), (1, TOL_SPLIT)):
        om, sm = run(torch, mo, BLOCKS, 1, 5, 0.0, prec)
        oa, sa = run(torch, ao, BLOCKS, 1, 5, 0.0, prec)
        assert (om - oa).abs().max().item() <= tol
        # two blocks of outer indices: every quartet is computed twice
        assert sm["quartets_kept"][0] == 2 * sa["quartets_kept"][0]
