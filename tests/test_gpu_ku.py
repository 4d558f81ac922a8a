"""Kramers-unrestricted input on the GPU (qdt_set_spinor_coefficients): every
block in both forms against the oracle, screened, through the Kramers-
restricted path when the spinors are Kramers pairs, and inside a batch."""
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


def ku_ctx(qdt, p):
    ctx = qdt.Context(0)
    ctx.set_basis(p.basis)
    ctx.set_spinor_coefficients(p.CL, p.CS)
    return ctx


def run(torch, ctx, blocks, s0, s1, tau, prec):
    out = torch.zeros(ctx.packed_size(list(blocks), s0, s1) // 8, dtype=torch.float64, device="cuda")
    st = ctx.transform(list(blocks), s0, s1, tau, prec, out)
    return out, st


@pytest.mark.parametrize("prec,tol", [(0, TOL_FP64), (1, TOL_SPLIT)])
def test_ku_all_blocks_against_oracle(oracle, torch_cuda, prec, tol):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    p = synth.ku_chain_problem(3, 4, seed=501, shells=(0, 1), nprim=2, blocks=BLOCKS, tau=0.0)
    ctx = ku_ctx(qdt, p)
    out, _ = run(torch, ctx, BLOCKS, 0, p.nK, 0.0, prec)
    got = out.cpu().numpy().reshape(len(BLOCKS), -1)
    tr = oracle.TransformKU(p)
    n = tr.n
    for i, b in enumerate(BLOCKS):
        assert np.abs(got[i] - tr.packed(b).reshape(-1)).max() <= tol
        full = torch.zeros(2 * n ** 4, dtype=torch.float64, device="cuda")
        ctx.unpack(out.view(len(BLOCKS), -1)[i].contiguous(), n, b, full)
        f = full.cpu().numpy().reshape(n, n, n, n, 2)
        assert np.abs(f[..., 0] + 1j * f[..., 1] - tr.full(b)).max() <= tol


def test_ku_screened_active_range(oracle, torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    p = synth.ku_chain_problem(8, 6, seed=502, shells=(0, 1), nprim=2, blocks=("coulomb",), tau=1e-9)
    ctx = ku_ctx(qdt, p)
    out, st = run(torch, ctx, ["coulomb"], 1, 5, p.tau, 0)
    tr = oracle.TransformKU(p, 1, 5)
    assert tr.mask("coulomb").mean() < 1.0
    assert st["quartets_kept"][0] == int(tr.mask("coulomb").sum())
    assert np.abs(out.cpu().numpy() - tr.packed("coulomb").reshape(-1)).max() <= TOL_FP64


def test_ku_of_kramers_pairs_matches_kramers_restricted(oracle, torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    pk = synth.chain_problem(3, 2, seed=503, shells=(0, 1), nprim=2, blocks=BLOCKS, tau=0.0)
    def c4(Cq):
        C = oracle.spinor_coefficients(Cq)
        return np.ascontiguousarray(np.stack([C[:, 0].real, C[:, 0].imag, C[:, 1].real, C[:, 1].imag], axis=-1))
    kr = qdt.Context(0)
    kr.set_basis(pk.basis)
    kr.set_coefficients(pk.CL, pk.CS)
    ku = qdt.Context(0)
    ku.set_basis(pk.basis)
    ku.set_spinor_coefficients(c4(pk.CL), c4(pk.CS))
    n = 2 * pk.nK
    okr, _ = run(torch, kr, BLOCKS, 0, pk.nK, 0.0, 0)
    oku, _ = run(torch, ku, BLOCKS, 0, n, 0.0, 0)
    for i, b in enumerate(BLOCKS):
        f1 = torch.zeros(2 * n ** 4, dtype=torch.float64, device="cuda")
        f2 = torch.zeros_like(f1)
        kr.unpack(okr.view(len(BLOCKS), -1)[i].contiguous(), pk.nK, b, f1)
        ku.unpack(oku.view(len(BLOCKS), -1)[i].contiguous(), n, b, f2)
        assert (f1 - f2).abs().max().item() <= TOL_FP64


def test_ku_and_kr_in_one_batch(torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    pu = synth.ku_chain_problem(4, 5, seed=504, shells=(0, 1), nprim=2, blocks=BLOCKS, tau=1e-11)
    pk = synth.chain_problem(4, 3, seed=505, shells=(0, 1), nprim=2, blocks=BLOCKS, tau=1e-11)
    cu, ck = ku_ctx(qdt, pu), qdt.Context(0)
    ck.set_basis(pk.basis)
    ck.set_coefficients(pk.CL, pk.CS)
    for prec in (0, 1):
        ru, _ = run(torch, cu, BLOCKS, 0, pu.nK, pu.tau, prec)
        rk, _ = run(torch, ck, BLOCKS, 0, pk.nK, pk.tau, prec)
        ou, ok = torch.zeros_like(ru), torch.zeros_like(rk)
        qdt.transform_batch([(cu, list(BLOCKS), 0, pu.nK, pu.tau, prec, ou),
                             (ck, list(BLOCKS), 0, pk.nK, pk.tau, prec, ok)])
        assert (ou - ru).abs().max().item() <= TOL_FP64
        assert (ok - rk).abs().max().item() <= TOL_FP64
