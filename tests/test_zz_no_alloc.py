"""qdt_second_half_noalloc: the second-half contraction without any device
allocation, for callers whose device memory is owned by another allocator or
that must avoid the synchronisation of a fresh cudaMalloc.  Its output must
equal what the allocating path (qdt_transform) produces.

This file is collected last on purpose: if the entry point misbehaves, a run
that stops at the first failure has already run every other test."""
import ctypes

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


def reference_packed(torch, p):
    """Packed Coulomb block from the allocating entry point qdt_transform."""
    from paper_2606_04316_gb300 import qdt
    ctx = qdt.Context(0)
    ctx.set_basis(p.basis)
    ctx.set_coefficients(p.CL, p.CS)
    out = torch.zeros(ctx.packed_size(["coulomb"], 0, p.nK) // 8, dtype=torch.float64, device="cuda")
    ctx.transform(["coulomb"], 0, p.nK, 0.0, 0, out)
    torch.cuda.synchronize()
    ctx.close()
    return out.cpu().numpy()


def operands(oracle, p):
    """Quaternion density Dq and first-half V = G Dq of the problem."""
    tr = oracle.Transform(p)
    D = tr.density("coulomb")
    V = tr.G("coulomb") @ D
    return D, V


def test_noalloc_matches_allocating_path_twice(oracle, torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    problems = [synth.chain_problem(3, 3, seed=501, shells=(0, 1), nprim=2, blocks=("coulomb",), tau=0.0),
                synth.chain_problem(2, 5, seed=502, shells=(0, 1), nprim=3, blocks=("coulomb",), tau=0.0)]
    for p in problems:                      # two calls in a row on the shared scratch
        D, V = operands(oracle, p)
        Dd = torch.from_numpy(D).cuda()
        Vd = torch.from_numpy(V).cuda()
        N = D.shape[1]
        O = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
        qdt.second_half_noalloc(Dd, Vd, O)
        torch.cuda.synchronize()
        got = oracle.pack_canonical(O.cpu().numpy(), p.nK).reshape(-1)
        ref = reference_packed(torch, p)
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL_FP64


def test_noalloc_rejects_oversized(torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    N = 2049
    Dd = torch.zeros((4, N), dtype=torch.float64, device="cuda")
    O = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(qdt.QdtError) as e:
        qdt.second_half_noalloc(Dd, Dd, O)
    assert e.value.code == -1 and "2048" in str(e.value)
