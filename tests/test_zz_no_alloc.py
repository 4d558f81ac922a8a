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


def test_noalloc_several_tiles_on_a_side_stream(oracle, torch_cuda):
    """N = 144 (three 64-wide tile rows and columns, several split-K slices of
    the shared array) on a non-default stream, twice in a row."""
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    p = synth.chain_problem(4, 8, seed=503, shells=(0, 1), nprim=2, blocks=("coulomb",), tau=0.0)
    D, V = operands(oracle, p)
    assert D.shape[1] == 144
    ref = reference_packed(torch, p)
    side = torch.cuda.Stream()
    for _ in range(2):
        with torch.cuda.stream(side):
            Dd = torch.from_numpy(D).to("cuda", non_blocking=False)
            Vd = torch.from_numpy(V).to("cuda", non_blocking=False)
            O = torch.full((144, 144), float("nan"), dtype=torch.float64, device="cuda")
        qdt.second_half_noalloc(Dd, Vd, O, stream=side)
        side.synchronize()
        got = oracle.pack_canonical(O.cpu().numpy(), p.nK).reshape(-1)
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL_FP64


def test_noalloc_wrapper_rejects_mismatched_operands(torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    D = torch.zeros((8, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        qdt.second_half_noalloc(D, torch.zeros((8, 15), dtype=torch.float64, device="cuda"),
                                torch.zeros((16, 16), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        qdt.second_half_noalloc(D, D, torch.zeros((15, 16), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        qdt.second_half_noalloc(D, D, torch.zeros((16, 16), dtype=torch.float64))
    with pytest.raises(ValueError):
        qdt.second_half_noalloc(D, D.float(), torch.zeros((16, 16), dtype=torch.float64, device="cuda"))


def test_noalloc_rejects_oversized(torch_cuda):
    """The C entry point refuses N > 2048 before launching anything."""
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    N = 2049
    Dd = torch.zeros((4, N), dtype=torch.float64, device="cuda")
    O = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    with pytest.raises(qdt.QdtError) as e:
        qdt.second_half_noalloc(Dd, Dd, O)
    assert e.value.code == -1 and "2048" in str(e.value)
    L = qdt.load()
    buf = ctypes.create_string_buffer(256)
    rc = L.qdt_second_half_noalloc(ctypes.c_void_p(Dd.data_ptr()), ctypes.c_void_p(Dd.data_ptr()), 4,
                                   3_100_000_000, ctypes.c_void_p(O.data_ptr()), None, buf, 256)
    assert rc == -1 and b"2048" in buf.value
