"""Failure detection without a GPU fault: the bounded wait that guards the
tensor-core pipeline gives up on an mbarrier that nothing arrives at, the
status word reports it as QDT_ERR_TIMEOUT, and the context stays usable."""
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


def test_bounded_wait_gives_up_and_context_survives(oracle, torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    p = synth.chain_problem(3, 2, seed=671, shells=(0, 1), nprim=2, tau=0.0)
    ctx = qdt.Context(0)
    ctx.set_basis(p.basis)
    ctx.set_coefficients(p.CL, p.CS)
    assert ctx.check_bounded_wait(0.05) == -6                 # QDT_ERR_TIMEOUT, as it should
    assert ctx.check_bounded_wait(0.0) == -1                  # bad limit
    out = torch.zeros(ctx.packed_size(["coulomb"], 0, 2) // 8, dtype=torch.float64, device="cuda")
    ctx.transform(["coulomb"], 0, 2, 0.0, 1, out)             # the split path reads the same status word
    ref = oracle.Transform(p).packed("coulomb").reshape(-1)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-10
