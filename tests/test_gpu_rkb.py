"""Restricted-kinetic-balance input on the GPU (qdt_set_rkb_coefficients,
Eq. RKB): the device expansion of c^S over the derivative functions, then the
transform, against the oracle's expansion and transform, for quaternion and
Kramers-unrestricted columns, in both forms."""
import dataclasses

import numpy as np
import pytest

from paper_2606_04316_gb300 import synth

pytestmark = pytest.mark.gpu
TOL_FP64, TOL_SPLIT = 1e-12, 1e-10
BLOCKS = ("coulomb", "gaunt", "gauge")
C_LIGHT = 137.035999084


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def run(torch, ctx, blocks, k0, k1, tau, prec):
    out = torch.zeros(ctx.packed_size(list(blocks), k0, k1) // 8, dtype=torch.float64, device="cuda")
    st = ctx.transform(list(blocks), k0, k1, tau, prec, out)
    return out, st


def expanded(oracle, p):
    """The problem with c^S expanded over the derivative functions by the oracle."""
    cs = oracle.rkb_to_derivative(p.CS, C_LIGHT, spinors=not p.kramers)
    return dataclasses.replace(p, CS=cs, rkb=False)


@pytest.mark.parametrize("kramers", [True, False])
@pytest.mark.parametrize("prec,tol", [(0, TOL_FP64), (1, TOL_SPLIT)])
def test_rkb_against_oracle(oracle, torch_cuda, kramers, prec, tol):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    n = 3 if kramers else 5
    p = synth.rkb_chain_problem(3, n, seed=621, shells=(0, 1), nprim=2, blocks=BLOCKS, tau=0.0,
                                kramers=kramers)
    ctx = qdt.Context(0)
    ctx.set_basis(p.basis)
    ctx.set_rkb_coefficients(p.CL, p.CS, C_LIGHT, spinors=not kramers)
    out, _ = run(torch, ctx, BLOCKS, 0, n, 0.0, prec)
    got = out.cpu().numpy().reshape(len(BLOCKS), -1)
    q = expanded(oracle, p)
    tr = oracle.Transform(q) if kramers else oracle.TransformKU(q)
    for i, b in enumerate(BLOCKS):
        ref = tr.packed(b).reshape(-1)
        assert np.abs(ref).max() > 1e-8
        assert np.abs(got[i] - ref).max() <= tol


@pytest.mark.parametrize("kramers", [True, False])
def test_rkb_equals_expanded_input(oracle, torch_cuda, kramers):
    """The device expansion gives the same coefficients as the oracle's (both
    scale each component by the correctly rounded 1/2c), so the transforms
    agree bit for bit; device-resident input takes the same path."""
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    n = 4
    p = synth.rkb_chain_problem(4, n, seed=622, shells=(0, 1), nprim=2, blocks=BLOCKS, tau=1e-11,
                                kramers=kramers)
    q = expanded(oracle, p)
    a, b = qdt.Context(0), qdt.Context(0)
    a.set_basis(p.basis)
    b.set_basis(p.basis)
    a.set_rkb_coefficients(torch.from_numpy(p.CL).cuda(), torch.from_numpy(p.CS).cuda(), C_LIGHT,
                           spinors=not kramers)
    if kramers:
        b.set_coefficients(q.CL, q.CS)
    else:
        b.set_spinor_coefficients(q.CL, q.CS)
    for prec in (0, 1):
        oa, sa = run(torch, a, BLOCKS, 0, n, p.tau, prec)
        ob, sb = run(torch, b, BLOCKS, 0, n, p.tau, prec)
        assert sa["quartets_kept"] == sb["quartets_kept"]
        assert torch.equal(oa, ob)


def test_rkb_rejects_bad_speed_of_light(torch_cuda):
    from paper_2606_04316_gb300 import qdt
    p = synth.rkb_chain_problem(2, 2, seed=623, shells=(0,), nprim=1)
    ctx = qdt.Context(0)
    ctx.set_basis(p.basis)
    for c in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(qdt.QdtError):
            ctx.set_rkb_coefficients(p.CL, p.CS, c)
