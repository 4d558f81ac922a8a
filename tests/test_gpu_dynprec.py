"""Split form with plain-FP32 integrals under an error budget: the measured
FP32 integral error stays inside the model the budget assumes, the FP32
quartets are in use, their bound is within the budget, the output stays
within the split form's tolerance, and a zero budget turns them off."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2606_04316_gb300 import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
F32_REL = 256.0 / 2 ** 24           # the error model: |FP32 - exact| <= F32_REL Q_A Q_C
BLOCKS = ("coulomb", "gaunt", "gauge")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def ctx_for(qdt, p):
    ctx = qdt.Context(0)
    ctx.set_basis(p.basis)
    ctx.set_coefficients(p.CL, p.CS)
    return ctx


@pytest.mark.parametrize("shells,nprim,seed", [((0, 1), 3, 681), ((0, 1, 2), 2, 682)])
def test_fp32_integral_error_within_model(torch_cuda, shells, nprim, seed):
    """Every kept integral (tau = 0 keeps all), Coulomb and gauge kernels, s/p/d
    shells (so S-function quartets up to L = 12): measured ratio 8x below the
    model's."""
    from paper_2606_04316_gb300 import qdt
    p = synth.chain_problem(3, 2, seed=seed, shells=shells, nprim=nprim, blocks=BLOCKS, tau=0.0)
    r = ctx_for(qdt, p).f32_error_ratio(list(BLOCKS), 0, 2, 0.0)
    print("measured max |FP32 - FP32 pairs| / (Q Q): Coulomb %.3e, L-S %.3e (model %.3e)" % (r[0], r[1], F32_REL))
    assert 0.0 < r[0] <= F32_REL / 8 and 0.0 < r[1] <= F32_REL / 8


def test_fp32_quartets_in_use_and_within_tolerance(oracle, torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    p = synth.chain_problem(8, 4, seed=683, shells=(0, 1), nprim=3, blocks=BLOCKS, tau=1e-12)
    ctx = ctx_for(qdt, p)
    n = ctx.packed_size(list(BLOCKS), 0, 4) // 8
    o_split = torch.zeros(n, dtype=torch.float64, device="cuda")
    o_fp64 = torch.zeros_like(o_split)
    st = ctx.transform(list(BLOCKS), 0, 4, p.tau, 1, o_split)
    ctx.transform(list(BLOCKS), 0, 4, p.tau, 0, o_fp64)
    assert st["quartets_f32"][0] > 0 and st["quartets_f32"][1] > 0
    assert 0.0 < st["f32_bound"] <= 3e-11
    assert 0.0 < st["flops_eri_f32"] < st["flops_eri"]
    assert (o_split - o_fp64).abs().max().item() <= 1e-10
    got = o_split.cpu().numpy().reshape(len(BLOCKS), -1)
    tr = oracle.Transform(p)
    for i, b in enumerate(BLOCKS):
        assert np.abs(got[i] - tr.packed(b).reshape(-1)).max() <= 1e-10


def test_zero_budget_turns_fp32_off(torch_cuda):
    code = r'''
import sys, torch
sys.path.insert(0, %r)
from paper_2606_04316_gb300 import qdt, synth
p = synth.chain_problem(6, 3, seed=684, shells=(0, 1), nprim=2, tau=1e-12)
ctx = qdt.Context(0); ctx.set_basis(p.basis); ctx.set_coefficients(p.CL, p.CS)
out = torch.zeros(ctx.packed_size(["coulomb"], 0, 3) // 8, dtype=torch.float64, device="cuda")
st = ctx.transform(["coulomb"], 0, 3, p.tau, 1, out)
print(st["quartets_f32"][0], st["f32_bound"])
''' % ROOT
    outs = {}
    for tag, env in (("default", {}), ("off", {"QDT_F32_BUDGET": "0"})):
        r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, **env), capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs[tag] = r.stdout.split()
    assert int(outs["default"][0]) > 0
    assert int(outs["off"][0]) == 0 and float(outs["off"][1]) == 0.0
