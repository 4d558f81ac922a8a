"""Full-size parity: the Coulomb block of the 40-centre s+p chain (nL 160,
nS 480, 40 Kramers pairs, Schwarz threshold 1e-12) on the GPU, in the launch
configuration the benchmark times (a context on its own stream, device
output), against values the oracle's row-streamed transform wrote
(tests/golden/make_golden.py): a seeded sample of 4000 packed entries plus the
96 largest, element by element (FP64 form <= 1e-12, split form <= 1e-10), the
kept shell-quartet count exactly, and whole-array checksums."""
import os

import numpy as np
import pytest

from paper_2606_04316_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "chain40_sp_coulomb_sample.txt")
TOL = {0: 1e-12, 1: 1e-10}


def read_golden():
    meta, idx, val = {}, [], []
    with open(GOLDEN) as f:
        for ln in f:
            if ln.startswith("#"):
                parts = ln[1:].split()
                if len(parts) >= 2 and parts[0] in ("doubles", "sum", "sum_abs", "sum_sq", "kept_shell_quartets"):
                    meta[parts[0]] = float(parts[1])
                continue
            i, v = ln.split()
            idx.append(int(i))
            val.append(float(v))
    return meta, np.array(idx, dtype=np.int64), np.array(val)


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def gpu_outputs(torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    p = synth.medium_dc()
    stream = torch.cuda.Stream()
    ctx = qdt.Context(0, stream=stream)
    ctx.set_basis(p.basis)
    ctx.set_coefficients(torch.from_numpy(p.CL).cuda(), torch.from_numpy(p.CS).cuda())
    n = ctx.packed_size(["coulomb"], 0, p.nK) // 8
    res = {}
    for prec in (0, 1):
        out = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = ctx.transform(["coulomb"], 0, p.nK, p.tau, prec, out)
        torch.cuda.synchronize()
        res[prec] = (out.cpu().numpy(), st)
    ctx.close()
    return res


@pytest.mark.parametrize("prec", [0, 1])
def test_chain40_coulomb_against_oracle(gpu_outputs, prec):
    meta, idx, ref = read_golden()
    got, st = gpu_outputs[prec]
    assert got.shape[0] == int(meta["doubles"])
    assert st["quartets_kept"][0] == int(meta["kept_shell_quartets"])
    err = np.abs(got[idx] - ref)
    assert err.max() <= TOL[prec], (prec, float(err.max()), int(idx[np.argmax(err)]))
    # whole-array checksums: every entry within the bar moves them by at most
    # doubles x bar (sum, sum_abs) and 2 bar sum|x| + doubles bar^2 (sum_sq)
    nd = got.shape[0]
    assert abs(got.sum() - meta["sum"]) <= nd * TOL[prec]
    assert abs(np.abs(got).sum() - meta["sum_abs"]) <= nd * TOL[prec]
    assert abs((got * got).sum() - meta["sum_sq"]) <= 2 * TOL[prec] * meta["sum_abs"] + nd * TOL[prec] ** 2
