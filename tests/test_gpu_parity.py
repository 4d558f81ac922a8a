"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element: FP64 form to 1e-12 absolute."""
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


def run_gpu(torch, p, blocks, k0, k1, tau, precision=0, host_out=False):
    from paper_2606_04316_gb300 import qdt
    ctx = qdt.Context(0)
    ctx.set_basis(p.basis)
    ctx.set_coefficients(p.CL, p.CS)
    n = ctx.packed_size(blocks, k0, k1) // 8
    if host_out:
        out = np.zeros(n)
    else:
        out = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = ctx.transform(blocks, k0, k1, tau, precision, out)
    res = out if host_out else out.cpu().numpy()
    return ctx, res.reshape(len(blocks), -1), st


def test_tiny_dirac_coulomb_packed_and_unpacked(oracle, torch_cuda):
    torch = torch_cuda
    p = synth.tiny_dc()
    ctx, got, st = run_gpu(torch, p, ["coulomb"], 0, p.nK, 0.0)
    tr = oracle.Transform(p)
    ref = tr.packed("coulomb")
    assert np.abs(got[0] - ref.reshape(-1)).max() <= TOL_FP64
    # unpack on the GPU vs the plain definition
    n = 2 * p.nK
    full = torch.zeros(2 * n ** 4, dtype=torch.float64, device="cuda")
    ctx.unpack(torch.from_numpy(got[0].copy()).cuda(), p.nK, "coulomb", full)
    f = full.cpu().numpy().reshape(n, n, n, n, 2)
    f = f[..., 0] + 1j * f[..., 1]
    assert np.abs(f - tr.full("coulomb")).max() <= TOL_FP64
    assert st["kernel_launches"] > 0


@pytest.mark.parametrize("nprim,shells", [(1, (0,)), (2, (0, 1)), (3, (0, 1))])
def test_small_dcb_all_blocks(oracle, torch_cuda, nprim, shells):
    torch = torch_cuda
    p = synth.chain_problem(3, 3, seed=101 + nprim, shells=shells, nprim=nprim,
                            blocks=("coulomb", "gaunt", "gauge"), tau=0.0)
    ctx, got, st = run_gpu(torch, p, list(p.blocks), 0, p.nK, 0.0)
    tr = oracle.Transform(p)
    for i, b in enumerate(p.blocks):
        ref = tr.packed(b).reshape(-1)
        err = np.abs(got[i] - ref).max()
        assert err <= TOL_FP64, (b, err, np.abs(ref).max())


def test_active_range_and_host_output(oracle, torch_cuda):
    torch = torch_cuda
    p = synth.chain_problem(3, 5, seed=77, shells=(0, 1), nprim=2, blocks=("coulomb", "gauge"), tau=0.0)
    ctx, got, st = run_gpu(torch, p, ["coulomb", "gauge"], 1, 4, 0.0, host_out=True)
    tr = oracle.Transform(p, k_begin=1, k_end=4)
    for i, b in enumerate(["coulomb", "gauge"]):
        assert np.abs(got[i] - tr.packed(b).reshape(-1)).max() <= TOL_FP64


def test_screened_chain_matches_oracle(oracle, torch_cuda):
    """A chain long enough for the density-weighted Schwarz screening to drop
    quartets; identical kept sets and results within the FP64 bar."""
    torch = torch_cuda
    p = synth.chain_problem(9, 4, seed=55, shells=(0, 1), nprim=2, blocks=("coulomb", "gaunt"), tau=1e-9)
    ctx, got, st = run_gpu(torch, p, ["coulomb", "gaunt"], 0, p.nK, p.tau)
    tr = oracle.Transform(p)
    kept_or = [int(tr.mask("coulomb").sum()), int(tr.mask("gaunt").sum())]
    assert kept_or[0] < tr.mask("coulomb").size          # screening is active
    assert st["quartets_kept"][0] == kept_or[0]
    assert st["quartets_kept"][1] == kept_or[1]
    for i, b in enumerate(["coulomb", "gaunt"]):
        assert np.abs(got[i] - tr.packed(b).reshape(-1)).max() <= TOL_FP64


TOL_SPLIT = 1e-10


@pytest.mark.parametrize("blocks", [("coulomb",), ("coulomb", "gaunt", "gauge")])
def test_split_form_small(oracle, torch_cuda, blocks):
    """Split (Ozaki BF16) form against the oracle within 1e-10."""
    torch = torch_cuda
    p = synth.chain_problem(3, 3, seed=202, shells=(0, 1), nprim=2, blocks=blocks, tau=0.0)
    ctx, got, st = run_gpu(torch, p, list(blocks), 0, p.nK, 0.0, precision=1)
    tr = oracle.Transform(p)
    for i, b in enumerate(blocks):
        ref = tr.packed(b).reshape(-1)
        err = np.abs(got[i] - ref).max()
        assert err <= TOL_SPLIT, (b, err)


def test_split_form_tiny_config(oracle, torch_cuda):
    torch = torch_cuda
    p = synth.tiny_dc()
    ctx, got, st = run_gpu(torch, p, ["coulomb"], 0, p.nK, 0.0, precision=1)
    ref = oracle.Transform(p).packed("coulomb").reshape(-1)
    assert np.abs(got[0] - ref).max() <= TOL_SPLIT
    assert st["slices"] == 6


@pytest.mark.slow
def test_multi_tile_screened_chain_both_forms(oracle, torch_cuda):
    """10-centre s+p chain, 6 Kramers pairs: ~8000 rows (63 row tiles of 128,
    ragged tail), 84 columns, Schwarz threshold 1e-9 (screening active);
    FP64 form <= 1e-12 and split form <= 1e-10 against the oracle."""
    torch = torch_cuda
    p = synth.chain_problem(10, 6, seed=303, shells=(0, 1), nprim=3, blocks=("coulomb",), tau=1e-9)
    tr = oracle.Transform(p)
    ref = tr.packed("coulomb").reshape(-1)
    assert tr.mask("coulomb").mean() < 1.0
    for prec, tol in ((0, TOL_FP64), (1, TOL_SPLIT)):
        ctx, got, st = run_gpu(torch, p, ["coulomb"], 0, p.nK, p.tau, precision=prec)
        assert np.abs(got[0] - ref).max() <= tol, (prec, np.abs(got[0] - ref).max())


@pytest.mark.slow
def test_full_size_chain40_properties(torch_cuda):
    """The 40-centre chain at full size (the benchmark's workload): the split
    form agrees with the FP64 form within 1e-10, and the Coulomb output, a
    Gram matrix of a positive-definite kernel, is positive semidefinite."""
    torch = torch_cuda
    from oracle import oracle as O
    p = synth.medium_dc()
    _, f64, st64 = run_gpu(torch, p, ["coulomb"], 0, p.nK, p.tau, precision=0)
    _, spl, stsp = run_gpu(torch, p, ["coulomb"], 0, p.nK, p.tau, precision=1)
    assert st64["quartets_kept"] == stsp["quartets_kept"]
    assert np.abs(f64 - spl).max() <= TOL_SPLIT
    nP = p.nK * (p.nK + 1) // 2
    full = np.zeros((nP, 4, nP, 4))
    iu, ju = np.triu_indices(nP)
    blk = f64[0].reshape(-1, 4, 4)
    full[iu, :, ju, :] = blk
    full[ju, :, iu, :] = blk.transpose(0, 2, 1)
    w = np.linalg.eigvalsh(full.reshape(4 * nP, 4 * nP))
    assert w.min() >= -1e-10 * w.max()


def test_d_shells_all_blocks(oracle, torch_cuda):
    """s, p and d shells (derivative functions up to f): both forms, all blocks."""
    torch = torch_cuda
    p = synth.chain_problem(2, 2, seed=601, shells=(0, 1, 2), nprim=2,
                            blocks=("coulomb", "gaunt", "gauge"), tau=0.0)
    tr = oracle.Transform(p)
    for prec, tol in ((0, TOL_FP64), (1, TOL_SPLIT)):
        ctx, got, st = run_gpu(torch, p, list(p.blocks), 0, p.nK, 0.0, precision=prec)
        for i, b in enumerate(p.blocks):
            err = np.abs(got[i] - tr.packed(b).reshape(-1)).max()
            assert err <= tol, (prec, b, err)


def test_single_kramers_pair_and_s_only(oracle, torch_cuda):
    torch = torch_cuda
    p = synth.chain_problem(4, 1, seed=602, shells=(0,), nprim=2, blocks=("coulomb", "gaunt"), tau=0.0)
    ctx, got, st = run_gpu(torch, p, ["coulomb", "gaunt"], 0, 1, 0.0)
    tr = oracle.Transform(p)
    for i, b in enumerate(["coulomb", "gaunt"]):
        assert np.abs(got[i] - tr.packed(b).reshape(-1)).max() <= TOL_FP64


def test_argument_errors(torch_cuda):
    torch = torch_cuda
    from paper_2606_04316_gb300 import qdt
    p = synth.chain_problem(2, 2, seed=603, shells=(0,), nprim=1, blocks=("coulomb",), tau=0.0)
    ctx = qdt.Context(0)
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(qdt.QdtError) as e:            # no basis yet
        ctx.transform(["coulomb"], 0, 1, 0.0, 0, out)
    assert e.value.code == -4
    ctx.set_basis(p.basis)
    ctx.set_coefficients(p.CL, p.CS)
    for args in [(0, 0, 0.0, 0), (1, 3, 0.0, 0), (0, 2, -1.0, 0), (0, 2, 0.0, 7)]:
        with pytest.raises(qdt.QdtError) as e:
            ctx.transform(["coulomb"], args[0], args[1], args[2], args[3], out)
        assert e.value.code == -1
    small = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(qdt.QdtError):
        ctx.transform(["coulomb"], 0, 2, 0.0, 0, small)
    bad = synth.chain_problem(1, 1, seed=604, shells=(3,), nprim=1, blocks=("coulomb",), tau=0.0)
    with pytest.raises(qdt.QdtError) as e:
        ctx.set_basis(bad.basis)                        # f shells are not accepted
    assert e.value.code == -1


def test_split_first_half_in_row_chunks(oracle, torch_cuda, monkeypatch):
    """The split form bounds its digit planes: the first half runs in row chunks
    of the integral rows and column chunks of the density, the second half in
    K chunks summed in FP64.  Row and column chunks must give the same bits as
    one call (same digits, same products); K chunks agree within the split
    form's bound."""
    torch = torch_cuda
    p = synth.chain_problem(6, 4, seed=311, shells=(0, 1), nprim=2, blocks=("coulomb", "gaunt", "gauge"),
                            tau=1e-12)
    _, whole, _ = run_gpu(torch, p, list(p.blocks), 0, p.nK, p.tau, precision=1)
    monkeypatch.setenv("QDT_SPLIT_CHUNK_ROWS", "128")
    _, chunked, st = run_gpu(torch, p, list(p.blocks), 0, p.nK, p.tau, precision=1)
    # column chunks of the density as well: the same tiles, the same products
    monkeypatch.setenv("QDT_SPLIT_CHUNK_COLS", "64")
    _, cols, _ = run_gpu(torch, p, list(p.blocks), 0, p.nK, p.tau, precision=1)
    monkeypatch.delenv("QDT_SPLIT_CHUNK_ROWS")
    monkeypatch.delenv("QDT_SPLIT_CHUNK_COLS")
    # second half in K chunks summed in FP64: a different summation order
    monkeypatch.setenv("QDT_SPLIT_KCHUNK", "128")
    _, kchunks, _ = run_gpu(torch, p, list(p.blocks), 0, p.nK, p.tau, precision=1)
    monkeypatch.delenv("QDT_SPLIT_KCHUNK")
    assert np.array_equal(chunked, whole)
    assert np.array_equal(cols, whole)
    # each K chunk has its own power-of-two scales: a second split evaluation, so
    # the two agree within the split form's bound, not bitwise
    assert np.abs(kchunks - whole).max() <= 1e-10
    tr = oracle.Transform(p)
    for i, b in enumerate(p.blocks):
        assert np.abs(chunked[i] - tr.packed(b).reshape(-1)).max() <= 1e-10
        assert np.abs(kchunks[i] - tr.packed(b).reshape(-1)).max() <= 1e-10


def test_integral_launch_shapes_change_no_bit(torch_cuda, monkeypatch):
    """The autotuner's candidates (CTA threads, ket positions per tile, tile
    order) change how the integral work is cut and scheduled, never the
    arithmetic of an integral: every pinned shape gives the same bits, for the
    Coulomb and the gauge kernel and both forms."""
    torch = torch_cuda
    p = synth.chain_problem(6, 3, seed=321, shells=(0, 1), nprim=2, blocks=("coulomb", "gaunt", "gauge"),
                            tau=1e-12)
    for prec in (0, 1):
        ref = None
        for shape in ("128,8,0", "256,4,1", "128,16,1", "256,8,0"):
            monkeypatch.setenv("QDT_ERI_LAUNCH", shape)
            _, got, _ = run_gpu(torch, p, list(p.blocks), 0, p.nK, p.tau, precision=prec)
            if ref is None:
                ref = got
            else:
                assert np.array_equal(got, ref), shape
        monkeypatch.delenv("QDT_ERI_LAUNCH")
