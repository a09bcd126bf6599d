"""The autotuner (gpspca_tune): it times every candidate sweep layout of a
shape, later solves of the shape run the fastest one and still match the FP64
oracle, and a saved table gives a new context the same layout (the same
bits)."""

import numpy as np
import pytest

import oracle
from paper_1312_6182_gb300 import binding, synth
from tests.compare import align_to_gpu_stop, assert_matches, gpu_arrays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = binding.Context(0)
    yield c
    c.close()


def _gammas(A64, form, rho):
    c = oracle.column_norms(A64).max()
    rho = np.atleast_1d(rho).astype(np.float64)
    return rho * c if form.endswith("1") else (rho * c) ** 2


def test_tune_block_m8_then_solve_and_reload(ctx, tmp_path):
    """Block L1 with 8 components on 1500 x 8000 float (candidates: one
    8-component pass, 5 + 3, 4 + 4, ... in clusters of 1-8, the tensor-core
    sweep); the tuned solve against the oracle (6 sweeps from the start); the
    saved table reproduces it in a new context."""
    m = 8
    At = synth.planted_spike(1500, 8000, m, [100.0 / np.sqrt(j) for j in range(1, m + 1)], support_frac=0.01,
                             seed=51, dtype=np.float32)
    A = At.astype(np.float64).T
    gam = list(_gammas(A, "BL1", [0.02] * m))
    mu = [1.0] * m
    dA = torch.from_numpy(At).cuda()
    nc, best, dflt = ctx.tune(dA, "BL1", gam, mu=mu, reps=3)
    assert nc >= 3
    assert 0.0 < best <= dflt
    ref = oracle.gpower(A, "BL1", gam, mu=mu, tol=0.0, maxit=6)
    res = ctx.solve(dA, "BL1", gam, mu=mu, tol=0.0, maxit=6)
    assert_matches("BL1", gpu_arrays(res), ref, oracle.column_norms(A), label="tuned BL1 m=8")
    path = tmp_path / "layouts.tsv"
    ctx.tune_save(path)
    lines = path.read_text().splitlines()
    assert lines[0] == "gpspca-tune 1" and len(lines) >= 2
    assert all(len(line.split("\t")) == 3 for line in lines[1:])
    other = binding.Context(0)
    try:
        other.tune_load(path)
        again = other.solve(dA, "BL1", gam, mu=mu, tol=0.0, maxit=6)
        assert torch.equal(res.Z, again.Z) and torch.equal(res.X, again.X)
        assert torch.equal(res.objective, again.objective)
    finally:
        other.close()


def test_tune_single_unit(ctx):
    """A single-unit shape (clusters of 1-8 as candidates): tuned solve
    against the oracle."""
    At = synth.planted_spike(2000, 6000, 2, [40.0, 20.0], support_frac=0.03, seed=52, dtype=np.float32)
    A = At.astype(np.float64).T
    gam = list(_gammas(A, "SL1", [0.1]))
    dA = torch.from_numpy(At).cuda()
    nc, best, dflt = ctx.tune(dA, "SL1", gam, reps=3)
    assert nc >= 1 and 0.0 < best <= dflt
    ref = oracle.gpower(A, "SL1", gam, tol=1e-6, maxit=500)
    res = ctx.solve(dA, "SL1", gam, tol=1e-6, maxit=500)
    g = gpu_arrays(res)
    ref = align_to_gpu_stop(A, "SL1", gam, None, ref, g, 1e-6)
    assert_matches("SL1", g, ref, oracle.column_norms(A), label="tuned SL1")


def test_tune_gamma_path_bf16(ctx):
    """A 16-value gamma path on bf16 storage, whose default is the
    tensor-core sweep (the CUDA-core passes are the other candidates); the
    tuned solve against the oracle on the stored values (4 sweeps)."""
    At = synth.planted_spike(1504, 6000, 3, [40.0, 20.0, 13.3], support_frac=0.02, seed=53, dtype=np.float32)
    tb = torch.from_numpy(At).to(torch.bfloat16)
    A = tb.float().numpy().astype(np.float64).T
    gam = list(_gammas(A, "SL1", synth.log_spaced_rho(16, 0.005, 0.2)))
    dA = tb.cuda()
    nc, best, dflt = ctx.tune(dA, "SL1", gam, reps=3)
    assert nc >= 2 and 0.0 < best <= dflt
    ref = oracle.gpower(A, "SL1", gam, tol=0.0, maxit=4)
    res = ctx.solve(dA, "SL1", gam, tol=0.0, maxit=4)
    assert_matches("SL1", gpu_arrays(res), ref, oracle.column_norms(A), label="tuned gamma path bf16")


def test_tune_load_rejects_other_files(ctx, tmp_path):
    bad = tmp_path / "bad.tsv"
    bad.write_text("not a table\n")
    with pytest.raises(binding.GpspcaError) as e:
        ctx.tune_load(bad)
    assert e.value.code == binding.EINVAL
    with pytest.raises(binding.GpspcaError) as e:
        ctx.tune_load(tmp_path / "missing.tsv")
    assert e.value.code == binding.ENOTFOUND
