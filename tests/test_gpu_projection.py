"""gpspca_project (S = B Z, samples onto sparse loadings) against the FP64
oracle.  The sums run in double-float (double for F64), so the stated bound is
float rounding of the output: per column ||S - S_ref|| <= 1e-6 ||S_ref||
(fp8: the entry q s is formed in float first, 2^-24 relative per entry)."""

import numpy as np
import pytest

import oracle
from paper_1312_6182_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = binding.Context(0)
    yield c
    c.close()


def _check(S, ref, tol=1e-6):
    S = S.double().cpu().numpy().T
    for j in range(ref.shape[1]):
        nr = np.linalg.norm(ref[:, j])
        if nr == 0:
            assert np.all(S[:, j] == 0)
        else:
            assert np.linalg.norm(S[:, j] - ref[:, j]) <= tol * nr, j


def test_project_training_and_new_samples(ctx):
    """Loadings from a solve (BL1 m = 4), scores of the training matrix and of
    new samples drawn from the same model (ragged q)."""
    At = synth.planted_spike(1203, 5003, 4, [40.0, 30.0, 22.0, 16.0], support_frac=0.02, seed=41, dtype=np.float32)
    A = At.astype(np.float64).T
    res = ctx.solve(torch.from_numpy(At).cuda(), "BL1", [0.1] * 4, mu=[1.0] * 4, gamma_relative=True)
    Z = res.Z.contiguous()
    _check(ctx.project(torch.from_numpy(At).cuda(), Z), oracle.project(A, Z.double().cpu().numpy().T))
    Bt = synth.planted_spike(777, 5003, 4, [40.0, 30.0, 22.0, 16.0], support_frac=0.02, seed=42, dtype=np.float32)
    _check(ctx.project(torch.from_numpy(Bt).cuda(), Z),
           oracle.project(Bt.astype(np.float64).T, Z.double().cpu().numpy().T))


@pytest.mark.parametrize("fmt", ["bf16", "fp8", "f64"])
def test_project_storage_types(ctx, fmt):
    rng = np.random.default_rng(43)
    Bt = rng.standard_normal((3001, 517)).astype(np.float32)
    Zn = np.where(rng.random((3001, 7)) < 0.1, rng.standard_normal((3001, 7)), 0.0)
    Zn[:, 3] = 0.0  # a zero loading
    Zn[:, 5] = rng.standard_normal(3001)  # a dense one
    kw = {}
    if fmt == "bf16":
        t = torch.from_numpy(Bt).to(torch.bfloat16)
        deq = t.float().numpy().astype(np.float64)
        Z = torch.from_numpy(Zn.T.astype(np.float32).copy()).cuda()
    elif fmt == "fp8":
        s = np.abs(Bt).max(axis=1).astype(np.float32) / 448.0
        t = torch.from_numpy(Bt / s[:, None]).to(torch.float8_e4m3fn)
        deq = t.float().numpy().astype(np.float64) * s[:, None]
        kw["col_scale"] = torch.from_numpy(s).cuda()
        Z = torch.from_numpy(Zn.T.astype(np.float32).copy()).cuda()
    else:
        t = torch.from_numpy(Bt.astype(np.float64))
        deq = Bt.astype(np.float64)
        Z = torch.from_numpy(Zn.T.copy()).cuda()
    S = ctx.project(t.cuda(), Z, **kw)
    Zref = Z.double().cpu().numpy().T
    _check(S, oracle.project(deq.T, Zref), tol=1e-12 if fmt == "f64" else 1e-6)


def test_project_host_buffers_and_64_components(ctx):
    rng = np.random.default_rng(44)
    Bt = rng.standard_normal((2000, 301)).astype(np.float32)
    Zn = np.where(rng.random((64, 2000)) < 0.05, rng.standard_normal((64, 2000)), 0.0).astype(np.float32)
    dev = ctx.project(torch.from_numpy(Bt).cuda(), torch.from_numpy(Zn).cuda())
    host = ctx.project(torch.from_numpy(Bt).pin_memory(), torch.from_numpy(Zn).pin_memory())
    assert torch.equal(dev.cpu(), host)
    _check(dev, oracle.project(Bt.astype(np.float64).T, Zn.astype(np.float64).T))
    with pytest.raises(ValueError):
        ctx.project(torch.from_numpy(Bt).cuda(), torch.from_numpy(Zn[:, :100]).cuda())
