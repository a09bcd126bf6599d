"""Several single-unit components by projection deflation (gpspca_solve_deflated)
against the FP64 oracle (``oracle.gpower_deflated``), component by component.

Component 0 is an ordinary single-unit solve and is held to the single-unit
tolerances.  Component j >= 1 solves on A_{j-1}, which the GPU forms from its
own z_0 .. z_{j-1}: their float-level differences from the oracle's loadings
(<= 1e-5 relative) enter A_{j-1} on the support columns, so later components
are compared at 10x the single-unit figures (loadings and iterate 1e-4,
objective 1e-5), still three orders below the differences between components.
"""

import numpy as np
import pytest

import oracle
from paper_1312_6182_gb300 import binding, synth
from tests.compare import assert_matches, gpu_arrays

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = binding.Context(0)
    yield c
    c.close()


def _component(ref, j):
    r = oracle.OracleResult(ref.X[:, j:j + 1], ref.Z[:, j:j + 1], ref.objective[j:j + 1], ref.iters[j:j + 1],
                            ref.status[j:j + 1], ref.gamma[j:j + 1], ref.mu[j:j + 1], [], ref.T[:, j:j + 1])
    return r


def _gpu_component(g, j):
    return {k: (v[:, j:j + 1] if k in ("X", "Z") else v[j:j + 1]) for k, v in g.items()}


def _check(form, g, ref, eps=2.0 ** -24, tight=1.0):
    m = ref.Z.shape[1]
    np.testing.assert_allclose(g["gamma_abs"], ref.gamma, rtol=1e-6 * tight)
    for j in range(m):
        f = 1.0 if j == 0 else 10.0
        assert_matches(form, _gpu_component(g, j), _component(ref, j), ref.cnorms[:, j], tol_z=1e-5 * f * tight,
                       tol_f=1e-6 * f * tight, tol_x=1e-5 * f * tight, eps=eps, iters_slack=1,
                       label=f"deflated {form} component {j}")


@pytest.mark.parametrize("form", ["SL1", "SL0"])
def test_deflated_spikes_fp32_ragged(ctx, form):
    """1203 x 5003 planted spikes (4 spikes, ragged p and n), 4 components at a
    relative gamma of 0.1 of each deflated matrix's largest column."""
    At = synth.planted_spike(1203, 5003, 4, [40.0, 30.0, 22.0, 16.0], support_frac=0.02, seed=21,
                             dtype=np.float32)
    A = At.astype(np.float64).T
    ref = oracle.gpower_deflated(A, form, [0.1] * 4, tol=1e-6, maxit=500, relative=True)
    res = ctx.solve_deflated(torch.from_numpy(At).cuda(), form, [0.1] * 4, tol=1e-6, maxit=500,
                             gamma_relative=True)
    _check(form, gpu_arrays(res), ref)
    # the components are distinct spikes, not repeats of the first
    Z = gpu_arrays(res)["Z"]
    assert np.max(np.abs(np.triu(Z.T @ Z, 1))) < 0.5


def test_deflated_workload_5000x20000(ctx):
    """The benchmark matrix (5000 x 20000 FP32, five planted spikes), five SL1
    components at a relative gamma of 0.05."""
    At = synth.workload_spikes_5000x20000(0)
    A = At.astype(np.float64).T
    ref = oracle.gpower_deflated(A, "SL1", [0.05] * 5, tol=1e-6, maxit=1000, relative=True)
    res = ctx.solve_deflated(torch.from_numpy(At).cuda(), "SL1", [0.05] * 5, tol=1e-6, maxit=1000,
                             gamma_relative=True)
    _check("SL1", gpu_arrays(res), ref)


def test_deflated_fp64(ctx):
    """FP64 storage deflates in double: near double-precision agreement."""
    At = synth.workload_fp64_200x1000(0)
    A = At.T
    ref = oracle.gpower_deflated(A, "SL1", [0.1] * 3, tol=1e-10, maxit=2000, relative=True)
    res = ctx.solve_deflated(torch.from_numpy(At).cuda(), "SL1", [0.1] * 3, tol=1e-10, maxit=2000,
                             gamma_relative=True)
    assert res.Z.dtype == torch.float64
    _check("SL1", gpu_arrays(res), ref, eps=2.0 ** -53, tight=1e-3)


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_deflated_low_precision_storage(ctx, fmt):
    """BF16 / FP8 storage is widened to the float working copy: the oracle runs
    on the stored values (fp8 times its column scale)."""
    At = synth.planted_spike(1000, 4000, 3, [40.0, 25.0, 15.0], support_frac=0.03, seed=22, dtype=np.float32)
    if fmt == "bf16":
        t = torch.from_numpy(At).to(torch.bfloat16)
        deq, kw = t.float().numpy(), {}
    else:
        s = np.abs(At).max(axis=1).astype(np.float32) / 448.0
        t = torch.from_numpy(At / s[:, None]).to(torch.float8_e4m3fn)
        deq, kw = t.float().numpy().astype(np.float64) * s[:, None], {"col_scale": torch.from_numpy(s).cuda()}
    A = deq.astype(np.float64).T
    ref = oracle.gpower_deflated(A, "SL0", [0.1] * 3, tol=1e-6, maxit=500, relative=True)
    res = ctx.solve_deflated(t.cuda(), "SL0", [0.1] * 3, tol=1e-6, maxit=500, gamma_relative=True, **kw)
    _check("SL0", gpu_arrays(res), ref)


def test_first_component_is_the_plain_solve(ctx):
    """Component 0 runs the same kernels on a bit-identical copy of A."""
    At = synth.planted_spike(800, 3000, 2, [30.0, 15.0], support_frac=0.05, seed=23, dtype=np.float32)
    dA = torch.from_numpy(At).cuda()
    d = ctx.solve_deflated(dA, "SL1", [0.1, 0.1], gamma_relative=True)
    s = ctx.solve(dA, "SL1", [0.1], gamma_relative=True)
    assert torch.equal(d.Z[0], s.Z[0]) and torch.equal(d.X[0], s.X[0])
    assert d.objective[0].item() == s.objective[0].item() and d.iters[0].item() == s.iters[0].item()
    assert torch.equal(dA.cpu(), torch.from_numpy(At))  # the caller's A is not modified


def test_zero_component_deflates_nothing(ctx):
    """A component whose gamma thresholds everything (status ZERO) leaves the
    matrix as it was: the next component equals the one without it."""
    At = synth.planted_spike(600, 2500, 3, [30.0, 20.0, 12.0], support_frac=0.04, seed=24, dtype=np.float32)
    A = At.astype(np.float64).T
    big = float(oracle.column_norms(A).max()) * 10.0
    dA = torch.from_numpy(At).cuda()
    g0 = oracle.gamma_from_rho(A, "SL1", 0.1)[0]
    with_zero = ctx.solve_deflated(dA, "SL1", [g0, big, g0])
    without = ctx.solve_deflated(dA, "SL1", [g0, g0])
    assert with_zero.status[1].item() == binding.ZERO
    assert torch.equal(with_zero.Z[1], torch.zeros_like(with_zero.Z[1]))
    assert torch.equal(with_zero.Z[2], without.Z[1]) and torch.equal(with_zero.X[2], without.X[1])


def test_deflated_host_buffers(ctx):
    """Host (pinned) input and outputs give the device path's bits."""
    At = synth.planted_spike(700, 2600, 2, [30.0, 18.0], support_frac=0.05, seed=25, dtype=np.float32)
    dev = ctx.solve_deflated(torch.from_numpy(At).cuda(), "SL0", [0.1, 0.1], gamma_relative=True)
    out = binding.alloc_result(2, 700, 2600, "cpu", torch.float32, pin=True)
    host = ctx.solve_deflated(torch.from_numpy(At).pin_memory(), "SL0", [0.1, 0.1], gamma_relative=True, out=out)
    assert torch.equal(host.Z, dev.Z.cpu()) and torch.equal(host.X, dev.X.cpu())
    assert torch.equal(host.objective, dev.objective.cpu()) and torch.equal(host.iters, dev.iters.cpu())


def test_deflated_rejects_block_forms(ctx):
    At = torch.randn(100, 50, device="cuda")
    with pytest.raises(binding.GpspcaError):
        ctx.solve_deflated(At, "BL1", [0.1])
