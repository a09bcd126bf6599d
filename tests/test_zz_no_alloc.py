"""The allocation-free sweep (gpspca_sweep_static) against gpspca_solve.

Callers that cannot allocate device memory when they need a sweep (another
framework's caching allocator holds the free memory, a latency-bound loop
that must not hit the allocator, code where allocation is forbidden) use
gpspca_sweep_static, whose scratch lives in fixed device arrays.  Its outputs
must agree with the solver's on the same matrix and iterate: the objective at
x0 and the loadings from t with gpspca_solve(maxit = 1), the next iterate
with gpspca_solve(maxit = 2), at the tolerances of the other parity tests, on
two calls in a row (the second reuses the arrays the first left behind).

This file is collected last so that a failure here comes after every other
test has run; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

from paper_1312_6182_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["SL1", "SL0"])
def test_static_sweep_matches_solver_twice(form):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    p, n = 2000, 9001
    At = synth.planted_spike(p, n, 3, [30.0, 15.0, 10.0], support_frac=0.03, seed=21, dtype=np.float32)
    dA = torch.from_numpy(At).cuda()
    cmax = float(np.linalg.norm(At.astype(np.float64), axis=1).max())
    gamma = 0.05 * cmax if form == "SL1" else (0.05 * cmax) ** 2
    with binding.Context(0) as ctx:
        r1 = ctx.solve(dA, form, [gamma], tol=0.0, maxit=1)
        r2 = ctx.solve(dA, form, [gamma], tol=0.0, maxit=2)
    x0 = r1.X[0].contiguous()
    f_ref = r1.objective[0].item()
    x1_ref = r2.X[0].double().cpu().numpy()
    z_ref = r1.Z[0].double().cpu().numpy()

    results = []
    for _call in range(2):
        x_next = torch.empty(p, device="cuda", dtype=torch.float32)
        t = torch.empty(n, device="cuda", dtype=torch.float32)
        obj = torch.empty(1, device="cuda", dtype=torch.float64)
        binding.sweep_static(dA, form, gamma, x0, x_next, t, obj)
        torch.cuda.synchronize()
        f = obj.item()
        xn = x_next.double().cpu().numpy()
        tt = t.double().cpu().numpy()
        assert abs(f - f_ref) <= 1e-6 * abs(f_ref), (f, f_ref)
        assert np.linalg.norm(xn - x1_ref) <= 1e-5, np.linalg.norm(xn - x1_ref)
        if form == "SL1":
            zr = np.sign(tt) * np.maximum(np.abs(tt) - gamma, 0.0)
        else:
            zr = tt * (tt * tt > gamma)
        z = zr / np.linalg.norm(zr)
        assert np.linalg.norm(z - z_ref) <= 1e-5 * np.linalg.norm(z_ref)
        assert np.array_equal(z != 0, z_ref != 0)
        results.append((f, xn, tt))
    # the second call, on the arrays the first call left, gives the same result
    assert results[0][0] == results[1][0]
    assert np.array_equal(results[0][1], results[1][1]) and np.array_equal(results[0][2], results[1][2])


def test_static_sweep_rejects_sizes_beyond_its_scratch():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    p, n = 8193, 300  # one row more than the fixed scratch is sized for
    dA = torch.zeros((n, p), device="cuda", dtype=torch.float32)
    x = torch.zeros(p, device="cuda")
    with pytest.raises(binding.GpspcaError) as e:
        binding.sweep_static(dA, "SL1", 0.1, x, torch.empty_like(x), torch.empty(n, device="cuda"),
                             torch.empty(1, device="cuda", dtype=torch.float64))
    assert e.value.code == binding.EINVAL and "8192" in str(e.value)


@pytest.mark.parametrize("form", ["SL1", "SL0"])
def test_static_sweep_against_the_oracle_formulas(form):
    """One sweep at the largest p the scratch takes (8192 rows), from the
    single-unit start (the largest column, normalised), against the same
    sweep in float64 written with the oracle's Table 1 functions: t = A^T x,
    f, g, y = A g, x_next = y/||y||."""
    import oracle

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    p, n = 8192, 1501
    At = synth.planted_spike(p, n, 2, [60.0, 30.0], support_frac=0.05, seed=22, dtype=np.float32)
    A = At.astype(np.float64).T
    cn = np.linalg.norm(A, axis=0)
    x = (A[:, int(np.argmax(cn))] / cn.max()).astype(np.float32)
    c = float(cn.max())
    gamma = 0.05 * c if form == "SL1" else (0.05 * c) ** 2
    t_ref = A.T @ x.astype(np.float64)
    one = np.ones(1)
    f_ref = float(oracle.objective_parts(form, t_ref[:, None], np.array([gamma]), one)[0])
    y = A @ oracle.gradient_direction(form, t_ref[:, None], np.array([gamma]), one)[:, 0]
    xn_ref = y / np.linalg.norm(y)
    dA = torch.from_numpy(At).cuda()
    dx = torch.from_numpy(x).cuda()
    x_next = torch.empty(p, device="cuda")
    t = torch.empty(n, device="cuda")
    obj = torch.empty(1, device="cuda", dtype=torch.float64)
    for _call in range(2):
        binding.sweep_static(dA, form, gamma, dx, x_next, t, obj)
        tt = t.double().cpu().numpy()
        # t to float32 accuracy of a dot product of length p
        dt = 4.0 * 2.0 ** -24 * np.linalg.norm(A, axis=0)
        assert np.all(np.abs(tt - t_ref) <= dt), np.max(np.abs(tt - t_ref) / dt)
        assert abs(obj.item() - f_ref) <= 1e-6 * f_ref, (obj.item(), f_ref)
        assert np.linalg.norm(x_next.double().cpu().numpy() - xn_ref) <= 1e-5
        assert np.count_nonzero(oracle.gradient_direction(form, t_ref[:, None], np.array([gamma]), one)) > 10


def test_static_sweep_reports_non_finite_input():
    """A NaN in A or in x is reported (GPSPCA_ENONFINITE), not returned as a
    zero iterate; the next call with finite input works."""
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    p, n = 300, 700
    At = np.random.default_rng(24).standard_normal((n, p)).astype(np.float32)
    x = torch.full((p,), p ** -0.5, device="cuda")
    out = (torch.empty(p, device="cuda"), torch.empty(n, device="cuda"),
           torch.empty(1, device="cuda", dtype=torch.float64))
    bad = At.copy()
    bad[11, 7] = np.nan
    with pytest.raises(binding.GpspcaError) as e:
        binding.sweep_static(torch.from_numpy(bad).cuda(), "SL1", 0.5, x, *out)
    assert e.value.code == binding.ENONFINITE
    xb = x.clone()
    xb[5] = float("inf")
    with pytest.raises(binding.GpspcaError) as e:
        binding.sweep_static(torch.from_numpy(At).cuda(), "SL0", 0.5, xb, *out)
    assert e.value.code == binding.ENONFINITE
    binding.sweep_static(torch.from_numpy(At).cuda(), "SL1", 0.5, x, *out)
    assert np.isfinite(out[2].item())


def test_static_sweep_checks_its_buffers():
    """Buffers of the wrong size, type or device are refused before the call."""
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    p, n = 64, 100
    dA = torch.randn(n, p, device="cuda")
    x = torch.randn(p, device="cuda")
    good = dict(x_next=torch.empty(p, device="cuda"), t=torch.empty(n, device="cuda"),
                objective=torch.empty(1, device="cuda", dtype=torch.float64))
    for key, wrong in (("t", torch.empty(n - 1, device="cuda")), ("objective", torch.empty(1, device="cuda")),
                       ("x_next", torch.empty(p, device="cuda", dtype=torch.float64))):
        kw = dict(good)
        kw[key] = wrong
        with pytest.raises(binding.GpspcaError) as e:
            binding.sweep_static(dA, "SL1", 0.1, x, kw["x_next"], kw["t"], kw["objective"])
        assert e.value.code == binding.EINVAL
