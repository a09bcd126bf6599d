"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Sizes span several column tiles, several clusters and ragged tails in both p
and n; the workload-sized cases (200 x 1000 FP64, 5000 x 20000 FP32) run in
the launch configuration the benchmark uses.
"""

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


def _dev(At, ld=None):
    """Device copy of At (n x p); ld > p pads each row (aligned fast path)."""
    n, p = At.shape
    if ld is None or ld == p:
        return torch.from_numpy(np.ascontiguousarray(At)).cuda()
    buf = np.zeros((n, ld), dtype=At.dtype)
    buf[:, :p] = At
    return torch.from_numpy(buf).cuda()


def _gammas(A64, form, rho):
    c = oracle.column_norms(A64).max()
    rho = np.atleast_1d(rho).astype(np.float64)
    return rho * c if form.endswith("1") else (rho * c) ** 2


def _run(ctx, At, form, gam, mu=None, tol=1e-6, maxit=1000, ld=None, x0=None, **kw):
    dA = _dev(At, ld)
    p = At.shape[1]
    res = ctx.solve(dA, form, list(gam), mu=mu, tol=tol, maxit=maxit, p=p, x0=x0, **kw)
    return gpu_arrays(res), res


def _converged(form, g, A, gam, mu, ref, tol, label, slack=2, **kw):
    """A solve run to convergence: where GPU and oracle stop a sweep apart
    (the decision sits on the tol boundary), compare with the oracle's state
    after the GPU's sweep count; then the stated limits."""
    ref = align_to_gpu_stop(A, form, gam, mu, ref, g, tol, slack=slack)
    assert_matches(form, g, ref, oracle.column_norms(A), label=label, **kw)


# ---------------------------------------------------------------- workload sizes

def test_fp64_200x1000_single_unit_l1(ctx):
    """200 x 1000 N(0,1), centred columns, FP64, SL1 at gamma = 0.1 max||a_i||,
    x0 = largest column, tol 1e-6, maxit 1000: computed in double on the GPU."""
    At = synth.workload_fp64_200x1000(0)
    A = At.T
    gam = _gammas(A, "SL1", 0.1)
    ref = oracle.gpower(A, "SL1", gam, tol=1e-6, maxit=1000)
    g, res = _run(ctx, At, "SL1", gam, tol=1e-6, maxit=1000)
    assert res.X.dtype == torch.float64
    assert_matches("SL1", g, ref, oracle.column_norms(A), tol_z=1e-9, tol_f=1e-11, tol_x=1e-9, iters_slack=0,
                   eps=2.0 ** -53)


@pytest.fixture(scope="module")
def spikes_full():
    At = synth.workload_spikes_5000x20000(0)
    return At, At.astype(np.float64).T


FULL_CASES = [
    ("SL1", None), ("SL0", None),
    ("BL1", [1.0] * 5), ("BL0", [1.0] * 5),
    ("BL1", [1.0, 0.9, 0.8, 0.7, 0.6]), ("BL0", [1.0, 0.9, 0.8, 0.7, 0.6]),
]


@pytest.mark.parametrize("form,mu", FULL_CASES)
def test_spikes_5000x20000_fp32(ctx, spikes_full, form, mu):
    """The four formulations on 5000 x 20000 planted spikes in FP32 against the
    FP64 oracle: loadings 1e-5, objective 1e-6, support outside the band."""
    At, A = spikes_full
    m = 1 if mu is None else 5
    gam = _gammas(A, form, [0.05] * m)
    ref = oracle.gpower(A, form, gam, mu=mu, tol=1e-6, maxit=1000)
    g, _ = _run(ctx, At, form, gam, mu=mu, tol=1e-6, maxit=1000)
    _converged(form, g, A, gam, mu, ref, 1e-6, f"5000x20000 {form} mu={mu}")


# ---------------------------------------------------------------- fixed sweep counts

RAGGED = dict(p=1237, n=3001)


@pytest.mark.parametrize("form", oracle.FORMS)
@pytest.mark.parametrize("ld", [1240, 1237])  # padded (bulk-copy path) and unpadded (element path)
def test_fixed_sweeps_ragged(ctx, form, ld):
    """tol = 0, 15 sweeps, ragged p and n, all four forms: per-step drift stays
    at float32 rounding.  ld = 1237 is not 16-byte aligned (element path)."""
    At = synth.planted_spike(RAGGED["p"], RAGGED["n"], 3, [25.0, 12.0, 8.0], support_frac=0.04, seed=5,
                             dtype=np.float32)
    A = At.astype(np.float64).T
    if form.startswith("S"):
        gam, mu = _gammas(A, form, [0.02, 0.08, 0.2]), None
    else:
        mu = [1.0, 0.8, 0.6]
        gam = _gammas(A, form, [0.03] * 3) * (np.array(mu) if form.endswith("1") else np.array(mu) ** 2)
    ref = oracle.gpower(A, form, gam, mu=mu, tol=0.0, maxit=15)
    g, _ = _run(ctx, At, form, gam, mu=mu, tol=0.0, maxit=15, ld=ld)
    assert_matches(form, g, ref, oracle.column_norms(A), label=f"ragged {form} ld={ld}")


@pytest.mark.parametrize("form", oracle.FORMS)
@pytest.mark.parametrize("tensor_cores", [True, False])
def test_long_columns(ctx, form, tensor_cores):
    """Float columns of 16384 rows or more: by default the tensor-core sweep
    for any m (here one or two components); with tensor_cores=False the
    CUDA-core sweep, which splits each column's rows over a cluster of CTAs
    whose partial dot products meet through distributed shared memory before
    the threshold.  16500 x 2003 planted spikes (rows ragged against the
    CTAs' slices and the 64-row chunks), 6 sweeps against the oracle; the two
    plans differ."""
    At = synth.planted_spike(16500, 2003, 2, [60.0, 35.0], support_frac=0.03, seed=64, dtype=np.float32)
    A = At.astype(np.float64).T
    m = 1 if form.startswith("S") else 2
    mu = None if m == 1 else [1.0, 0.8]
    gam = _gammas(A, form, [0.05] * m)
    dA = torch.from_numpy(At).cuda()
    plans = [ctx.plan_launches(dA, form, list(gam), mu=mu, tensor_cores=tc) for tc in (True, False)]
    assert plans[0][1] != plans[1][1], plans
    ref = oracle.gpower(A, form, gam, mu=mu, tol=0.0, maxit=6)
    res = ctx.solve(dA, form, list(gam), mu=mu, tol=0.0, maxit=6, tensor_cores=tensor_cores)
    assert_matches(form, gpu_arrays(res), ref, oracle.column_norms(A),
                   label=f"long columns {form} {'tensor cores' if tensor_cores else 'CUDA cores'}")


@pytest.mark.parametrize("form", ["SL1", "SL0"])
def test_gamma_path_64(ctx, form):
    """A 64-value gamma path (log-spaced over [0.001, 0.5] max||a_i||) on one
    A: 64 independent single-unit solves in 8 passes of the fused sweep."""
    At = synth.planted_spike(1500, 6000, 3, [40.0, 20.0, 13.3], support_frac=0.02, seed=1, dtype=np.float32)
    A = At.astype(np.float64).T
    gam = _gammas(A, form, synth.log_spaced_rho(64))
    ref = oracle.gpower(A, form, gam, tol=1e-6, maxit=300)
    g, _ = _run(ctx, At, form, gam, tol=1e-6, maxit=300)
    _converged(form, g, A, gam, None, ref, 1e-6, f"gamma path 64 {form} (CUDA cores)")


@pytest.mark.parametrize("p,n,m", [(1500, 8000, 16), (2000, 12000, 32)])
def test_block_many_components(ctx, p, n, m):
    """Block L1 with m = 16 and 32 components on as many planted spikes
    (theta_j = 100/sqrt(j), 1% supports): several component passes per sweep,
    a 16x16 / 32x32 FP64 Jacobi polar step, the PCA start; 8 sweeps."""
    At = synth.planted_spike(p, n, m, [100.0 / np.sqrt(j) for j in range(1, m + 1)], support_frac=0.01, seed=7,
                             dtype=np.float32)
    A = At.astype(np.float64).T
    gam = _gammas(A, "BL1", [0.02] * m)
    ref = oracle.gpower(A, "BL1", gam, mu=[1.0] * m, tol=0.0, maxit=8)
    g, _ = _run(ctx, At, "BL1", gam, mu=[1.0] * m, tol=0.0, maxit=8)
    assert_matches("BL1", g, ref, oracle.column_norms(A), label=f"BL1 m={m} {p}x{n}")


@pytest.mark.parametrize("m", [6, 8])
@pytest.mark.parametrize("tensor_cores", [True, False])
def test_block_six_to_eight_float_components(ctx, m, tensor_cores):
    """Float block L1 with 6 and 8 components on as many planted spikes: by
    default on the tensor cores (float read in place and split into bf16
    planes), and with tensor_cores=False in one 8-wide CUDA-core pass; both
    against the oracle, 6 sweeps from the PCA start.  The two plans differ
    (their per-iteration kernel counts are not the same)."""
    p, n = 1500, 8000
    At = synth.planted_spike(p, n, m, [80.0 / np.sqrt(j) for j in range(1, m + 1)], support_frac=0.02, seed=71,
                             dtype=np.float32)
    A = At.astype(np.float64).T
    gam = _gammas(A, "BL1", [0.03] * m)
    mu = [1.0] * m
    dA = torch.from_numpy(At).cuda()
    plans = [ctx.plan_launches(dA, "BL1", list(gam), mu=mu, tensor_cores=tc) for tc in (True, False)]
    assert plans[0][1] != plans[1][1], plans
    ref = oracle.gpower(A, "BL1", gam, mu=mu, tol=0.0, maxit=6)
    res = ctx.solve(dA, "BL1", list(gam), mu=mu, tol=0.0, maxit=6, tensor_cores=tensor_cores)
    assert_matches("BL1", gpu_arrays(res), ref, oracle.column_norms(A),
                   label=f"BL1 m={m} {p}x{n} {'tensor cores' if tensor_cores else 'CUDA cores'}")


# ---------------------------------------------------------------- tensor-core (tcgen05) sweep

@pytest.mark.parametrize("form,p,n,m", [("BL1", 1496, 8008, 16), ("BL0", 2048, 6000, 16), ("BL1", 1504, 9000, 32)])
def test_tensor_core_sweep_block_matches_oracle(ctx, form, p, n, m):
    """BF16 storage with 16 or more components runs the two-pass tcgen05
    sweep (p, n ragged against its 64-row and 128-column tiles); the oracle
    runs on the stored values.  8 sweeps from the PCA start."""
    At = synth.planted_spike(p, n, m, [100.0 / np.sqrt(j) for j in range(1, m + 1)], support_frac=0.01, seed=8,
                             dtype=np.float32)
    tb, deq = _bf16(At)
    A = deq.astype(np.float64).T
    gam = _gammas(A, form, [0.02] * m)
    mu = [1.0] * m
    ref = oracle.gpower(A, form, gam, mu=mu, tol=0.0, maxit=8)
    res = ctx.solve(tb.cuda(), form, list(gam), mu=mu, tol=0.0, maxit=8)
    assert_matches(form, gpu_arrays(res), ref, oracle.column_norms(A), label=f"tc bf16 {form} m={m} {p}x{n}")


@pytest.mark.parametrize("form", ["SL1", "SL0"])
def test_tensor_core_gamma_path_64(ctx, form):
    """A 64-value gamma path on BF16 storage: all 64 columns in one tcgen05
    contraction per sweep (N = 3 x 64), against the oracle's 64 solves."""
    At = synth.planted_spike(1504, 6000, 3, [40.0, 20.0, 13.3], support_frac=0.02, seed=1, dtype=np.float32)
    tb, deq = _bf16(At)
    A = deq.astype(np.float64).T
    gam = _gammas(A, form, synth.log_spaced_rho(64))
    ref = oracle.gpower(A, form, gam, tol=1e-6, maxit=300)
    res = ctx.solve(tb.cuda(), form, list(gam), tol=1e-6, maxit=300)
    _converged(form, gpu_arrays(res), A, gam, None, ref, 1e-6, f"tc gamma path 64 {form} bf16")


@pytest.mark.parametrize("form", ["BL1", "SL0"])
@pytest.mark.parametrize("p", [1200, 1204])  # aligned and unaligned column strides
def test_tensor_core_sweep_fp8_storage(ctx, form, p):
    """FP8 E4M3 storage with per-column scales and 16 components / gamma
    values: the tensor cores read the fp8 values as bf16 (exact) and the
    scales enter the threshold; oracle on the dequantised matrix."""
    At = synth.planted_spike(p, 5000, 16, [100.0 / np.sqrt(j) for j in range(1, 17)], support_frac=0.01, seed=13,
                             dtype=np.float32)
    q, sc, deq = _fp8(At)
    A = deq.astype(np.float64).T
    m = 16
    rho = [0.02] * m if form.startswith("B") else list(synth.log_spaced_rho(m, 0.005, 0.3))
    gam = _gammas(A, form, rho)
    mu = [1.0] * m if form.startswith("B") else None
    ref = oracle.gpower(A, form, gam, mu=mu, tol=0.0, maxit=6)
    res = ctx.solve(q.cuda(), form, list(gam), mu=mu, tol=0.0, maxit=6, col_scale=sc.cuda())
    assert_matches(form, gpu_arrays(res), ref, oracle.column_norms(A), label=f"tc fp8 {form} p={p}")


@pytest.mark.parametrize("dtype,form,p,n,m", [
    ("bf16", "BL1", 40, 100, 6),     # p below one 64-row chunk, n below one 128-column tile
    ("bf16", "SL0", 37, 1000, 8),    # unaligned bf16 stride: padded copy for TMA
    ("f32", "SL1", 70, 300, 9),      # float: three bf16 planes
    ("f32", "BL0", 256, 2000, 64),   # N = 192, the largest tensor-memory layout
])
def test_tensor_core_sweep_edge_shapes(ctx, dtype, form, p, n, m):
    """Shapes at the edges of the tensor-core sweep's tiles, layouts and
    widths, against the oracle on the stored values (3 sweeps from the start).
    The 64-component case has 64 planted spikes (31 columns each, theta_j =
    60 - j/2), so that every component is determined by the data rather than
    by rounding."""
    k = min(m, 4)
    if m == 64:
        At = synth.planted_spike(p, n, m, [60.0 - 0.5 * j for j in range(m)], support_size=31, seed=95,
                                 dtype=np.float32)
    else:
        At = synth.planted_spike(p, n, k, [30.0 / (j + 1) for j in range(k)], support_frac=0.05, seed=31 + m,
                                 dtype=np.float32)
    if dtype == "bf16":
        tA, deq = _bf16(At)
        tA = tA.cuda()
    else:
        tA, deq = torch.from_numpy(At).cuda(), At
    A = deq.astype(np.float64).T
    block = form.startswith("B")
    rho = ([0.05] if m == 64 else [0.01]) * m if block else list(synth.log_spaced_rho(m, 0.005, 0.2))
    gam = _gammas(A, form, rho)
    mu = [1.0] * m if block else None
    ref = oracle.gpower(A, form, gam, mu=mu, tol=0.0, maxit=3)
    res = ctx.solve(tA, form, list(gam), mu=mu, tol=0.0, maxit=3, allow_degenerate=True)
    if block and 4 < m < 64:
        # more components than spikes: compare only the well-determined objective
        assert abs(res.objective.sum().item() - ref.total) / ref.total < 1e-6
        X = res.X.double().cpu().numpy().T
        assert np.abs(X.T @ X - np.eye(m)).max() < 1e-5
    else:
        assert_matches(form, gpu_arrays(res), ref, oracle.column_norms(A), label=f"tc edge {dtype} {form} m={m}")


@pytest.mark.parametrize("dtype,form,p,n,m", [
    ("f32", "BL1", 2100, 3000, 16),     # float read in place; 4 row ranges, the last one shorter
    ("f32", "SL1", 8000, 2000, 16),     # 8 row ranges (the most)
    ("f32-ld", "SL0", 2100, 3000, 16),  # float with an odd column stride: planes copied once per solve
    ("bf16", "SL1", 3000, 2500, 64),    # N = 192 on bf16 storage
])
def test_tensor_core_t_pass_row_ranges(ctx, dtype, form, p, n, m):
    """Long columns on few 128-column tiles: the T pass splits each tile's rows
    into ranges (partial T summed in range order before the threshold).
    Against the oracle on the stored values, 4 sweeps from the start; two runs
    give the same bits."""
    block = form.startswith("B")
    k = m if block else 3
    At = synth.planted_spike(p, n, k, [100.0 / np.sqrt(j) for j in range(1, k + 1)], support_frac=0.02, seed=41,
                             dtype=np.float32)
    if dtype == "bf16":
        tA, deq = _bf16(At)
        tA = tA.cuda()
    elif dtype == "f32-ld":
        wide = torch.zeros(n, p + 1)
        wide[:, :p] = torch.from_numpy(At)
        tA, deq = wide.cuda()[:, :p], At
    else:
        tA, deq = torch.from_numpy(At).cuda(), At
    A = deq.astype(np.float64).T
    rho = [0.02] * m if block else list(synth.log_spaced_rho(m, 0.005, 0.2))
    gam = _gammas(A, form, rho)
    mu = [1.0] * m if block else None
    ref = oracle.gpower(A, form, gam, mu=mu, tol=0.0, maxit=4)
    res = ctx.solve(tA, form, list(gam), mu=mu, tol=0.0, maxit=4)
    assert_matches(form, gpu_arrays(res), ref, oracle.column_norms(A), label=f"tc row ranges {dtype} {form} {p}x{n}")
    again = ctx.solve(tA, form, list(gam), mu=mu, tol=0.0, maxit=4)
    assert torch.equal(res.Z, again.Z) and torch.equal(res.X, again.X)


@pytest.mark.parametrize("form,p,n,m,frac", [
    ("BL0", 1500, 4099, 9, 0.02),    # 18% of the columns active
    ("BL1", 2100, 3001, 16, 0.01),   # 16%: 480 listed columns, 7.5 chunks of 64
    ("BL1", 777, 1601, 10, 0.03),    # 30%, p ragged against the 128-row blocks
])
def test_tensor_core_listed_columns(ctx, form, p, n, m, frac):
    """Float storage on the tensor cores: a threshold sweep's rank update
    Y = A G reads only the columns with some G_ij != 0 (gathered by TMA from
    the list of active columns), the others contributing nothing.  m planted
    spikes of theta_j = 60/sqrt(j), 4 sweeps from the PCA start, against the
    oracle at the stated limits."""
    At = synth.planted_spike(p, n, m, [60.0 / np.sqrt(j + 1) for j in range(m)], support_frac=frac, seed=61,
                             dtype=np.float32)
    A = At.astype(np.float64).T
    rho = {9: 0.05, 16: 0.05, 10: 0.06}[m]
    gam = _gammas(A, form, [rho] * m)
    ref = oracle.gpower(A, form, gam, mu=[1.0] * m, tol=0.0, maxit=4)
    res = ctx.solve(torch.from_numpy(At).cuda(), form, list(gam), mu=[1.0] * m, tol=0.0, maxit=4)
    assert_matches(form, gpu_arrays(res), ref, oracle.column_norms(A), label=f"tc listed {form} {p}x{n} m={m}")
    again = ctx.solve(torch.from_numpy(At).cuda(), form, list(gam), mu=[1.0] * m, tol=0.0, maxit=4)
    assert torch.equal(res.Z, again.Z) and torch.equal(res.X, again.X)


@pytest.mark.parametrize("storage,form,p,n,m", [
    ("bf16", "BL1", 2100, 3001, 16),      # bf16 read in place (column stride a multiple of 8)
    ("bf16", "BL0", 777, 1601, 10),       # p ragged: the last pieces of each column zero-filled
    ("bf16-odd", "BL1", 1501, 2999, 12),  # unaligned stride: the padded bf16 copy
    ("fp8", "BL1", 1200, 3001, 16),       # fp8 values (bf16 copy), column scales in G
    ("f32-odd", "BL0", 1203, 2501, 16),   # float with an unaligned stride: three bf16 planes copied
])
def test_tensor_core_listed_columns_bf16_planes(ctx, storage, form, p, n, m):
    """The rank update over the listed active columns in the tensor-core
    sweep that reads bf16 planes (bf16 storage, fp8 values, copied float
    planes): the listed columns are copied piece by piece into the swizzled
    layout of a tile load.  m planted spikes (theta_j = 60/sqrt(j), 2%
    supports: 20-32% of the columns active, below the 60% up to which the
    sweep lists them), 4 sweeps from the PCA start, against the oracle on the
    stored values; a second solve gives the same bits."""
    At = synth.planted_spike(p, n, m, [60.0 / np.sqrt(j + 1) for j in range(m)], support_frac=0.02, seed=63,
                             dtype=np.float32)
    scale = None
    if storage.startswith("bf16"):
        tb, deq = _bf16(At)
        if storage == "bf16-odd":
            wide = torch.zeros((n, p + 2), dtype=torch.bfloat16)  # stride 1503: not a multiple of 8
            wide[:, :p] = tb
            dA = wide.cuda()
        else:
            dA = tb.cuda()
    elif storage == "fp8":
        q, sc, deq = _fp8(At)
        dA, scale = q.cuda(), sc.cuda()
    else:
        deq = At
        wide = torch.zeros((n, p + 2), dtype=torch.float32)  # stride 1205: not a multiple of 4
        wide[:, :p] = torch.from_numpy(At)
        dA = wide.cuda()
    A = deq.astype(np.float64).T
    gam = _gammas(A, form, [0.05] * m)
    mu = [1.0] * m
    ref = oracle.gpower(A, form, gam, mu=mu, tol=0.0, maxit=4)
    res = ctx.solve(dA, form, list(gam), mu=mu, tol=0.0, maxit=4, p=p, col_scale=scale)
    active = np.count_nonzero(np.any(ref.Z != 0, axis=1)) / n
    assert active <= 0.4, active
    assert_matches(form, gpu_arrays(res), ref, oracle.column_norms(A),
                   label=f"tc listed {storage} {form} {p}x{n} m={m} ({active:.0%} active)")
    again = ctx.solve(dA, form, list(gam), mu=mu, tol=0.0, maxit=4, p=p, col_scale=scale)
    assert torch.equal(res.Z, again.Z) and torch.equal(res.X, again.X)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("maxit", [1, 2])
def test_first_sweep_from_the_rotation_step(ctx, storage, maxit):
    """The first sweep after a block start on the tensor cores forms T from
    the A^T Q its Rayleigh-Ritz step kept, times the rotation (no read of A
    for T): one and two sweeps from the PCA start against the oracle, and
    the host-driven launches give the graph's bits."""
    p, n, m = 1500, 4099, 16
    At = synth.planted_spike(p, n, m, [60.0 / np.sqrt(j + 1) for j in range(m)], support_frac=0.01, seed=65,
                             dtype=np.float32)
    if storage == "bf16":
        tb, deq = _bf16(At)
        dA, A = tb.cuda(), deq.astype(np.float64).T
    else:
        dA, A = torch.from_numpy(At).cuda(), At.astype(np.float64).T
    gam = _gammas(A, "BL1", [0.05] * m)
    mu = [1.0] * m
    ref = oracle.gpower(A, "BL1", gam, mu=mu, tol=0.0, maxit=maxit)
    res = ctx.solve(dA, "BL1", list(gam), mu=mu, tol=0.0, maxit=maxit)
    assert_matches("BL1", gpu_arrays(res), ref, oracle.column_norms(A),
                   label=f"first sweep from the rotation {storage} maxit={maxit}")
    eager = ctx.solve(dA, "BL1", list(gam), mu=mu, tol=0.0, maxit=maxit, eager=True)
    assert torch.equal(res.Z, eager.Z) and torch.equal(res.X, eager.X)
    assert torch.equal(res.objective, eager.objective) and torch.equal(res.iters, eager.iters)


def test_tensor_core_all_thresholded(ctx):
    """Float storage, 16 components, gamma above every |a_i^T x|: no column is
    active, the first sweep's objective is 0 (status ZERO, one sweep)."""
    At = np.random.default_rng(62).standard_normal((1000, 300)).astype(np.float32)
    A = At.astype(np.float64).T
    c = oracle.column_norms(A).max() * (1.0 + 1e-6)
    res = ctx.solve(torch.from_numpy(At).cuda(), "BL1", [c] * 16, mu=[1.0] * 16)
    assert np.all(res.status.cpu().numpy() == binding.ZERO) and np.all(res.iters.cpu().numpy() == 1)
    assert torch.all(res.Z == 0) and torch.all(res.objective == 0)


def test_tensor_core_and_cuda_core_sweeps_agree(ctx):
    """The same solve with and without the tensor cores: float-rounding
    differences only, on the well-determined quantities (the objective, and
    the components of the four planted spikes; the other twelve fit noise
    with near-equal eigenvalues and move freely at rounding level)."""
    At = synth.planted_spike(1024, 4096, 4, [40.0, 28.0, 23.0, 20.0], support_frac=0.02, seed=5, dtype=np.float32)
    dA = _bf16(At)[0].cuda()
    gam = [0.03] * 16
    a = ctx.solve(dA, "BL1", gam, mu=[1.0] * 16, tol=0.0, maxit=4, gamma_relative=True, tensor_cores=False)
    b = ctx.solve(dA, "BL1", gam, mu=[1.0] * 16, tol=0.0, maxit=4, gamma_relative=True)
    assert ((a.objective[:4] - b.objective[:4]).abs() / a.objective[:4].abs()).max().item() < 1e-5
    assert abs(a.objective.sum().item() - b.objective.sum().item()) / a.objective.sum().item() < 1e-6
    # the planted subspace: projector onto the leading four columns
    Xa, Xb = a.X[:4].double(), b.X[:4].double()
    assert (Xa.T @ Xa - Xb.T @ Xb).abs().max().item() < 1e-5


# ---------------------------------------------------------------- storage precisions

def _bf16(At):
    t = torch.from_numpy(At).to(torch.bfloat16)
    return t, t.float().numpy()


def _fp8(At):
    s = np.abs(At).max(axis=1).astype(np.float32) / 448.0
    s[s == 0] = 1.0
    q = torch.from_numpy(At / s[:, None]).to(torch.float8_e4m3fn)
    deq = q.float().numpy() * s[:, None]
    return q, torch.from_numpy(s), deq


@pytest.mark.parametrize("form", oracle.FORMS)
def test_bf16_storage_matches_oracle_on_stored_values(ctx, form):
    """BF16 storage: the oracle runs on the exactly upcast BF16 values, so the
    only differences are float32 accumulation."""
    At = synth.planted_spike(2000, 7001, 3, [30.0, 15.0, 10.0], support_frac=0.03, seed=11, dtype=np.float32)
    tb, deq = _bf16(At)
    A = deq.astype(np.float64).T
    m = 1 if form.startswith("S") else 3
    mu = None if m == 1 else [1.0, 0.8, 0.6]
    gam = _gammas(A, form, [0.05] * m)
    ref = oracle.gpower(A, form, gam, mu=mu, tol=1e-6, maxit=500)
    res = ctx.solve(tb.cuda(), form, list(gam), mu=mu, tol=1e-6, maxit=500)
    _converged(form, gpu_arrays(res), A, gam, mu, ref, 1e-6, f"bf16 storage {form}")


@pytest.mark.parametrize("form", ["SL0", "BL1"])
def test_fp8_storage_matches_oracle_on_stored_values(ctx, form):
    """FP8 E4M3 with per-column scales: oracle on the dequantised matrix."""
    At = synth.planted_spike(1800, 6000, 3, [30.0, 15.0, 10.0], support_frac=0.03, seed=12, dtype=np.float32)
    q, s, deq = _fp8(At)
    A = deq.astype(np.float64).T
    m = 1 if form.startswith("S") else 3
    mu = None if m == 1 else [1.0, 1.0, 1.0]
    gam = _gammas(A, form, [0.05] * m)
    ref = oracle.gpower(A, form, gam, mu=mu, tol=1e-6, maxit=500)
    res = ctx.solve(q.cuda(), form, list(gam), mu=mu, tol=1e-6, maxit=500, col_scale=s.cuda())
    _converged(form, gpu_arrays(res), A, gam, mu, ref, 1e-6, f"fp8 storage {form}")


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_low_precision_then_fp32_refinement(ctx, fmt):
    """Precision path: converge on BF16 / FP8 storage, then 3 FP32 sweeps from
    the converged X on the FP32 matrix; against the oracle on the FP32 matrix
    the loadings are within 1e-3."""
    At = synth.planted_spike(2000, 8000, 4, [40.0, 28.0, 23.0, 20.0], support_frac=0.01, seed=2,
                             dtype=np.float32)
    A = At.astype(np.float64).T
    mu = [1.0] * 4
    gam = _gammas(A, "BL1", [0.05] * 4)
    ref = oracle.gpower(A, "BL1", gam, mu=mu, tol=1e-6, maxit=1000)
    if fmt == "bf16":
        low = ctx.solve(_bf16(At)[0].cuda(), "BL1", list(gam), mu=mu, tol=1e-6, maxit=1000)
    else:
        q, s, _ = _fp8(At)
        low = ctx.solve(q.cuda(), "BL1", list(gam), mu=mu, tol=1e-6, maxit=1000, col_scale=s.cuda())
    x0 = low.X.contiguous()
    fine = ctx.solve(torch.from_numpy(At).cuda(), "BL1", list(gam), mu=mu, tol=0.0, maxit=3, x0=x0)
    g = gpu_arrays(fine)
    # stated: loadings and iterate 1e-3 after the low-precision solve and the
    # refinement, objective 1e-6, support outside the band; the band and the
    # objective limit also carry the iterate's own difference (each t_i moves
    # by at most ||a_i|| ||x_j - x_j^oracle||)
    dx = np.linalg.norm(g["X"] - ref.X, axis=0)
    assert_matches("BL1", g, ref, oracle.column_norms(A), tol_z=1e-3, tol_x=1e-3, tol_f=1e-6, check_status=False,
                   iters_slack=10 ** 6, dx=dx, label=f"{fmt} + 3 fp32 sweeps")


# ---------------------------------------------------------------- API behaviour

def test_host_buffers_equal_device_buffers(ctx):
    """The C ABI with host (pinned) input and outputs gives the bit-identical
    result of the device path."""
    At = synth.planted_spike(1000, 4000, 2, [30.0, 15.0], support_frac=0.05, seed=4, dtype=np.float32)
    gam = _gammas(At.astype(np.float64).T, "SL1", 0.05)
    dev = ctx.solve(torch.from_numpy(At).cuda(), "SL1", list(gam))
    hA = torch.from_numpy(At).pin_memory()
    out = binding.alloc_result(1, 1000, 4000, "cpu", torch.float32, pin=True)
    host = ctx.solve(hA, "SL1", list(gam), out=out)
    assert torch.equal(host.Z, dev.Z.cpu()) and torch.equal(host.X, dev.X.cpu())
    assert torch.equal(host.objective, dev.objective.cpu())


def test_relative_gamma_is_scaled_on_device(ctx):
    At = synth.planted_spike(800, 3000, 2, [30.0, 15.0], support_frac=0.05, seed=8, dtype=np.float32)
    A = At.astype(np.float64).T
    for form in ("SL1", "BL0"):
        m = 1 if form.startswith("S") else 2
        rho = [0.07] * m
        res = ctx.solve(torch.from_numpy(At).cuda(), form, rho, mu=None if m == 1 else [1.0, 1.0],
                        gamma_relative=True)
        ga = res.gamma_abs.cpu().numpy()
        np.testing.assert_allclose(ga, oracle.gamma_from_rho(A, form, rho), rtol=1e-12)
        mu = None if m == 1 else [1.0, 1.0]
        ref = oracle.gpower(A, form, ga, mu=mu)
        _converged(form, gpu_arrays(res), A, ga, mu, ref, 1e-6, f"relative gamma {form}")


def test_relative_gamma_on_the_tensor_cores(ctx):
    """The fused float tensor-core sweep sums the column norms in the start's
    first power step (no pass of its own); the largest is then re-normed
    exactly, so a relative gamma matches the oracle's scale to rounding, and
    the solve matches the oracle at the stated limits."""
    m = 16
    At = synth.planted_spike(900, 3100, m, [60.0 / np.sqrt(j + 1) for j in range(m)], support_frac=0.01, seed=63,
                             dtype=np.float32)
    A = At.astype(np.float64).T
    for form in ("BL1", "BL0"):
        res = ctx.solve(torch.from_numpy(At).cuda(), form, [0.05] * m, mu=[1.0] * m, gamma_relative=True, tol=0.0,
                        maxit=4)
        ga = res.gamma_abs.cpu().numpy()
        np.testing.assert_allclose(ga, oracle.gamma_from_rho(A, form, [0.05] * m), rtol=1e-12)
        ref = oracle.gpower(A, form, ga, mu=[1.0] * m, tol=0.0, maxit=4)
        assert_matches(form, gpu_arrays(res), ref, oracle.column_norms(A), label=f"tc relative gamma {form}")


def test_warm_start_x0(ctx):
    """A caller's start near the solution (the planted directions u_j plus
    noise of the same norm), projected on the Stiefel manifold, then 12
    sweeps.  (From a purely random start this matrix first settles near a
    point where the objective still creeps up by 7e-11 per sweep, a direction
    so flat that float rounding of each sweep adds up along it instead of
    dying out; the split of the objective between the two components is then
    not determined to 1e-6.)"""
    At, meta = synth.planted_spike(700, 2500, 2, [25.0, 12.0], support_frac=0.05, seed=9, dtype=np.float32,
                                   with_meta=True)
    A = At.astype(np.float64).T
    gam = _gammas(A, "BL0", [0.05, 0.05])
    U = meta.U.T
    noise = np.random.default_rng(5).standard_normal((700, 2))
    x0 = (U + np.linalg.norm(U, axis=0) / np.sqrt(700) * noise).astype(np.float32)
    ref = oracle.gpower(A, "BL0", gam, mu=[1.0, 1.0], tol=0.0, maxit=12, x0=x0.astype(np.float64))
    g, _ = _run(ctx, At, "BL0", gam, mu=[1.0, 1.0], tol=0.0, maxit=12,
                x0=torch.from_numpy(np.ascontiguousarray(x0.T)).cuda())
    assert_matches("BL0", g, ref, oracle.column_norms(A), label="warm start x0 BL0")


@pytest.mark.parametrize("cond", [1e6, 1e8, 1e10])
def test_polar_factor_of_ill_conditioned_start(ctx, cond):
    """The block polar step X = Y (Y^T Y)^{-1/2} (Section 2, Stiefel
    projection) on a caller's start Y whose Gram matrix has condition `cond`
    (up to 1e10; the degenerate limit is 1e12).  The GPU forms Y^T Y in double,
    solves the m x m eigenproblem by Jacobi in double-float (about 48
    significant bits), so its smallest eigenvalue carries an error of about
    2^-48 cond relative to itself, and applies W = (Y^T Y)^{-1/2} with
    compensated float arithmetic (one rounding of Y W to float); the bound
    below is that, against the FP64 polar factor (SVD).  An FP64 Gram + eigh
    polar factor is printed beside it for scale."""
    p, m = 1200, 4
    rng = np.random.default_rng(27)
    Q, _ = np.linalg.qr(rng.standard_normal((p, m)))
    R, _ = np.linalg.qr(rng.standard_normal((m, m)))
    s = np.geomspace(1.0, cond ** -0.5, m)
    Y = ((Q * s) @ R.T).astype(np.float32)  # p x m
    Y64 = Y.astype(np.float64)
    X_svd, degenerate = oracle.polar(Y64)
    assert not degenerate
    w, V = np.linalg.eigh(Y64.T @ Y64)
    X_eigh = Y64 @ (V / np.sqrt(w)) @ V.T
    At = synth.planted_spike(p, 3000, 2, [30.0, 15.0], support_frac=0.05, seed=28, dtype=np.float32)
    gam = list(_gammas(At.astype(np.float64).T, "BL1", [0.05] * m))
    res = ctx.solve(torch.from_numpy(At).cuda(), "BL1", gam, mu=[1.0] * m, tol=0.0, maxit=1,
                    x0=torch.from_numpy(np.ascontiguousarray(Y.T)).cuda())
    X = res.X.double().cpu().numpy().T
    err = np.abs(X - X_svd).max()
    orth = np.abs(X.T @ X - np.eye(m)).max()
    bound = 4.0 * (2.0 ** -24 * np.sqrt(m) + 2.0 ** -46 * cond)
    print(f"[polar] cond {cond:.0e}: gpu {err:.2e}, orthogonality {orth:.2e}, fp64 gram+eigh "
          f"{np.abs(X_eigh - X_svd).max():.2e}, bound {bound:.1e}")
    assert err <= bound and orth <= bound


def test_deterministic(ctx):
    At = synth.planted_spike(1500, 5000, 3, [30.0, 15.0, 10.0], support_frac=0.03, seed=10, dtype=np.float32)
    dA = torch.from_numpy(At).cuda()
    gam = list(_gammas(At.astype(np.float64).T, "BL1", [0.04] * 3))
    a = ctx.solve(dA, "BL1", gam, mu=[1.0, 1.0, 1.0])
    b = ctx.solve(dA, "BL1", gam, mu=[1.0, 1.0, 1.0])
    assert torch.equal(a.Z, b.Z) and torch.equal(a.X, b.X) and torch.equal(a.objective, b.objective)


@pytest.mark.parametrize("form", ["SL1", "BL0"])
def test_eager_launches_equal_graph(ctx, form):
    """The host-driven launch mode (for profilers) runs the same kernels: bit-identical results."""
    At = synth.planted_spike(1500, 5000, 3, [30.0, 15.0, 10.0], support_frac=0.03, seed=11, dtype=np.float32)
    dA = torch.from_numpy(At).cuda()
    m = 1 if form == "SL1" else 3
    gam = list(_gammas(At.astype(np.float64).T, form, [0.04] * m))
    mu = None if m == 1 else [1.0, 0.8, 0.6]
    a = ctx.solve(dA, form, gam, mu=mu)
    b = ctx.solve(dA, form, gam, mu=mu, eager=True)
    for k in ("X", "Z", "support", "objective", "iters", "status"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k


# ---------------------------------------------------------------- edge cases

def test_tiny_shapes(ctx):
    rng = np.random.default_rng(3)
    for p, n, form in ((1, 9, "SL0"), (9, 1, "SL1"), (3, 5, "BL1"), (5, 40, "BL0")):
        At = rng.standard_normal((n, p)).astype(np.float32)
        A = At.astype(np.float64).T
        m = 1 if form.startswith("S") else min(2, p, n)
        mu = None if m == 1 else [1.0] * m
        gam = _gammas(A, form, [0.1] * m)
        ref = oracle.gpower(A, form, gam, mu=mu, tol=0.0, maxit=6)
        g, _ = _run(ctx, At, form, gam, mu=mu, tol=0.0, maxit=6)
        assert_matches(form, g, ref, oracle.column_norms(A), label=f"tiny {p}x{n} {form}")


def test_zero_matrix_and_large_gamma(ctx):
    At = np.zeros((50, 30), dtype=np.float32)
    g, res = _run(ctx, At, "SL1", [0.1])
    assert g["status"][0] == binding.ZERO and g["iters"][0] == 0 and np.all(g["Z"] == 0)
    At = np.random.default_rng(1).standard_normal((200, 64)).astype(np.float32)
    A = At.astype(np.float64).T
    for form in oracle.FORMS:
        m = 1 if form.startswith("S") else 2
        # gamma just above the bound max |a_i^T x| <= max ||a_i||: exactly at it,
        # the start column's own t sits on the threshold, inside the band of
        # 1e-6 gamma where float and double may decide the tie differently
        c = oracle.column_norms(A).max() * (1.0 + 1e-6)
        gam = [c] * m if form.endswith("1") else [c * c] * m
        g, _ = _run(ctx, At, form, gam, mu=None if m == 1 else [1.0, 1.0])
        assert np.all(g["status"] == binding.ZERO) and np.all(g["iters"] == 1)
        assert np.all(g["Z"] == 0) and np.all(g["objective"] == 0)


def test_empty_matrix(ctx):
    At = torch.zeros((0, 16), device="cuda")
    res = ctx.solve(At, "SL1", [0.1], p=16)
    assert res.status.item() == binding.ZERO and res.iters.item() == 0


@pytest.mark.parametrize("form", ["SL1", "BL1", "BL0"])
def test_nonfinite_input_is_reported(ctx, form):
    """A NaN entry (or one whose square overflows) is reported as ENONFINITE:
    by the column-norm pass, or for block starts on the CUDA cores by the
    first power step, which forms the column norms."""
    At = np.random.default_rng(2).standard_normal((100, 40)).astype(np.float32)
    m = 1 if form.startswith("S") else 2
    mu = None if m == 1 else [1.0] * m
    for bad in (np.nan, 3e19):
        At[17, 3] = bad
        with pytest.raises(binding.GpspcaError) as e:
            ctx.solve(torch.from_numpy(At).cuda(), form, [0.1] * m, mu=mu)
        assert e.value.code == binding.ENONFINITE
    # the context stays usable
    At[17, 3] = 0.0
    ctx.solve(torch.from_numpy(At).cuda(), form, [0.1] * m, mu=mu)


@pytest.mark.parametrize("eager", [False, True])
def test_timeout_status_maps_to_etimedout(ctx, eager):
    """A solve whose device state carries the timeout bit (set on the host
    after the solve ran: the INJECT_TIMEOUT test hook; no device wait is made
    to expire) returns GPSPCA_ETIMEDOUT, and the context's next solve is the
    one it would have been without it."""
    At = synth.planted_spike(600, 2000, 2, [30.0, 15.0], support_frac=0.05, seed=26, dtype=np.float32)
    dA = torch.from_numpy(At).cuda()
    with pytest.raises(binding.GpspcaError) as e:
        ctx.solve(dA, "BL1", [0.05, 0.05], mu=[1.0, 1.0], gamma_relative=True, eager=eager,
                  extra_flags=binding.INJECT_TIMEOUT)
    assert e.value.code == binding.ETIMEDOUT and "gave up" in str(e.value)
    after = ctx.solve(dA, "BL1", [0.05, 0.05], mu=[1.0, 1.0], gamma_relative=True, eager=eager)
    with binding.Context(0) as fresh:
        ref = fresh.solve(dA, "BL1", [0.05, 0.05], mu=[1.0, 1.0], gamma_relative=True, eager=eager)
    assert after.rc == binding.OK
    assert torch.equal(after.Z, ref.Z) and torch.equal(after.X, ref.X) and torch.equal(after.iters, ref.iters)


def test_nonfinite_input_on_the_tensor_cores(ctx):
    """Float storage with 16 components runs the fused tensor-core sweep,
    whose first power step of the start sums the column norms: a NaN (or an
    entry whose square overflows) is reported as ENONFINITE there, and the
    context stays usable."""
    At = np.random.default_rng(3).standard_normal((700, 200)).astype(np.float32)
    for bad in (np.nan, 3e19):
        At[301, 77] = bad
        with pytest.raises(binding.GpspcaError) as e:
            ctx.solve(torch.from_numpy(At).cuda(), "BL0", [0.1] * 16, mu=[1.0] * 16, gamma_relative=True)
        assert e.value.code == binding.ENONFINITE
    At[301, 77] = 0.0
    ctx.solve(torch.from_numpy(At).cuda(), "BL0", [0.1] * 16, mu=[1.0] * 16, gamma_relative=True)


def test_degenerate_polar_status(ctx):
    At = np.random.default_rng(20).standard_normal((30, 12)).astype(np.float32)
    A = At.astype(np.float64).T
    c = oracle.column_norms(A).max()
    gam = [0.1 * c, 2.0 * c]
    ref = oracle.gpower(A, "BL1", gam, mu=[1.0, 1.0])
    res = ctx.solve(torch.from_numpy(At).cuda(), "BL1", gam, mu=[1.0, 1.0])
    assert res.rc == binding.EDEGENERATE
    g = gpu_arrays(res)
    assert_matches("BL1", g, ref, oracle.column_norms(A), label="degenerate polar")


def test_invalid_arguments(ctx):
    dA = torch.randn(40, 8, device="cuda")
    for kw in (dict(form="BL1", gamma=[0.1] * 9, mu=[1.0] * 9),   # m > p
               dict(form="SL1", gamma=[-1.0]),
               dict(form="BL0", gamma=[0.1, 0.1], mu=[1.0, 0.0]),
               dict(form="SL1", gamma=[0.1] * 65)):
        with pytest.raises(binding.GpspcaError) as e:
            ctx.solve(dA, **kw)
        assert e.value.code == binding.EINVAL


def test_time_sweep(ctx):
    At = synth.planted_spike(2000, 8000, 2, [30.0, 15.0], support_frac=0.05, seed=4, dtype=np.float32)
    ms = ctx.time_sweep(torch.from_numpy(At).cuda(), "SL1", [0.05], gamma_relative=True, reps=5)
    assert 0 < ms < 100


# ---------------------------------------------------------------- serving

def test_batch_equals_solo_solves(ctx):
    """gpspca_solve_batch: independent solves of different shapes, forms and
    storage (more than its 8 concurrent slots) give the bit-identical results
    of solo solves, and the batch is ordered on the context's stream."""
    rng = np.random.default_rng(5)
    items = []
    for i in range(11):
        p = int(rng.integers(200, 1500))
        n = int(rng.integers(800, 5000))
        form = oracle.FORMS[i % 4]
        m = 1 if form.startswith("S") else int(rng.integers(2, 7))
        At = synth.planted_spike(p, n, m, [30.0 / (j + 1) for j in range(m)], support_frac=0.05, seed=200 + i,
                                 dtype=np.float32)
        dA = torch.from_numpy(At).cuda()
        if i % 3 == 2:
            dA = dA.to(torch.bfloat16)
        items.append(dict(At=dA, form=form, gamma=[float(rng.uniform(0.02, 0.2))] * m,
                          mu=None if m == 1 else [1.0] * m, gamma_relative=True))
    solo = [ctx.solve(**{k: v for k, v in it.items()}) for it in items]
    got = ctx.solve_batch(items)
    for ref, out in zip(solo, got):
        assert torch.equal(out.Z, ref.Z) and torch.equal(out.X, ref.X)
        assert torch.equal(out.objective, ref.objective) and torch.equal(out.iters, ref.iters)
    with pytest.raises(binding.GpspcaError):
        ctx.solve_batch([dict(At=items[0]["At"], form="SL1", gamma=[-1.0])])


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_groups_same_shape_solves(ctx, dtype):
    """Same-shape single-unit requests of a batch (here 40 of 300 x 2000, SL1
    and SL0, each with its own data, gamma, tolerance and sweep limit) run
    as groups, one launch per step for all members.  Every member against
    the oracle at the stated limits (members stop on their own tests); the
    same requests in two groups of another composition give the same bits;
    a request of another shape in the batch runs on its own (the bits of its
    solo solve)."""
    rng = np.random.default_rng(66)
    p, n = 300, 2000
    tdt = torch.float32 if dtype == "f32" else torch.float64
    items, mats = [], []
    for i in range(40):
        At = synth.planted_spike(p, n, 2, [30.0, 15.0], support_frac=0.05, seed=300 + i, dtype=np.float32)
        mats.append(At)
        items.append(dict(At=torch.from_numpy(At).to(tdt).cuda(), form="SL1" if i % 2 else "SL0",
                          gamma=[float(rng.uniform(0.03, 0.15))], gamma_relative=True,
                          tol=1e-6 if i % 5 else 0.0, maxit=1000 if i % 5 else 3 + i % 4))
    other = synth.planted_spike(400, 1500, 2, [30.0, 15.0], support_frac=0.05, seed=399, dtype=np.float32)
    items.append(dict(At=torch.from_numpy(other).to(tdt).cuda(), form="SL1", gamma=[0.05], gamma_relative=True))
    got = ctx.solve_batch(items)
    solo_other = ctx.solve(**items[40])
    assert torch.equal(got[40].Z, solo_other.Z) and torch.equal(got[40].X, solo_other.X)
    # another composition: the odd members first, in a batch of their own, then the even ones
    again = {}
    for half in (list(range(1, 40, 2)), list(range(0, 40, 2))):
        for i, r in zip(half, ctx.solve_batch([items[i] for i in half])):
            again[i] = r
    for i in range(40):
        assert torch.equal(got[i].Z, again[i].Z) and torch.equal(got[i].X, again[i].X), i
        assert torch.equal(got[i].objective, again[i].objective) and torch.equal(got[i].iters, again[i].iters), i
    its = np.array([int(r.iters[0]) for r in got[:40]])
    assert len(set(its.tolist())) > 1  # the members stopped on their own tests
    for i in range(40):
        A = mats[i].astype(np.float64).T
        form = items[i]["form"]
        gam = _gammas(A, form, items[i]["gamma"])
        ref = oracle.gpower(A, form, gam, tol=items[i]["tol"], maxit=items[i]["maxit"])
        g = gpu_arrays(got[i])
        if items[i]["tol"] > 0:
            _converged(form, g, A, gam, None, ref, items[i]["tol"], f"group member {i} {dtype}")
        else:
            assert_matches(form, g, ref, oracle.column_norms(A), label=f"group member {i} {dtype}")


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_batch_groups_low_precision_storage(ctx, storage):
    """Groups of bf16 and fp8 (per-column scales) requests: 8 members of
    256 x 3000, SL1, against the oracle on the stored values; the same
    requests split over two batches give the same bits."""
    p, n = 256, 3000
    items, deqs = [], []
    for i in range(8):
        At = synth.planted_spike(p, n, 2, [25.0, 12.0], support_frac=0.05, seed=500 + i, dtype=np.float32)
        if storage == "bf16":
            tb, deq = _bf16(At)
            items.append(dict(At=tb.cuda(), form="SL1", gamma=[0.08], gamma_relative=True, tol=0.0, maxit=5))
        else:
            q, sc, deq = _fp8(At)
            items.append(dict(At=q.cuda(), col_scale=sc.cuda(), form="SL1", gamma=[0.08], gamma_relative=True,
                              tol=0.0, maxit=5))
        deqs.append(deq)
    got = ctx.solve_batch(items)
    again = ctx.solve_batch(items[4:]) + ctx.solve_batch(items[:4])
    again = again[4:] + again[:4]
    for i in range(8):
        assert torch.equal(got[i].Z, again[i].Z) and torch.equal(got[i].X, again[i].X), i
        A = deqs[i].astype(np.float64).T
        gam = _gammas(A, "SL1", [0.08])
        ref = oracle.gpower(A, "SL1", gam, tol=0.0, maxit=5)
        assert_matches("SL1", gpu_arrays(got[i]), ref, oracle.column_norms(A), label=f"group {storage} member {i}")


def test_batch_group_with_a_failing_member(ctx):
    """A member with a NaN in its matrix reports GPSPCA_ENONFINITE; the other
    members of its group (host outputs for some of them) give the bits they
    give in a group without it."""
    p, n = 256, 1024
    items = []
    for i in range(6):
        At = synth.planted_spike(p, n, 1, [25.0], support_frac=0.05, seed=400 + i, dtype=np.float32)
        if i == 3:
            At[17, 5] = np.nan
        out = binding.alloc_result(1, p, n, "cpu" if i % 2 else "cuda", torch.float32, pin=bool(i % 2))
        items.append(dict(At=torch.from_numpy(At).cuda(), form="SL1", gamma=[0.08], gamma_relative=True, out=out))
    with pytest.raises(binding.GpspcaError) as e:
        ctx.solve_batch(items)
    assert e.value.code == binding.ENONFINITE
    good = (0, 1, 2, 4, 5)
    refs = ctx.solve_batch([{k: v for k, v in items[i].items() if k != "out"} for i in good])
    for i, ref in zip(good, refs):
        got = items[i]["out"]
        assert torch.equal(got.Z.cpu(), ref.Z.cpu()) and torch.equal(got.X.cpu(), ref.X.cpu()), i
        assert torch.equal(got.objective.cpu(), ref.objective.cpu()), i


def test_batch_shares_host_matrix(ctx):
    """Requests of a batch that share one pinned host matrix (the library copies
    it once) give the device batch's bits, with host or device outputs, for
    float and fp8 (host scales) storage."""
    At = synth.planted_spike(900, 3100, 3, [30.0, 20.0, 12.0], support_frac=0.05, seed=31, dtype=np.float32)
    s = np.abs(At).max(axis=1).astype(np.float32) / 448.0
    q = torch.from_numpy(At / s[:, None]).to(torch.float8_e4m3fn)
    for hA, hs in ((torch.from_numpy(At).pin_memory(), None), (q.pin_memory(), torch.from_numpy(s).pin_memory())):
        cases = [("SL1", None), ("BL0", [1.0] * 3), ("SL0", None), ("BL1", [1.0, 0.9, 0.8])]
        dev_items, host_items = [], []
        for k, (form, mu) in enumerate(cases):
            m = 1 if mu is None else 3
            common = dict(form=form, gamma=[0.05] * m, mu=mu, gamma_relative=True)
            dev_items.append(dict(At=hA.cuda(), col_scale=None if hs is None else hs.cuda(), **common))
            out = binding.alloc_result(m, 900, 3100, "cpu", torch.float32, pin=True) if k % 2 else None
            host_items.append(dict(At=hA, col_scale=hs, out=out, **common))
        dev = ctx.solve_batch(dev_items)
        host = ctx.solve_batch(host_items)
        for a, b in zip(dev, host):
            assert torch.equal(a.Z.cpu(), b.Z.cpu()) and torch.equal(a.X.cpu(), b.X.cpu())
            assert torch.equal(a.objective.cpu(), b.objective.cpu()) and torch.equal(a.iters.cpu(), b.iters.cpu())


def test_batch_shares_column_norms_of_a_device_matrix(ctx):
    """Single-unit requests of a batch on one device matrix take its column
    norms from one pass the batch makes for them: their results are
    bit-identical to solo solves (a block request on the same matrix keeps
    its own norms), and a non-finite entry is still reported by each of them
    (each copies the shared norms with the check its own pass would make)."""
    At = synth.planted_spike(2000, 6000, 3, [30.0, 20.0, 12.0], support_frac=0.05, seed=41, dtype=np.float32)
    dA = torch.from_numpy(At).cuda()
    items = [dict(At=dA, form="SL1", gamma=[0.05], gamma_relative=True),
             dict(At=dA, form="SL0", gamma=[0.05], gamma_relative=True),
             dict(At=dA, form="BL1", gamma=[0.05] * 3, mu=[1.0] * 3, gamma_relative=True),
             dict(At=dA, form="SL1", gamma=[0.1], gamma_relative=True)]
    solo = [ctx.solve(**it) for it in items]
    got = ctx.solve_batch(items)
    for ref, out in zip(solo, got):
        assert torch.equal(out.Z, ref.Z) and torch.equal(out.X, ref.X)
        assert torch.equal(out.objective, ref.objective) and torch.equal(out.iters, ref.iters)
    bad = At.copy()
    bad[17, 3] = np.nan
    dB = torch.from_numpy(bad).cuda()
    for order in (("SL1", "SL0"), ("SL0", "SL1")):  # the first request's code is the one raised
        with pytest.raises(binding.GpspcaError) as e:
            ctx.solve_batch([dict(At=dB, form=f, gamma=[0.05], gamma_relative=True) for f in order])
        assert e.value.code == binding.ENONFINITE
    again = ctx.solve_batch(items[:2])  # the context stays usable
    assert torch.equal(again[0].Z, solo[0].Z) and torch.equal(again[1].Z, solo[1].Z)


def test_upload_then_solve_equals_device_solve(ctx):
    """gpspca_upload copies a pinned host matrix into a device tensor (same
    stride; a wider stride, re-strided by the copy; fp8 with its scales);
    a solve on the destination gives the bits of a solve on a device copy
    made by PyTorch."""
    p, n = 900, 3100
    At = synth.planted_spike(p, n, 3, [30.0, 20.0, 12.0], support_frac=0.05, seed=32, dtype=np.float32)
    ref = ctx.solve(torch.from_numpy(At).cuda(), "BL1", [0.05] * 3, mu=[1.0] * 3, gamma_relative=True)
    for ld in (p, p + 36):
        dst = torch.zeros((n, ld), device="cuda")
        ctx.upload(torch.from_numpy(At).pin_memory(), dst, p=p)
        got = ctx.solve(dst, "BL1", [0.05] * 3, mu=[1.0] * 3, gamma_relative=True, p=p)
        assert torch.equal(got.Z, ref.Z) and torch.equal(got.X, ref.X), ld
        assert torch.equal(got.objective, ref.objective)
    s = np.abs(At).max(axis=1).astype(np.float32) / 448.0
    q = torch.from_numpy(At / s[:, None]).to(torch.float8_e4m3fn)
    ref8 = ctx.solve(q.cuda(), "SL0", [0.05], gamma_relative=True, col_scale=torch.from_numpy(s).cuda())
    dq = torch.empty((n, p), dtype=torch.float8_e4m3fn, device="cuda")
    ds = torch.zeros(n, device="cuda")
    ctx.upload(q.pin_memory(), dq, host_scale=torch.from_numpy(s).pin_memory(), dev_scale=ds)
    got8 = ctx.solve(dq, "SL0", [0.05], gamma_relative=True, col_scale=ds)
    assert torch.equal(got8.Z, ref8.Z) and torch.equal(got8.objective, ref8.objective)


def test_upload_double_buffered_batches(ctx):
    """The pattern of a pipelined loop: the copy of step k + 1's matrix is
    issued before the batch of step k, into the other of two device buffers,
    and the matrices alternate between two different ones, so a solve that
    did not wait for its copy would read the previous matrix (or part of
    it).  Every step's results equal those of its matrix solved from a
    device copy; outputs go to pinned host buffers."""
    p, n = 2000, 25000  # 200 MB per copy
    mats = [synth.planted_spike(p, n, 2, [40.0, 20.0], support_frac=0.02, seed=33 + k, dtype=np.float32)
            for k in range(2)]
    hosts = [torch.from_numpy(a).pin_memory() for a in mats]
    cases = [("SL1", None), ("BL1", [1.0, 1.0])]
    refs = []
    for a in mats:
        dA = torch.from_numpy(a).cuda()
        refs.append([ctx.solve(dA, f, [0.05] * (1 if mu is None else 2), mu=mu, gamma_relative=True)
                     for f, mu in cases])
        del dA
    bufs = [torch.zeros((n, p), device="cuda") for _ in range(2)]
    steps = 6
    ctx.upload(hosts[0], bufs[0])
    for k in range(steps):
        if k + 1 < steps:
            ctx.upload(hosts[(k + 1) % 2], bufs[(k + 1) % 2])
        items = []
        for f, mu in cases:
            m = 1 if mu is None else 2
            out = binding.alloc_result(m, p, n, "cpu", torch.float32, pin=True)
            items.append(dict(At=bufs[k % 2], form=f, gamma=[0.05] * m, mu=mu, gamma_relative=True, out=out))
        res = ctx.solve_batch(items)
        for a, b in zip(res, refs[k % 2]):
            assert torch.equal(a.Z, b.Z.cpu()) and torch.equal(a.X, b.X.cpu()), k
            assert torch.equal(a.objective, b.objective.cpu()), k


def test_upload_rejects_mismatched_descriptors(ctx):
    h = torch.zeros((10, 8)).pin_memory()
    with pytest.raises(binding.GpspcaError) as e:
        ctx.upload(h, torch.zeros((10, 7), device="cuda"))
    assert e.value.code == binding.EINVAL
    with pytest.raises(binding.GpspcaError) as e:
        ctx.upload(h, torch.zeros((10, 8), device="cuda", dtype=torch.float64))
    assert e.value.code == binding.EINVAL
    with pytest.raises(ValueError):
        ctx.upload(h, torch.zeros((10, 8)))


def test_submitted_requests_equal_solo_solves(ctx):
    """Requests of different shapes and formulations submitted together (and so
    overlapping on the device) give the bit-identical results of solo solves."""
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(10):
        p = int(rng.integers(200, 1500))
        n = int(rng.integers(800, 5000))
        form = oracle.FORMS[i % 4]
        m = 1 if form.startswith("S") else int(rng.integers(2, 6))
        At = synth.planted_spike(p, n, m, [30.0 / (j + 1) for j in range(m)], support_frac=0.05, seed=100 + i,
                                 dtype=np.float32)
        reqs.append((torch.from_numpy(At).cuda(), form, [float(rng.uniform(0.02, 0.2))] * m,
                     None if m == 1 else [1.0] * m))
    solo = [ctx.solve(dA, f, g, mu=mu, gamma_relative=True) for dA, f, g, mu in reqs]
    tickets = [ctx.submit(dA, f, g, mu=mu, gamma_relative=True) for dA, f, g, mu in reqs]
    for (t, out), ref in zip(tickets, solo):
        rc = ctx.poll(t, wait_us=-1)
        assert rc in (binding.OK, binding.EDEGENERATE)
        assert torch.equal(out.Z, ref.Z) and torch.equal(out.X, ref.X)
        assert torch.equal(out.objective, ref.objective) and torch.equal(out.iters, ref.iters)
    assert ctx.poll(tickets[0][0], 0) == binding.ENOTFOUND


def test_submit_admission_by_footprint():
    """Requests are admitted by their HBM footprint (matrix, outputs and the
    solve's workspace) under the context budget: with a budget that holds
    one 24 MB request at a time, four submitted requests wait for each other
    and each result equals its solo solve; a request whose own matrix and
    outputs exceed the budget is refused with ENOMEM."""
    reqs = []
    for i in range(4):
        At = synth.planted_spike(1500, 4000, 2, [30.0, 15.0], support_frac=0.05, seed=300 + i, dtype=np.float32)
        reqs.append((torch.from_numpy(At).cuda(), oracle.FORMS[i % 4]))
    solo = []
    with binding.Context(0) as big:
        for dA, form in reqs:
            m = 1 if form.startswith("S") else 2
            solo.append(big.solve(dA, form, [0.05] * m, mu=None if m == 1 else [1.0, 1.0], gamma_relative=True))
    with binding.Context(0, budget_bytes=40 << 20) as small:
        tickets = []
        for dA, form in reqs:
            m = 1 if form.startswith("S") else 2
            tickets.append(small.submit(dA, form, [0.05] * m, mu=None if m == 1 else [1.0, 1.0], gamma_relative=True))
        for (t, out), ref in zip(tickets, solo):
            assert small.poll(t, wait_us=-1) == binding.OK
            assert torch.equal(out.Z, ref.Z) and torch.equal(out.X, ref.X)
            assert torch.equal(out.objective, ref.objective)
        huge = torch.zeros((6000, 2000), device="cuda")  # 48 MB
        with pytest.raises(binding.GpspcaError) as e:
            small.submit(huge, "SL1", [0.05], gamma_relative=True)
        assert e.value.code == binding.ENOMEM
