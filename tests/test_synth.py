"""The seeded input generators: Philox4x32-10 against the published
known-answer vectors (Salmon et al., SC'11, Random123 distribution), the
host twin of the device generator, and the serving request mix."""

import numpy as np
import pytest

from paper_1312_6182_gb300 import synth


@pytest.mark.parametrize("ctr,key,expect", [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
])
def test_philox_known_answers(ctr, key, expect):
    out = synth.philox4x32_10(*ctr, *key)
    assert tuple(int(w) for w in out) == expect


def test_philox_vectorised_equals_scalar():
    c0 = np.arange(50, dtype=np.uint32)
    vec = synth.philox4x32_10(c0, 7, 0, 1, 123, 456)
    for i in (0, 17, 49):
        sc = synth.philox4x32_10(int(c0[i]), 7, 0, 1, 123, 456)
        assert all(int(vec[w][i]) == int(sc[w]) for w in range(4))


def test_uniform23_open_interval_and_exact():
    w = np.array([0, 511, 512, 0xFFFFFFFF], dtype=np.uint32)
    u = synth._uniform23(w)
    assert u.dtype == np.float32
    assert np.all(u > 0) and np.all(u < 1)
    assert u[0] == u[1] == np.float32(0.5 * 2.0 ** -23)
    assert u[2] == np.float32(1.5 * 2.0 ** -23)
    assert float(u[3]) == (2 ** 23 - 0.5) * 2.0 ** -23


def test_counter_spikes_structure():
    p, n, k, frac = 400, 6000, 3, 0.05
    theta = [40.0, 20.0, 13.0]
    A1 = synth.counter_spikes(p, n, k, theta, frac, seed=77)
    A2 = synth.counter_spikes(p, n, k, theta, frac, seed=77)
    A0 = synth.counter_spikes(p, n, 0, [], frac, seed=77)  # noise only
    assert A1.shape == (n, p) and A1.dtype == np.float32
    assert np.array_equal(A1, A2)
    assert not np.array_equal(A1, synth.counter_spikes(p, n, k, theta, frac, seed=78))
    # noise ~ N(0, 1)
    assert abs(A0.mean()) < 0.01 and abs(A0.std() - 1.0) < 0.01
    # spike columns: disjoint supports of expected size frac * n, rank-one excess
    diff = A1.astype(np.float64) - A0
    cols = np.nonzero(np.abs(diff).sum(axis=1) > 0)[0]
    assert abs(len(cols) - k * frac * n) < 5 * np.sqrt(k * frac * n)
    s = round(frac * n)
    norms = np.linalg.norm(diff[cols], axis=1)
    assert np.all(norms > 0)
    # every spike column is +-theta_j / sqrt(s) u_j for one j: rank <= k
    sv = np.linalg.svd(diff[cols], compute_uv=False)
    assert sv[k] < 1e-4 * sv[0]
    assert abs(sv[0] - theta[0] * np.sqrt(p) * np.sqrt(len(cols) / k) / np.sqrt(s)) < 0.2 * sv[0]


def test_counter_spikes_bf16_rounding():
    A = synth.counter_spikes(64, 100, 1, [10.0], 0.1, seed=5)
    B = synth.counter_spikes(64, 100, 1, [10.0], 0.1, seed=5, dtype="bf16")
    assert np.all(B.view(np.uint32) & np.uint32(0xFFFF) == 0)
    assert np.all(np.abs(B - A) <= np.abs(A) * 2.0 ** -8 + 1e-30)


def test_serving_mix():
    rq = synth.serving_requests()
    assert len(rq) == 2000
    arr = np.array([r.arrival_s for r in rq])
    assert arr[0] == 0 and np.all(np.diff(arr) >= 0)
    assert abs(len(rq) / arr[-1] - 200) < 20  # Poisson at 200/s
    assert all(256 <= r.p <= 8192 and 1024 <= r.n <= 65536 and 1 <= r.m <= 16 for r in rq)
    assert {r.form for r in rq} == {"SL1", "SL0", "BL1", "BL0"} and {r.dtype for r in rq} == {"f32", "bf16"}
    assert all(0.02 <= r.rho <= 0.2 for r in rq)
    r = next(q for q in rq if q.form.startswith("S") and q.m > 2)
    g = r.gammas()
    assert len(g) == r.m and abs(g[0] - r.rho / 2) < 1e-12 and abs(g[-1] - r.rho) < 1e-12


def test_block_sample_equals_the_columns_of_the_whole_matrix():
    """A sample of noise blocks is bit-identical to those columns of the whole
    planted-spike matrix (the CPU baselines time the oracle on such a
    sample of the 20000 x 100000 workload)."""
    kw = dict(support_frac=0.05, seed=4, noise_streams=16)
    full = synth.planted_spike(300, 1600, 3, [40.0, 20.0, 10.0], **kw)
    part = synth.planted_spike(300, 1600, 3, [40.0, 20.0, 10.0], blocks=(2, 5), **kw)
    assert np.array_equal(full[200:500], part)
    assert not np.array_equal(full[:300], part)
