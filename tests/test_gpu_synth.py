"""The device generator (gpspca_synth_spikes) against its host twin: the
same counters and float32 arithmetic, so every entry agrees up to the
last-ulp differences of the float32 log / sin / cos implementations."""

import numpy as np
import pytest

from paper_1312_6182_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("p,n,k,ld", [(1001, 5003, 4, None), (256, 1024, 16, 260), (8, 3, 0, None)])
def test_device_generator_matches_host_twin(dtype, p, n, k, ld):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    theta = [40.0 / (j + 1) for j in range(k)]
    frac, seed = 0.05, 1000 + 17
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    buf = torch.full((n, ld or p), 7.0, device="cuda", dtype=tdt)  # padding must stay untouched
    binding.synth_spikes(buf, k, theta, frac, seed, p=p)
    torch.cuda.synchronize()
    got = buf[:, :p].float().cpu().numpy()
    ref = synth.counter_spikes(p, n, k, theta, frac, seed, dtype=dtype)
    if ld:
        assert torch.all(buf[:, p:] == 7.0)
    if dtype == "bf16":
        # one bfloat16 ulp (2^-7 relative) where rounding sits on a boundary, plus
        # the absolute float32 error of cos / sin near their zeros
        excess = np.abs(got - ref) - (2.0 ** -7 * np.abs(ref) + 1e-5)
        assert excess.max() <= 0, excess.max()
    else:
        err = np.abs(got - ref) / (1.0 + np.abs(ref))
        assert err.max() <= 1e-5, err.max()
    assert np.mean(got == ref) > 0.5  # same counters: most entries bit-identical (a wrong counter gives ~0)


def test_device_generator_rejects_bad_arguments():
    buf = torch.empty((10, 10), device="cuda")
    with pytest.raises(binding.GpspcaError):
        binding.synth_spikes(buf, 3, [1.0, 1.0, 1.0], 0.5, 1)  # 3 * 0.5 > 1: supports cannot be disjoint
