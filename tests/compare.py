"""Comparison of a GPU result with the FP64 oracle, at the stated tolerances.

Tolerances (per column j):
  loadings   ||z_gpu - z_orc|| / ||z_orc||     <= tol_z   (1e-5 for float32 compute)
  objective  |f_gpu - f_orc| / f_orc            <= tol_f   (1e-6)
  support    identical, except entries whose threshold margin in the oracle's
             T is within 1e-6 * gamma (L1: |mu|t| - gamma|, L0: |(mu t)^2 - gamma|)
  iterate    ||X_gpu - X_orc||_F / sqrt(m)      <= tol_x
"""

import numpy as np


def unpack_support(words, n):
    w = np.asarray(words).astype(np.uint32)
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(bool)
    return bits.reshape(w.shape[0], -1)[:, :n].T  # n x m


def near_threshold(form, T, gamma, mu, band=1e-6):
    if form.endswith("1"):
        margin = np.abs(mu * np.abs(T) - gamma)
    else:
        margin = np.abs((mu * T) ** 2 - gamma)
    return margin <= band * np.maximum(gamma, 1e-300)


def gpu_arrays(res):
    """GPU result tensors -> numpy in the paper's orientation (X p x m, Z n x m)."""
    return dict(
        X=res.X.double().cpu().numpy().T,
        Z=res.Z.double().cpu().numpy().T,
        support=res.support.cpu().numpy(),
        objective=res.objective.cpu().numpy(),
        iters=res.iters.cpu().numpy(),
        status=res.status.cpu().numpy(),
        gamma_abs=res.gamma_abs.cpu().numpy(),
    )


def assert_matches(form, g, ref, tol_z=1e-5, tol_f=1e-6, tol_x=1e-5, iters_slack=1, check_support=True,
                   check_status=True):
    n, m = ref.Z.shape
    if check_status:
        np.testing.assert_array_equal(g["status"], ref.status)
    assert np.all(np.abs(g["iters"] - ref.iters) <= iters_slack), (g["iters"], ref.iters)
    for j in range(m):
        zr = ref.Z[:, j]
        nz = np.linalg.norm(zr)
        if nz == 0:
            assert np.all(g["Z"][:, j] == 0), f"column {j}: oracle zero, gpu not"
        else:
            err = np.linalg.norm(g["Z"][:, j] - zr) / nz
            assert err <= tol_z, f"column {j}: loadings rel err {err:.3e} > {tol_z:.1e}"
        fr = ref.objective[j]
        if fr != 0:
            ef = abs(g["objective"][j] - fr) / abs(fr)
            assert ef <= tol_f, f"column {j}: objective rel err {ef:.3e} > {tol_f:.1e}"
        else:
            assert g["objective"][j] == 0
    if ref.total != 0:
        et = abs(np.sum(g["objective"]) - ref.total) / abs(ref.total)
        assert et <= tol_f, f"total objective rel err {et:.3e}"
    ex = np.linalg.norm(g["X"] - ref.X) / np.sqrt(m)
    assert ex <= tol_x, f"iterate err {ex:.3e} > {tol_x:.1e}"
    if check_support:
        sup = unpack_support(g["support"], n)
        exempt = near_threshold(form, ref.T, ref.gamma, ref.mu)
        diff = (sup != (ref.Z != 0)) & ~exempt
        assert not diff.any(), f"support differs at {np.argwhere(diff)[:5].tolist()}"
        assert np.array_equal(sup, g["Z"] != 0)
