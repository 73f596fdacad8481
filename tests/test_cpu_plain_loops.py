"""The plain CPU loops the benchmark times as its "plain CPU" baseline (not a
reference: uncompensated sums in the data's own precision) compute the same
operations as the oracle, within FP32 / FP64 rounding."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_plain_loops_agree_with_the_oracle(storage):
    tol = 1e-5 if storage == "f32" else 1e-12
    n = 10_007
    y = synth.uniform(n, 1, storage).numpy()
    z = synth.uniform(n, 2, storage).numpy()
    assert np.array_equal(oracle.plain_copy(y), y)
    x = oracle.plain_axpy(y, z, 0.5)
    # alpha = 0.5: one rounding either way, so the plain loop is bit-exact
    assert np.array_equal(x.astype(np.float64), oracle.round_to(oracle.axpy(y, z, 0.5), storage))
    ref = oracle.dot(y, z)
    scale = np.linalg.norm(y.astype(np.float64)) * np.linalg.norm(z.astype(np.float64))
    assert abs(oracle.plain_dot(y, z) - ref) <= tol * scale
    m, k = 37, 411
    A = synth.normal((m, k), 3, storage).numpy().ravel()
    xg = synth.uniform(k, 4, storage).numpy()
    ref = oracle.gemv(A, xg, m, k, k, "row")
    got = oracle.plain_gemv(A, xg, m, k, k, "row").astype(np.float64)
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    At = np.ascontiguousarray(A.reshape(m, k).T).ravel()        # column-major storage of A
    got = oracle.plain_gemv(At, xg, m, k, m, "col").astype(np.float64)
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    rp, ci, v = synth.laplacian_3d(12, storage)
    xs = synth.uniform(12 ** 3, 5, storage).numpy()
    ref = oracle.csr_spmv(rp, ci, v, xs)
    got = oracle.plain_csr(rp.numpy(), ci.numpy(), v.numpy(), xs).astype(np.float64)
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
