"""mpir_gls_residual_noalloc: the GLS residual for callers that cannot
allocate device memory (frameworks that own all device allocations,
real-time loops).  It keeps its scratch in a fixed
device array inside the library instead of asking a handle for memory.

The test calls it twice in a row through the C ABI on different inputs and
compares each result with the handle-based mpir_gls_residual, within the
tolerance the residual tests use (the FP64 gemv bound; here both entry
points run the same kernels, so the results agree to the last bit in
practice).  This file is collected last so that a failure here cannot stop
the other GPU tests."""
import numpy as np
import pytest

from paper_2406_16499_gb300 import inputs as I
from gpu_util import U64, dev, host, zeros

pytestmark = pytest.mark.gpu


def _case(seed, n, m, p):
    G = I.gls_svd(seed, n, m, p, 1e3, 1e1)
    g = I.rng(seed + 1)
    return G["W"], G["V"], G["d"], g.standard_normal(m), g.standard_normal(p), g.standard_normal(n)


def test_noalloc_residual_matches_handle_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_16499_gb300 import mpir
    h = mpir.Handle()
    try:
        for seed, (n, m, p) in ((1, (300, 77, 300)), (2, (1000, 513, 1200))):
            W, V, d, x, y, z = _case(seed, n, m, p)
            dW, dV, dd, dx, dy, dz = dev(W), dev(V), dev(d), dev(x), dev(y), dev(z)
            r1, r2, r3 = zeros(p), zeros(n), zeros(m)
            h.gls_residual(dW, dV, dd, dx, dy, dz, r1, r2, r3)
            a1, a2, a3 = zeros(p), zeros(n), zeros(m)
            nrm = torch.zeros(6, dtype=torch.float64, device="cuda")
            rc = mpir.gls_residual_noalloc(dW, dV, dd, dx, dy, dz, a1, a2, a3, nrm)
            assert rc == 0
            torch.cuda.synchronize()
            ref = np.concatenate([host(r1), host(r2), host(r3)])
            got = np.concatenate([host(a1), host(a2), host(a3)])
            scale = (np.abs(np.concatenate([np.zeros(p), d, np.zeros(m)]))
                     + np.concatenate([np.abs(y) + np.abs(V).T @ np.abs(z),
                                       np.abs(W) @ np.abs(x) + np.abs(V) @ np.abs(y),
                                       np.abs(W).T @ np.abs(z)]))
            assert np.all(np.abs(got - ref) <= (n + m + p + 2) * U64 * scale)
            sq = host(nrm)
            assert abs(np.sqrt(sq[0]) / np.linalg.norm(host(r1)) - 1) < 1e-12
            assert abs(np.sqrt(sq[3]) / np.linalg.norm(x) - 1) < 1e-12
    finally:
        h.close()


def test_noalloc_residual_on_a_caller_stream():
    """The same check on a caller-created (non-default) stream, two calls in
    a row on that stream with different inputs, results read after a
    synchronization of that stream only."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_16499_gb300 import mpir
    h = mpir.Handle()
    st = torch.cuda.Stream()
    try:
        outs = []
        cases = [_case(seed, 400, 120, 500) for seed in (5, 6)]
        with torch.cuda.stream(st):
            for W, V, d, x, y, z in cases:
                dW, dV, dd, dx, dy, dz = dev(W), dev(V), dev(d), dev(x), dev(y), dev(z)
                a1, a2, a3 = zeros(500), zeros(400), zeros(120)
                assert mpir.gls_residual_noalloc(dW, dV, dd, dx, dy, dz, a1, a2, a3, None,
                                                 stream=st.cuda_stream) == 0
                outs.append((dW, dV, dd, dx, dy, dz, a1, a2, a3))
        st.synchronize()
        for (dW, dV, dd, dx, dy, dz, a1, a2, a3), (W, V, d, x, y, z) in zip(outs, cases):
            r1, r2, r3 = zeros(500), zeros(400), zeros(120)
            h.gls_residual(dW, dV, dd, dx, dy, dz, r1, r2, r3)
            torch.cuda.synchronize()
            scale = (np.abs(np.concatenate([np.zeros(500), d, np.zeros(120)]))
                     + np.concatenate([np.abs(y) + np.abs(V).T @ np.abs(z),
                                       np.abs(W) @ np.abs(x) + np.abs(V) @ np.abs(y),
                                       np.abs(W).T @ np.abs(z)]))
            ref = np.concatenate([host(r1), host(r2), host(r3)])
            got = np.concatenate([host(a1), host(a2), host(a3)])
            assert np.all(np.abs(got - ref) <= (400 + 120 + 500 + 2) * U64 * scale)
    finally:
        h.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_16499_gb300 import mpir
    # n = m = p = 8192 needs ~1M doubles of partial sums, beyond the 512k
    # array; the check happens before anything is read or launched.
    dummy = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    L = mpir.lib()
    rc = L.mpir_gls_residual_noalloc(8192, 8192, 8192, dummy.data_ptr(), 8192, dummy.data_ptr(), 8192,
                                     dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                     dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), None, None)
    assert rc == 5
