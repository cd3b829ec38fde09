"""The tensor-core block-reflector application (tcgen05 GEMMs, xLARFB with a
128-reflector block, the trailing update of Lemma 4.5 / 4.6's
factorizations) against the same product in FP64 on the CPU:
    C <- (I - V X V^T) C,  X = T^T or T,  V unit lower trapezoidal.
FP32 mode (three TF32 products) must be FP32-class; TF32 mode TF32-class;
BF16 mode (kind::f16, bfloat16 operands, FP32 accumulation) BF16-class, and
equal to a bfloat16 emulation of the same two products.
Shapes cover ragged M, N (partial 128-tiles), K < 128 and split-K."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_16499_gb300 import mpir
    hd = mpir.Handle()
    yield hd
    hd.close()


def dev32(a, ld=None):
    import torch
    a = np.asarray(a, dtype=np.float32)
    rows, cols = a.shape
    ld = ld or ((rows + 31) // 32) * 32
    buf = torch.zeros((cols, ld), dtype=torch.float32, device="cuda")
    buf[:, :rows] = torch.from_numpy(np.ascontiguousarray(a.T)).cuda()
    return buf.t()[:rows, :]


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("tf32", 3e-3), ("bf16", 1.2e-2)])
@pytest.mark.parametrize("M,N,K,trans", [(300, 200, 128, True), (1000, 513, 77, False), (4096, 1024, 128, True),
                                         (129, 33, 5, True)])
def test_larfb_tc_matches_fp64(h, prec, tol, M, N, K, trans):
    import torch
    g = np.random.default_rng(M * 7 + N + K)
    Vp = g.standard_normal((M, K)) / np.sqrt(M)
    Vu = np.tril(Vp, -1)[:, :K]
    Vu[np.arange(K), np.arange(K)] = 1.0
    T = np.triu(g.standard_normal((K, K))) / np.sqrt(K)
    C = g.standard_normal((M, N))
    X = T.T if trans else T
    Vp32 = Vp.astype(np.float32).astype(np.float64)
    Vu32 = np.tril(Vp32, -1)[:, :K]
    Vu32[np.arange(K), np.arange(K)] = 1.0
    T32 = T.astype(np.float32).astype(np.float64)
    C32 = C.astype(np.float32).astype(np.float64)
    X32 = T32.T if trans else T32
    ref = C32 - Vu32 @ (X32 @ (Vu32.T @ C32))
    Td = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    Td[:K, :K] = torch.from_numpy(T.astype(np.float32).T.copy()).cuda().t()
    Td = Td.t().contiguous().t()          # column-major, ld 128
    Cd = dev32(C)
    h.larfb(dev32(Vp), Td, Cd, trans=trans, prec=prec)
    torch.cuda.synchronize()
    got = Cd.cpu().numpy().astype(np.float64)
    scale = np.linalg.norm(C32) + np.linalg.norm(Vu32) ** 2 * np.linalg.norm(X32) * np.linalg.norm(C32) / np.sqrt(M)
    err = np.linalg.norm(got - ref) / scale
    assert err < tol, err


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), as float64."""
    x = np.asarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("M,N,K,trans", [(1000, 513, 77, False), (4096, 1024, 128, True)])
def test_larfb_bf16_is_bfloat16(h, M, N, K, trans):
    """The BF16 path rounds V, C and W = X V^T C to bfloat16 and accumulates
    in FP32: it matches that emulation far more closely than it matches the
    exact product (whose distance is the bfloat16 rounding itself)."""
    import torch
    g = np.random.default_rng(M + 3 * N + K)
    Vp = g.standard_normal((M, K)) / np.sqrt(M)
    T = np.triu(g.standard_normal((K, K))) / np.sqrt(K)
    C = g.standard_normal((M, N))
    Vp32 = Vp.astype(np.float32).astype(np.float64)
    Vu32 = np.tril(Vp32, -1)[:, :K]
    Vu32[np.arange(K), np.arange(K)] = 1.0
    T32 = T.astype(np.float32).astype(np.float64)
    C32 = C.astype(np.float32).astype(np.float64)
    X32 = T32.T if trans else T32
    ref = C32 - Vu32 @ (X32 @ (Vu32.T @ C32))
    Vb = bf16(Vu32)
    W = X32 @ (Vb.T @ bf16(C32))
    emu = C32 - Vb @ bf16(W)
    Td = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    Td[:K, :K] = torch.from_numpy(T.astype(np.float32).T.copy()).cuda().t()
    Td = Td.t().contiguous().t()
    Cd = dev32(C)
    h.larfb(dev32(Vp), Td, Cd, trans=trans, prec="bf16")
    torch.cuda.synchronize()
    got = Cd.cpu().numpy().astype(np.float64)
    scale = np.linalg.norm(C32) + np.linalg.norm(Vu32) ** 2 * np.linalg.norm(X32) * np.linalg.norm(C32) / np.sqrt(M)
    e_emu = np.linalg.norm(got - emu) / scale
    e_ref = np.linalg.norm(got - ref) / scale
    assert e_emu < 4e-4 and e_ref > 5 * e_emu, (e_emu, e_ref)
