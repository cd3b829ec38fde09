"""The large LSE workload (m = 16384, n = 8192, p = 1024; cond(A) in 1e1,
1e4, 1e8, cond(B) = 1e2) at full size.  The oracle's factorization is too
slow at this size, so the checks are the size-independent properties the
FP64-level bar is defined by, evaluated by the oracle's double-double
residual: eq. lse-stop ratios (eta) and the constraint residual
||Bx-d|| / (||B|| ||x|| + ||d||), both <= 1e-14."""
import numpy as np
import pytest

from paper_2406_16499_gb300 import inputs as I

pytestmark = pytest.mark.gpu

M, N, P = 16384, 8192, 1024


@pytest.fixture(scope="module")
def h():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_16499_gb300 import mpir
    hd = mpir.Handle()
    yield hd
    hd.close()


@pytest.mark.parametrize("cond,fact,refine", [(1e1, "fp32", "classical"), (1e4, "tf32", "classical"),
                                              (1e8, "fp32", "gmres")])
def test_lse_large_full_size(h, oracle_mod, cond, fact, refine):
    import torch
    from paper_2406_16499_gb300 import mpir
    T = I.lse_svd_torch(20243623 + int(np.log10(cond)), M, N, P, cond, 1e2, "cuda")
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    r = torch.zeros(M, dtype=torch.float64, device="cuda")
    v = torch.zeros(P, dtype=torch.float64, device="cuda")
    st, info = h.lse_solve(T["A"], T["B"], T["b"], T["d"], x, r, v, mpir.make_opts(fact=fact, refine=refine))
    assert st == 0, (st, info.as_dict())
    A = T["A"].cpu().numpy()
    B = T["B"].cpu().numpy()
    met = oracle_mod.lse_metrics(A, B, T["b"].cpu().numpy(), T["d"].cpu().numpy(), x.cpu().numpy(),
                                 r.cpu().numpy(), v.cpu().numpy())
    print(cond, fact, refine, info.as_dict()["iters"], info.as_dict()["escalated"], met["eta"], met["e_con"])
    assert met["eta"] <= 1e-14 and met["e_con"] <= 1e-14, met
