"""The benchmark's algorithmic work counts (the numerator of its roofline)
against the textbook Householder flop counts.

QR of an M x N matrix (M >= N): 2 M N^2 - 2 N^3 / 3 flops; applying its N
reflectors to K columns: 4 M N K - 2 N^2 K.  The GQR of the n = p = 4096,
m = 1024 GLS workload is then 7.87e9 (QR of W) + 6.01e10 (Q^T V) + 9.16e10
(RQ of the n x p C) = 1.60e11 flops; the blocked compact-WY form adds the
small triangular products of each panel (a few per cent).
"""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def qr_flops(M, N):
    return 2.0 * M * N * N - 2.0 * N ** 3 / 3.0


@pytest.mark.parametrize("M,N", [(4096, 1024), (4096, 4096), (2000, 300)])
def test_blocked_qr_count_matches_householder(M, N):
    """At least the unblocked count, and above it by the compact-WY overhead,
    which is of order nb / N (nb = 32 reflectors per panel)."""
    pf, lf = bench.qr_work(M, N)
    assert pf > 0 and lf > 0
    excess = (pf + lf) / qr_flops(M, N) - 1
    assert 0 <= excess <= 4 * 32 / N


def test_gls_workload_count_matches_the_gqr():
    n, m, p = 4096, 1024, 4096
    w = bench.gls_work(n, m, p)
    textbook = qr_flops(n, m) + (4.0 * n * m * p - 2.0 * m * m * p) + qr_flops(p, n)
    assert abs(textbook / 1.60e11 - 1) < 0.005
    assert abs(w["factor_flops"] / textbook - 1) < 0.03
    assert w["panel_flops"] < 0.02 * w["factor_flops"]        # the panels are ~1 % of the work
    assert w["resid_bytes"] == 8.0 * (n * m + n * p)            # one FP64 read of W and V


def test_fp32_simt_peak_from_unit_counts():
    assert bench.fp32_simt_peak(2070.0) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


def test_lse_workload_count_matches_the_grq():
    """LSE m = 16384, n = 8192, p = 1024: QR of the n x p B~ (1.65e10), its
    reflectors applied to the m columns of X (5.15e11), QR of the m x n
    A Q^T (1.83e12): 2.37e12 flops; the split into panel, inner (SIMT) and
    tensor-core parts sums to the total."""
    m, n, p = 16384, 8192, 1024
    w = bench.lse_work(m, n, p)
    textbook = qr_flops(n, p) + (4.0 * n * p * m - 2.0 * p * p * m) + qr_flops(m, n)
    assert abs(textbook / 2.37e12 - 1) < 0.005
    assert abs(w["factor_flops"] / textbook - 1) < 0.03
    assert w["panel_flops"] + w["inner_flops"] + w["tc_flops"] == pytest.approx(w["factor_flops"])
    assert w["tc_flops"] > 0.9 * w["factor_flops"]
    assert w["resid_bytes"] == 8.0 * (m * n + p * n)


def test_tf32_peak_from_measured_bf16():
    peaks = {"bf16_tflops": 1920.0, "bf16_tflops_sustained": 1697.3}
    assert bench.tf32_peak(peaks, sustained=False) == pytest.approx(1920.0 * 1.1 / 2.25)
    assert bench.tf32_peak(peaks, sustained=True) == pytest.approx(1697.3 * 1.1 / 2.25)


def test_paper_shape_lists_follow_sec_6():
    """Sec. 6.2: n in {1024, 2048, 3072} with (m, p) = (8n, n/32), (8n, n/64),
    (10n, n/32), (10n, n/64), (12n, n/32), (12n, n/64) at four condition
    numbers; n in {128, 192, 256} with (m, p) = (128n, n/8), (128n, n/4),
    (128n, n/2), (256n, n/8), (256n, n/4), (256n, n/2) at 1e5.  Sec. 6.3:
    (p, m) = (8n, n/32) ... (12n, n/64) for the same n and conditionings."""
    lse1, lse2, gls = bench.paper_shape_list(True)
    assert len(lse1) == 72 and len(lse2) == 18 and len(gls) == 72
    assert ((3072, 36864, 48), 1e9) in lse1 and ((128, 16384, 16), 1e5) in lse2
    assert ((2048, 64, 16384), 1e5) in gls
    for (n, m, p), _ in lse1 + lse2:
        assert p <= n <= m                       # LSE shapes (m >= n >= p)
    for (n, m, p), _ in gls:
        assert m <= n <= p                       # GLS shapes (m <= n <= p)
    small = bench.paper_shape_list(False)
    assert all(set(a) <= set(b) for a, b in zip(small, (lse1, lse2, gls)))
