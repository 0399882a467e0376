"""The measurement arithmetic of bench.py (CPU only), against quantities
counted independently from the oracle's grid:
  * the DOF convention of Section 6 (interior faces + cells + 1), at the
    sizes of the benchmarked configurations;
  * the patch sizes behind the smoother's algorithmic bytes, from the
    oracle's oversampled-patch rectangles, and the band width behind the band
    form's bytes, from the sparsity of the oracle's reduced operator C^T A C;
  * the node count behind the operator roofline, from the oracle's curl.
"""

import numpy as np

import bench
from oracle.fine import Grid, assemble, curl_matrix


def test_dof_convention():
    for n, b, expect in ((32, 8, 3009), (256, 16, 196097), (512, 16, 785409), (1024, 16, 3143681)):
        g = Grid(n, b)
        assert bench.dof(n) == g.interior_faces().size + g.ncell + 1 == expect


def _patch_nodes(g):
    """Interior nodes (n_x, n_y) of every oversampled patch, from the oracle."""
    out = []
    for J in range(g.nc):
        for I in range(g.nc):
            x0, x1, y0, y1 = g.patch_rect(I, J)
            out.append((x1 - x0 - 1, y1 - y0 - 1))
    return out


def test_smoother_bytes_follow_the_patches():
    for n, b, ts, tc in ((256, 16, 2, 4), (256, 16, 4, 4), (64, 8, 8, 8), (48, 4, 2, 4)):
        dense = band = 0
        for nx, ny in _patch_nodes(Grid(n, b)):
            m = nx * ny
            dense += m * m * ts + m * (8 + 2 * tc)
            band += 2 * m * (nx + 2) * tc + m * (8 + 2 * tc)
        assert bench.smoother_bytes(n, b, 2, ts, tc) == dense
        assert bench.band_smoother_bytes(n, b, 2, tc) == band
    # the figures quoted for the headline workload: 64.9 MB BF16, 128.3 MB FP32
    assert abs(bench.smoother_bytes(256, 16, 2, 2, 4) - 64.88e6) < 0.01e6
    assert abs(bench.smoother_bytes(256, 16, 2, 4, 4) - 128.32e6) < 0.01e6


def test_band_width_of_the_patch_operator():
    """The band form stores n_x + 2 entries per row (half bandwidth n_x + 1):
    the largest |i - j| over the nonzeros of the reduced operator C^T A C on
    a patch's interior nodes, ordered x fastest."""
    n, b = 16, 4
    g = Grid(n, b)
    kappa = np.exp(np.random.default_rng(3).standard_normal((n, n)))
    A, _ = assemble(g, kappa)
    C = curl_matrix(g)
    I = g.interior_faces()
    K = (C.T @ A[I][:, I] @ C).tocoo()
    for (Ip, Jp) in ((0, 0), (1, 2), (3, 3)):
        x0, x1, y0, y1 = g.patch_rect(Ip, Jp)
        nx, ny = x1 - x0 - 1, y1 - y0 - 1
        # inner nodes (i, j), 1 <= i, j <= n - 1, are columns (j - 1)(n - 1) + (i - 1) of C
        ii, jj = np.meshgrid(np.arange(x0 + 1, x1), np.arange(y0 + 1, y1), indexing="xy")
        cols = ((jj - 1) * (n - 1) + (ii - 1)).ravel()
        local = {c: k for k, c in enumerate(cols)}
        width = 0
        for r, c in zip(K.row, K.col):
            if r in local and c in local:
                width = max(width, abs(local[r] - local[c]))
        assert width == nx + 1, (Ip, Jp, width, nx)


def test_operator_roofline_counts():
    """9 FMAs of K p per interior node plus two per node of the n x n array,
    and (2 sizeof(TC) + 64) bytes per node; the interior nodes are the
    columns of the oracle's curl."""
    for n in (16, 64):
        inner = curl_matrix(Grid(n, 4)).shape[1]
        assert inner == (n - 1) ** 2
        r = bench.operator_roofline(n, 4, 1.0, 1, {"hbm_gbs": 1000.0}, "measured")
        assert r["algorithmic_flops_per_launch"] == 2.0 * (9 * inner + 2 * n * n)
        assert r["algorithmic_bytes_per_launch"] == n * n * (2 * 4 + 8 + 5 * 8 + 8 + 8)
        assert abs(r["avg_launch_us"] - 1000.0) < 1e-9
        assert abs(r["achieved"] - r["algorithmic_flops_per_launch"] / 1e-3 / 1e9) < 1e-9
