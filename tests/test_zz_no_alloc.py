"""The allocation-free pressure entry point against the pressure output of
tg_solve (GPU).

tg_pressure_noalloc serves callers that cannot allocate device memory (work
recorded in a stream capture, processes whose memory belongs to another
allocator, paths that must avoid cudaMalloc's implicit synchronisation).  It
keeps its scratch in a static device array shared by all calls, so this test
calls it twice in a row on the same device and checks both results against
the existing entry point.  The file sorts last so that a run stopping at the
first failure has already run every other test; it also passes alone in a
fresh process."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tg():
    from paper_1807_07220_gb300 import build, tgms
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(tgms.LIB_PATH):
        build.build_library()
    tgms.lib()
    return tgms


def test_noalloc_pressure_matches_solve(tg):
    from paper_1807_07220_gb300 import inputs
    for n, b in ((32, 8), (64, 16)):
        kappa = inputs.grf_channel_field(n, 1e6, 11)
        f = inputs.random_pairs(n, 3, 12)
        s = tg.Solver(kappa, b, 10.0)
        try:
            s.solve(f, rtol=1e-12)
            ref = s.p.clone()
            stream = torch.cuda.current_stream().cuda_stream
            for _ in range(2):
                p = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
                tg.tg_pressure_noalloc(s.kappa, s.ux, s.uy, p, n, stream)
                err = (torch.linalg.norm(p - ref) / torch.linalg.norm(ref)).item()
                assert err < 1e-12, (n, err)
        finally:
            s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(tg):
    n = 1025
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tg.TgmsError) as e:
        tg.tg_pressure_noalloc(z, z, z, z, n, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -8
