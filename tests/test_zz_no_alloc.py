"""The allocation-free pressure entry point against the pressure output of
tg_solve (GPU).

tg_pressure_noalloc serves callers that cannot allocate device memory:
processes whose device memory belongs to another allocator or to a fixed
arena, and paths that must avoid cudaMalloc's implicit synchronisation.  It
keeps its scratch in a static device array shared by all calls, so this test
calls it twice in a row on the same device and checks both results against
the existing entry point, checks that the calls leave the device's memory
use unchanged, that an invalid permeability is reported without
poisoning the next call, and that a call on a stream being captured is
refused without invalidating the capture.  The file sorts last so that a run stopping at the
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


def _solved(tg, n, b):
    from paper_1807_07220_gb300 import inputs
    kappa = inputs.grf_channel_field(n, 1e6, 11)
    f = inputs.random_pairs(n, 3, 12)
    s = tg.Solver(kappa, b, 10.0)
    s.solve(f, rtol=1e-12)
    return s


def _rel(p, ref):
    return (torch.linalg.norm(p - ref) / torch.linalg.norm(ref)).item()


def test_noalloc_pressure_matches_solve(tg):
    for n, b in ((32, 8), (64, 16)):
        s = _solved(tg, n, b)
        try:
            ref = s.p.clone()
            stream = torch.cuda.current_stream().cuda_stream
            for _ in range(2):
                p = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
                tg.tg_pressure_noalloc(s.kappa, s.ux, s.uy, p, n, stream)
                assert _rel(p, ref) < 1e-12, n
        finally:
            s.close()


def test_noalloc_allocates_nothing(tg):
    """Neither torch's allocator nor the device's free memory moves across
    repeated calls (one call first, so that the kernels are loaded)."""
    n, b = 64, 16
    s = _solved(tg, n, b)
    try:
        stream = torch.cuda.current_stream().cuda_stream
        outs = [torch.zeros((n, n), dtype=torch.float64, device="cuda") for _ in range(3)]
        tg.tg_pressure_noalloc(s.kappa, s.ux, s.uy, outs[0], n, stream)
        torch.cuda.synchronize()
        torch_before = torch.cuda.memory_allocated()
        free_before = torch.cuda.mem_get_info()[0]
        for p in outs[1:]:
            tg.tg_pressure_noalloc(s.kappa, s.ux, s.uy, p, n, stream)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == torch_before
        assert torch.cuda.mem_get_info()[0] == free_before
        for p in outs:
            assert _rel(p, s.p) < 1e-12
    finally:
        s.close()


def test_noalloc_invalid_kappa_then_valid_call(tg):
    """A kappa <= 0 cell gives TG_ERR_INVALID_ARG; the status word is cleared
    for the next call, which succeeds."""
    n, b = 32, 8
    s = _solved(tg, n, b)
    try:
        stream = torch.cuda.current_stream().cuda_stream
        bad = s.kappa.clone()
        bad.view(-1)[n * 5 + 7] = 0.0
        p = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        with pytest.raises(tg.TgmsError) as e:
            tg.tg_pressure_noalloc(bad, s.ux, s.uy, p, n, stream)
        assert e.value.code == -1
        tg.tg_pressure_noalloc(s.kappa, s.ux, s.uy, p, n, stream)
        assert _rel(p, s.p) < 1e-12
    finally:
        s.close()


def test_noalloc_refuses_a_capturing_stream(tg):
    """The call reads its status on the host and synchronises its stream, so
    it cannot be recorded in a graph: on a capturing stream it returns
    TG_ERR_UNSUPPORTED before enqueuing anything, the capture still ends in a
    graph that replays, and the next call on an ordinary stream succeeds."""
    n, b = 32, 8
    s = _solved(tg, n, b)
    try:
        p = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        x = torch.arange(64, dtype=torch.float64, device="cuda")
        side = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        code = None
        with torch.cuda.graph(graph, stream=side):
            y = 2.0 * x
            try:
                tg.tg_pressure_noalloc(s.kappa, s.ux, s.uy, p, n, side.cuda_stream)
            except tg.TgmsError as e:
                code = e.code
        assert code == -8
        y.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(y, 2.0 * x)
        assert not p.any()   # nothing of the refused call ran
        tg.tg_pressure_noalloc(s.kappa, s.ux, s.uy, p, n, torch.cuda.current_stream().cuda_stream)
        assert _rel(p, s.p) < 1e-12
    finally:
        s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(tg):
    n = 1025
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tg.TgmsError) as e:
        tg.tg_pressure_noalloc(z, z, z, z, n, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -8
