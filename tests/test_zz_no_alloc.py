"""The no-allocation wave-space entry point.

fsd_apply_wave_noalloc serves callers that cannot allocate device memory (a
captured CUDA graph, a memory pool they do not own, an allocation-free
real-time loop): it keeps every intermediate in one fixed-size device array
inside the library.  This test calls it through the C ABI twice in a row,
with different inputs, and checks each result against the context-based
wave-space operator (fsd_apply_mobility, part 2, FP32) within the FP32
operator tolerance of the parity tests (2e-5 relative L2).  The file is named
so that pytest collects it last."""

import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


def test_noalloc_wave_matches_context_operator():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g

    g.build()
    import paper_2607_25161_gb300 as pkg

    lib = pkg.load()
    pos, body, L = synth.suspension(48, 5, 0.08, 21)
    nt = len(pos)
    grid, P, xi = 40, 8, 0.5
    s = pkg.Suspension(pos, body, L, xi=xi, grid=grid, P=P)
    rng = np.random.default_rng(22)
    dpos = torch.tensor(pos, dtype=torch.float64, device="cuda")
    dout = torch.empty((nt, 11), dtype=torch.float64, device="cuda")
    for call in range(2):
        F = rng.normal(size=(nt, 11))
        ref = s.apply_mobility(F, part=2, precision=pkg.FSD_MIXED)
        dF = torch.tensor(F, dtype=torch.float64, device="cuda")
        dout.fill_(float("nan"))
        torch.cuda.synchronize()
        st = lib.fsd_apply_wave_noalloc(nt, ctypes.c_void_p(dpos.data_ptr()),
                                        ctypes.c_void_p(dF.data_ptr()),
                                        ctypes.c_void_p(dout.data_ptr()), L, xi, grid, P, 0.0,
                                        1.0, 1.0, None)
        torch.cuda.synchronize()
        assert st == pkg.FSD_OK
        got = dout.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, ref) < 2e-5, (call, rel(got, ref))
    s.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    pytest.importorskip("torch")
    import paper_2607_25161_gb300 as pkg

    lib = pkg.load()
    # limits are checked before any pointer is touched or any work is queued
    assert lib.fsd_apply_wave_noalloc(5000, None, None, None, 20.0, 0.5, 32, 8, 0.0, 1.0, 1.0,
                                      None) == pkg.FSD_EINVAL
    assert lib.fsd_apply_wave_noalloc(10, None, None, None, 20.0, 0.5, 60, 8, 0.0, 1.0, 1.0,
                                      None) == pkg.FSD_EINVAL
