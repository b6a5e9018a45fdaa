"""The no-allocation wave-space entry point.

fsd_apply_wave_noalloc serves callers that cannot allocate device memory
(device memory owned by an allocator or pool they do not control, a plug-in
that must not grow the device footprint after start-up, an allocation-free
real-time loop): it keeps every intermediate in one fixed-size device array
inside the library.  These tests call it through the C ABI twice in a row,
with different inputs, and check each result against the context-based
wave-space operator (fsd_apply_mobility, part 2, FP32) within the FP32
operator tolerance of the parity tests (2e-5 relative L2), once at a middle
size and once at the largest accepted one (48^3 grid, 4096 beads), whose
layout comes closest to the array's 10 MiB.  A third test uses the entry
point the way it exists to be used: one plain call, then a second call
captured into a CUDA graph on a side stream (torch's default, global capture
mode), replayed after the positions and moments in the captured buffers have
been rewritten.  The file is named so that pytest collects it last."""

import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


# xi is chosen so that the grid resolves it (the window deconvolution factor
# exp(k^2/(2 alpha) - k^2/(4 xi^2)) decays towards the grid's corner); on a grid
# too coarse for xi that factor amplifies FP32 rounding, and two FP32 codes
# that sum in different orders no longer agree to 2e-5
@pytest.mark.parametrize("n_agg,n_b,phi,grid,P,xi", [(48, 5, 0.08, 40, 8, 0.5),
                                                     (512, 8, 0.05, 48, 8, 0.25)])
def test_noalloc_wave_matches_context_operator(n_agg, n_b, phi, grid, P, xi):
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g

    g.build()
    import paper_2607_25161_gb300 as pkg

    lib = pkg.load()
    pos, body, L = synth.suspension(n_agg, n_b, phi, 21)
    nt = len(pos)
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


def test_noalloc_replays_inside_captured_graph():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g

    g.build()
    import paper_2607_25161_gb300 as pkg

    lib = pkg.load()
    xi, grid, P = 0.5, 40, 8
    # two configurations of the same bead count and box: the replays must read
    # the positions in the captured buffer, not those of the captured call
    configs = [synth.suspension(48, 5, 0.08, seed) for seed in (31, 32)]
    L = configs[0][2]
    assert configs[1][2] == L and len(configs[1][0]) == len(configs[0][0])
    nt = len(configs[0][0])
    rng = np.random.default_rng(33)
    dpos = torch.tensor(configs[0][0], dtype=torch.float64, device="cuda")
    dF = torch.tensor(rng.normal(size=(nt, 11)), dtype=torch.float64, device="cuda")
    dout = torch.empty((nt, 11), dtype=torch.float64, device="cuda")

    def call(stream):
        return lib.fsd_apply_wave_noalloc(nt, ctypes.c_void_p(dpos.data_ptr()),
                                          ctypes.c_void_p(dF.data_ptr()),
                                          ctypes.c_void_p(dout.data_ptr()), L, xi, grid, P, 0.0,
                                          1.0, 1.0, stream)

    torch.cuda.synchronize()
    assert call(None) == pkg.FSD_OK
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(graph, stream=side):
        st = call(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == pkg.FSD_OK
    for rep, (pos, body, _) in enumerate(configs + configs[::-1]):
        F = rng.normal(size=(nt, 11))
        s = pkg.Suspension(pos, body, L, xi=xi, grid=grid, P=P)
        ref = s.apply_mobility(F, part=2, precision=pkg.FSD_MIXED)
        s.close()
        dpos.copy_(torch.tensor(pos, dtype=torch.float64))
        dF.copy_(torch.tensor(F, dtype=torch.float64))
        dout.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        got = dout.cpu().numpy()
        assert np.all(np.isfinite(got)), rep
        assert rel(got, ref) < 2e-5, (rep, rel(got, ref))
    del graph


def test_noalloc_rejects_sizes_beyond_its_limits():
    pytest.importorskip("torch")
    import paper_2607_25161_gb300 as pkg

    lib = pkg.load()
    # limits are checked before any pointer is touched or any work is queued
    assert lib.fsd_apply_wave_noalloc(5000, None, None, None, 20.0, 0.5, 32, 8, 0.0, 1.0, 1.0,
                                      None) == pkg.FSD_EINVAL
    assert lib.fsd_apply_wave_noalloc(10, None, None, None, 20.0, 0.5, 60, 8, 0.0, 1.0, 1.0,
                                      None) == pkg.FSD_EINVAL
