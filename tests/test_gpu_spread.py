"""GPU checks of the FP32 wave-space kernels on grids of different shapes.

FP32 spreading is grid-centric: the grid is cut into 8^3 tiles, and each
tile gathers the window contributions of the beads listed for it (a grid
side of 50 leaves partial tiles at the upper faces, 48 does not).  The FP32
wave-space operator must agree with the FP64 operator at the same grid
within 1e-5 (relative L2), and with the oracle's wave-space sum to the
accuracy of the grid rule, on grids with and without partial tiles; the
fused (planar) and separate (interleaved) FFT passes are checked the same
way."""

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g

    g.build()
    import paper_2607_25161_gb300 as p

    return p


def test_spreading_with_full_and_partial_tiles_agrees(pkg):
    pos, body, L = synth.mixed_suspension(40, 0.1, 31, size_hi=8)
    rng = np.random.default_rng(7)
    F = rng.normal(size=(len(pos), 11))
    xi = 1.2  # the xerr = 1e-8 rule asks for 43 points per side here
    ref = O.mobility_wave_dense(pos, L, xi, 2.0 * xi * np.sqrt(46.0)).reshape(11 * len(pos), -1) @ F.reshape(-1)
    for grid in (48, 50):  # 48: full 8^3 tiles; 50: partial tiles at the upper faces
        s = pkg.Suspension(pos, body, L, xi=xi, grid=grid, P=12)
        w64 = s.apply_mobility(F, part=2, precision=FP64).reshape(-1)
        w32 = s.apply_mobility(F, part=2, precision=MIXED).reshape(-1)
        s.close()
        assert rel(w32, w64) < 1e-5
        assert rel(w64, ref) < 1e-5


def test_fused_and_separate_fft_passes_agree(pkg):
    # FP32 planes up to n ~ 170 run the fused x + y kernels with planar
    # fields; larger grids take separate x and y passes with interleaved
    # fields.  Both must match the FP64 operator (separate passes) at the
    # same grid.
    pos, body, L = synth.mixed_suspension(40, 0.1, 31, size_hi=8)
    rng = np.random.default_rng(8)
    F = rng.normal(size=(len(pos), 11))
    for grid in (96, 180):
        s = pkg.Suspension(pos, body, L, xi=1.2, grid=grid, P=12)
        w64 = s.apply_mobility(F, part=2, precision=FP64).reshape(-1)
        w32 = s.apply_mobility(F, part=2, precision=MIXED).reshape(-1)
        s.close()
        assert rel(w32, w64) < 1e-5


def test_wave_operator_on_grids_beyond_the_default_line_counts(pkg):
    # n = 300: the FP64 z pass no longer fits four kx columns of six lines in
    # shared memory and takes fewer per block; FP32 at n = 300 takes the
    # separate x and y passes.  Both precisions must agree.
    import numpy as np

    rng = np.random.default_rng(31)
    pos = rng.uniform(0.0, 40.0, size=(16, 3))
    pos[:, 0] = np.arange(16) * 2.5 + 0.5
    s = pkg.Suspension(pos, np.arange(16), 40.0, xi=0.5, grid=300)
    assert s.params["grid"] == 300
    F = rng.normal(size=(16, 11))
    u64 = s.apply_mobility(F, part=2, precision=pkg.FSD_FP64)
    u32 = s.apply_mobility(F, part=2, precision=pkg.FSD_MIXED)
    s.close()
    assert np.abs(u64).max() > 0
    assert np.linalg.norm(u32 - u64) < 1e-5 * np.linalg.norm(u64)
