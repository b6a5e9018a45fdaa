"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/fsd.h declares; argument validation that runs before any CUDA call
(CPU only: no compute calls)."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g

    g.build()
    import paper_2607_25161_gb300 as pkg

    return pkg.load()


def test_header_symbols_exported(lib):
    hdr = open(os.path.join(ROOT, "include", "fsd.h")).read()
    names = set(re.findall(r"\b(fsd_[a-z_0-9]+)\s*\(", hdr))
    assert len(names) >= 13
    for n in sorted(names):
        assert hasattr(lib, n), n
    import paper_2607_25161_gb300 as pkg

    assert set(pkg.EXPORTS) == names


def test_default_params(lib):
    import paper_2607_25161_gb300 as pkg

    p = pkg.default_params(box=10.0)
    assert p.a == 1.0 and p.eta == 1.0 and p.box == 10.0
    assert p.P == 0 and p.restart == 30 and abs(p.tol - 1e-6) < 1e-20
    assert abs(p.precond_cutoff - 2.1) < 1e-15 and p.precision == pkg.FSD_FP64


def test_setup_rejects_bad_arguments_before_device_work(lib):
    import paper_2607_25161_gb300 as pkg

    p = pkg.default_params(box=10.0)
    ctx = ctypes.c_void_p()
    pos = np.zeros((1, 3))
    ids = np.zeros(1, dtype=np.int32)
    st = lib.fsd_setup(ctypes.byref(ctx), 0, pos.ctypes.data_as(ctypes.c_void_p),
                       ids.ctypes.data_as(ctypes.c_void_p), ctypes.byref(p), None)
    assert st == pkg.FSD_EINVAL
    assert b"n_beads" in lib.fsd_last_error(None)
    assert not ctx.value
    p.box = -1.0
    st = lib.fsd_setup(ctypes.byref(ctx), 1, pos.ctypes.data_as(ctypes.c_void_p),
                       ids.ctypes.data_as(ctypes.c_void_p), ctypes.byref(p), None)
    assert st == pkg.FSD_EINVAL
    st = lib.fsd_setup(None, 1, None, None, None, None)
    assert st == pkg.FSD_EINVAL
    # calls on a NULL context are rejected
    assert lib.fsd_solve(None, None, 0.0, None, None, None) == pkg.FSD_EINVAL
    assert lib.fsd_apply_saddle(None, None, None, 0) == pkg.FSD_EINVAL
    lib.fsd_destroy(None)


def test_struct_layout_matches_header(lib):
    # the ctypes mirrors list the header's fields in order
    import paper_2607_25161_gb300 as pkg

    hdr = open(os.path.join(ROOT, "include", "fsd.h")).read()
    body = hdr[hdr.index("typedef struct {\n  double a;"):hdr.index("} fsd_params;")]
    fields = re.findall(r"\b(?:double|int)\s+([a-zA-Z_0-9]+)\s*;", body)
    assert fields == [f for f, _ in pkg.FsdParams._fields_]
    body = hdr[hdr.index("typedef struct {\n  int iters;"):hdr.index("} fsd_stats;")]
    fields = re.findall(r"\b(?:double|int|int64_t)\s+([a-zA-Z_0-9]+)\s*;", body)
    assert fields == [f for f, _ in pkg.FsdStats._fields_]


def test_binding_passes_an_empty_suspension_to_the_library_checks(lib):
    import paper_2607_25161_gb300 as pkg

    with pytest.raises(pkg.FsdError, match="n_beads"):
        pkg.Suspension(np.zeros((0, 3)), np.zeros(0, dtype=np.int32), 20.0)
