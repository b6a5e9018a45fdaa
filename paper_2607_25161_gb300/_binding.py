"""ctypes binding of the FSD C ABI (include/fsd.h): argument marshalling only.

Every array argument may be a NumPy array (host) or a torch CUDA tensor
(device); device tensors are passed by pointer and used on the context's
stream.  Nothing here computes any part of the method: all arithmetic runs in
the CUDA library.  Loading fails loudly when the library is missing."""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfsd.so")

FSD_OK, FSD_EINVAL, FSD_ENOMEM, FSD_ECUDA, FSD_ENOCONV, FSD_ENUMERIC, FSD_EOVERLAP, FSD_ETIMEOUT = range(8)
FSD_FP64, FSD_MIXED = 0, 1
FSD_FLAG_WARM_START = 1
FSD_FLAG_COMOVING = 2
FSD_FLAG_GRAPH = 4
FSD_FLAG_AUTOTUNE = 8
FSD_FLAG_LEES_EDWARDS = 16
FSD_FLAG_FP32_KRYLOV = 32
FSD_DRIFT_RFD, FSD_DRIFT_FIXMAN = 0, 1
FSD_NF_LANCZOS, FSD_NF_PAIRWISE = 0, 1
STATUS_NAMES = {0: "FSD_OK", 1: "FSD_EINVAL", 2: "FSD_ENOMEM", 3: "FSD_ECUDA", 4: "FSD_ENOCONV",
                5: "FSD_ENUMERIC", 6: "FSD_EOVERLAP", 7: "FSD_ETIMEOUT"}

# every entry point declared in include/fsd.h
EXPORTS = (
    "fsd_default_params", "fsd_setup", "fsd_solve", "fsd_step", "fsd_get_beads",
    "fsd_apply_mobility", "fsd_apply_saddle", "fsd_apply_precond", "fsd_apply_lubrication",
    "fsd_rhs", "fsd_get_params", "fsd_profile_enable", "fsd_profile_read",
    "fsd_profile_group_name", "fsd_apply_wave_noalloc", "fsd_last_error", "fsd_destroy",
    "fsd_setup_batch", "fsd_batch_info", "fsd_solve_batch", "fsd_step_batch", "fsd_batch_get_beads",
    "fsd_batch_system", "fsd_batch_last_error", "fsd_destroy_batch", "fsd_brownian", "fsd_drift",
    "fsd_contact_forces", "fsd_set_tilt", "fsd_fma_throughput", "fsd_interparticle_forces",
)
PROF_GROUPS = 10


class FsdParams(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double), ("eta", ctypes.c_double), ("box", ctypes.c_double),
        ("xi", ctypes.c_double), ("xerr", ctypes.c_double), ("rc", ctypes.c_double),
        ("grid", ctypes.c_int), ("P", ctypes.c_int), ("m_shape", ctypes.c_double),
        ("lub_cutoff", ctypes.c_double), ("precond_cutoff", ctypes.c_double),
        ("lub_hmin", ctypes.c_double), ("tol", ctypes.c_double), ("restart", ctypes.c_int),
        ("max_iter", ctypes.c_int), ("precision", ctypes.c_int), ("inner_restart", ctypes.c_int),
        ("inner_tol", ctypes.c_double), ("flags", ctypes.c_int), ("tile", ctypes.c_int),
        ("lanczos_tol", ctypes.c_double), ("lanczos_max_iter", ctypes.c_int),
        ("tilt", ctypes.c_double), ("nf_sampler", ctypes.c_int),
        ("rough_alpha", ctypes.c_double), ("rough_h0", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FsdPairForces(ctypes.Structure):
    _fields_ = [
        ("kn", ctypes.c_double), ("hamaker", ctypes.c_double), ("zeta", ctypes.c_double),
        ("kappa", ctypes.c_double), ("h_c", ctypes.c_double), ("r_cut", ctypes.c_double),
    ]


class FsdStats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("matvec64", ctypes.c_int),
        ("matvec32", ctypes.c_int), ("rel_residual", ctypes.c_double), ("ms_total", ctypes.c_double),
        ("n_pairs", ctypes.c_int64), ("n_lub", ctypes.c_int64), ("grid", ctypes.c_int),
        ("P", ctypes.c_int), ("xi", ctypes.c_double), ("rc", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path=LIB_PATH):
    """Load libfsd.so and declare the signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("FSD CUDA library not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    lib.fsd_default_params.argtypes = [ctypes.POINTER(FsdParams)]
    lib.fsd_default_params.restype = None
    lib.fsd_setup.argtypes = [ctypes.POINTER(P), ctypes.c_int64, P, P, ctypes.POINTER(FsdParams), P]
    lib.fsd_solve.argtypes = [P, P, D, P, P, ctypes.POINTER(FsdStats)]
    lib.fsd_step.argtypes = [P, P, D, D, P, ctypes.POINTER(FsdStats)]
    lib.fsd_get_beads.argtypes = [P, P, P]
    lib.fsd_apply_mobility.argtypes = [P, P, P, I, I]
    lib.fsd_apply_saddle.argtypes = [P, P, P, I]
    lib.fsd_apply_precond.argtypes = [P, P, P]
    lib.fsd_apply_lubrication.argtypes = [P, P, P, I]
    lib.fsd_rhs.argtypes = [P, P, D, P]
    lib.fsd_get_params.argtypes = [P, ctypes.POINTER(FsdParams)]
    lib.fsd_profile_enable.argtypes = [P, I]
    lib.fsd_profile_read.argtypes = [P, P, P, I]
    lib.fsd_profile_group_name.argtypes = [I]
    lib.fsd_profile_group_name.restype = ctypes.c_char_p
    lib.fsd_apply_wave_noalloc.argtypes = [ctypes.c_int64, P, P, P, D, D, I, I, D, D, D, P]
    lib.fsd_last_error.argtypes = [P]
    lib.fsd_last_error.restype = ctypes.c_char_p
    lib.fsd_destroy.argtypes = [P]
    lib.fsd_destroy.restype = None
    lib.fsd_setup_batch.argtypes = [ctypes.POINTER(P), I, P, P, P, P, P]
    lib.fsd_batch_info.argtypes = [P, P, P, P]
    lib.fsd_solve_batch.argtypes = [P, P, P, P, P, P]
    lib.fsd_step_batch.argtypes = [P, P, P, D, P, P]
    lib.fsd_batch_get_beads.argtypes = [P, P, P]
    lib.fsd_batch_system.argtypes = [P, I]
    lib.fsd_batch_system.restype = P
    lib.fsd_batch_last_error.argtypes = [P]
    lib.fsd_batch_last_error.restype = ctypes.c_char_p
    lib.fsd_brownian.argtypes = [P, D, D, ctypes.c_uint64, ctypes.c_uint64, P, P, P, P, P,
                                 ctypes.POINTER(FsdStats)]
    lib.fsd_drift.argtypes = [P, I, D, D, D, ctypes.c_uint64, ctypes.c_uint64, P, P, P, P,
                              ctypes.POINTER(FsdStats)]
    lib.fsd_contact_forces.argtypes = [P, D, P]
    lib.fsd_interparticle_forces.argtypes = [P, ctypes.POINTER(FsdPairForces), P]
    lib.fsd_set_tilt.argtypes = [P, D]
    lib.fsd_fma_throughput.argtypes = [I, ctypes.POINTER(D), P]
    lib.fsd_destroy_batch.argtypes = [P]
    lib.fsd_destroy_batch.restype = None
    for name in EXPORTS:
        if name not in ("fsd_default_params", "fsd_last_error", "fsd_destroy",
                        "fsd_profile_group_name", "fsd_batch_system", "fsd_batch_last_error",
                        "fsd_destroy_batch"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class FsdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _ptr(arr):
    """Pointer of a NumPy array or torch tensor (None passes through)."""
    if arr is None:
        return None
    if hasattr(arr, "data_ptr"):
        if not arr.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(arr.data_ptr())
    if not arr.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return arr.ctypes.data_as(ctypes.c_void_p)


def default_params(**kw):
    lib = load()
    p = FsdParams()
    lib.fsd_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def fma_throughput(fp_bits, stream=None):
    """fsd_fma_throughput: measured FP32 (32) or FP64 (64) FMA rate of the
    current device in flop/s (2 per FMA)."""
    lib = load()
    out = ctypes.c_double()
    st = lib.fsd_fma_throughput(int(fp_bits), ctypes.byref(out), stream)
    if st != FSD_OK:
        raise FsdError(st, "fsd_fma_throughput failed")
    return out.value


class Suspension:
    """One suspension behind an fsd_ctx (fsd_setup ... fsd_destroy)."""

    def __init__(self, bead_pos, agg_id, box, stream=None, **params):
        self.lib = load()
        self._keep = []
        pos = bead_pos if hasattr(bead_pos, "data_ptr") else np.ascontiguousarray(bead_pos, dtype=np.float64)
        ids = agg_id if hasattr(agg_id, "data_ptr") else np.ascontiguousarray(agg_id, dtype=np.int32)
        self.n_beads = int(pos.shape[0])
        # an empty suspension reaches fsd_setup, which rejects it (FSD_EINVAL)
        self.n_agg = int(ids.max()) + 1 if self.n_beads > 0 else 0
        self.params_in = default_params(box=float(box), **params)
        self.ctx = ctypes.c_void_p()
        st = self.lib.fsd_setup(ctypes.byref(self.ctx), self.n_beads, _ptr(pos), _ptr(ids),
                                ctypes.byref(self.params_in), stream)
        if st != FSD_OK:
            raise FsdError(st, self.lib.fsd_last_error(None).decode())

    def _check(self, st, allow=(FSD_OK,)):
        if st not in allow:
            raise FsdError(st, self.lib.fsd_last_error(self.ctx).decode())
        return st

    @property
    def params(self):
        p = FsdParams()
        self._check(self.lib.fsd_get_params(self.ctx, ctypes.byref(p)))
        return p.as_dict()

    def solve(self, ft=None, shear=0.0, vel=None, stresslet=None, allow=(FSD_OK, FSD_EOVERLAP)):
        """fsd_solve; returns (velocity [N,6], stresslet [N,3,3], stats dict, status)."""
        if vel is None:
            vel = np.zeros((self.n_agg, 6))
        if stresslet is None:
            stresslet = np.zeros((self.n_agg, 3, 3))
        st_ = FsdStats()
        st = self.lib.fsd_solve(self.ctx, _ptr(ft), float(shear), _ptr(vel), _ptr(stresslet),
                                ctypes.byref(st_))
        self._check(st, allow)
        return vel, stresslet, st_.as_dict(), st

    def step(self, ft=None, shear=0.0, dt=1e-3, vel=None, allow=(FSD_OK, FSD_EOVERLAP)):
        st_ = FsdStats()
        st = self.lib.fsd_step(self.ctx, _ptr(ft), float(shear), float(dt), _ptr(vel),
                               ctypes.byref(st_))
        self._check(st, allow)
        return st_.as_dict(), st

    def beads(self):
        pos = np.zeros((self.n_beads, 3))
        q = np.zeros((self.n_agg, 4))
        self._check(self.lib.fsd_get_beads(self.ctx, _ptr(pos), _ptr(q)))
        return pos, q

    def apply_mobility(self, F, part=3, precision=FSD_FP64, out=None):
        F = F if hasattr(F, "data_ptr") else np.ascontiguousarray(F, dtype=np.float64)
        if out is None:
            out = np.zeros((self.n_beads, 11))
        self._check(self.lib.fsd_apply_mobility(self.ctx, _ptr(F), _ptr(out), int(part), int(precision)))
        return out

    def apply_saddle(self, x, precision=FSD_FP64, out=None):
        x = x if hasattr(x, "data_ptr") else np.ascontiguousarray(x, dtype=np.float64)
        if out is None:
            out = np.zeros(11 * self.n_beads + 6 * self.n_agg)
        self._check(self.lib.fsd_apply_saddle(self.ctx, _ptr(x), _ptr(out), int(precision)))
        return out

    def apply_precond(self, r, out=None):
        r = r if hasattr(r, "data_ptr") else np.ascontiguousarray(r, dtype=np.float64)
        if out is None:
            out = np.zeros(11 * self.n_beads + 6 * self.n_agg)
        self._check(self.lib.fsd_apply_precond(self.ctx, _ptr(r), _ptr(out)))
        return out

    def apply_lubrication(self, dU, precision=FSD_FP64, out=None):
        dU = dU if hasattr(dU, "data_ptr") else np.ascontiguousarray(dU, dtype=np.float64)
        if out is None:
            out = np.zeros((self.n_agg, 6))
        self._check(self.lib.fsd_apply_lubrication(self.ctx, _ptr(dU), _ptr(out), int(precision)))
        return out

    def rhs(self, ft=None, shear=0.0, out=None):
        if ft is not None and not hasattr(ft, "data_ptr"):
            ft = np.ascontiguousarray(ft, dtype=np.float64)
        if out is None:
            out = np.zeros(11 * self.n_beads + 6 * self.n_agg)
        self._check(self.lib.fsd_rhs(self.ctx, _ptr(ft), float(shear), _ptr(out)))
        return out

    def brownian(self, kT, dt, seed=0, step=0, wave_field=None, psi_real=None, psi_nf=None,
                 outputs=True):
        """fsd_brownian: Brownian terms of the next solve; returns (slip
        [Nt, 11], near-field force [Nt, 6], stats) (None, None, stats when
        outputs is false)."""
        def prep(a):
            if a is None or hasattr(a, "data_ptr"):
                return a
            return np.ascontiguousarray(a, dtype=np.float64)
        if wave_field is not None and not hasattr(wave_field, "data_ptr"):
            wave_field = np.ascontiguousarray(np.stack([np.asarray(wave_field).real,
                                                        np.asarray(wave_field).imag], -1))
        slip = np.zeros((self.n_beads, 11)) if outputs else None
        fnf = np.zeros((self.n_beads, 6)) if outputs else None
        st_ = FsdStats()
        self._check(self.lib.fsd_brownian(self.ctx, float(kT), float(dt), int(seed), int(step),
                                          _ptr(wave_field), _ptr(prep(psi_real)), _ptr(prep(psi_nf)),
                                          _ptr(slip), _ptr(fnf), ctypes.byref(st_)))
        return slip, fnf, st_.as_dict()

    def drift(self, method, kT, dt=0.0, param=0.0, seed=0, step=0, dq=None, outputs=True,
              allow=(FSD_OK, FSD_EOVERLAP)):
        """fsd_drift: Brownian drift added to the next solve; returns (drift
        [N, 6], Brownian velocity [N, 6] (Fixman), Brownian stresslet
        [N, 3, 3], stats, status) (None for the arrays when outputs is false)."""
        if dq is not None and not hasattr(dq, "data_ptr"):
            dq = np.ascontiguousarray(dq, dtype=np.float64)
        d = np.zeros((self.n_agg, 6)) if outputs else None
        ub = np.zeros((self.n_agg, 6)) if outputs else None
        sb = np.zeros((self.n_agg, 3, 3)) if outputs else None
        st_ = FsdStats()
        st = self.lib.fsd_drift(self.ctx, int(method), float(kT), float(dt), float(param), int(seed),
                                int(step), _ptr(dq), _ptr(d), _ptr(ub), _ptr(sb), ctypes.byref(st_))
        self._check(st, allow)
        return d, ub, sb, st_.as_dict(), st

    def set_tilt(self, tilt):
        """fsd_set_tilt: Lees-Edwards offset of the box."""
        self._check(self.lib.fsd_set_tilt(self.ctx, float(tilt)))

    def contact(self, kn, out=None):
        """fsd_contact_forces: Hertz contact force / torque per aggregate [N, 6]."""
        if out is None:
            out = np.zeros((self.n_agg, 6))
        self._check(self.lib.fsd_contact_forces(self.ctx, float(kn), _ptr(out)))
        return out

    def interparticle(self, kn=0.0, hamaker=0.0, zeta=0.0, kappa=1.0, h_c=0.0, r_cut=0.0, out=None):
        """fsd_interparticle_forces: Hertz + DLVO force / torque per aggregate [N, 6]."""
        if out is None:
            out = np.zeros((self.n_agg, 6))
        pf = FsdPairForces(float(kn), float(hamaker), float(zeta), float(kappa), float(h_c), float(r_cut))
        self._check(self.lib.fsd_interparticle_forces(self.ctx, ctypes.byref(pf), _ptr(out)))
        return out

    def profile(self, on=True):
        self._check(self.lib.fsd_profile_enable(self.ctx, 1 if on else 0))

    def profile_read(self):
        """{group: (device ms, timed launches)} since profile(True)."""
        ms = np.zeros(PROF_GROUPS)
        cnt = np.zeros(PROF_GROUPS, dtype=np.int64)
        self._check(self.lib.fsd_profile_read(self.ctx, _ptr(ms), _ptr(cnt), PROF_GROUPS))
        return {self.lib.fsd_profile_group_name(g).decode(): (float(ms[g]), int(cnt[g]))
                for g in range(PROF_GROUPS)}

    @classmethod
    def borrowed(cls, ctx, n_beads, n_agg):
        """A view of a context owned elsewhere (a batch system); close() does
        not destroy it."""
        self = cls.__new__(cls)
        self.lib = load()
        self._keep = []
        self.ctx = ctypes.c_void_p(ctx)
        self.n_beads = int(n_beads)
        self.n_agg = int(n_agg)
        self._borrowed = True
        return self

    def close(self):
        if self.ctx and not getattr(self, "_borrowed", False):
            self.lib.fsd_destroy(self.ctx)
        self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent suspensions behind an fsd_batch (fsd_setup_batch ...
    fsd_destroy_batch).  systems: list of (bead_pos [n,3], agg_id [n], box);
    params: one dict for all systems or a list of dicts."""

    def __init__(self, systems, params=None, stream=None):
        self.lib = load()
        n = len(systems)
        plist = params if isinstance(params, (list, tuple)) else [params or {}] * n
        pos = np.ascontiguousarray(np.concatenate([np.asarray(s[0], dtype=np.float64) for s in systems]))
        ids = np.ascontiguousarray(np.concatenate([np.asarray(s[1], dtype=np.int32) for s in systems]))
        self.bead_off = np.zeros(n + 1, dtype=np.int64)
        self.bead_off[1:] = np.cumsum([len(s[0]) for s in systems])
        arr = (FsdParams * n)()
        for i, (s, kw) in enumerate(zip(systems, plist)):
            arr[i] = default_params(box=float(s[2]), **kw)
        self.ctx = ctypes.c_void_p()
        st = self.lib.fsd_setup_batch(ctypes.byref(self.ctx), n, _ptr(self.bead_off), _ptr(pos),
                                      _ptr(ids), ctypes.cast(arr, ctypes.c_void_p), stream)
        if st != FSD_OK:
            raise FsdError(st, self.lib.fsd_batch_last_error(None).decode())
        self.n_sys = n
        self.agg_off = np.zeros(n + 1, dtype=np.int64)
        used = (FsdParams * n)()
        self._check(self.lib.fsd_batch_info(self.ctx, None, _ptr(self.agg_off),
                                            ctypes.cast(used, ctypes.c_void_p)))
        self.params = [used[i].as_dict() for i in range(n)]
        self.n_beads = int(self.bead_off[-1])
        self.n_agg = int(self.agg_off[-1])

    def _check(self, st, allow=(FSD_OK,)):
        if st not in allow:
            raise FsdError(st, self.lib.fsd_batch_last_error(self.ctx).decode())
        return st

    def _stats(self, arr):
        return [arr[i].as_dict() for i in range(self.n_sys)]

    def solve(self, ft=None, shear=0.0, allow=(FSD_OK, FSD_EOVERLAP)):
        """fsd_solve_batch; returns (velocity [A,6], stresslet [A,3,3], [stats], status)."""
        rates = np.ascontiguousarray(np.broadcast_to(np.asarray(shear, dtype=np.float64), (self.n_sys,)))
        if ft is not None and not hasattr(ft, "data_ptr"):
            ft = np.ascontiguousarray(ft, dtype=np.float64)
        vel = np.zeros((self.n_agg, 6))
        S = np.zeros((self.n_agg, 3, 3))
        stats = (FsdStats * self.n_sys)()
        st = self.lib.fsd_solve_batch(self.ctx, _ptr(ft), _ptr(rates), _ptr(vel), _ptr(S),
                                      ctypes.cast(stats, ctypes.c_void_p))
        self._check(st, allow)
        return vel, S, self._stats(stats), st

    def step(self, ft=None, shear=0.0, dt=1e-3, vel=None, allow=(FSD_OK, FSD_EOVERLAP)):
        rates = np.ascontiguousarray(np.broadcast_to(np.asarray(shear, dtype=np.float64), (self.n_sys,)))
        if ft is not None and not hasattr(ft, "data_ptr"):
            ft = np.ascontiguousarray(ft, dtype=np.float64)
        stats = (FsdStats * self.n_sys)()
        st = self.lib.fsd_step_batch(self.ctx, _ptr(ft), _ptr(rates), float(dt), _ptr(vel),
                                     ctypes.cast(stats, ctypes.c_void_p))
        self._check(st, allow)
        return self._stats(stats), st

    def beads(self):
        pos = np.zeros((self.n_beads, 3))
        q = np.zeros((self.n_agg, 4))
        self._check(self.lib.fsd_batch_get_beads(self.ctx, _ptr(pos), _ptr(q)))
        return pos, q

    def system(self, s):
        """Suspension view of system s (owned by the batch)."""
        ctx = self.lib.fsd_batch_system(self.ctx, int(s))
        if not ctx:
            raise IndexError(s)
        return Suspension.borrowed(ctx, self.bead_off[s + 1] - self.bead_off[s],
                                   self.agg_off[s + 1] - self.agg_off[s])

    def close(self):
        if self.ctx:
            self.lib.fsd_destroy_batch(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
