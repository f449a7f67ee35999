"""Python binding of the C ABI in include/rpb.h (argument marshalling only).

Every computation runs in the CUDA library librpb.so; this module only checks tensor
shapes/dtypes/devices, passes raw device pointers and the current torch CUDA stream, and turns
error codes into exceptions.  There is no CPU fallback: if the library cannot be built or loaded,
load() raises.

Vectors are torch float64 CUDA tensors of shape (3N,) in structure-of-arrays layout
[x_0..x_{N-1} | y_0..y_{N-1} | z_0..z_{N-1}] (use inputs.to_soa / from_soa to convert from the
particle-major (N, 3) arrays of the paper's notation).
"""
import ctypes
import os

from . import build as _build

RPB_OK, RPB_EINVAL, RPB_ENOMEM, RPB_ECUDA, RPB_ENOCONV, RPB_ETIMEOUT = 0, 1, 2, 3, 4, 5
RPB_FP64, RPB_FP32 = 0, 1
PRECISIONS = {"fp64": RPB_FP64, "fp32": RPB_FP32}

# Every entry point the header declares (checked by the tests against include/rpb.h).
EXPORTS = ("rpb_create", "rpb_destroy", "rpb_set_stream", "rpb_mobility_apply", "rpb_lanczos_sqrt_apply",
           "rpb_rfd_drift", "rpb_forces", "rpb_philox_normal", "rpb_ab_step", "rpb_last_error",
           "rpb_launch_count", "rpb_mobility_apply_noalloc", "rpb_batch_create", "rpb_batch_destroy",
           "rpb_batch_set_stream", "rpb_batch_mobility_apply", "rpb_batch_ab_step", "rpb_step", "rpb_batch_run",
           "rpb_set_periodic", "rpb_set_preconditioner", "rpb_fma_peak", "rpb_run", "rpb_mobility_apply2",
           "rpb_mobility_apply_rows", "rpb_set_product_hook", "rpb_batch_set_tiles", "rpb_batch_get_tiles",
           "rpb_batch_tune", "rpb_mobility_apply_part")
SCHEMES = {"AB": 0, "EM": 1}
RFDS = {"centred": 0, "one-sided": 1}
PRECONDITIONERS = {"none": 0, "block-diagonal": 1}
NOALLOC_MAX_N = 16384


class RpbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rpb error {code}: {msg}")
        self.code = code


class NoConvergence(RpbError):
    pass


class Params(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("eta", ctypes.c_double), ("kT", ctypes.c_double), ("precision", ctypes.c_int),
                ("wall", ctypes.c_int)]

    def __init__(self, a=1.0, eta=1.0, kT=1.0, precision=0, wall=1):
        super().__init__(a, eta, kT, precision, wall)


class ForceParams(ctypes.Structure):
    _fields_ = [("weight", ctypes.c_double), ("U0", ctypes.c_double), ("b", ctypes.c_double),
                ("torque", ctypes.c_double * 3)]


class StepStats(ctypes.Structure):
    _fields_ = [("lanczos_iters", ctypes.c_int), ("lanczos_err", ctypes.c_double), ("converged", ctypes.c_int)]


# int hook(void *user, int64_t N, const double *pos, const double *F, const double *T, double *U)
PRODUCT_HOOK = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p)


class BatchTiles(ctypes.Structure):
    _fields_ = [("seg_tiles", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("symmetric", ctypes.c_int)]

    def as_dict(self):
        return dict(seg_tiles=self.seg_tiles, ctas_per_sm=self.ctas_per_sm, symmetric=bool(self.symmetric))


class StepOptions(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("rfd", ctypes.c_int)]


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load librpb.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; build it with paper_1612_00474_gb300/build.py")
    L = ctypes.CDLL(path)
    vp, i64, i32, d, u32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint32, \
        ctypes.c_uint64
    L.rpb_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params), i64, i32, vp]
    L.rpb_destroy.argtypes = [vp]
    L.rpb_set_stream.argtypes = [vp, vp]
    L.rpb_set_periodic.argtypes = [vp, d, d]
    L.rpb_set_preconditioner.argtypes = [vp, i32]
    L.rpb_mobility_apply.argtypes = [vp, i64, vp, vp, vp, vp]
    L.rpb_lanczos_sqrt_apply.argtypes = [vp, i64, vp, vp, vp, d, i32, ctypes.POINTER(i32), ctypes.POINTER(d)]
    L.rpb_rfd_drift.argtypes = [vp, i64, vp, vp, d, vp]
    L.rpb_forces.argtypes = [vp, i64, vp, ctypes.POINTER(ForceParams), vp]
    L.rpb_philox_normal.argtypes = [vp, i64, u64, u32, u32, u32, vp]
    L.rpb_ab_step.argtypes = [vp, i64, vp, vp, i64, u64, d, d, d, i32, ctypes.POINTER(ForceParams),
                              ctypes.POINTER(StepStats)]
    L.rpb_step.argtypes = [vp, i64, vp, vp, i64, u64, d, d, d, i32, ctypes.POINTER(ForceParams),
                           ctypes.POINTER(StepOptions), ctypes.POINTER(StepStats)]
    L.rpb_last_error.argtypes = []
    L.rpb_last_error.restype = ctypes.c_char_p
    L.rpb_launch_count.argtypes = []
    L.rpb_launch_count.restype = ctypes.c_uint64
    L.rpb_mobility_apply_noalloc.argtypes = [i64, vp, vp, vp, vp, ctypes.POINTER(Params), vp]
    L.rpb_fma_peak.argtypes = [i32, vp, ctypes.POINTER(d), ctypes.POINTER(d)]
    L.rpb_mobility_apply2.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
    L.rpb_mobility_apply_rows.argtypes = [vp, i64, vp, vp, vp, i64, i64, vp]
    L.rpb_mobility_apply_part.argtypes = [vp, i64, vp, vp, vp, i32, i32, vp]
    L.rpb_set_product_hook.argtypes = [vp, PRODUCT_HOOK, vp]
    L.rpb_batch_set_tiles.argtypes = [vp, ctypes.POINTER(BatchTiles)]
    L.rpb_batch_get_tiles.argtypes = [vp, ctypes.POINTER(BatchTiles)]
    L.rpb_batch_tune.argtypes = [vp, i32, ctypes.POINTER(i64), vp, i32, ctypes.POINTER(BatchTiles), i32,
                                 ctypes.POINTER(BatchTiles), ctypes.POINTER(d), ctypes.POINTER(i32)]
    L.rpb_run.argtypes = [vp, i64, vp, vp, i64, u64, i32, d, d, d, i32, ctypes.POINTER(ForceParams),
                          ctypes.POINTER(StepOptions), ctypes.POINTER(StepStats), ctypes.POINTER(i64)]
    pi64 = ctypes.POINTER(i64)
    L.rpb_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params), i64, i32, i32, vp]
    L.rpb_batch_destroy.argtypes = [vp]
    L.rpb_batch_set_stream.argtypes = [vp, vp]
    L.rpb_batch_mobility_apply.argtypes = [vp, i32, pi64, vp, vp, vp, vp]
    L.rpb_batch_ab_step.argtypes = [vp, i32, pi64, vp, vp, pi64, ctypes.POINTER(u64), d, d, d, i32,
                                    ctypes.POINTER(ForceParams), ctypes.POINTER(StepStats)]
    L.rpb_batch_run.argtypes = [vp, i32, pi64, vp, vp, pi64, ctypes.POINTER(u64), i32, d, d, d, i32,
                                ctypes.POINTER(ForceParams), ctypes.POINTER(StepStats), pi64]
    for name in EXPORTS:
        if name not in ("rpb_last_error", "rpb_launch_count"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def last_error():
    return load().rpb_last_error().decode()


def launch_count():
    """Kernel launches the library has enqueued so far (rpb_launch_count)."""
    return int(load().rpb_launch_count())


PEAK_KINDS = {"ffma2": 0, "ffma": 1, "dfma": 2}


def fma_peak(kind="ffma2"):
    """Measured fused-multiply-add rate of the current device (rpb_fma_peak): (TFLOP/s, ms per launch)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().rpb_fma_peak(PEAK_KINDS[kind], _stream(), ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def mobility_apply_noalloc(pos, F=None, T=None, a=1.0, eta=1.0, precision="fp64", out=None):
    """U = M_tt F + M_tr T without a context and without any allocation in the library
    (rpb_mobility_apply_noalloc), for callers that cannot allocate device memory; N <= NOALLOC_MAX_N.
    out must be given by such callers (it is allocated here only as a convenience)."""
    import torch

    n = pos.numel()
    out = torch.empty(n, dtype=torch.float64, device=pos.device) if out is None else out
    p = Params(float(a), float(eta), 0.0, PRECISIONS[precision])
    _check(load().rpb_mobility_apply_noalloc(n // 3, _ptr(pos, n, "pos"), _ptr(F, n, "F"), _ptr(T, n, "T"),
                                             _ptr(out, n, "U"), ctypes.byref(p), _stream()))
    return out


def _check(rc):
    if rc == RPB_OK:
        return
    msg = last_error()
    if rc == RPB_ENOCONV:
        raise NoConvergence(rc, msg)
    raise RpbError(rc, msg)


def _ptr(t, n=None, name="tensor"):
    """Device pointer of a contiguous float64 CUDA tensor (None passes through as NULL)."""
    if t is None:
        return None
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _force_params(weight, U0, b, torque):
    fp = ForceParams()
    fp.weight, fp.U0, fp.b = float(weight), float(U0), float(b)
    for k in range(3):
        fp.torque[k] = float(torque[k])
    return fp


class Context:
    """A library context (rpb_create) bound to the current CUDA device."""

    def __init__(self, max_N, a=1.0, eta=1.0, kT=1.0, precision="fp64", max_iter=64, wall=True):
        L = load()
        p = Params(float(a), float(eta), float(kT), PRECISIONS[precision], 1 if wall else 0)
        h = ctypes.c_void_p()
        _check(L.rpb_create(ctypes.byref(h), ctypes.byref(p), int(max_N), int(max_iter), _stream()))
        self._h = h
        self.max_N = int(max_N)
        self.max_iter = int(max_iter)
        self.params = dict(a=a, eta=eta, kT=kT, precision=precision)

    def close(self):
        if self._h:
            h, self._h = self._h, None  # never destroyed twice, even when destroy reports an error
            _check(load().rpb_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind_stream(self):
        _check(load().rpb_set_stream(self._h, _stream()))

    def set_periodic(self, Lx, Ly):
        """Pseudo-periodic boundaries with periods (Lx, Ly); (0, 0) switches them off (rpb_set_periodic)."""
        _check(load().rpb_set_periodic(self._h, float(Lx), float(Ly)))

    def set_preconditioner(self, kind):
        """Lanczos preconditioner: "none" (default) or "block-diagonal" (rpb_set_preconditioner)."""
        _check(load().rpb_set_preconditioner(self._h, PRECONDITIONERS[kind]))

    @staticmethod
    def _empty(n, like):
        import torch

        return torch.empty(n, dtype=torch.float64, device=like.device)

    def mobility_apply(self, pos, F=None, T=None, out=None):
        """U = M_tt F + M_tr T (rpb_mobility_apply)."""
        n = pos.numel()
        out = self._empty(n, pos) if out is None else out
        self._bind_stream()
        _check(load().rpb_mobility_apply(self._h, n // 3, _ptr(pos, n, "pos"), _ptr(F, n, "F"), _ptr(T, n, "T"),
                                         _ptr(out, n, "U")))
        return out

    def mobility_apply_rows(self, pos, F, T, row0, row1, out=None):
        """Rows row0 .. row1 - 1 of M_tt F + M_tr T, as a (3 (row1 - row0),) SoA tensor
        (rpb_mobility_apply_rows); row0 a multiple of 128."""
        n = pos.numel()
        nr = int(row1) - int(row0)
        out = self._empty(3 * nr, pos) if out is None else out
        self._bind_stream()
        _check(load().rpb_mobility_apply_rows(self._h, n // 3, _ptr(pos, n, "pos"), _ptr(F, n, "F"), _ptr(T, n, "T"),
                                              int(row0), int(row1), _ptr(out, 3 * nr, "U_rows")))
        return out

    def mobility_apply_part(self, pos, F, T, part, nparts, out=None):
        """Share `part` of `nparts` of M_tt F + M_tr T, a (3N,) SoA tensor (rpb_mobility_apply_part): the
        shares of parts 0 .. nparts - 1 add up to the product."""
        n = pos.numel()
        out = self._empty(n, pos) if out is None else out
        self._bind_stream()
        _check(load().rpb_mobility_apply_part(self._h, n // 3, _ptr(pos, n, "pos"), _ptr(F, n, "F"), _ptr(T, n, "T"),
                                              int(part), int(nparts), _ptr(out, n, "U")))
        return out

    def set_product_hook(self, fn):
        """Delegate every product of this context to fn(N, pos, F, T, U) -> int, called with raw device
        pointers (0 for a missing F or T) on the context's stream (rpb_set_product_hook); None
        restores the library's own products."""
        if fn is None:
            self._hook = None
            _check(load().rpb_set_product_hook(self._h, PRODUCT_HOOK(), None))
            return
        self._hook = PRODUCT_HOOK(lambda user, N, pos, F, T, U: fn(int(N), pos or 0, F or 0, T or 0, U or 0))
        _check(load().rpb_set_product_hook(self._h, self._hook, None))

    def mobility_apply2(self, pos, F, T, P, out=None, out2=None):
        """(M_tt F + M_tr T, M_tt P) at the same positions, in one pass where the context can
        (rpb_mobility_apply2)."""
        n = pos.numel()
        out = self._empty(n, pos) if out is None else out
        out2 = self._empty(n, pos) if out2 is None else out2
        self._bind_stream()
        _check(load().rpb_mobility_apply2(self._h, n // 3, _ptr(pos, n, "pos"), _ptr(F, n, "F"), _ptr(T, n, "T"),
                                          _ptr(P, n, "P"), _ptr(out, n, "U"), _ptr(out2, n, "U2")))
        return out, out2

    def lanczos_sqrt_apply(self, pos, W, tol=1e-3, max_iter=None, out=None, raise_on_noconv=True):
        """g ~ M^{1/2} W (rpb_lanczos_sqrt_apply); returns (g, iterations, eps, converged)."""
        n = pos.numel()
        out = self._empty(n, pos) if out is None else out
        it = ctypes.c_int(0)
        err = ctypes.c_double(0.0)
        self._bind_stream()
        rc = load().rpb_lanczos_sqrt_apply(self._h, n // 3, _ptr(pos, n, "pos"), _ptr(W, n, "W"), _ptr(out, n, "g"),
                                           float(tol), int(max_iter or self.max_iter), ctypes.byref(it),
                                           ctypes.byref(err))
        if rc == RPB_ENOCONV and not raise_on_noconv:
            return out, it.value, err.value, False
        _check(rc)
        return out, it.value, err.value, True

    def rfd_drift(self, pos, Wt, delta=1e-6, out=None):
        n = pos.numel()
        out = self._empty(n, pos) if out is None else out
        self._bind_stream()
        _check(load().rpb_rfd_drift(self._h, n // 3, _ptr(pos, n, "pos"), _ptr(Wt, n, "Wt"), float(delta),
                                    _ptr(out, n, "drift")))
        return out

    def forces(self, pos, weight=1.0, U0=1.0, b=0.1, torque=(0.0, 1.0, 0.0), out=None):
        n = pos.numel()
        out = self._empty(n, pos) if out is None else out
        fp = _force_params(weight, U0, b, torque)
        self._bind_stream()
        _check(load().rpb_forces(self._h, n // 3, _ptr(pos, n, "pos"), ctypes.byref(fp), _ptr(out, n, "F")))
        return out

    def philox_normal(self, N, seed, step, stream_id, instance=0, out=None, device="cuda"):
        import torch

        out = torch.empty(3 * N, dtype=torch.float64, device=device) if out is None else out
        self._bind_stream()
        _check(load().rpb_philox_normal(self._h, int(N), int(seed), int(step), int(stream_id), int(instance),
                                        _ptr(out, 3 * N, "out")))
        return out

    def ab_step(self, pos, U_prev, step, seed, dt=0.01, delta=1e-6, tol=1e-3, max_iter=None, weight=1.0, U0=1.0,
                b=0.1, torque=(0.0, 1.0, 0.0), raise_on_noconv=True):
        """One stochastic Adams-Bashforth step in place (rpb_ab_step); returns the step statistics."""
        n = pos.numel()
        fp = _force_params(weight, U0, b, torque)
        stats = StepStats()
        self._bind_stream()
        rc = load().rpb_ab_step(self._h, n // 3, _ptr(pos, n, "pos"), _ptr(U_prev, n, "U_prev"), int(step),
                                int(seed), float(dt), float(delta), float(tol), int(max_iter or self.max_iter),
                                ctypes.byref(fp), ctypes.byref(stats))
        if not (rc == RPB_ENOCONV and not raise_on_noconv):
            _check(rc)
        return dict(m=stats.lanczos_iters, eps=stats.lanczos_err, converged=bool(stats.converged))

    def step(self, pos, U_prev, step, seed, scheme="AB", rfd="centred", dt=0.01, delta=1e-6, tol=1e-3,
             max_iter=None, weight=1.0, U0=1.0, b=0.1, torque=(0.0, 1.0, 0.0), raise_on_noconv=True):
        """One time step in place with the chosen integrator ("AB" or "EM") and RFD difference
        ("centred" or "one-sided") (rpb_step); returns the step statistics."""
        n = pos.numel()
        fp = _force_params(weight, U0, b, torque)
        opts = StepOptions(SCHEMES[scheme], RFDS[rfd])
        stats = StepStats()
        self._bind_stream()
        rc = load().rpb_step(self._h, n // 3, _ptr(pos, n, "pos"), _ptr(U_prev, n, "U_prev"), int(step), int(seed),
                             float(dt), float(delta), float(tol), int(max_iter or self.max_iter), ctypes.byref(fp),
                             ctypes.byref(opts), ctypes.byref(stats))
        if not (rc == RPB_ENOCONV and not raise_on_noconv):
            _check(rc)
        return dict(m=stats.lanczos_iters, eps=stats.lanczos_err, converged=bool(stats.converged))

    def run(self, pos, U_prev, step, seed, nsteps, scheme="AB", rfd="centred", dt=0.01, delta=1e-6, tol=1e-3,
            max_iter=None, weight=1.0, U0=1.0, b=0.1, torque=(0.0, 1.0, 0.0), raise_on_noconv=True):
        """nsteps time steps in place from one launch of a CUDA graph (a loop node around the step) with
        the Lanczos stop decided on the device (rpb_run); the same results as nsteps calls of step().  Returns (last step's statistics,
        number of steps whose Lanczos did not converge)."""
        n = pos.numel()
        fp = _force_params(weight, U0, b, torque)
        opts = StepOptions(SCHEMES[scheme], RFDS[rfd])
        stats = StepStats()
        unconv = ctypes.c_int64(0)
        self._bind_stream()
        rc = load().rpb_run(self._h, n // 3, _ptr(pos, n, "pos"), _ptr(U_prev, n, "U_prev"), int(step), int(seed),
                            int(nsteps), float(dt), float(delta), float(tol), int(max_iter or self.max_iter),
                            ctypes.byref(fp), ctypes.byref(opts), ctypes.byref(stats), ctypes.byref(unconv))
        if not (rc == RPB_ENOCONV and not raise_on_noconv):
            _check(rc)
        return (dict(m=stats.lanczos_iters, eps=stats.lanczos_err, converged=bool(stats.converged)),
                int(unconv.value))


class BatchContext:
    """A ragged-batch context (rpb_batch_create): one call advances many independent suspensions,
    each kept in its own (3 N_b,) float64 CUDA tensors."""

    def __init__(self, max_total_N, max_B, a=1.0, eta=1.0, kT=1.0, precision="fp32", max_iter=64):
        L = load()
        p = Params(float(a), float(eta), float(kT), PRECISIONS[precision])
        h = ctypes.c_void_p()
        _check(L.rpb_batch_create(ctypes.byref(h), ctypes.byref(p), int(max_total_N), int(max_B), int(max_iter),
                                  _stream()))
        self._h = h
        self.max_total_N = int(max_total_N)
        self.max_B = int(max_B)
        self.max_iter = int(max_iter)
        self.params = dict(a=a, eta=eta, kT=kT, precision=precision)

    def close(self):
        if self._h:
            h, self._h = self._h, None  # never destroyed twice, even when destroy reports an error
            _check(load().rpb_batch_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind_stream(self):
        _check(load().rpb_batch_set_stream(self._h, _stream()))

    @staticmethod
    def _ptrs(ts, name, nullable=False):
        if ts is None:
            if nullable:
                return None
            raise ValueError(f"{name} is required")
        arr = (ctypes.c_void_p * len(ts))()
        for k, t in enumerate(ts):
            arr[k] = _ptr(t, None, f"{name}[{k}]").value
        return arr

    def mobility_apply(self, pos, F=None, T=None, out=None):
        """U_b = M_tt F_b + M_tr T_b for each instance (rpb_batch_mobility_apply); lists of tensors."""
        import torch

        B = len(pos)
        Ns = (ctypes.c_int64 * B)(*[p.numel() // 3 for p in pos])
        out = [torch.empty_like(p) for p in pos] if out is None else out
        self._bind_stream()
        _check(load().rpb_batch_mobility_apply(self._h, B, Ns, self._ptrs(pos, "pos"), self._ptrs(F, "F", True),
                                               self._ptrs(T, "T", True), self._ptrs(out, "U")))
        return out

    def set_tiles(self, seg_tiles=8, ctas_per_sm=5, symmetric=True):
        """Tile schedule of the float32 products (rpb_batch_set_tiles)."""
        t = BatchTiles(int(seg_tiles), int(ctas_per_sm), 1 if symmetric else 0)
        _check(load().rpb_batch_set_tiles(self._h, ctypes.byref(t)))

    def get_tiles(self):
        t = BatchTiles()
        _check(load().rpb_batch_get_tiles(self._h, ctypes.byref(t)))
        return t.as_dict()

    def tune(self, pos, reps=3):
        """Time every candidate tile schedule on this batch and keep the fastest (rpb_batch_tune);
        returns dict(best=..., candidates=[(schedule, weighted ms), ...])."""
        B = len(pos)
        Ns = (ctypes.c_int64 * B)(*[p.numel() // 3 for p in pos])
        best = BatchTiles()
        cand = (BatchTiles * 16)()
        ms = (ctypes.c_double * 16)()
        nc = ctypes.c_int(0)
        self._bind_stream()
        _check(load().rpb_batch_tune(self._h, B, Ns, self._ptrs(pos, "pos"), int(reps), ctypes.byref(best), 16, cand,
                                     ms, ctypes.byref(nc)))
        return dict(best=best.as_dict(), candidates=[(cand[k].as_dict(), ms[k]) for k in range(min(nc.value, 16))])

    def ab_step(self, pos, U_prev, steps, seeds, dt=0.01, delta=1e-6, tol=1e-3, max_iter=None, weight=1.0, U0=1.0,
                b=0.1, torque=(0.0, 1.0, 0.0), raise_on_noconv=True):
        """One AB step of every instance in place (rpb_batch_ab_step); returns per-instance statistics."""
        B = len(pos)
        Ns = (ctypes.c_int64 * B)(*[p.numel() // 3 for p in pos])
        st = (ctypes.c_int64 * B)(*[int(s) for s in steps])
        sd = (ctypes.c_uint64 * B)(*[int(s) for s in seeds])
        stats = (StepStats * B)()
        fp = _force_params(weight, U0, b, torque)
        self._bind_stream()
        rc = load().rpb_batch_ab_step(self._h, B, Ns, self._ptrs(pos, "pos"), self._ptrs(U_prev, "U_prev"), st, sd,
                                      float(dt), float(delta), float(tol), int(max_iter or self.max_iter),
                                      ctypes.byref(fp), stats)
        if not (rc == RPB_ENOCONV and not raise_on_noconv):
            _check(rc)
        return [dict(m=s.lanczos_iters, eps=s.lanczos_err, converged=bool(s.converged)) for s in stats]

    def run(self, pos, U_prev, steps, seeds, nsteps, lanczos_iters=16, dt=0.01, delta=1e-6, tol=1e-3, weight=1.0,
            U0=1.0, b=0.1, torque=(0.0, 1.0, 0.0), raise_on_noconv=True):
        """nsteps AB steps of every instance with the step replayed from a CUDA graph (rpb_batch_run);
        returns (last step's statistics, number of unconverged instance-steps)."""
        B = len(pos)
        Ns = (ctypes.c_int64 * B)(*[p.numel() // 3 for p in pos])
        st = (ctypes.c_int64 * B)(*[int(s) for s in steps])
        sd = (ctypes.c_uint64 * B)(*[int(s) for s in seeds])
        stats = (StepStats * B)()
        unconv = ctypes.c_int64(0)
        fp = _force_params(weight, U0, b, torque)
        self._bind_stream()
        rc = load().rpb_batch_run(self._h, B, Ns, self._ptrs(pos, "pos"), self._ptrs(U_prev, "U_prev"), st, sd,
                                  int(nsteps), float(dt), float(delta), float(tol), int(lanczos_iters),
                                  ctypes.byref(fp), stats, ctypes.byref(unconv))
        if not (rc == RPB_ENOCONV and not raise_on_noconv):
            _check(rc)
        return [dict(m=s.lanczos_iters, eps=s.lanczos_err, converged=bool(s.converged)) for s in stats], unconv.value
