"""ctypes binding of libtwa (include/twa.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module loads it, converts
Python arguments to C types and turns status codes into exceptions. PyTorch is
used only for device buffers and the current CUDA stream. If libtwa.so is
missing the import of ``lib()`` fails loudly: there is no CPU fallback.
"""
import ctypes
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtwa.so")

TWA_OK = 0
ERRORS = {-1: "TWA_EINVAL", -2: "TWA_ENOTPSD", -3: "TWA_ENOMEM", -4: "TWA_ECUDA", -5: "TWA_ETIMEOUT",
          -6: "TWA_ENONFINITE", -7: "TWA_ESTATE", -8: "TWA_EUNSUPPORTED"}
PRECISION = {"fp64": 0, "bf16": 1, "bf16x3": 2, "tf32": 3, "fp32": 4, "bf16x2": 5, "bf16l2": 6, "bf16b": 7}


class TWAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code
        self.name = ERRORS.get(code, "?")


# twa_alloc_fn / twa_free_fn of include/twa.h
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("init_state", ctypes.c_int), ("window_start", ctypes.c_double),
                ("renormalize", ctypes.c_int), ("clip_negative", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("traj_offset", ctypes.c_int64), ("ws_route", ctypes.c_int), ("noise_route", ctypes.c_int),
                ("sample_stride", ctypes.c_int64), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", ctypes.c_void_p), ("integrator", ctypes.c_int)]


def torch_allocator():
    """(alloc, free) C callbacks that take a context's device memory from
    torch's caching allocator, on the stream the library passes. Keep the
    returned pair alive as long as the context (TWA does that itself)."""
    import torch

    def alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ALLOC_FN(alloc), FREE_FN(free)


def _allocator(allocator):
    """None, "torch", or a pair (alloc(nbytes, stream) -> int, free(ptr, stream))."""
    if allocator is None:
        return None
    if allocator == "torch":
        return torch_allocator()
    a, f = allocator
    return (ALLOC_FN(lambda n, s, u: a(int(n), int(s or 0)) or None),
            FREE_FN(lambda p, s, u: f(int(p), int(s or 0))))


ROUTE = {"dense": 0, "fft": 1, "resident": 2}
RESIDENT_MAX_N = 512
NOISE = {"cholesky": 0, "circulant": 1}
INTEGRATOR = {"heun": 0, "midpoint": 1}


class Obs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("Sz", "Sz_se", "sigma_z", "sigma_z_se", "SpSm", "SpSm_se",
                                                  "G2num", "G2num_se", "g2", "g2_se")] + \
               [(n, ctypes.c_int64) for n in ("M", "steps", "samples")] + \
               [(n, ctypes.c_double) for n in ("w_max", "w_min", "w_tilde", "stability", "min_pivot")] + \
               [(n, ctypes.c_int64) for n in ("clipped", "nonfinite")] + [("factor_residual", ctypes.c_double)] + \
               [(n, ctypes.c_int64) for n in ("fft_length", "fft_ctas")]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class GradReq(ctypes.Structure):
    _fields_ = [("objective", ctypes.c_int), ("want_alpha", ctypes.c_int), ("M", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("checkpoint", ctypes.c_int64)]


class GradOut(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("J", "dJ_dw", "dJ_dw_se", "dJ_dalpha", "dJ_dalpha_se")] + \
               [(n, ctypes.c_int64) for n in ("M", "steps", "samples")] + [("mu", ctypes.c_double * 5)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "mu"}
        d["mu"] = list(self.mu)
        return d


OBJECTIVE = {"SpSm": 0, "g2": 1}
MATRIX = {"W": 0, "L": 1}


class Point(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("alpha", ctypes.c_double), ("w", ctypes.c_double),
                ("Gamma", ctypes.c_double), ("dt", ctypes.c_double), ("steps", ctypes.c_int64),
                ("window_start", ctypes.c_double), ("means", ctypes.c_void_p)]

class CorrReq(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("prep_steps", ctypes.c_int64), ("lag_steps", ctypes.c_int64),
                ("lag_stride", ctypes.c_int64), ("eps", ctypes.c_double), ("n_omega", ctypes.c_int64),
                ("omega_max", ctypes.c_double)]


class CorrOut(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("n_lags", ctypes.c_int64)] + \
               [(n, ctypes.c_double) for n in ("dtau", "fwhm", "fwhm_se", "omega_peak", "S_peak", "spsm_tau0")]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_SIGNATURES = {
    "twa_version": (ctypes.c_char_p, []),
    "twa_opts_default": (ctypes.c_int, [ctypes.POINTER(Opts)]),
    "twa_init": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.POINTER(Opts)]),
    "twa_run": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64]),
    "twa_sync": (ctypes.c_int, [_P]),
    "twa_observables": (ctypes.c_int, [_P, ctypes.POINTER(Obs)]),
    "twa_get_state": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
    "twa_set_state": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, ctypes.c_int]),
    "twa_get_state_f32": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
    "twa_set_state_f32": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, ctypes.c_int]),
    "twa_get_moments": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "twa_field": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64]),
    "twa_contract": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int64]),
    "twa_reduce_moments": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(Obs)]),
    "twa_reduce_moments_noalloc": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(Obs)]),
    "twa_grad": (ctypes.c_int, [_P, ctypes.POINTER(GradReq), ctypes.POINTER(GradOut), _P]),
    "twa_batch_run": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(Opts),
                                     _P, _P]),
    "twa_correlation": (ctypes.c_int, [_P, ctypes.POINTER(CorrReq), ctypes.POINTER(CorrOut), _P, _P, _P, _P]),
    "twa_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "twa_wait_probe": (ctypes.c_int, [_P, ctypes.c_int64]),
    "twa_profile_read": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "twa_last_error": (ctypes.c_char_p, [_P]),
    "twa_destroy": (None, [_P]),
}


def lib():
    """Load libtwa.so (built in-tree by paper_2608_10075_b300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libtwa.so not built: run `python -m paper_2608_10075_b300.build` (%s)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error(ctx=None):
    return lib().twa_last_error(ctx).decode()


def _ptr(x, dtype="float64"):
    """Device or host address of a torch tensor / numpy array (contiguous, of
    element type `dtype`)."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(x.dtype) != "torch." + dtype:
            raise ValueError("expected a %s tensor" % dtype)
        return ctypes.c_void_p(x.data_ptr()), bool(x.is_cuda)
    import numpy as np
    if not (isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"] and x.dtype == np.dtype(dtype)):
        raise ValueError("expected a C-contiguous %s numpy array or a torch tensor" % dtype)
    return ctypes.c_void_p(x.ctypes.data), False


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class TWA:
    """One context of the C library: parameters, pump matrix, factor, trajectories.

    Mirrors twa_init / twa_run / twa_observables; see include/twa.h.
    """

    def __init__(self, N, alpha, w, Gamma, dt, seed=0, precision="fp64", init_state=-1, window_start=0.0,
                 renormalize=True, clip_negative=False, stream=None, traj_offset=0, ws_route="dense",
                 noise_route="cholesky", sample_stride=1, allocator=None, integrator="heun"):
        L = lib()
        o = Opts()
        L.twa_opts_default(ctypes.byref(o))
        o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        o.init_state = int(init_state)
        o.window_start = float(window_start)
        o.renormalize = 1 if renormalize else 0
        o.clip_negative = 1 if clip_negative else 0
        o.stream = _stream_handle(stream)
        o.traj_offset = int(traj_offset)
        o.ws_route = ROUTE[ws_route] if isinstance(ws_route, str) else int(ws_route)
        o.noise_route = NOISE[noise_route] if isinstance(noise_route, str) else int(noise_route)
        o.sample_stride = int(sample_stride)
        o.integrator = INTEGRATOR[integrator] if isinstance(integrator, str) else int(integrator)
        # device memory from the caller's allocator (kept alive with the context)
        self._alloc = _allocator(allocator)
        if self._alloc is not None:
            o.alloc, o.free = self._alloc
        self._stream = stream
        h = ctypes.c_void_p()
        a = float(alpha)
        rc = L.twa_init(ctypes.byref(h), int(N), a, float(w), float(Gamma), float(dt),
                        int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(o))
        if rc != TWA_OK:
            raise TWAError(rc, last_error(None))
        self._h = h
        self.N, self.alpha, self.w, self.Gamma, self.dt = int(N), a, float(w), float(Gamma), float(dt)
        self.seed, self.precision = int(seed), precision
        self.M = None

    def _check(self, rc):
        if rc != TWA_OK:
            raise TWAError(rc, last_error(self._h))

    def run(self, M, steps):
        self._check(lib().twa_run(self._h, int(M), int(steps)))
        self.M = int(M)
        return self

    def sync(self):
        self._check(lib().twa_sync(self._h))

    def observables(self):
        o = Obs()
        self._check(lib().twa_observables(self._h, ctypes.byref(o)))
        return o.as_dict()

    def get_state(self, out=None, device=None):
        """Spins as three [M][N] float64 arrays: torch CUDA tensors when `device`
        is given (or `out` holds CUDA tensors), numpy arrays otherwise."""
        M, N = self.M, self.N
        if out is None:
            if device is not None:
                import torch
                out = tuple(torch.empty((M, N), dtype=torch.float64, device=device) for _ in range(3))
            else:
                import numpy as np
                out = tuple(np.empty((M, N)) for _ in range(3))
        (px, dx), (py, _), (pz, _) = (_ptr(a) for a in out)
        self._check(lib().twa_get_state(self._h, px, py, pz, 1 if dx else 0))
        return out

    def set_state(self, sx, sy, sz):
        """Replace the spins from three [M][N] arrays (numpy or torch, host or
        CUDA): float64 through twa_set_state, float32 through twa_set_state_f32."""
        f32 = str(sx.dtype).endswith("float32")
        (px, dx), (py, _), (pz, _) = (_ptr(a, "float32" if f32 else "float64") for a in (sx, sy, sz))
        M = int(sx.shape[0])
        fn = lib().twa_set_state_f32 if f32 else lib().twa_set_state
        self._check(fn(self._h, M, px, py, pz, 1 if dx else 0))
        self.M = M

    def get_state_f32(self, out=None, device=None):
        """Spins as three [M][N] float32 arrays (twa_get_state_f32; tensor-core
        precisions): torch CUDA tensors when `device` is given, numpy otherwise."""
        M, N = self.M, self.N
        if out is None:
            if device is not None:
                import torch
                out = tuple(torch.empty((M, N), dtype=torch.float32, device=device) for _ in range(3))
            else:
                import numpy as np
                out = tuple(np.empty((M, N), dtype=np.float32) for _ in range(3))
        (px, dx), (py, _), (pz, _) = (_ptr(a, "float32") for a in out)
        self._check(lib().twa_get_state_f32(self._h, px, py, pz, 1 if dx else 0))
        return out

    def moments(self):
        """Per-trajectory window means [M][5]: S^z, A, A^2, A S^z, (S^z)^2."""
        import numpy as np
        out = np.empty((self.M, 5))
        self._check(lib().twa_get_moments(self._h, ctypes.c_void_p(out.ctypes.data), 0))
        return out

    def field(self, s, out=None):
        """P[k] = W s[k] for a CUDA float64 tensor s of shape [K][N]."""
        import torch
        if out is None:
            out = torch.empty_like(s)
        (ps, ds), (po, do) = _ptr(s), _ptr(out)
        if not (ds and do):
            raise ValueError("field() takes CUDA tensors")
        self._check(lib().twa_field(self._h, ps, po, int(s.shape[0])))
        return out

    def contract(self, s, matrix="W", out=None):
        """P[k] = A s[k] for a CUDA float64 tensor s of shape [K][N], A = W
        (matrix="W") or the noise factor L (matrix="L"), in the arithmetic of
        the context's step (twa_contract)."""
        import torch
        if out is None:
            out = torch.empty_like(s)
        (ps, ds), (po, do) = _ptr(s), _ptr(out)
        if not (ds and do):
            raise ValueError("contract() takes CUDA tensors")
        self._check(lib().twa_contract(self._h, MATRIX[matrix], ps, po, int(s.shape[0])))
        return out

    def grad(self, objective, M, steps, checkpoint=64, want_alpha=True, per_traj=False):
        """Pathwise dJ/dw and dJ/dalpha at fixed noise (twa_grad). With per_traj,
        also the [M][2] per-trajectory samples whose mean is the derivative."""
        import numpy as np
        r = GradReq(OBJECTIVE[objective], 1 if want_alpha else 0, int(M), int(steps), int(checkpoint))
        o = GradOut()
        buf = np.empty((int(M), 2)) if per_traj else None
        p = ctypes.c_void_p(buf.ctypes.data) if per_traj else None
        self._check(lib().twa_grad(self._h, ctypes.byref(r), ctypes.byref(o), p))
        d = o.as_dict()
        if per_traj:
            d["per_traj"] = buf
        return d

    def correlation(self, M, prep_steps, lag_steps, lag_stride, eps, n_omega, omega_max):
        """Two-time correlation, spectrum and linewidth (twa_correlation).
        Returns a dict: the twa_corr_out fields, "C" (complex [n_lags]),
        "C_se" ([n_lags][2]), "S" ([n_omega]), "omega" ([n_omega]), "parts"
        ([n_lags][8])."""
        import numpy as np
        r = CorrReq(int(M), int(prep_steps), int(lag_steps), int(lag_stride), float(eps), int(n_omega),
                    float(omega_max))
        # buffers sized for a valid request; the library rejects the others
        n_lags = 1 + max(int(lag_steps), 0) // max(int(lag_stride), 1)
        C = np.empty((n_lags, 2))
        Cse = np.empty((n_lags, 2))
        S = np.empty(max(int(n_omega), 1))
        parts = np.empty((n_lags, 8))
        o = CorrOut()
        self._check(lib().twa_correlation(self._h, ctypes.byref(r), ctypes.byref(o), ctypes.c_void_p(C.ctypes.data),
                                          ctypes.c_void_p(S.ctypes.data), ctypes.c_void_p(parts.ctypes.data),
                                          ctypes.c_void_p(Cse.ctypes.data)))
        d = o.as_dict()
        d.update(C=C[:, 0] + 1j * C[:, 1], C_se=Cse, S=S, parts=parts,
                 omega=np.array([-omega_max + j * (2.0 * omega_max / (n_omega - 1)) for j in range(n_omega - 1)]
                                + [omega_max]))
        return d

    def wait_probe(self, limit_us):
        """Enqueue one bounded device wait that runs out (twa_wait_probe); the
        next synchronising call raises TWA_ETIMEOUT."""
        self._check(lib().twa_wait_probe(self._h, int(limit_us)))

    def profile(self, enable=True):
        self._check(lib().twa_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{kind: (total ms, launches, tensor-core FLOPs issued, algorithmic
        FLOPs)} of the kernels timed since profile()."""
        ms = (ctypes.c_double * len(PROF_KINDS))()
        n = (ctypes.c_int64 * len(PROF_KINDS))()
        fl = (ctypes.c_double * len(PROF_KINDS))()
        fa = (ctypes.c_double * len(PROF_KINDS))()
        self._check(lib().twa_profile_read(self._h, ms, n, fl, fa))
        return {k: (ms[i], n[i], fl[i], fa[i]) for i, k in enumerate(PROF_KINDS)}

    def close(self):
        if getattr(self, "_h", None):
            lib().twa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


PROF_KINDS = ("noise", "predict", "correct", "close", "gemm64", "elem64", "noise_factor", "resident")


def reduce_moments(means, N):
    """Observables of per-trajectory window means [M][5] (host float64), e.g. the
    concatenated shards of one ensemble, reduced on the device."""
    import numpy as np
    a = np.ascontiguousarray(means, dtype=np.float64)
    o = Obs()
    rc = lib().twa_reduce_moments(ctypes.c_void_p(a.ctypes.data), int(a.shape[0]), int(N), ctypes.byref(o))
    if rc != TWA_OK:
        raise TWAError(rc, last_error(None))
    return o.as_dict()


def batch_run(points, M, seed=0, precision="bf16x3", stream=None, allocator=None, integrator="heun",
              means=False, ws_route="dense"):
    """twa_batch_run: points = list of dicts with N, alpha, w, Gamma, dt, steps,
    window_start. Returns (list of observables dicts, (BN, K-stage config));
    with means=True every dict also holds "means", the point's per-trajectory
    window means [M][5]."""
    import numpy as np
    arr = (Point * len(points))()
    bufs = [np.empty((int(M), 5)) if means else None for _ in points]
    for k, p in enumerate(points):
        arr[k] = Point(int(p["N"]), float(p["alpha"]), float(p["w"]), float(p["Gamma"]), float(p["dt"]),
                       int(p["steps"]), float(p.get("window_start", 0.0)),
                       ctypes.c_void_p(bufs[k].ctypes.data) if means else None)
    o = Opts()
    lib().twa_opts_default(ctypes.byref(o))
    o.precision = PRECISION[precision]
    o.integrator = INTEGRATOR[integrator]
    o.ws_route = ROUTE[ws_route]
    o.stream = _stream_handle(stream)
    alloc = _allocator(allocator)
    if alloc is not None:
        o.alloc, o.free = alloc
    out = (Obs * len(points))()
    tiles = (ctypes.c_int * 2)()
    rc = lib().twa_batch_run(ctypes.cast(arr, ctypes.c_void_p), len(points), int(M), int(seed) & (2 ** 64 - 1),
                             ctypes.byref(o), ctypes.cast(out, ctypes.c_void_p), ctypes.cast(tiles, ctypes.c_void_p))
    if rc != TWA_OK:
        raise TWAError(rc, last_error(None))
    res = [x.as_dict() for x in out]
    if means:
        for d, b in zip(res, bufs):
            d["means"] = b
    return res, (tiles[0], tiles[1])


NOALLOC_MAX_M = 65536


def reduce_moments_noalloc(means, N):
    """Same as reduce_moments, for callers that cannot allocate device memory:
    the library stages the data in a fixed device array of NOALLOC_MAX_M
    trajectories (see twa_reduce_moments_noalloc in include/twa.h). Calls on one
    device share that array, so concurrent callers must serialise."""
    import numpy as np
    a = np.ascontiguousarray(means, dtype=np.float64)
    o = Obs()
    rc = lib().twa_reduce_moments_noalloc(ctypes.c_void_p(a.ctypes.data), int(a.shape[0]), int(N), ctypes.byref(o))
    if rc != TWA_OK:
        raise TWAError(rc, last_error(None))
    return o.as_dict()


def header_functions():
    """Names of the functions include/twa.h declares (for the export check)."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "twa.h")
    with open(hdr) as f:
        return re.findall(r"^TWA_API [^(]*?\b(twa_\w+)\(", f.read(), flags=re.M)


INF = math.inf
