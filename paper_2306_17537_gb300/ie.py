"""Thin ctypes binding of the C ABI in ``include/ie.h`` (argument marshalling only).

Every function here forwards to the same-named ``extern "C"`` entry point of ``libie_gb300.so``;
all computation happens in that library's CUDA kernels. Host arrays are numpy arrays (complex
fields as complex128, interleaved re/im like the ABI); device arrays are anything exposing a device
pointer via ``data_ptr()`` (torch tensors) or a plain integer address. Importing this module loads
the library and raises ``ImportError`` if it has not been built (``__graft_entry__.build()``):
there is no fallback path.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libie_gb300.so")

IE_OK, IE_EINVAL, IE_ENOMEM, IE_ECUDA, IE_ENOCONV, IE_ESTATE = range(6)
IE_DD_NONE, IE_DD_JACOBI, IE_DD_GAUSS_SEIDEL = range(3)
IE_PREC_MIXED, IE_PREC_FP64, IE_PREC_DFLOAT = range(3)
IE_MAX_HISTORY = 128
KERNEL_CLASSES = ("P1_c64", "P2_c64", "P3_c64", "P4_c64", "P5_c64", "P1_c128", "P2_c128", "P3_c128", "P4_c128",
                  "P5_c128", "dots", "update", "krylov_misc", "field", "setup")
STATUS_NAMES = {0: "IE_OK", 1: "IE_EINVAL", 2: "IE_ENOMEM", 3: "IE_ECUDA", 4: "IE_ENOCONV", 5: "IE_ESTATE"}


class ie_grid(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32), ("origin", ct.c_double * 3)]


class ie_dipole(ct.Structure):
    _fields_ = [("pos", ct.c_double * 3), ("moment", ct.c_double * 3)]


class ie_opts(ct.Structure):
    _fields_ = [("n_blocks", ct.c_int32), ("z_split", ct.POINTER(ct.c_int32)), ("restart", ct.c_int32),
                ("max_outer", ct.c_int32), ("max_inner", ct.c_int32), ("precision", ct.c_int32),
                ("adaptive", ct.c_int32), ("fixed_tol", ct.c_double), ("contraction", ct.c_int32),
                ("graph", ct.c_int32), ("outer_krylov", ct.c_int32), ("outer_restart", ct.c_int32),
                ("outer_inner_tol", ct.c_double), ("concurrent_blocks", ct.c_int32)]


class ie_batch_item(ct.Structure):
    _fields_ = [("ctx", ct.c_void_p), ("sigma6", ct.POINTER(ct.c_double)), ("n_src", ct.c_int32),
                ("src", ct.POINTER(ie_dipole)), ("n_rx", ct.c_int32), ("rx_xyz", ct.POINTER(ct.c_double)),
                ("dd_mode", ct.c_int32), ("tol", ct.c_double), ("opts", ct.POINTER(ie_opts)),
                ("H_out", ct.POINTER(ct.c_double)), ("info", ct.c_void_p), ("status", ct.c_int),
                ("E_init_dev", ct.c_void_p)]


class ie_info(ct.Structure):
    _fields_ = [("outer_iters", ct.c_int32), ("gmres_iters_total", ct.c_int32), ("matvecs", ct.c_int32),
                ("n_history", ct.c_int32), ("final_rel_residual", ct.c_double), ("seconds", ct.c_double),
                ("residual_history", ct.c_double * IE_MAX_HISTORY),
                ("sweep_gmres_iters", ct.c_int32 * IE_MAX_HISTORY), ("reorth_passes", ct.c_int32),
                ("warm_start_used", ct.c_int32), ("cold_rel_residual", ct.c_double),
                ("warm_rel_residual", ct.c_double), ("active_blocks", ct.c_int32)]

    def history(self):
        return list(self.residual_history[: self.n_history])


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
_lib = ct.CDLL(LIB_PATH)

_P = ct.c_void_p
_D = ct.POINTER(ct.c_double)
_SIGS = {
    "ie_default_opts": (None, [ct.POINTER(ie_opts)]),
    "ie_create": (ct.c_int, [ct.POINTER(ie_grid), ct.c_double, ct.c_double, ct.c_double, ct.POINTER(_P)]),
    "ie_set_stream": (ct.c_int, [_P, _P]),
    "ie_set_contrast": (ct.c_int, [_P, _D]),
    "ie_set_contrast_dev": (ct.c_int, [_P, _P]),
    "ie_solve": (ct.c_int, [_P, ct.c_int32, ct.POINTER(ie_dipole), ct.c_int32, _D, ct.c_int32, ct.c_double,
                            ct.POINTER(ie_opts), _D, ct.POINTER(ie_info)]),
    "ie_get_field": (ct.c_int, [_P, _D]),
    "ie_get_field_dev": (ct.c_int, [_P, _P]),
    "ie_incident_field_dev": (ct.c_int, [_P, ct.POINTER(ie_dipole), _P]),
    "ie_set_initial_field_dev": (ct.c_int, [_P, _P]),
    "ie_solve_batch": (ct.c_int, [ct.c_int32, ct.POINTER(ie_batch_item), ct.c_int32]),
    "ie_matvec": (ct.c_int, [_P, ct.c_int32, ct.c_int32, ct.c_int32, _D, _D]),
    "ie_matvec_dev": (ct.c_int, [_P, ct.c_int32, ct.c_int32, _P, _P]),
    "ie_matvec_contraction": (ct.c_int, [_P, ct.c_int32, ct.c_int32, ct.c_int32, _D, _D]),
    "ie_matvec_dev_noalloc": (ct.c_int, [_P, ct.c_int32, ct.c_int32, _P, _P]),
    "ie_interaction": (ct.c_int, [_P, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, _D, _D]),
    "ie_gmres": (ct.c_int, [_P, ct.c_int32, ct.c_int32, ct.c_int32, _D, _D, ct.c_double, ct.c_int32, ct.c_int32, _D,
                            ct.POINTER(ct.c_int32), _D]),
    "ie_green_spectrum": (ct.c_int, [_P, ct.c_int32, ct.c_int32, _D, ct.POINTER(ct.c_int32)]),
    "ie_incident_field": (ct.c_int, [_P, ct.POINTER(ie_dipole), _D]),
    "ie_receiver_fields": (ct.c_int, [_P, _D, ct.POINTER(ie_dipole), ct.c_int32, _D, _D]),
    "ie_fft_dims": (ct.c_int, [_P, ct.c_int32, ct.POINTER(ct.c_int32)]),
    "ie_profile_enable": (ct.c_int, [_P, ct.c_int32]),
    "ie_profile_read": (ct.c_int, [_P, ct.c_int32, ct.POINTER(ct.c_int64), _D, _D]),
    "ie_tuned_tiles": (ct.c_int32, [ct.c_char_p, ct.c_int32]),
    "ie_last_error": (ct.c_char_p, [_P]),
    "ie_debug_fail_allocation": (None, [ct.c_int32]),
    "ie_debug_force_tile": (ct.c_int32, [ct.c_int32, ct.c_int32]),
    "ie_destroy": (None, [_P]),
    # include/ie_fno.h
    "ie_fno_create": (ct.c_int, [ct.c_int32] * 9 + [ct.POINTER(_P)]),
    "ie_fno_param_count": (ct.c_int64, [_P]),
    "ie_fno_set_stream": (ct.c_int, [_P, _P]),
    "ie_fno_set_tensor_cores": (ct.c_int, [_P, ct.c_int32]),
    "ie_fno_set_params": (ct.c_int, [_P, ct.POINTER(ct.c_float)]),
    "ie_fno_get_params": (ct.c_int, [_P, ct.POINTER(ct.c_float)]),
    "ie_fno_forward": (ct.c_int, [_P, ct.c_int32, _P, _P]),
    "ie_fno_backward": (ct.c_int, [_P, ct.c_int32, _P, _P, ct.POINTER(ct.c_float)]),
    "ie_fno_train_step": (ct.c_int, [_P, ct.c_int32, _P, _P, ct.c_float, ct.POINTER(ct.c_float)]),
    "ie_fno_encode": (ct.c_int, [_P, _P, ct.c_double, _P, _P, _P]),
    "ie_fno_encode_target": (ct.c_int, [_P, _P, _P, _P, _P]),
    "ie_fno_decode": (ct.c_int, [_P, _P, _P, _P, _P]),
    "ie_fno_last_error": (ct.c_char_p, [_P]),
    "ie_fno_destroy": (None, [_P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class IEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _c128(a, n=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} complex values, got {a.size}")
    return a


def _addr(x) -> int:
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    return int(x)


def _dipole(d) -> ie_dipole:
    pos, mom = (d.pos, d.moment) if hasattr(d, "pos") else d
    return ie_dipole((ct.c_double * 3)(*pos), (ct.c_double * 3)(*mom))


def ie_default_opts() -> ie_opts:
    o = ie_opts()
    _lib.ie_default_opts(ct.byref(o))
    return o


class Context:
    """Owns one ``ie_ctx*``; methods are the ABI calls of the same name (without the prefix)."""

    def __init__(self, grid, h: float, sigma0: float, freq: float):
        g = ie_grid(int(grid.nx), int(grid.ny), int(grid.nz), (ct.c_double * 3)(*grid.origin))
        p = _P()
        st = _lib.ie_create(ct.byref(g), float(h), float(sigma0), float(freq), ct.byref(p))
        if st != IE_OK:
            raise IEError(st, "ie_create failed")
        self.ptr = p
        self.nx, self.ny, self.nz = int(grid.nx), int(grid.ny), int(grid.nz)
        self.n = self.nx * self.ny * self.nz
        self._keep = []

    # ---------------------------------------------------------------- helpers
    def _check(self, st, allow=(IE_OK,)):
        if st not in allow:
            raise IEError(st, _lib.ie_last_error(self.ptr).decode())
        return st

    def close(self):
        if getattr(self, "ptr", None):
            _lib.ie_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- ABI calls
    def set_stream(self, stream):
        """``stream``: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(_lib.ie_set_stream(self.ptr, _P(handle or 0)))

    def set_contrast(self, sigma6: np.ndarray):
        s = np.ascontiguousarray(sigma6, dtype=np.float64)
        if s.size != 6 * self.n:
            raise ValueError("sigma6 must hold nz*ny*nx*6 values")
        self._check(_lib.ie_set_contrast(self.ptr, _dptr(s)))

    def set_contrast_dev(self, sigma6_dev):
        self._check(_lib.ie_set_contrast_dev(self.ptr, _P(_addr(sigma6_dev))))

    def solve(self, sources, receivers, dd_mode=IE_DD_NONE, tol=1e-6, opts: ie_opts | None = None,
              allow_noconv=False):
        src = (ie_dipole * max(1, len(sources)))(*[_dipole(d) for d in sources])
        rx = np.ascontiguousarray(np.asarray(receivers, dtype=np.float64).reshape(-1, 3))
        H = np.zeros((len(sources), len(rx), 3), dtype=np.complex128)
        info = ie_info()
        allow = (IE_OK, IE_ENOCONV) if allow_noconv else (IE_OK,)
        st = _lib.ie_solve(self.ptr, len(sources), src, len(rx), _dptr(rx), int(dd_mode), float(tol),
                           ct.byref(opts) if opts is not None else None, _dptr(H), ct.byref(info))
        self._check(st, allow)
        return H, info, st

    def get_field(self) -> np.ndarray:
        E = np.zeros((3, self.nz, self.ny, self.nx), dtype=np.complex128)
        self._check(_lib.ie_get_field(self.ptr, _dptr(E)))
        return E

    def get_field_dev(self, E_dev):
        self._check(_lib.ie_get_field_dev(self.ptr, _P(_addr(E_dev))))

    def incident_field_dev(self, src, E0_dev):
        d = _dipole(src)
        self._check(_lib.ie_incident_field_dev(self.ptr, ct.byref(d), _P(_addr(E0_dev))))

    def set_initial_field_dev(self, E_dev):
        """Initial guess for the next solve (complex128 [3][nz][ny][nx] device tensor), or None."""
        self._check(_lib.ie_set_initial_field_dev(self.ptr, _P(_addr(E_dev)) if E_dev is not None else None))

    def matvec(self, x: np.ndarray, z0=0, nz=None, precision=IE_PREC_MIXED) -> np.ndarray:
        nz = self.nz if nz is None else nz
        n = 3 * nz * self.ny * self.nx
        xx = _c128(x, n)
        y = np.zeros(n, dtype=np.complex128)
        self._check(_lib.ie_matvec(self.ptr, int(precision), int(z0), int(nz), _dptr(xx), _dptr(y)))
        return y.reshape(3, nz, self.ny, self.nx)

    def matvec_contraction(self, x: np.ndarray, z0=0, nz=None, precision=IE_PREC_MIXED) -> np.ndarray:
        """y = (M - G dsigma M) x on the slab (ie_matvec_contraction)."""
        nz = self.nz if nz is None else nz
        n = 3 * nz * self.ny * self.nx
        xx = _c128(x, n)
        y = np.zeros(n, dtype=np.complex128)
        self._check(_lib.ie_matvec_contraction(self.ptr, int(precision), int(z0), int(nz), _dptr(xx), _dptr(y)))
        return y.reshape(3, nz, self.ny, self.nx)

    def matvec_dev(self, x_dev, y_dev, z0=0, nz=None):
        nz = self.nz if nz is None else nz
        self._check(_lib.ie_matvec_dev(self.ptr, int(z0), int(nz), _P(_addr(x_dev)), _P(_addr(y_dev))))

    def matvec_dev_noalloc(self, x_dev, y_dev, z0=0, nz=None):
        """ie_matvec_dev without any device allocation, for callers with a fixed device-memory budget:
        the FFT intermediates use a fixed 16 MiB library-owned array per GPU (see ie.h)."""
        nz = self.nz if nz is None else nz
        self._check(_lib.ie_matvec_dev_noalloc(self.ptr, int(z0), int(nz), _P(_addr(x_dev)), _P(_addr(y_dev))))

    def interaction(self, x: np.ndarray, zs0, nzs, zt0, nzt) -> np.ndarray:
        xx = _c128(x, 3 * nzs * self.ny * self.nx)
        y = np.zeros((3, nzt, self.ny, self.nx), dtype=np.complex128)
        self._check(_lib.ie_interaction(self.ptr, int(zs0), int(nzs), int(zt0), int(nzt), _dptr(xx), _dptr(y)))
        return y

    def gmres(self, b, x0=None, z0=0, nz=None, tol=1e-6, restart=30, max_iter=600, precision=IE_PREC_MIXED):
        nz = self.nz if nz is None else nz
        n = 3 * nz * self.ny * self.nx
        bb = _c128(b, n)
        xx0 = _c128(x0, n) if x0 is not None else None
        x = np.zeros(n, dtype=np.complex128)
        it = ct.c_int32(0)
        rel = ct.c_double(0.0)
        st = _lib.ie_gmres(self.ptr, int(precision), int(z0), int(nz), _dptr(bb),
                           _dptr(xx0) if xx0 is not None else None, float(tol), int(restart), int(max_iter),
                           _dptr(x), ct.byref(it), ct.byref(rel))
        self._check(st, (IE_OK, IE_ENOCONV))
        return x.reshape(3, nz, self.ny, self.nx), it.value, rel.value, st

    def green_spectrum(self, comp: int, nz_set=None):
        nz_set = self.nz if nz_set is None else nz_set
        dims = (ct.c_int32 * 3)()
        self._check(_lib.ie_fft_dims(self.ptr, int(nz_set), dims))
        Lx, Ly, Lz = dims
        out = np.zeros((Lz // 2 + 1, Ly // 2 + 1, Lx // 2 + 1), dtype=np.complex128)
        self._check(_lib.ie_green_spectrum(self.ptr, int(nz_set), int(comp), _dptr(out), dims))
        return out, (Lx, Ly, Lz)

    def incident_field(self, src) -> np.ndarray:
        E = np.zeros((3, self.nz, self.ny, self.nx), dtype=np.complex128)
        d = _dipole(src)
        self._check(_lib.ie_incident_field(self.ptr, ct.byref(d), _dptr(E)))
        return E

    def receiver_fields(self, E, src, receivers) -> np.ndarray:
        EE = _c128(E, 3 * self.n)
        rx = np.ascontiguousarray(np.asarray(receivers, dtype=np.float64).reshape(-1, 3))
        H = np.zeros((len(rx), 3), dtype=np.complex128)
        d = _dipole(src)
        self._check(_lib.ie_receiver_fields(self.ptr, _dptr(EE), ct.byref(d), len(rx), _dptr(rx), _dptr(H)))
        return H

    def profile_enable(self, on=True):
        self._check(_lib.ie_profile_enable(self.ptr, int(bool(on))))

    def profile_read(self):
        """{class name: (launches, device ms, algorithmic bytes)} since the last profile_enable."""
        out = {}
        for k, name in enumerate(KERNEL_CLASSES):
            n = ct.c_int64(0)
            ms = ct.c_double(0.0)
            by = ct.c_double(0.0)
            self._check(_lib.ie_profile_read(self.ptr, k, ct.byref(n), ct.byref(ms), ct.byref(by)))
            out[name] = (n.value, ms.value, by.value)
        return out

    def fft_dims(self, nz_set=None):
        dims = (ct.c_int32 * 3)()
        self._check(_lib.ie_fft_dims(self.ptr, int(self.nz if nz_set is None else nz_set), dims))
        return tuple(dims)


def solve_batch(problems, max_concurrent=0):
    """ie_solve_batch on a list of dicts with keys ctx (Context), sources, receivers and optionally
    sigma6 (host array set on the context before that item), dd_mode, tol, opts, E_init_dev (device
    complex128 initial guess, see Context.set_initial_field_dev). Items sharing a
    context run in order; different contexts run concurrently. Returns [(H, info, status)]."""
    n = len(problems)
    items = (ie_batch_item * max(1, n))()
    keep, outs = [], []
    for i, p in enumerate(problems):
        ctx = p["ctx"]
        src = (ie_dipole * max(1, len(p["sources"])))(*[_dipole(d) for d in p["sources"]])
        rx = np.ascontiguousarray(np.asarray(p["receivers"], dtype=np.float64).reshape(-1, 3))
        H = np.zeros((len(p["sources"]), len(rx), 3), dtype=np.complex128)
        info = ie_info()
        s6 = p.get("sigma6")
        s6 = np.ascontiguousarray(s6, dtype=np.float64) if s6 is not None else None
        it = items[i]
        it.ctx = ctx.ptr
        it.sigma6 = _dptr(s6) if s6 is not None else None
        it.n_src, it.src = len(p["sources"]), src
        it.n_rx, it.rx_xyz = len(rx), _dptr(rx)
        it.dd_mode, it.tol = int(p.get("dd_mode", IE_DD_NONE)), float(p.get("tol", 1e-6))
        o = p.get("opts")
        it.opts = ct.pointer(o) if o is not None else None
        it.H_out = _dptr(H)
        it.info = ct.cast(ct.pointer(info), ct.c_void_p)
        init = p.get("E_init_dev")
        it.E_init_dev = _addr(init) if init is not None else None
        keep += [src, rx, s6, o, info]
        outs.append((H, info))
    _lib.ie_solve_batch(n, items, int(max_concurrent))
    return [(H, info, items[i].status) for i, (H, info) in enumerate(outs)]


class FNO:
    """Owns one ``ie_fno*`` (include/ie_fno.h); methods are the ABI calls of the same name.

    Device arguments are torch tensors (or raw addresses) on the current device; parameters travel as
    flat FP32 numpy vectors in the order and layout of the header."""

    def __init__(self, n, modes=12, width=32, layers=4, cin=12, cout=6, hidden=128, batch_max=8, bf16=True):
        p = _P()
        st = _lib.ie_fno_create(int(n), int(modes), int(width), int(layers), int(cin), int(cout), int(hidden),
                                int(batch_max), int(bool(bf16)), ct.byref(p))
        if st != IE_OK:
            raise IEError(st, "ie_fno_create failed")
        self.ptr = p
        self.n, self.modes, self.width, self.layers = int(n), int(modes), int(width), int(layers)
        self.cin, self.cout, self.hidden, self.batch_max = int(cin), int(cout), int(hidden), int(batch_max)

    def _check(self, st):
        if st != IE_OK:
            raise IEError(st, _lib.ie_fno_last_error(self.ptr).decode())

    def close(self):
        if getattr(self, "ptr", None):
            _lib.ie_fno_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def param_count(self) -> int:
        return int(_lib.ie_fno_param_count(self.ptr))

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        self._check(_lib.ie_fno_set_stream(self.ptr, _P(handle or 0)))

    def set_tensor_cores(self, on: bool):
        """ie_fno_set_tensor_cores: BF16 pointwise maps on the tcgen05 tensor cores (default) or CUDA cores."""
        self._check(_lib.ie_fno_set_tensor_cores(self.ptr, int(bool(on))))

    def set_params(self, flat: np.ndarray):
        v = np.ascontiguousarray(flat, dtype=np.float32)
        if v.size != self.param_count():
            raise ValueError(f"expected {self.param_count()} parameters, got {v.size}")
        self._check(_lib.ie_fno_set_params(self.ptr, v.ctypes.data_as(ct.POINTER(ct.c_float))))

    def get_params(self) -> np.ndarray:
        v = np.zeros(self.param_count(), dtype=np.float32)
        self._check(_lib.ie_fno_get_params(self.ptr, v.ctypes.data_as(ct.POINTER(ct.c_float))))
        return v

    def forward(self, batch, a_dev, u_dev):
        self._check(_lib.ie_fno_forward(self.ptr, int(batch), _P(_addr(a_dev)), _P(_addr(u_dev))))

    def backward(self, batch, a_dev, du_dev, want_host=True):
        g = np.zeros(self.param_count(), dtype=np.float32) if want_host else None
        self._check(_lib.ie_fno_backward(self.ptr, int(batch), _P(_addr(a_dev)), _P(_addr(du_dev)),
                                         g.ctypes.data_as(ct.POINTER(ct.c_float)) if want_host else None))
        return g

    def train_step(self, batch, a_dev, t_dev, lr, want_loss=True):
        loss = ct.c_float(0.0)
        self._check(_lib.ie_fno_train_step(self.ptr, int(batch), _P(_addr(a_dev)), _P(_addr(t_dev)), float(lr),
                                           ct.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def encode(self, sigma6_dev, sigma0, b_dev, a_dev, bnorm_dev):
        self._check(_lib.ie_fno_encode(self.ptr, _P(_addr(sigma6_dev)), float(sigma0), _P(_addr(b_dev)),
                                       _P(_addr(a_dev)), _P(_addr(bnorm_dev))))

    def encode_target(self, E_dev, b_dev, bnorm_dev, t_dev):
        self._check(_lib.ie_fno_encode_target(self.ptr, _P(_addr(E_dev)), _P(_addr(b_dev)), _P(_addr(bnorm_dev)),
                                              _P(_addr(t_dev))))

    def decode(self, u_dev, b_dev, bnorm_dev, x0_dev):
        self._check(_lib.ie_fno_decode(self.ptr, _P(_addr(u_dev)), _P(_addr(b_dev)), _P(_addr(bnorm_dev)),
                                       _P(_addr(x0_dev))))


def fno_flat(params) -> np.ndarray:
    """Flatten a parameter set (lists of arrays in the header's order; complex arrays interleaved)."""
    parts = []
    for arr in params:
        a = np.asarray(arr)
        if np.iscomplexobj(a):
            a = np.stack([a.real, a.imag], axis=-1)
        parts.append(a.astype(np.float32).ravel())
    return np.concatenate(parts)


def debug_fail_allocation(after: int):
    """ie_debug_fail_allocation: make the device allocation after `after` more successful ones report
    out-of-memory (testing hook; negative switches it off)."""
    _lib.ie_debug_fail_allocation(int(after))


def debug_force_tile(pass_: int, variant: int):
    """ie_debug_force_tile: run pass 2, 3 or 4 (P2, P3, P4) in the given tile variant in every later
    convolution of this process (-1: back to the autotuner). Testing hook."""
    st = _lib.ie_debug_force_tile(int(pass_), int(variant))
    if st != IE_OK:
        raise IEError(st, f"ie_debug_force_tile({pass_}, {variant})")


def tuned_tiles() -> str:
    """Tile shapes chosen so far by the library's FFT-tile autotuner (ie_tuned_tiles)."""
    n = _lib.ie_tuned_tiles(None, 0)
    buf = ct.create_string_buffer(n)
    _lib.ie_tuned_tiles(buf, n)
    return buf.value.decode()


def make_opts(n_blocks=1, z_split=None, restart=30, max_outer=50, max_inner=600, precision=IE_PREC_MIXED,
              adaptive=True, fixed_tol=1e-6, contraction=False, graph=False, outer_krylov=False, outer_restart=10,
              outer_inner_tol=0.1, concurrent_blocks=False) -> ie_opts:
    o = ie_default_opts()
    o.n_blocks = int(n_blocks)
    if z_split is not None:
        arr = (ct.c_int32 * len(z_split))(*[int(v) for v in z_split])
        o._z_split_keep = arr  # keep alive with the struct
        o.z_split = ct.cast(arr, ct.POINTER(ct.c_int32))
        o.n_blocks = len(z_split) - 1
    o.restart, o.max_outer, o.max_inner = int(restart), int(max_outer), int(max_inner)
    o.precision, o.adaptive, o.fixed_tol = int(precision), int(bool(adaptive)), float(fixed_tol)
    o.contraction = int(bool(contraction))
    o.graph = int(bool(graph))
    o.outer_krylov, o.outer_restart, o.outer_inner_tol = int(bool(outer_krylov)), int(outer_restart), float(outer_inner_tol)
    o.concurrent_blocks = int(bool(concurrent_blocks))
    return o


EXPORTED = tuple(_SIGS)
