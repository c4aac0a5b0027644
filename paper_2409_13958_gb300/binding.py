"""ctypes binding of libpmfem (include/pmfem.h): same names, argument marshalling only.

Device buffers may be torch CUDA tensors (their data_ptr() is passed) or raw integer
addresses; host buffers are NumPy arrays or pinned torch CPU tensors.  Streams may be
torch.cuda.Stream objects, raw cudaStream_t integers, or None (library stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PMFEM_FP64, PMFEM_FP32, PMFEM_BF16SPLIT = 0, 1, 2
PMFEM_EX, PMFEM_MS, PMFEM_AP, PMFEM_AN, PMFEM_ALL = 1, 2, 4, 8, 15
(PMFEM_BF16_PRECORRECTION, PMFEM_BF16_PROJECTION, PMFEM_BF16_CHARGES, PMFEM_BF16_GRADIENT,
 PMFEM_BF16_EXCHANGE) = 1, 2, 4, 8, 16

_ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EMESH", -5: "ENONFINITE", -6: "ETIMEOUT", -7: "ESTATE",
           -8: "ENOCONV"}

_c = ctypes
_vp, _i32, _i64, _dbl = _c.c_void_p, _c.c_int32, _c.c_int64, _c.c_double
_pi32, _pi64, _pdbl = _c.POINTER(_c.c_int32), _c.POINTER(_c.c_int64), _c.POINTER(_c.c_double)

# name -> (restype, argtypes); every exported symbol of include/pmfem.h
SIGNATURES = {
    "pmfem_version": (_c.c_char_p, []),
    "pmfem_last_error": (_c.c_char_p, [_vp]),
    "pmfem_create_mesh": (_c.c_int, [_c.POINTER(_vp), _vp, _i64, _vp, _i64, _dbl, _dbl, _dbl]),
    "pmfem_set_aim": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _dbl]),
    "pmfem_set_periodicity": (_c.c_int, [_vp, _dbl, _dbl, _dbl]),
    "pmfem_set_layout": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int, _c.c_int]),
    "pmfem_set_setup_device": (_c.c_int, [_vp, _c.c_int]),
    "pmfem_set_exchange_per_tet": (_c.c_int, [_vp, _vp]),
    "pmfem_set_anisotropy": (_c.c_int, [_vp, _vp, _c.c_int, _vp, _vp, _vp, _vp]),
    "pmfem_set_precision": (_c.c_int, [_vp, _c.c_int]),
    "pmfem_set_bf16_operators": (_c.c_int, [_vp, _c.c_int]),
    "pmfem_set_applied_field": (_c.c_int, [_vp, _dbl, _dbl, _dbl]),
    "pmfem_num_unknowns": (_c.c_int, [_vp, _pi64]),
    "pmfem_lca_map": (_c.c_int, [_vp, _vp]),
    "pmfem_field": (_c.c_int, [_vp, _vp, _vp, _c.c_int, _vp]),
    "pmfem_field_host": (_c.c_int, [_vp, _vp, _vp, _c.c_int, _vp]),
    "pmfem_field_noalloc": (_c.c_int, [_vp, _vp, _vp, _c.c_int, _vp]),
    "pmfem_set_m": (_c.c_int, [_vp, _vp, _vp]),
    "pmfem_get_m": (_c.c_int, [_vp, _vp, _vp]),
    "pmfem_llg_step": (_c.c_int, [_vp, _dbl, _c.c_int, _vp]),
    "pmfem_llg_step_implicit": (_c.c_int, [_vp, _dbl, _c.c_int, _vp, _vp, _vp]),
    "pmfem_profile": (_c.c_int, [_vp, _c.c_int]),
    "pmfem_profile_read": (_c.c_int, [_vp, _vp, _vp, _c.c_int]),
    "pmfem_sync": (_c.c_int, [_vp]),
    "pmfem_destroy": (_c.c_int, [_vp]),
    "pmfem_operator_info": (_c.c_int, [_vp, _c.c_int, _pi64, _pi64, _c.POINTER(_c.c_int)]),
    "pmfem_operator_export": (_c.c_int, [_vp, _c.c_int, _vp, _vp, _vp]),
    "pmfem_device_info": (_c.c_int, [_vp, _vp, _c.c_int]),
    "pmfem_surrogate_set_params": (_c.c_int, [_vp, _vp, _i64, _dbl, _dbl, _c.c_int]),
    "pmfem_surrogate_get_params": (_c.c_int, [_vp, _vp]),
    "pmfem_surrogate_apply": (_c.c_int, [_vp, _vp, _vp, _vp]),
    "pmfem_surrogate_grad": (_c.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pmfem_surrogate_train": (_c.c_int, [_vp, _vp, _vp, _i64, _c.c_int, _c.c_int, _dbl, _vp, _vp]),
    "pmfem_grid_pair": (_c.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pmfem_surrogate_enable": (_c.c_int, [_vp, _c.c_int]),
    "pmfem_surrogate_stats": (_c.c_int, [_vp, _vp]),
    "pmfem_batch_create": (_c.c_int, [_c.POINTER(_vp), _vp, _c.c_int]),
    "pmfem_batch_destroy": (_c.c_int, [_vp]),
    "pmfem_batch_last_error": (_c.c_char_p, [_vp]),
    "pmfem_batch_offsets": (_c.c_int, [_vp, _vp]),
    "pmfem_batch_autotune": (_c.c_int, [_vp, _c.c_int]),
    "pmfem_batch_tiles": (_c.c_int, [_vp, _vp]),
    "pmfem_batch_set_applied_field": (_c.c_int, [_vp, _c.c_int, _dbl, _dbl, _dbl, _vp]),
    "pmfem_batch_field": (_c.c_int, [_vp, _vp, _vp, _c.c_int, _vp]),
    "pmfem_batch_set_m": (_c.c_int, [_vp, _vp, _vp]),
    "pmfem_batch_get_m": (_c.c_int, [_vp, _vp, _vp]),
    "pmfem_batch_llg_step": (_c.c_int, [_vp, _dbl, _c.c_int, _vp]),
    "pmfem_batch_sync": (_c.c_int, [_vp]),
    "pmfem_batch_profile": (_c.c_int, [_vp, _c.c_int]),
    "pmfem_batch_profile_read": (_c.c_int, [_vp, _vp, _vp, _c.c_int]),
    "pmfem_setup_times": (_c.c_int, [_vp, _vp, _c.c_int]),
    "pmfem_debug_fail_alloc": (_c.c_int, [_c.c_int]),
    "pmfem_build_flags": (_c.c_int, []),
    "pmfem_bloch_spectrum": (_c.c_int, [_vp, _vp, _vp, _vp]),
    "pmfem_bloch_convolve": (_c.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pmfem_grid_info": (_c.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pmfem_export_spectrum": (_c.c_int, [_vp, _vp]),
    "pmfem_folded_positions": (_c.c_int, [_vp, _vp]),
}
SYMBOLS = tuple(SIGNATURES)

_LIB = None
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpmfem.so")


def _open(p: str):
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with __graft_entry__.build() "
                           "(paper_2409_13958_gb300._build.build()); there is no CPU fallback")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load_library(path: str | None = None):
    """Load libpmfem.so (raises when it has not been built; there is no fallback)."""
    global _LIB
    if _LIB is None:
        _LIB = _open(path or LIB_PATH)
    return _LIB


def load_variant(path: str):
    """Another build of the library (e.g. the bounds-checked one), for handles created with
    Pmfem.create_mesh(..., lib=...)."""
    return _open(path)


class ImplicitOpts(ctypes.Structure):
    """pmfem_implicit_opts (include/pmfem.h); zero fields select the defaults."""
    _fields_ = [("newton_tol", ctypes.c_double), ("krylov_tol", ctypes.c_double), ("restart", ctypes.c_int),
                ("max_newton", ctypes.c_int), ("max_krylov", ctypes.c_int)]


class PmfemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


def _addr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


class Pmfem:
    """One periodic unit cell (a pmfem_t handle)."""

    def __init__(self, handle, lib=None):
        self._lib = lib if lib is not None else load_library()
        self.h = handle

    def _ck(self, rc: int):
        if rc != 0:
            msg = self._lib.pmfem_last_error(self.h).decode()
            raise PmfemError(rc, msg)

    # ------------------------------------------------------------------ set-up
    @classmethod
    def create_mesh(cls, xyz, tets, Ms: float, A: float, alpha: float, lib=None) -> "Pmfem":
        lib = lib if lib is not None else load_library()
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        h = _vp()
        rc = lib.pmfem_create_mesh(ctypes.byref(h), xyz.ctypes.data, xyz.shape[0], tets.ctypes.data,
                                   tets.shape[0], Ms, A, alpha)
        if rc != 0:
            raise PmfemError(rc, lib.pmfem_last_error(None).decode())
        return cls(h, lib)

    def set_aim(self, Nx=0, Ny=0, Nz=0, order_p=0, near_boxes=0, near_elem_factor=0.0):
        self._ck(self._lib.pmfem_set_aim(self.h, Nx, Ny, Nz, order_p, near_boxes, near_elem_factor))

    def set_periodicity(self, L1=0.0, L2=0.0, L3=0.0):
        self._ck(self._lib.pmfem_set_periodicity(self.h, L1, L2, L3))

    def set_exchange_per_tet(self, A_tet=None):
        a = None if A_tet is None else np.ascontiguousarray(A_tet, dtype=np.float64)
        self._ck(self._lib.pmfem_set_exchange_per_tet(self.h, None if a is None else a.ctypes.data))

    def set_anisotropy(self, tet_grain=None, axes=None, K1=None, Ku=None, u=None):
        if tet_grain is None:
            self._ck(self._lib.pmfem_set_anisotropy(self.h, None, 0, None, None, None, None))
            return
        tg = np.ascontiguousarray(tet_grain, dtype=np.int32)
        ax = np.ascontiguousarray(axes, dtype=np.float64).reshape(-1, 9)
        k1 = None if K1 is None else np.ascontiguousarray(K1, dtype=np.float64)
        ku = None if Ku is None else np.ascontiguousarray(Ku, dtype=np.float64)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
        addr = lambda x: None if x is None else x.ctypes.data
        self._ck(self._lib.pmfem_set_anisotropy(self.h, tg.ctypes.data, ax.shape[0], addr(k1), ax.ctypes.data,
                                                addr(ku), addr(uu)))

    def set_setup_device(self, use_gpu: bool):
        self._ck(self._lib.pmfem_set_setup_device(self.h, int(bool(use_gpu))))

    def set_layout(self, tile_y=0, tile_z=0, sort_window=0, col_bits=0):
        self._ck(self._lib.pmfem_set_layout(self.h, tile_y, tile_z, sort_window, col_bits))

    def set_precision(self, mode: int):
        self._ck(self._lib.pmfem_set_precision(self.h, mode))

    def set_bf16_operators(self, mask: int):
        self._ck(self._lib.pmfem_set_bf16_operators(self.h, mask))

    def set_applied_field(self, Hx=0.0, Hy=0.0, Hz=0.0):
        self._ck(self._lib.pmfem_set_applied_field(self.h, Hx, Hy, Hz))

    def num_unknowns(self) -> int:
        n = _i64()
        self._ck(self._lib.pmfem_num_unknowns(self.h, ctypes.byref(n)))
        return int(n.value)

    def lca_map(self, n_nodes: int) -> np.ndarray:
        out = np.empty(n_nodes, dtype=np.int32)
        self._ck(self._lib.pmfem_lca_map(self.h, out.ctypes.data))
        return out

    # ------------------------------------------------------------------ compute
    def field(self, m, H, components: int = PMFEM_ALL, stream=None):
        self._ck(self._lib.pmfem_field(self.h, _addr(m), _addr(H), components, _stream(stream)))

    def field_host(self, m_host, H_host, components: int = PMFEM_ALL, stream=None):
        self._ck(self._lib.pmfem_field_host(self.h, _addr(m_host), _addr(H_host), components, _stream(stream)))

    def field_noalloc(self, m, H, components: int = PMFEM_ALL, stream=None):
        self._ck(self._lib.pmfem_field_noalloc(self.h, _addr(m), _addr(H), components, _stream(stream)))

    def set_m(self, m, stream=None):
        self._ck(self._lib.pmfem_set_m(self.h, _addr(m), _stream(stream)))

    def get_m(self, m, stream=None):
        self._ck(self._lib.pmfem_get_m(self.h, _addr(m), _stream(stream)))

    # ------------------------------------------------------------------ surrogate
    NET_PARAMS = 57121

    def surrogate_set_params(self, params, sq: float, su: float, act_bf16: bool = False):
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        self._ck(self._lib.pmfem_surrogate_set_params(self.h, p.ctypes.data, p.size, sq, su, 1 if act_bf16 else 0))

    def surrogate_get_params(self) -> np.ndarray:
        out = np.empty(self.NET_PARAMS, dtype=np.float32)
        self._ck(self._lib.pmfem_surrogate_get_params(self.h, out.ctypes.data))
        return out

    def surrogate_apply(self, Q, U, stream=None):
        self._ck(self._lib.pmfem_surrogate_apply(self.h, _addr(Q), _addr(U), _stream(stream)))

    def surrogate_grad(self, Q, U):
        g = np.empty(self.NET_PARAMS, dtype=np.float32)
        loss = _c.c_double()
        self._ck(self._lib.pmfem_surrogate_grad(self.h, _addr(Q), _addr(U), g.ctypes.data, ctypes.byref(loss)))
        return float(loss.value), g

    def surrogate_train(self, Q, U, npairs: int, epochs: int = 1, batch: int = 1, lr: float = 1e-3, stream=None):
        losses = np.zeros(epochs)
        self._ck(self._lib.pmfem_surrogate_train(self.h, _addr(Q), _addr(U), npairs, epochs, batch, lr,
                                                 losses.ctypes.data, _stream(stream)))
        return losses

    def grid_pair(self, m, Q, U, stream=None):
        self._ck(self._lib.pmfem_grid_pair(self.h, _addr(m), _addr(Q), _addr(U), _stream(stream)))

    def surrogate_enable(self, every_k: int):
        self._ck(self._lib.pmfem_surrogate_enable(self.h, every_k))

    def surrogate_stats(self) -> dict:
        out = np.zeros(4)
        self._ck(self._lib.pmfem_surrogate_stats(self.h, out.ctypes.data))
        return {"steps": int(out[0]), "net_stages": int(out[1]), "judged_stages": int(out[2]),
                "judged_rel_l2": float(out[3])}

    def llg_step_implicit(self, dt: float, nsteps: int = 1, newton_tol: float = 0.0, krylov_tol: float = 0.0,
                          restart: int = 0, max_newton: int = 0, max_krylov: int = 0, stream=None) -> dict:
        """Implicit midpoint steps (Newton-GMRES); returns the iteration counts."""
        o = ImplicitOpts(newton_tol, krylov_tol, restart, max_newton, max_krylov)
        st = np.zeros(4, dtype=np.int64)
        rc = self._lib.pmfem_llg_step_implicit(self.h, dt, nsteps, ctypes.byref(o), st.ctypes.data, _stream(stream))
        out = {"newton": int(st[0]), "krylov": int(st[1]), "field_evals": int(st[2]), "steps": int(st[3])}
        self._ck(rc)
        return out

    def llg_step(self, dt: float, nsteps: int = 1, stream=None):
        self._ck(self._lib.pmfem_llg_step(self.h, dt, nsteps, _stream(stream)))

    KERNELS = ("charges", "projection", "fft_x_fwd", "fft_y_fwd", "fft_z_conv", "fft_y_inv", "fft_x_inv",
               "interp_precorr", "gradient_exchange", "grid_clear", "permute", "interp_stencil",
               "surrogate_in", "surrogate_hidden", "surrogate_out")

    def profile(self, enable: bool = True):
        self._ck(self._lib.pmfem_profile(self.h, 1 if enable else 0))

    def profile_read(self) -> dict:
        n = len(self.KERNELS)
        counts = np.zeros(n, dtype=np.int64)
        ms = np.zeros(n, dtype=np.float64)
        self._ck(self._lib.pmfem_profile_read(self.h, counts.ctypes.data, ms.ctypes.data, n))
        return {k: (int(c), float(t)) for k, c, t in zip(self.KERNELS, counts, ms)}

    def sync(self):
        self._ck(self._lib.pmfem_sync(self.h))

    def destroy(self):
        if self.h:
            self._lib.pmfem_destroy(self.h)
            self.h = None

    # ------------------------------------------------------------------ introspection
    def operator_export(self, which: int):
        rows, nnz, comps = _i64(), _i64(), _c.c_int()
        self._ck(self._lib.pmfem_operator_info(self.h, which, ctypes.byref(rows), ctypes.byref(nnz),
                                                 ctypes.byref(comps)))
        rp = np.empty(rows.value + 1, dtype=np.int32)
        col = np.empty(nnz.value, dtype=np.int32)
        vals = np.empty((nnz.value, comps.value), dtype=np.float64)
        self._ck(self._lib.pmfem_operator_export(self.h, which, rp.ctypes.data, col.ctypes.data, vals.ctypes.data))
        return rp, col, vals

    def device_info(self) -> dict:
        out = np.zeros(13, dtype=np.int64)
        self._ck(self._lib.pmfem_device_info(self.h, out.ctypes.data, 13))
        names = ("adjacency", "precorrection", "projection")
        d = {n: {"entries": int(out[3 * k]), "padded": int(out[3 * k + 1]), "col_bits": int(out[3 * k + 2])}
             for k, n in enumerate(names)}
        d["projection_exceptions"] = int(out[9])
        d["tile"] = (int(out[10]), int(out[11]))
        d["projection"]["rows"] = int(out[12])
        return d

    def setup_times(self) -> dict:
        out = np.zeros(7)
        self._ck(self._lib.pmfem_setup_times(self.h, out.ctypes.data, 7))
        keys = ("pairing", "operators", "grid", "spectrum", "near_elements", "precorrection", "device")
        return dict(zip(keys, out.tolist()))

    def bloch_spectrum(self, k0):
        """Real spectrum of the twisted Bloch kernel, shape (fft z, fft y, fft x), and the
        largest imaginary part of the transform."""
        dims, fft, _, _ = self.grid_info()
        k = np.ascontiguousarray(k0, dtype=np.float64)
        out = np.empty((fft[2], fft[1], fft[0]), dtype=np.float64)
        mi = ctypes.c_double(0.0)
        self._ck(self._lib.pmfem_bloch_spectrum(self.h, k.ctypes.data, out.ctypes.data, ctypes.byref(mi)))
        return out, mi.value

    def bloch_convolve(self, k0, Q, U, stream=None):
        k = np.ascontiguousarray(k0, dtype=np.float64)
        self._ck(self._lib.pmfem_bloch_convolve(self.h, k.ctypes.data, _addr(Q), _addr(U), _stream(stream)))

    def grid_info(self):
        dims = np.zeros(3, np.int32)
        fft = np.zeros(3, np.int32)
        origin = np.zeros(3)
        delta = np.zeros(3)
        self._ck(self._lib.pmfem_grid_info(self.h, dims.ctypes.data, fft.ctypes.data, origin.ctypes.data,
                                           delta.ctypes.data))
        return dims, fft, origin, delta

    def export_spectrum(self) -> np.ndarray:
        dims, fft, _, _ = self.grid_info()
        shape = (fft[2] // 2 + 1, fft[1] // 2 + 1, fft[0] // 2 + 1)   # z, y, x (x fastest)
        out = np.empty(shape, dtype=np.float64)
        self._ck(self._lib.pmfem_export_spectrum(self.h, out.ctypes.data))
        return out

    def folded_positions(self) -> np.ndarray:
        out = np.empty((self.num_unknowns(), 3), dtype=np.float64)
        self._ck(self._lib.pmfem_folded_positions(self.h, out.ctypes.data))
        return out

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class PmfemBatch:
    """A batch of set-up cells (pmfem_batch_t): one launch per pass over all cells, RK4 steps
    replayed from a captured CUDA graph, FP32.  Keeps the cells alive while it exists."""

    def __init__(self, cells):
        self._lib = load_library()
        self.cells = list(cells)
        arr = (_vp * len(self.cells))(*[c.h for c in self.cells])
        b = _vp()
        rc = self._lib.pmfem_batch_create(ctypes.byref(b), arr, len(self.cells))
        if rc != 0:
            raise PmfemError(rc, "pmfem_batch_create failed")
        self.b = b

    def _ck(self, rc: int):
        if rc != 0:
            raise PmfemError(rc, self._lib.pmfem_batch_last_error(self.b).decode())

    def offsets(self) -> np.ndarray:
        out = np.zeros(len(self.cells) + 1, dtype=np.int64)
        self._ck(self._lib.pmfem_batch_offsets(self.b, out.ctypes.data))
        return out

    def autotune(self, reps: int = 5):
        self._ck(self._lib.pmfem_batch_autotune(self.b, reps))

    def tiles(self) -> np.ndarray:
        out = np.zeros((len(self.cells), 2), dtype=np.int32)
        self._ck(self._lib.pmfem_batch_tiles(self.b, out.ctypes.data))
        return out

    def set_applied_field(self, cell: int, Hx=0.0, Hy=0.0, Hz=0.0, stream=None):
        self._ck(self._lib.pmfem_batch_set_applied_field(self.b, cell, Hx, Hy, Hz, _stream(stream)))

    def field(self, m, H, components: int = PMFEM_ALL, stream=None):
        self._ck(self._lib.pmfem_batch_field(self.b, _addr(m), _addr(H), components, _stream(stream)))

    def set_m(self, m, stream=None):
        self._ck(self._lib.pmfem_batch_set_m(self.b, _addr(m), _stream(stream)))

    def get_m(self, m, stream=None):
        self._ck(self._lib.pmfem_batch_get_m(self.b, _addr(m), _stream(stream)))

    # ------------------------------------------------------------------ surrogate
    NET_PARAMS = 57121

    def surrogate_set_params(self, params, sq: float, su: float, act_bf16: bool = False):
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        self._ck(self._lib.pmfem_surrogate_set_params(self.h, p.ctypes.data, p.size, sq, su, 1 if act_bf16 else 0))

    def surrogate_get_params(self) -> np.ndarray:
        out = np.empty(self.NET_PARAMS, dtype=np.float32)
        self._ck(self._lib.pmfem_surrogate_get_params(self.h, out.ctypes.data))
        return out

    def surrogate_apply(self, Q, U, stream=None):
        self._ck(self._lib.pmfem_surrogate_apply(self.h, _addr(Q), _addr(U), _stream(stream)))

    def surrogate_grad(self, Q, U):
        g = np.empty(self.NET_PARAMS, dtype=np.float32)
        loss = _c.c_double()
        self._ck(self._lib.pmfem_surrogate_grad(self.h, _addr(Q), _addr(U), g.ctypes.data, ctypes.byref(loss)))
        return float(loss.value), g

    def surrogate_train(self, Q, U, npairs: int, epochs: int = 1, batch: int = 1, lr: float = 1e-3, stream=None):
        losses = np.zeros(epochs)
        self._ck(self._lib.pmfem_surrogate_train(self.h, _addr(Q), _addr(U), npairs, epochs, batch, lr,
                                                 losses.ctypes.data, _stream(stream)))
        return losses

    def grid_pair(self, m, Q, U, stream=None):
        self._ck(self._lib.pmfem_grid_pair(self.h, _addr(m), _addr(Q), _addr(U), _stream(stream)))

    def surrogate_enable(self, every_k: int):
        self._ck(self._lib.pmfem_surrogate_enable(self.h, every_k))

    def surrogate_stats(self) -> dict:
        out = np.zeros(4)
        self._ck(self._lib.pmfem_surrogate_stats(self.h, out.ctypes.data))
        return {"steps": int(out[0]), "net_stages": int(out[1]), "judged_stages": int(out[2]),
                "judged_rel_l2": float(out[3])}

    def llg_step(self, dt: float, nsteps: int = 1, stream=None):
        self._ck(self._lib.pmfem_batch_llg_step(self.b, dt, nsteps, _stream(stream)))

    def profile(self, enable: bool = True):
        self._ck(self._lib.pmfem_batch_profile(self.b, 1 if enable else 0))

    def profile_read(self) -> dict:
        n = len(Pmfem.KERNELS)
        counts = np.zeros(n, dtype=np.int64)
        ms = np.zeros(n, dtype=np.float64)
        self._ck(self._lib.pmfem_batch_profile_read(self.b, counts.ctypes.data, ms.ctypes.data, n))
        return {k: (int(c), float(t)) for k, c, t in zip(Pmfem.KERNELS, counts, ms)}

    def sync(self):
        self._ck(self._lib.pmfem_batch_sync(self.b))

    def destroy(self):
        if self.b:
            self._lib.pmfem_batch_destroy(self.b)
            self.b = None
