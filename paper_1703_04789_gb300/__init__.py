"""GB300 (sm_103a) spin-projected MPS library: Python binding of ``libspmps.so``.

The binding marshals arguments only: every contraction, the Davidson solver and the
decimation run in the library's CUDA kernels.  PyTorch provides device buffers and streams.
There is no CPU fallback: importing works without a GPU, but creating a handle without the
built library or without a CUDA device raises ``SpmpsError``.

Names follow the C ABI in ``include/spmps.h`` (spmps_create -> ``Spmps(...)``,
spmps_apply_heff -> ``Spmps.apply_heff`` ...).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["Spmps", "SpmpsError", "load_library", "library_path", "STATUS"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libspmps.so")
_lib = None

STATUS = {
    0: "OK", 1: "BAD_INPUT", 2: "NOT_CONVERGED", 3: "SINGULAR_METRIC", 4: "OOM", 5: "TIMEOUT",
    6: "CUDA", 7: "NAN", 8: "STATE", 9: "UNSUPPORTED",
}


class SpmpsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Options(C.Structure):
    _fields_ = [
        ("batched", C.c_int), ("precond", C.c_int), ("cg_steps", C.c_int),
        ("dav_tol_r", C.c_double), ("dav_tol_theta", C.c_double),
        ("dav_max_sub", C.c_int), ("dav_max_iter", C.c_int), ("device", C.c_int),
        ("jacobi_smem_max", C.c_int), ("precision", C.c_int), ("autotune", C.c_int),
        ("metric_max_dim", C.c_int), ("tc_wait_polls", C.c_int), ("tensor_core_kernel", C.c_int),
        ("m_screen", C.c_double), ("fp64_tensor_cores", C.c_int),
    ]


def library_path() -> str:
    return _LIB_PATH


def load_library(path: str | None = None):
    """Load libspmps.so (built by ``paper_1703_04789_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise SpmpsError(6, f"{p} is missing: build it with paper_1703_04789_gb300.build.build()")
    lib = C.CDLL(p)
    H = C.c_void_p
    i, d, i64 = C.c_int, C.c_double, C.c_int64
    P = C.POINTER
    sig = {
        "spmps_default_options": (None, [P(Options)]),
        "spmps_create": (i, [i, i, i, i, i, i, P(Options), P(H)]),
        "spmps_destroy": (i, [H]),
        "spmps_last_error": (C.c_char_p, [H]),
        "spmps_set_hubbard": (i, [H, d, d]),
        "spmps_set_hamiltonian": (i, [H, P(d), P(d), d]),
        "spmps_set_mpo": (i, [H, P(i), C.c_void_p]),
        "spmps_init_determinant": (i, [H, P(C.c_int8)]),
        "spmps_expect_mpo": (i, [H, P(i), C.c_void_p, P(d)]),
        "spmps_fragment_energies": (i, [H, P(d)]),
        "spmps_rdm1": (i, [H, P(d)]),
        "spmps_spin_correlation": (i, [H, P(i), i, P(i), i, P(d)]),
        "spmps_seniority": (i, [H, P(d)]),
        "spmps_init_random": (i, [H, C.c_uint64]),
        "spmps_save": (i, [H, C.c_char_p]),
        "spmps_load": (i, [H, C.c_char_p]),
        "spmps_mpo_from_integrals": (i, [i, P(d), P(d), d, P(i), C.c_void_p]),
        "spmps_set_mps": (i, [H, P(i), P(i), P(P(d)), i]),
        "spmps_x_layout": (i, [H, i, P(i64), P(i), P(i), P(i64), P(i), P(i)]),
        "spmps_apply_heff": (i, [H, i, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
        "spmps_apply_heff_host": (i, [H, i, P(d), P(d), P(d)]),
        "spmps_apply_heff_timed": (i, [H, i, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, P(d)]),
        "spmps_apply_heff_noalloc": (i, [H, i, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
        "spmps_apply_flops": (i, [H, i, P(d)]),
        "spmps_device_fp64_peak": (i, [i, P(d)]),
        "spmps_device_tf32_peak": (i, [i, i, i, P(d)]),
        "spmps_apply_costs": (i, [H, i, P(d), P(d)]),
        "spmps_add_lower_state": (i, [H, P(i), P(i), C.c_void_p]),
        "spmps_clear_lower_states": (i, [H]),
        "spmps_lower_overlap": (i, [H, i, P(d)]),
        "spmps_two_site": (i, [H, i, C.c_void_p]),
        "spmps_canonicalize": (i, [H]),
        "spmps_sweep": (i, [H, i, P(d)]),
        "spmps_optimize_step": (i, [H, i, i, P(d), P(i)]),
        "spmps_energy": (i, [H, P(d), P(d)]),
        "spmps_expect_s2": (i, [H, P(d)]),
        "spmps_stats": (i, [H, P(i64), P(d)]),
        "spmps_davidson_stats": (i, [H, P(i64), P(i64)]),
        "spmps_quadrature": (i, [H, P(d), P(d)]),
        "spmps_get_mps": (i, [H, P(i), P(i), C.c_void_p, P(i)]),
        "spmps_stream": (i, [H, P(C.c_void_p)]),
        "spmps_profile": (i, [H, i]),
        "spmps_kernel_stats": (i, [H, i, P(i64), P(d), P(d)]),
        "spmps_mlp_harvest": (i, [H, i, i, i64]),
        "spmps_mlp_data": (i, [H, P(i64), P(C.c_float), P(C.c_float)]),
        "spmps_mlp_params": (i, [H, P(C.c_float), i]),
        "spmps_mlp_loss_grad": (i, [H, P(C.c_float), P(C.c_float), i, P(d), P(C.c_float)]),
        "spmps_mlp_train": (i, [H, i, i, d, C.c_uint64, i, P(d), P(d)]),
        "spmps_mlp_infer": (i, [H, P(d), P(d), P(d), d, i64, P(d), i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Spmps:
    """One SP-MPS problem on one GPU (spmps_create ... spmps_destroy)."""

    def __init__(self, K, N, twoM, twoS, n_beta, D, *, batched=True, precond="diag", cg_steps=5,
                 dav_tol_r=1e-6, dav_tol_theta=1e-10, dav_max_sub=20, dav_max_iter=200, device=0,
                 jacobi_smem_max=0, precision="fp64", autotune=False, metric_max_dim=0,
                 tc_wait_polls=0, tensor_core_kernel="tcgen05", m_screen=0.0, fp64_tensor_cores=False):
        self.lib = load_library()
        o = Options()
        self.lib.spmps_default_options(C.byref(o))
        o.batched = 1 if batched else 0
        o.precond = {"diag": 0, "metric": 1, "learned": 2, "olsen": 3, "metric_block": 4}[precond]
        o.cg_steps, o.dav_tol_r, o.dav_tol_theta = cg_steps, dav_tol_r, dav_tol_theta
        o.dav_max_sub, o.dav_max_iter, o.device = dav_max_sub, dav_max_iter, device
        o.jacobi_smem_max = jacobi_smem_max
        o.precision = {"fp64": 0, "tf32": 1, "3xtf32": 2}[precision]
        o.autotune = 1 if autotune else 0
        o.metric_max_dim = metric_max_dim
        o.tc_wait_polls = tc_wait_polls
        o.tensor_core_kernel = {"tcgen05": 0, "mma_sync": 1}[tensor_core_kernel]
        o.m_screen = m_screen
        o.fp64_tensor_cores = 1 if fp64_tensor_cores else 0
        h = C.c_void_p()
        self._h = None
        self._check(self.lib.spmps_create(K, N, twoM, twoS, n_beta, D, C.byref(o), C.byref(h)), None)
        self._h = h
        self.K, self.N, self.twoM, self.twoS, self.n_beta, self.D = K, N, twoM, twoS, n_beta, D

    def _check(self, st, h=...):
        if st != 0:
            hh = self._h if h is ... else h
            msg = self.lib.spmps_last_error(hh).decode()
            raise SpmpsError(st, msg)
        return st

    def close(self):
        if self._h is not None:
            self.lib.spmps_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- problem definition ----------------------------------------------------------------
    def set_hubbard(self, t: float, U: float):
        self._check(self.lib.spmps_set_hubbard(self._h, t, U))

    def set_hamiltonian(self, h1: np.ndarray, h2: np.ndarray | None = None, ecore: float = 0.0):
        h1 = np.ascontiguousarray(h1, dtype=np.float64)
        h2p = None
        if h2 is not None:
            h2 = np.ascontiguousarray(h2, dtype=np.float64)
            h2p = _dptr(h2)
        self._check(self.lib.spmps_set_hamiltonian(self._h, _dptr(h1), h2p, ecore))

    def init_determinant(self, occ):
        """Product-state MPS of a determinant: occ[k] in {0, 1 (beta), 2 (alpha), 3 (both)}."""
        o = np.ascontiguousarray(occ, dtype=np.int8)
        self._check(self.lib.spmps_init_determinant(self._h, o.ctypes.data_as(C.POINTER(C.c_int8))))

    def init_random(self, seed: int):
        self._check(self.lib.spmps_init_random(self._h, seed))

    def save(self, path: str):
        self._check(self.lib.spmps_save(self._h, os.fsencode(path)))

    def load(self, path: str):
        self._check(self.lib.spmps_load(self._h, os.fsencode(path)))

    def set_mpo(self, sites):
        """Hamiltonian as an MPO: sites[k] of shape (Dl, Dr, 4, 4)."""
        ws = [np.ascontiguousarray(w, dtype=np.float64) for w in sites]
        dims = np.array([1] + [w.shape[1] for w in ws], dtype=np.int32)
        arr = (C.POINTER(C.c_double) * self.K)(*[_dptr(w) for w in ws])
        self._check(self.lib.spmps_set_mpo(self._h, dims.ctypes.data_as(C.POINTER(C.c_int)), C.cast(arr, C.c_void_p)))

    def set_mps(self, labels, tensors, center: int = 0):
        """labels: K+1 arrays (D_i, 2) of (n, 2m); tensors: K dense (D_i, 4, D_i+1) arrays."""
        dims = np.array([l.shape[0] for l in labels], dtype=np.int32)
        lab = np.ascontiguousarray(np.concatenate([np.asarray(l, dtype=np.int32).reshape(-1, 2) for l in labels]))
        ts = [np.ascontiguousarray(t, dtype=np.float64) for t in tensors]
        arr = (C.POINTER(C.c_double) * len(ts))(*[_dptr(t) for t in ts])
        self._check(self.lib.spmps_set_mps(self._h, dims.ctypes.data_as(C.POINTER(C.c_int)),
                                           lab.ctypes.data_as(C.POINTER(C.c_int)), arr, center))
        self._keep = ts

    # ---- excited states ------------------------------------------------------------------------
    def add_lower_state(self, labels, tensors):
        """A lower state to stay orthogonal to (in the projected metric, Eq. orthoB); format of set_mps."""
        dims = np.array([l.shape[0] for l in labels], dtype=np.int32)
        lab = np.ascontiguousarray(np.concatenate([np.asarray(l, dtype=np.int32).reshape(-1, 2) for l in labels]))
        ts = [np.ascontiguousarray(t, dtype=np.float64) for t in tensors]
        arr = (C.POINTER(C.c_double) * len(ts))(*[_dptr(t) for t in ts])
        self._check(self.lib.spmps_add_lower_state(self._h, dims.ctypes.data_as(C.POINTER(C.c_int)),
                                                   lab.ctypes.data_as(C.POINTER(C.c_int)), arr))

    def clear_lower_states(self):
        self._check(self.lib.spmps_clear_lower_states(self._h))

    def lower_overlap(self, j: int = 0) -> float:
        """<Psi_j| P |Psi> of the current MPS."""
        v = C.c_double()
        self._check(self.lib.spmps_lower_overlap(self._h, j, C.byref(v)))
        return v.value

    # ---- layout -------------------------------------------------------------------------------
    def x_layout(self, site: int):
        """Block table of the two-site tensor at (site, site+1): dict with n_x, blocks
        (n_blocks x 5: left label, s, column offset, rows, cols), row_off, width."""
        n = C.c_int64()
        nb = C.c_int()
        nl = C.c_int()
        self._check(self.lib.spmps_x_layout(self._h, site, C.byref(n), C.byref(nb), None, None, None, C.byref(nl)))
        blocks = np.zeros((max(nb.value, 1), 5), dtype=np.int32)
        ro = np.zeros(max(nl.value, 1), dtype=np.int64)
        wd = np.zeros(max(nl.value, 1), dtype=np.int32)
        self._check(self.lib.spmps_x_layout(self._h, site, C.byref(n), C.byref(nb),
                                            blocks.ctypes.data_as(C.POINTER(C.c_int)),
                                            ro.ctypes.data_as(C.POINTER(C.c_int64)),
                                            wd.ctypes.data_as(C.POINTER(C.c_int)), C.byref(nl)))
        return {"n_x": n.value, "blocks": blocks[:nb.value], "row_off": ro[:nl.value], "width": wd[:nl.value]}

    @staticmethod
    def pack(dense: np.ndarray, layout, ql: np.ndarray, qr: np.ndarray) -> np.ndarray:
        """Dense (Dl, 4, 4, Dr) two-site tensor -> row-block vector (index shuffling only)."""
        out = np.zeros(layout["n_x"])
        lab_l = _label_ranges(ql)
        lab_r = _label_ranges(qr)
        lq = [q for q, _, _ in lab_l]
        for la, s, col, rows, cols in layout["blocks"]:
            qa, a0, _ = lab_l[la]
            s1, s2 = divmod(int(s), 4)
            qb = (qa[0] + _LN[s1] + _LN[s2], qa[1] + _LM[s1] + _LM[s2])
            b0 = _find(lab_r, qb)
            blk = dense[a0:a0 + rows, s1, s2, b0:b0 + cols]
            w = layout["width"][la]
            ro = layout["row_off"][la]
            for i in range(rows):
                out[ro + i * w + col: ro + i * w + col + cols] = blk[i]
        del lq
        return out

    @staticmethod
    def unpack(vec: np.ndarray, layout, ql: np.ndarray, qr: np.ndarray) -> np.ndarray:
        dense = np.zeros((ql.shape[0], 4, 4, qr.shape[0]))
        lab_l = _label_ranges(ql)
        lab_r = _label_ranges(qr)
        for la, s, col, rows, cols in layout["blocks"]:
            qa, a0, _ = lab_l[la]
            s1, s2 = divmod(int(s), 4)
            qb = (qa[0] + _LN[s1] + _LN[s2], qa[1] + _LM[s1] + _LM[s2])
            b0 = _find(lab_r, qb)
            w = layout["width"][la]
            ro = layout["row_off"][la]
            for i in range(rows):
                dense[a0 + i, s1, s2, b0:b0 + cols] = vec[ro + i * w + col: ro + i * w + col + cols]
        return dense

    # ---- the hot path ----------------------------------------------------------------------
    def apply_heff(self, site: int, x, y=None, z=None, stream=None):
        """Device apply: x, y, z are CUDA torch tensors (float64, n_x) or raw pointers."""
        def ptr(t):
            if t is None:
                return None
            return C.c_void_p(t if isinstance(t, int) else t.data_ptr())
        s = None
        if stream is not None:
            s = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        self._check(self.lib.spmps_apply_heff(self._h, site, ptr(x), ptr(y), ptr(z), s))

    def apply_heff_noalloc(self, site: int, x, y=None, z=None, stream=None):
        """The projected action with no device allocation (intermediates in the library's fixed
        static scratch); needs a previous apply_heff for the same site."""
        def ptr(t):
            return None if t is None else C.c_void_p(t if isinstance(t, int) else t.data_ptr())
        s = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        self._check(self.lib.spmps_apply_heff_noalloc(self._h, site, ptr(x), ptr(y), ptr(z), s))

    def apply_heff_timed(self, site: int, x, y, z, stream=None):
        """Device apply with per-phase CUDA-event times (ms): [zero fill, A, B, C]; y or z may be
        None (that operator is then not applied)."""
        ms = np.zeros(4)
        s = None if stream is None else C.c_void_p(stream.cuda_stream)
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        self._check(self.lib.spmps_apply_heff_timed(self._h, site, ptr(x), ptr(y), ptr(z), s, _dptr(ms)))
        return ms

    def apply_flops(self, site: int):
        f = np.zeros(3)
        self._check(self.lib.spmps_apply_flops(self._h, site, _dptr(f)))
        return f

    def apply_costs(self, site: int):
        """Algorithmic (flops, bytes), each [[A, B, C] of H, [A, B, C] of N], of one projected
        action at `site`."""
        fl, by = np.zeros(6), np.zeros(6)
        self._check(self.lib.spmps_apply_costs(self._h, site, fl.ctypes.data_as(C.POINTER(C.c_double)),
                                               by.ctypes.data_as(C.POINTER(C.c_double))))
        return fl.reshape(2, 3), by.reshape(2, 3)

    def apply_heff_host(self, site: int, x: np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        z = np.zeros_like(x)
        self._check(self.lib.spmps_apply_heff_host(self._h, site, _dptr(x), _dptr(y), _dptr(z)))
        return y, z

    def two_site(self, site: int, x):
        self._check(self.lib.spmps_two_site(self._h, site, C.c_void_p(x if isinstance(x, int) else x.data_ptr())))

    def canonicalize(self):
        self._check(self.lib.spmps_canonicalize(self._h))

    def sweep(self, n_sweeps: int, allow_not_converged: bool = True):
        e = np.zeros(max(n_sweeps, 1))
        st = self.lib.spmps_sweep(self._h, n_sweeps, _dptr(e))
        if st != 0 and not (allow_not_converged and st == 2):
            self._check(st)
        return e[:n_sweeps], st

    def optimize_step(self, site: int, move_right: bool, allow_not_converged: bool = False):
        th = C.c_double()
        it = C.c_int()
        st = self.lib.spmps_optimize_step(self._h, site, 1 if move_right else 0, C.byref(th), C.byref(it))
        if st != 0 and not (allow_not_converged and st == 2):
            self._check(st)
        return th.value, it.value

    def energy(self):
        E = C.c_double()
        nP = C.c_double()
        self._check(self.lib.spmps_energy(self._h, C.byref(E), C.byref(nP)))
        return E.value, nP.value

    def expect_s2(self):
        v = C.c_double()
        self._check(self.lib.spmps_expect_s2(self._h, C.byref(v)))
        return v.value

    # ---- spin-free properties (Eq. PropSpinFree) ----------------------------------------------
    def expect_mpo(self, sites):
        ws = [np.ascontiguousarray(w, dtype=np.float64) for w in sites]
        dims = np.array([1] + [w.shape[1] for w in ws], dtype=np.int32)
        arr = (C.POINTER(C.c_double) * self.K)(*[_dptr(w) for w in ws])
        v = C.c_double()
        self._check(self.lib.spmps_expect_mpo(self._h, dims.ctypes.data_as(C.POINTER(C.c_int)), C.cast(arr, C.c_void_p),
                                              C.byref(v)))
        return v.value

    def fragment_energies(self):
        e = np.zeros(self.K)
        self._check(self.lib.spmps_fragment_energies(self._h, _dptr(e)))
        return e

    def rdm1(self):
        g = np.zeros((self.K, self.K))
        self._check(self.lib.spmps_rdm1(self._h, _dptr(g)))
        return g

    def spin_correlation(self, X, Y):
        x = np.ascontiguousarray(X, dtype=np.int32)
        y = np.ascontiguousarray(Y, dtype=np.int32)
        v = C.c_double()
        self._check(self.lib.spmps_spin_correlation(self._h, x.ctypes.data_as(C.POINTER(C.c_int)), len(x),
                                                    y.ctypes.data_as(C.POINTER(C.c_int)), len(y), C.byref(v)))
        return v.value

    def seniority(self):
        v = C.c_double()
        self._check(self.lib.spmps_seniority(self._h, C.byref(v)))
        return v.value

    def stats(self):
        c = (C.c_int64 * 3)()
        v = (C.c_double * 3)()
        self._check(self.lib.spmps_stats(self._h, c, v))
        return {"davidson_iterations": c[0], "applies": c[1], "launches": c[2],
                "apply_flops": v[0], "discarded_weight": v[1], "apply_flops_total": v[2]}

    def davidson_stats(self):
        """(iterations, FP64 refinement iterations) of the last sweep."""
        a = C.c_int64()
        b = C.c_int64()
        self._check(self.lib.spmps_davidson_stats(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def get_mps(self):
        """Checkpoint: (labels, tensors, center) in the format set_mps reads."""
        dims = np.zeros(self.K + 1, dtype=np.int32)
        cen = C.c_int()
        self._check(self.lib.spmps_get_mps(self._h, dims.ctypes.data_as(C.POINTER(C.c_int)), None, None, C.byref(cen)))
        lab = np.zeros(2 * int(dims.sum()), dtype=np.int32)
        ts = [np.zeros((int(dims[k]), 4, int(dims[k + 1]))) for k in range(self.K)]
        arr = (C.POINTER(C.c_double) * self.K)(*[_dptr(t) for t in ts])
        self._check(self.lib.spmps_get_mps(self._h, dims.ctypes.data_as(C.POINTER(C.c_int)),
                                           lab.ctypes.data_as(C.POINTER(C.c_int)), C.cast(arr, C.c_void_p),
                                           C.byref(cen)))
        labels, off = [], 0
        for b in range(self.K + 1):
            labels.append(lab[2 * off: 2 * (off + int(dims[b]))].reshape(-1, 2).astype(np.int64))
            off += int(dims[b])
        return labels, ts, cen.value

    def stream_handle(self) -> int:
        p = C.c_void_p()
        self._check(self.lib.spmps_stream(self._h, C.byref(p)))
        return p.value or 0

    def profile(self, enable: bool):
        self._check(self.lib.spmps_profile(self._h, 1 if enable else 0))

    def kernel_stats(self, kind: int):
        n = C.c_int64()
        ms = C.c_double()
        fl = C.c_double()
        self._check(self.lib.spmps_kernel_stats(self._h, kind, C.byref(n), C.byref(ms), C.byref(fl)))
        return {"launches": n.value, "ms": ms.value, "flops": fl.value}

    # ---- learned Davidson correction --------------------------------------------------------
    def mlp_harvest(self, enable=True, samples_per_iteration=512, capacity=1 << 21):
        """Harvest (features, target) pairs during Davidson solves; disabling keeps the pairs."""
        self._check(self.lib.spmps_mlp_harvest(self._h, 1 if enable else 0, samples_per_iteration,
                                               capacity if enable else 0))

    def mlp_data(self):
        n = C.c_int64()
        self._check(self.lib.spmps_mlp_data(self._h, C.byref(n), None, None))
        X = np.zeros((max(n.value, 1), 4), dtype=np.float32)
        T = np.zeros(max(n.value, 1), dtype=np.float32)
        self._check(self.lib.spmps_mlp_data(self._h, C.byref(n), X.ctypes.data_as(C.POINTER(C.c_float)),
                                            T.ctypes.data_as(C.POINTER(C.c_float))))
        return X[:n.value], T[:n.value]

    def mlp_set_params(self, flat):
        p = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(self.lib.spmps_mlp_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), 1))

    def mlp_get_params(self):
        p = np.zeros(67329, dtype=np.float32)
        self._check(self.lib.spmps_mlp_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), 0))
        return p

    def mlp_loss_grad(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        g = np.zeros(67329, dtype=np.float32)
        loss = C.c_double()
        self._check(self.lib.spmps_mlp_loss_grad(self._h, X.ctypes.data_as(C.POINTER(C.c_float)),
                                                 T.ctypes.data_as(C.POINTER(C.c_float)), X.shape[0], C.byref(loss),
                                                 g.ctypes.data_as(C.POINTER(C.c_float))))
        return loss.value, g

    def mlp_train(self, steps, batch=4096, lr=1e-3, seed=5, reinit=True):
        a = C.c_double()
        b = C.c_double()
        self._check(self.lib.spmps_mlp_train(self._h, steps, batch, lr, seed, 1 if reinit else 0, C.byref(a), C.byref(b)))
        return a.value, b.value

    def mlp_infer(self, r, dh, dn, theta, tensor_cores=True):
        r = np.ascontiguousarray(r, dtype=np.float64)
        dh = np.ascontiguousarray(dh, dtype=np.float64)
        dn = np.ascontiguousarray(dn, dtype=np.float64)
        t = np.zeros_like(r)
        self._check(self.lib.spmps_mlp_infer(self._h, _dptr(r), _dptr(dh), _dptr(dn), theta, r.shape[0], _dptr(t),
                                             1 if tensor_cores else 0))
        return t

    def quadrature(self):
        b = np.zeros(self.n_beta)
        c = np.zeros(self.n_beta)
        self._check(self.lib.spmps_quadrature(self._h, _dptr(b), _dptr(c)))
        return b, c


def mpo_from_integrals(h1, h2=None, ecore: float = 0.0):
    """The library's general MPO for integrals h1 (K x K) and chemist h2 (K^4): a list of
    (Dl, Dr, 4, 4) site tensors.  Host only."""
    lib = load_library()
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    K = h1.shape[0]
    h2p = None
    if h2 is not None:
        h2 = np.ascontiguousarray(h2, dtype=np.float64)
        h2p = h2.ctypes.data_as(C.POINTER(C.c_double))
    dims = np.zeros(K + 1, dtype=np.int32)
    st = lib.spmps_mpo_from_integrals(K, h1.ctypes.data_as(C.POINTER(C.c_double)), h2p, ecore,
                                      dims.ctypes.data_as(C.POINTER(C.c_int)), None)
    if st != 0:
        raise SpmpsError(st, lib.spmps_last_error(None).decode())
    ws = [np.zeros((int(dims[k]), int(dims[k + 1]), 4, 4)) for k in range(K)]
    arr = (C.POINTER(C.c_double) * K)(*[_dptr(w) for w in ws])
    st = lib.spmps_mpo_from_integrals(K, h1.ctypes.data_as(C.POINTER(C.c_double)), h2p, ecore,
                                      dims.ctypes.data_as(C.POINTER(C.c_int)), C.cast(arr, C.c_void_p))
    if st != 0:
        raise SpmpsError(st, lib.spmps_last_error(None).decode())
    return ws


def device_tf32_peak(kind: int, sms: int = 0, device: int = 0) -> float:
    """Measured dense tensor-core throughput (TFLOP/s): kind 0 = TF32 mma.sync.m16n8k8, kind 1 =
    tcgen05.mma kind::tf32, kind 2 = INT8 mma.sync.m16n8k32 (TOP/s); on `sms` SMs (0 = all)."""
    lib = load_library()
    v = C.c_double()
    st = lib.spmps_device_tf32_peak(device, kind, sms, C.byref(v))
    if st != 0:
        raise SpmpsError(st, "TF32 peak measurement failed")
    return v.value


def device_fp64_peak(device: int = 0) -> float:
    """Measured FP64 FMA throughput (TFLOP/s) of the device."""
    lib = load_library()
    v = C.c_double()
    st = lib.spmps_device_fp64_peak(device, C.byref(v))
    if st != 0:
        raise SpmpsError(st, lib.spmps_last_error(None).decode())
    return v.value


_LN = (0, 1, 1, 2)
_LM = (0, -1, 1, 0)


def _label_ranges(q: np.ndarray):
    """[(label, start, dim)] of a per-index label array sorted by (n, 2m)."""
    out = []
    q = np.asarray(q)
    i = 0
    while i < q.shape[0]:
        j = i
        while j < q.shape[0] and q[j, 0] == q[i, 0] and q[j, 1] == q[i, 1]:
            j += 1
        out.append(((int(q[i, 0]), int(q[i, 1])), i, j - i))
        i = j
    return out


def _find(ranges, q):
    for lab, start, _ in ranges:
        if lab == q:
            return start
    raise KeyError(q)
