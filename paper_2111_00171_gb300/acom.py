"""Thin ctypes binding of libacom (include/acom.h).

Argument marshalling only: every step of the match runs in the library's CUDA
kernels.  PyTorch tensors supply device memory and the current CUDA stream.
The binding refuses to run when the compiled library is missing.
"""

from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

ACOM_OK = 0
ACOM_PREC_FP32 = 0
ACOM_PREC_BF16 = 1
ACOM_PREC_FP16 = 2
ACOM_PREC_FP8 = 3
STATUS = {0: "ACOM_OK", 1: "ACOM_ERR_INVALID_ARG", 2: "ACOM_ERR_OOM", 3: "ACOM_ERR_CUDA",
          4: "ACOM_ERR_TIMEOUT", 5: "ACOM_ERR_UNSUPPORTED", 6: "ACOM_ERR_BAD_INPUT"}

EXPORTED = ("acom_plan_create", "acom_plan_destroy", "acom_plan_get_info",
            "acom_plan_get_zone_axes", "acom_plan_get_spectra", "acom_match",
            "acom_polar_spectra", "acom_bounds", "acom_bounds_static", "acom_status_str",
            "acom_last_error",
            "acom_version", "acom_profile_enable", "acom_profile_reset", "acom_profile_read",
            "acom_kernel_launches", "acom_plan_concat", "acom_plan_get_phases", "acom_refine",
            "acom_refine_defaults", "acom_kinematical_score", "acom_kinematical_score_strain",
            "acom_match_multi",
            "acom_match_async", "acom_sync", "acom_autotune", "acom_device_allocations",
            "acom_set_device_wait_limit")


class AcomError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Crystal(C.Structure):
    _fields_ = [("lattice", (C.c_double * 3) * 3), ("n_atoms", C.c_int32),
                ("frac_pos", C.POINTER(C.c_double)), ("ff_A", C.POINTER(C.c_double)),
                ("ff_B", C.POINTER(C.c_double))]


class ZaGrid(C.Structure):
    _fields_ = [("v", (C.c_double * 3) * 3), ("step_deg", C.c_double),
                ("solid_angle", C.c_double)]


class Shells(C.Structure):
    _fields_ = [("n_shells", C.c_int32), ("dq", C.c_double)]


class PlanOpts(C.Structure):
    _fields_ = [("delta", C.c_double), ("gamma_pow", C.c_double), ("omega", C.c_double),
                ("lambda_", C.c_double), ("q_max", C.c_double), ("precision", C.c_int32)]


class PlanInfo(C.Structure):
    _fields_ = [("n_za", C.c_int32), ("n_shells", C.c_int32), ("n_phi", C.c_int32),
                ("n_freq", C.c_int32), ("n_reflections", C.c_int32), ("precision", C.c_int32),
                ("device_bytes", C.c_int64), ("last_evaluated", C.c_int64),
                ("n_phases", C.c_int32), ("last_refine_pairs", C.c_int64), ("k0", C.c_int32)]


class PeaksCSR(C.Structure):
    _fields_ = [("n_patterns", C.c_int64), ("row_ptr", C.c_void_p), ("qx", C.c_void_p),
                ("qy", C.c_void_p), ("I", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("za_idx", C.c_void_p), ("phi3_bin", C.c_void_p), ("mirror", C.c_void_p),
                ("score", C.c_void_p), ("score_cos", C.c_void_p), ("phi3", C.c_void_p),
                ("orient", C.c_void_p), ("za_scores", C.c_void_p), ("phase", C.c_void_p),
                ("phase_score", C.c_void_p), ("runner_za", C.c_void_p),
                ("runner_score", C.c_void_p), ("runner_orient", C.c_void_p)]


class MatchOpts(C.Structure):
    _fields_ = [("refine", C.c_int32), ("chunk", C.c_int32), ("exhaustive", C.c_int32),
                ("rescore_top", C.c_int32), ("tile_order", C.c_int32), ("cta_pairs", C.c_int32)]


class TuneResult(C.Structure):
    _fields_ = [("chunk", C.c_int32), ("tile_order", C.c_int32), ("cta_pairs", C.c_int32),
                ("ms", C.c_float)]


class RefineOpts(C.Structure):
    _fields_ = [("steps", C.c_int32), ("rho_start", C.c_float), ("rho_end", C.c_float),
                ("damping", C.c_float), ("max_step_deg", C.c_float), ("twin", C.c_int32)]


_LIB = None


def library_path():
    return _build.LIB


def load_library():
    """Load the in-tree libacom.so; raise if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libacom is not built ({path} missing): run "
                           "python -c 'import __graft_entry__ as g; g.build()'")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.acom_plan_create.argtypes = [C.POINTER(Crystal), C.POINTER(ZaGrid), C.POINTER(Shells),
                                     C.c_int32, C.c_double, C.POINTER(PlanOpts), P,
                                     C.POINTER(P)]
    lib.acom_plan_destroy.argtypes = [P]
    lib.acom_plan_get_info.argtypes = [P, C.POINTER(PlanInfo)]
    lib.acom_plan_concat.argtypes = [C.POINTER(P), C.c_int32, P, C.POINTER(P)]
    lib.acom_plan_get_phases.argtypes = [P, C.POINTER(C.c_int32)]
    lib.acom_refine.argtypes = [P, C.POINTER(PeaksCSR), C.POINTER(RefineOpts), P, P, P, P, P]
    lib.acom_refine_defaults.restype = RefineOpts
    lib.acom_kinematical_score.argtypes = [P, C.POINTER(PeaksCSR), P, P, C.c_float, P, P, P, P]
    lib.acom_kinematical_score_strain.argtypes = [P, C.POINTER(PeaksCSR), P, P, P, C.c_float, P,
                                                  P, P, P, P]
    lib.acom_match_multi.argtypes = [P, C.POINTER(PeaksCSR), C.POINTER(MatchOpts), C.c_int32,
                                     C.c_float, C.POINTER(Result), P]
    lib.acom_match_async.argtypes = [P, C.POINTER(PeaksCSR), C.POINTER(MatchOpts),
                                     C.POINTER(Result), P]
    lib.acom_sync.argtypes = [P, P]
    lib.acom_autotune.argtypes = [P, C.POINTER(PeaksCSR), C.POINTER(MatchOpts),
                                  C.POINTER(TuneResult), C.POINTER(TuneResult), P]
    lib.acom_plan_get_zone_axes.argtypes = [P, P]
    lib.acom_plan_get_spectra.argtypes = [P, P, P]
    lib.acom_match.argtypes = [P, C.POINTER(PeaksCSR), C.POINTER(MatchOpts), C.POINTER(Result), P]
    lib.acom_polar_spectra.argtypes = [P, C.POINTER(PeaksCSR), P, P, P]
    lib.acom_bounds.argtypes = [P, C.POINTER(PeaksCSR), P, P]
    lib.acom_bounds_static.argtypes = [P, C.POINTER(PeaksCSR), P, P]
    lib.acom_profile_enable.argtypes = [C.c_int32]
    lib.acom_profile_enable.restype = None
    lib.acom_profile_reset.restype = None
    lib.acom_kernel_launches.restype = C.c_int64
    lib.acom_device_allocations.restype = C.c_int64
    lib.acom_set_device_wait_limit.argtypes = [C.c_int64]
    lib.acom_set_device_wait_limit.restype = None
    lib.acom_status_str.restype = C.c_char_p
    lib.acom_status_str.argtypes = [C.c_int]
    lib.acom_last_error.restype = C.c_char_p
    lib.acom_version.restype = C.c_int32
    for name in ("acom_plan_create", "acom_plan_destroy", "acom_plan_get_info",
                 "acom_plan_concat", "acom_plan_get_phases", "acom_refine",
                 "acom_kinematical_score", "acom_kinematical_score_strain", "acom_match_multi",
                 "acom_match_async", "acom_sync",
                 "acom_autotune",
                 "acom_plan_get_zone_axes", "acom_plan_get_spectra", "acom_match",
                 "acom_polar_spectra", "acom_bounds", "acom_bounds_static"):
        getattr(lib, name).restype = C.c_int
    _LIB = lib
    return lib


def _check(status):
    if status != ACOM_OK:
        msg = load_library().acom_last_error().decode()
        raise AcomError(status, msg)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


@dataclass
class CrystalSpec:
    """Lattice rows (Angstrom), fractional basis and single-Gaussian form
    factors f_n(q) = A_n exp(-B_n q^2)."""
    lattice: np.ndarray
    frac_pos: np.ndarray
    ff_A: np.ndarray
    ff_B: np.ndarray


def cubic_triangle():
    """[001], [011], [111]; the m-3m standard triangle covers 4 pi / 48."""
    return [[0, 0, 1], [0, 1, 1], [1, 1, 1]], 4 * math.pi / 48


def hexagonal_triangle():
    """[0001], a axis, 30 degrees in the basal plane; 1/24 of the sphere."""
    return [[0, 0, 1], [1, 0, 0], [math.cos(math.pi / 6), math.sin(math.pi / 6), 0]], \
        4 * math.pi / 24


class Plan:
    """Orientation plan on the current CUDA device (acom_plan_create)."""

    def __init__(self, crystal: CrystalSpec, za_vectors, solid_angle, step_deg, n_shells, dq,
                 n_phi, delta=0.08, gamma_pow=1.0, omega=1.0, lam=0.01969, q_max=1.5,
                 sigma_exc=0.02, precision=ACOM_PREC_FP32, stream=None):
        import torch  # noqa: F401  (device context)
        lib = load_library()
        self._lib = lib
        lat = np.ascontiguousarray(crystal.lattice, dtype=np.float64)
        self._pos = np.ascontiguousarray(crystal.frac_pos, dtype=np.float64).reshape(-1, 3)
        self._A = np.ascontiguousarray(crystal.ff_A, dtype=np.float64).reshape(-1)
        self._B = np.ascontiguousarray(crystal.ff_B, dtype=np.float64).reshape(-1)
        cr = Crystal()
        for i in range(3):
            for j in range(3):
                cr.lattice[i][j] = float(lat[i, j])
        cr.n_atoms = len(self._pos)
        dp = C.POINTER(C.c_double)
        cr.frac_pos = self._pos.ctypes.data_as(dp)
        cr.ff_A = self._A.ctypes.data_as(dp)
        cr.ff_B = self._B.ctypes.data_as(dp)
        g = ZaGrid()
        for i in range(3):
            for j in range(3):
                g.v[i][j] = float(za_vectors[i][j])
        g.step_deg = float(step_deg)
        g.solid_angle = float(solid_angle)
        sh = Shells(int(n_shells), float(dq))
        op = PlanOpts(float(delta), float(gamma_pow), float(omega), float(lam), float(q_max),
                      int(precision))
        h = C.c_void_p()
        _check(lib.acom_plan_create(C.byref(cr), C.byref(g), C.byref(sh), int(n_phi),
                                    float(sigma_exc), C.byref(op), _stream_ptr(stream),
                                    C.byref(h)))
        self.handle = h
        self.step_deg = float(step_deg)
        self.info = self.get_info()

    @classmethod
    def concat(cls, plans, stream=None):
        """One plan over the zone axes of several phases' plans
        (acom_plan_concat); the inputs stay owned by the caller."""
        lib = load_library()
        arr = (C.c_void_p * len(plans))(*(p.handle.value for p in plans))
        h = C.c_void_p()
        _check(lib.acom_plan_concat(arr, len(plans), _stream_ptr(stream), C.byref(h)))
        self = cls.__new__(cls)
        self._lib = lib
        self.handle = h
        self.step_deg = plans[0].step_deg
        self.info = self.get_info()
        return self

    def phases(self):
        """Phase offsets [n_phases + 1]: phase p owns axes [off[p], off[p+1])."""
        out = (C.c_int32 * (self.info["n_phases"] + 1))()
        _check(self._lib.acom_plan_get_phases(self.handle, out))
        return np.array(out[:], dtype=np.int64)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            _check(self._lib.acom_plan_destroy(self.handle))
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def get_info(self):
        inf = PlanInfo()
        _check(self._lib.acom_plan_get_info(self.handle, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in PlanInfo._fields_}

    def zone_axes(self):
        out = np.empty((self.info["n_za"], 3), dtype=np.float64)
        _check(self._lib.acom_plan_get_zone_axes(self.handle, out.ctypes.data_as(C.c_void_p)))
        return out

    def spectra(self, stream=None):
        import torch
        i = self.info
        out = torch.empty((i["n_za"], i["n_shells"], i["n_freq"], 2), dtype=torch.float32,
                          device="cuda")
        _check(self._lib.acom_plan_get_spectra(self.handle, _ptr(out), _stream_ptr(stream)))
        return out

    @staticmethod
    def _csr(row_ptr, qx, qy, I):
        import torch
        for t, dt in ((row_ptr, torch.int64), (qx, torch.float32), (qy, torch.float32),
                      (I, torch.float32)):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise ValueError("peaks must be contiguous CUDA tensors: row_ptr int64, "
                                 "qx/qy/I float32")
        return PeaksCSR(row_ptr.numel() - 1, row_ptr.data_ptr(), qx.data_ptr(), qy.data_ptr(),
                        I.data_ptr())

    def polar_spectra(self, row_ptr, qx, qy, I, stream=None):
        """[B][S][F][2] spectra of the sparse polar images and ||X||_2."""
        import torch
        pk = self._csr(row_ptr, qx, qy, I)
        i = self.info
        out = torch.empty((pk.n_patterns, i["n_shells"], i["n_freq"], 2), dtype=torch.float32,
                          device="cuda")
        xn = torch.empty((pk.n_patterns,), dtype=torch.float32, device="cuda")
        _check(self._lib.acom_polar_spectra(self.handle, C.byref(pk), _ptr(out), _ptr(xn),
                                            _stream_ptr(stream)))
        return out, xn.sqrt()

    def bounds(self, row_ptr, qx, qy, I, stream=None):
        """[B][Z] spectral bounds of the contraction (acom_bounds)."""
        import torch
        pk = self._csr(row_ptr, qx, qy, I)
        out = torch.empty((pk.n_patterns, self.info["n_za"]), dtype=torch.float32, device="cuda")
        _check(self._lib.acom_bounds(self.handle, C.byref(pk), _ptr(out), _stream_ptr(stream)))
        return out

    def bounds_static(self, row_ptr, qx, qy, I, out, stream=None):
        """acom_bounds_static into the caller's [B][Z] tensor ``out`` (no device
        allocation inside the library call).  ``out`` must be a contiguous
        float32 CUDA tensor of shape (B, n_za) on the device current for the
        plan: the library writes B x n_za values through its pointer."""
        import torch
        pk = self._csr(row_ptr, qx, qy, I)
        shape = (pk.n_patterns, self.info["n_za"])
        if (not isinstance(out, torch.Tensor) or not out.is_cuda
                or out.device.index != torch.cuda.current_device()
                or out.dtype != torch.float32 or not out.is_contiguous()
                or tuple(out.shape) != shape):
            raise ValueError(f"out must be a contiguous float32 CUDA tensor of shape {shape} "
                             "on the current device")
        _check(self._lib.acom_bounds_static(self.handle, C.byref(pk), _ptr(out),
                                            _stream_ptr(stream)))
        return out

    def alloc_result(self, n, za_scores=False, orient=True, phase_scores=False, runner=False):
        import torch
        dev = "cuda"
        r = {"za_idx": torch.empty(n, dtype=torch.int32, device=dev),
             "phi3_bin": torch.empty(n, dtype=torch.int32, device=dev),
             "mirror": torch.empty(n, dtype=torch.uint8, device=dev),
             "score": torch.empty(n, dtype=torch.float32, device=dev),
             "score_cos": torch.empty(n, dtype=torch.float32, device=dev)}
        if orient:
            r["phi3"] = torch.empty(n, dtype=torch.float32, device=dev)
            r["orient"] = torch.empty((n, 3, 3), dtype=torch.float32, device=dev)
        if za_scores:
            r["za_scores"] = torch.empty((n, self.info["n_za"]), dtype=torch.float32, device=dev)
        if runner:
            r["runner_za"] = torch.empty(n, dtype=torch.int32, device=dev)
            r["runner_score"] = torch.empty(n, dtype=torch.float32, device=dev)
            r["runner_orient"] = torch.empty((n, 3, 3), dtype=torch.float32, device=dev)
        if phase_scores:
            r["phase"] = torch.empty(n, dtype=torch.int32, device=dev)
            r["phase_score"] = torch.empty((n, self.info["n_phases"]), dtype=torch.float32,
                                           device=dev)
        return r

    def match(self, row_ptr, qx, qy, I, refine=True, chunk=0, za_scores=False, out=None,
              exhaustive=False, phase_scores=False, runner=False, rescore_top=0, tile_order=0,
              cta_pairs=0, stream=None):
        """acom_match on device CSR tensors; returns a dict of device tensors
        (with phase_scores: the phase of each winner and every phase's best;
        with runner: the runner-up axis, score and grid orientation;
        cta_pairs=1: the tensor-core contraction on CTA pairs instead of one
        CTA per MMA)."""
        pk = self._csr(row_ptr, qx, qy, I)
        r = out if out is not None else self.alloc_result(pk.n_patterns, za_scores=za_scores,
                                                          phase_scores=phase_scores,
                                                          runner=runner)
        res = Result(*(_ptr(r.get(k)) for k, _ in Result._fields_))
        opts = MatchOpts(1 if refine else 0, int(chunk), 1 if exhaustive else 0, int(rescore_top),
                         int(tile_order), int(cta_pairs))
        _check(self._lib.acom_match(self.handle, C.byref(pk), C.byref(opts), C.byref(res),
                                    _stream_ptr(stream)))
        return r


    def match_async(self, row_ptr, qx, qy, I, out, refine=True, chunk=0, exhaustive=False,
                    rescore_top=0, tile_order=0, stream=None):
        """acom_match_async into the result dict ``out`` (alloc_result): the
        work is only enqueued; sync() returns its status.  Capturable into a
        CUDA graph once a synchronous match has sized the workspace."""
        pk = self._csr(row_ptr, qx, qy, I)
        res = Result(*(_ptr(out.get(k)) for k, _ in Result._fields_))
        opts = MatchOpts(1 if refine else 0, int(chunk), 1 if exhaustive else 0, int(rescore_top),
                         int(tile_order))
        _check(self._lib.acom_match_async(self.handle, C.byref(pk), C.byref(opts), C.byref(res),
                                          _stream_ptr(stream)))
        return out

    def autotune(self, row_ptr, qx, qy, I, stream=None):
        """acom_autotune on a sample of peaks: (best, trials), each a dict of
        chunk, tile_order, cta_pairs and ms."""
        pk = self._csr(row_ptr, qx, qy, I)
        best = TuneResult()
        trials = (TuneResult * 12)()
        _check(self._lib.acom_autotune(self.handle, C.byref(pk), None, C.byref(best), trials,
                                       _stream_ptr(stream)))
        as_dict = lambda t: {"chunk": t.chunk, "tile_order": t.tile_order,
                             "cta_pairs": t.cta_pairs, "ms": t.ms}
        return as_dict(best), [as_dict(t) for t in trials]

    def sync(self, stream=None):
        """acom_sync: wait for the stream; the status of the last async match."""
        _check(self._lib.acom_sync(self.handle, _stream_ptr(stream)))

    def match_multi(self, row_ptr, qx, qy, I, n_matches=3, r_del=0.04, refine=True, chunk=0,
                    exhaustive=False, stream=None):
        """acom_match_multi: up to n_matches orientations per pattern by
        iterative peak deletion; returns one result dict per match (score and
        score_cos of the original pattern; za_idx -1 where nothing was left)."""
        pk = self._csr(row_ptr, qx, qy, I)
        outs = [self.alloc_result(pk.n_patterns) for _ in range(n_matches)]
        arr = (Result * n_matches)(*[Result(*(_ptr(r.get(k)) for k, _ in Result._fields_))
                                     for r in outs])
        opts = MatchOpts(1 if refine else 0, int(chunk), 1 if exhaustive else 0)
        _check(self._lib.acom_match_multi(self.handle, C.byref(pk), C.byref(opts),
                                          int(n_matches), float(r_del), arr,
                                          _stream_ptr(stream)))
        return outs

    # ---- continuous refinement (acom_refine, acom_kinematical_score)

    def refine(self, row_ptr, qx, qy, I, orient, orient_alt=None, steps=20, rho_start=0.15,
               rho_end=0.03, damping=0.3, max_step_deg=1.0, twin=True, stream=None):
        """acom_refine: ascent of the kinematical score from ``orient``
        ([B][3][3] FP32 CUDA tensor, overwritten with the refined m) and, if
        given, from ``orient_alt`` (e.g. the match's runner_orient); returns
        (orient, score [B], winning start [B] uint8: bit 0 twin, bit 1 alt)."""
        import torch
        pk = self._csr(row_ptr, qx, qy, I)
        if orient.dtype != torch.float32 or not orient.is_cuda or not orient.is_contiguous():
            raise ValueError("orient must be a contiguous float32 CUDA tensor [B][3][3]")
        score = torch.empty(pk.n_patterns, dtype=torch.float32, device="cuda")
        tw = torch.empty(pk.n_patterns, dtype=torch.uint8, device="cuda")
        opts = RefineOpts(int(steps), float(rho_start), float(rho_end), float(damping),
                          float(max_step_deg), 1 if twin else 0)
        alt = None if orient_alt is None else orient_alt.contiguous()
        _check(self._lib.acom_refine(self.handle, C.byref(pk), C.byref(opts), _ptr(orient),
                                     _ptr(alt), _ptr(score), _ptr(tw), _stream_ptr(stream)))
        return orient, score, tw

    def kinematical_score(self, row_ptr, qx, qy, I, orient, r=None, rho=0.03, strain=None,
                          stream=None):
        """acom_kinematical_score at Exp(r) m^T: (score [B], dS/dr [B][3],
        Gauss-Newton matrix [B][6]); with ``strain`` ([B][6] reciprocal-lattice
        strain xx xy xz yy yz zz, acom_kinematical_score_strain) also dS/de
        [B][6] as a fourth element."""
        import torch
        pk = self._csr(row_ptr, qx, qy, I)
        n = pk.n_patterns
        score = torch.empty(n, dtype=torch.float32, device="cuda")
        grad = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        gn = torch.empty((n, 6), dtype=torch.float32, device="cuda")
        rr = None if r is None else r.detach().to(torch.float32).contiguous()
        if strain is None:
            _check(self._lib.acom_kinematical_score(self.handle, C.byref(pk),
                                                    _ptr(orient.contiguous()), _ptr(rr),
                                                    float(rho), _ptr(score), _ptr(grad),
                                                    _ptr(gn), _stream_ptr(stream)))
            return score, grad, gn
        ee = strain.detach().to(torch.float32).contiguous()
        if tuple(ee.shape) != (n, 6) or not ee.is_cuda:
            raise ValueError("strain must be a CUDA tensor [B][6]")
        de = torch.empty((n, 6), dtype=torch.float32, device="cuda")
        _check(self._lib.acom_kinematical_score_strain(self.handle, C.byref(pk),
                                                       _ptr(orient.contiguous()), _ptr(rr),
                                                       _ptr(ee), float(rho), _ptr(score),
                                                       _ptr(grad), _ptr(gn), _ptr(de),
                                                       _stream_ptr(stream)))
        return score, grad, gn, de


def _autograd_function():
    import torch

    class KinematicalScore(torch.autograd.Function):
        """S(r) = kinematical score at Exp(r) m^T for each pattern, with its
        hand-written gradient dS/dr from the same kernel launch."""

        @staticmethod
        def forward(ctx, r, plan, peaks, orient, rho):
            s, g, _ = plan.kinematical_score(*peaks, orient, r=r, rho=rho)
            ctx.save_for_backward(g)
            return s

        @staticmethod
        def backward(ctx, gs):
            (g,) = ctx.saved_tensors
            return gs[:, None] * g, None, None, None, None

    class KinematicalScoreStrain(torch.autograd.Function):
        """S(r, e) with the reciprocal lattice strained by e ([B][6]), with
        dS/dr and dS/de from the same kernel launch."""

        @staticmethod
        def forward(ctx, r, e, plan, peaks, orient, rho):
            s, g, _, de = plan.kinematical_score(*peaks, orient, r=r, rho=rho, strain=e)
            ctx.save_for_backward(g, de)
            return s

        @staticmethod
        def backward(ctx, gs):
            g, de = ctx.saved_tensors
            return gs[:, None] * g, gs[:, None] * de, None, None, None, None

    return KinematicalScore, KinematicalScoreStrain


def kinematical_score(r, plan, peaks, orient, rho=0.03):
    """Differentiable S(r) (torch.autograd.Function): ``peaks`` is the
    (row_ptr, qx, qy, I) tuple of CUDA tensors, ``orient`` the [B][3][3] base
    orientations, ``r`` [B][3] axis-angle vectors."""
    global _KIN
    if _KIN is None:
        _KIN = _autograd_function()
    return _KIN[0].apply(r, plan, peaks, orient, rho)


def kinematical_score_strain(r, e, plan, peaks, orient, rho=0.03):
    """Differentiable S(r, e): as kinematical_score, with ``e`` [B][6] the
    reciprocal-lattice strain (xx, xy, xz, yy, yz, zz) of each pattern."""
    global _KIN
    if _KIN is None:
        _KIN = _autograd_function()
    return _KIN[1].apply(r, e, plan, peaks, orient, rho)


_KIN = None


def au_crystal(a=4.08):
    """fcc Au, f(q) = 79 exp(-0.25 q^2)."""
    return CrystalSpec(np.eye(3) * a,
                       np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], float),
                       np.full(4, 79.0), np.full(4, 0.25))


def mg_crystal(a=3.21, c=5.21):
    """hcp Mg-like P6_3/mmc, f(q) = 12 exp(-0.3 q^2)."""
    L = np.array([[a, 0, 0], [-a / 2, a * math.sqrt(3) / 2, 0], [0, 0, c]])
    return CrystalSpec(L, np.array([[1 / 3, 2 / 3, .25], [2 / 3, 1 / 3, .75]]),
                       np.full(2, 12.0), np.full(2, 0.3))
