"""Thin ctypes binding of liblhc (argument marshalling only).

Every computation runs in the CUDA library.  If ``liblhc.so`` has not been built
this module raises at load time; there is no CPU fallback.

Tensors are torch tensors (complex128 or complex64, C-contiguous) on a CUDA
device or on the host; the library stages host buffers itself.  Layouts are the
ones of ``include/lhc.h``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblhc.so")

KERNEL_PROJECT, KERNEL_CONTRACT, KERNEL_FUSED, KERNEL_REDUCE, KERNEL_COMBINE = range(5)
KERNEL_NAMES = ("project_f64", "contract", "fused_mma", "reduce_f64", "combine")
OK, EINVAL, ENOMEM, EBUDGET, ETIMEOUT, ECUDA, EBUSY, ENOTFOUND, ECANCELED = range(9)
FP64, MIXED = 0, 1
C128, C64 = 0, 1
MESON, BARYON = 0, 1
PRECISIONS = {"fp64": FP64, "mixed": MIXED}


class LhcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"liblhc status {status}: {msg}")
        self.status = status


class Lattice(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("T", ctypes.c_int), ("dtype", ctypes.c_int)]


class Call(ctypes.Structure):
    """One call of a batch (lhc_call)."""
    _fields_ = [("part", ctypes.c_int), ("lat", Lattice), ("S", ctypes.c_void_p), ("GB", ctypes.c_void_p),
                ("vec", ctypes.c_void_p), ("n_r", ctypes.c_int), ("t_lo", ctypes.c_int), ("t_hi", ctypes.c_int),
                ("r", ctypes.c_int * 4), ("k", ctypes.POINTER(ctypes.c_int)), ("nq", ctypes.c_int),
                ("out", ctypes.c_void_p)]


JOB_INSERTION, JOB_SPECTATOR, JOB_THREEPT = range(3)
JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED, JOB_CANCELED = range(5)


class Job(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("kind", ctypes.c_int), ("prec", ctypes.c_int),
                ("prop", ctypes.c_uint64), ("prop_b", ctypes.c_uint64),
                ("psi", ctypes.c_void_p), ("eta", ctypes.c_void_p), ("n_r", ctypes.c_int),
                ("t_lo", ctypes.c_int), ("t_hi", ctypes.c_int), ("t_sink", ctypes.c_int),
                ("r", ctypes.c_int * 4), ("k", ctypes.POINTER(ctypes.c_int)), ("nq", ctypes.c_int),
                ("out_ins", ctypes.c_void_p), ("out_spec", ctypes.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                               "(paper_1711_02384_gb300/build.py) first")
        L = ctypes.CDLL(LIB_PATH)
        vp, ci, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(Lattice)
        L.lhc_strerror.restype = ctypes.c_char_p
        L.lhc_strerror.argtypes = [ci]
        L.lhc_last_error.restype = ctypes.c_char_p
        L.lhc_last_error.argtypes = []
        L.lhc_version.restype = ci
        L.lhc_launch_count.restype = ctypes.c_ulonglong
        L.lhc_launch_count.argtypes = []
        L.lhc_create.argtypes = [ctypes.POINTER(vp), ci, sz]
        L.lhc_destroy.argtypes = [vp]
        L.lhc_set_gamma5.argtypes = [vp, ip]
        L.lhc_momenta.argtypes = [ci, ci, ip, ci, ip]
        L.lhc_insertion.argtypes = [vp, lp, vp, vp, ci, ci, ci, ip, ip, ci, ci, vp, vp]
        L.lhc_spectator.argtypes = [vp, lp, ci, vp, vp, vp, ci, ci, ip, ip, ci, ci, vp, vp]
        L.lhc_combine.argtypes = [vp, ci, vp, ci, vp, ci, ci, ci, vp, vp, vp, ci, ci, vp, vp]
        L.lhc_sync.argtypes = [vp, vp]
        u64 = ctypes.c_uint64
        L.lhc_release_workspace.argtypes = [vp]
        L.lhc_selftest_timeout.argtypes = [vp, ci, vp]
        L.lhc_selftest_flag.argtypes = [vp, ci, vp]
        L.lhc_serve_start.argtypes = [vp, ci]
        L.lhc_serve_stop.argtypes = [vp]
        L.lhc_prop_register.argtypes = [vp, vp, lp, ctypes.POINTER(u64)]
        L.lhc_prop_release.argtypes = [vp, u64]
        L.lhc_submit.argtypes = [vp, ctypes.POINTER(Job), ctypes.POINTER(u64)]
        L.lhc_poll.argtypes = [vp, u64, ip]
        L.lhc_wait.argtypes = [vp, u64, ci]
        L.lhc_cancel.argtypes = [vp, u64]
        dp = ctypes.POINTER(ctypes.c_double)
        L.lhc_job_times.argtypes = [vp, u64, dp, dp, dp]
        L.lhc_job_device_times.argtypes = [vp, u64, dp, dp]
        L.lhc_serve_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t), ip, ip]
        L.lhc_profile.argtypes = [vp, ci]
        L.lhc_profile_read.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]
        L.lhc_wilson_apply.argtypes = [vp, lp, ctypes.c_double, vp, ci, vp, vp, ci, vp]
        L.lhc_wilson_solve.argtypes = [vp, lp, ctypes.c_double, vp, vp, vp, ci, ctypes.c_double, ci, ip,
                                       ctypes.POINTER(ctypes.c_double), vp]
        L.lhc_combine_open.argtypes = [vp, vp, ci, vp, ci, ci, ci, vp, ci, vp, ci, ci, vp, vp]
        L.lhc_combine_open_baryon.argtypes = [vp, vp, ci, vp, ci, ci, ci, vp, ci, vp, ci, ci, vp, vp]
        L.lhc_set_projection.argtypes = [vp, ci]
        L.lhc_prop_stage.argtypes = [vp, lp, vp, ci, ci, vp]
        L.lhc_prop_unstage.argtypes = [vp, vp]
        L.lhc_batch.argtypes = [vp, ctypes.POINTER(Call), ci, vp]
        L.lhc_set_tuning.argtypes = [vp, ci, ctypes.c_char_p]
        L.lhc_tuning_table.argtypes = [ip, ci, ip]
        L.lhc_tuning_load.argtypes = [ctypes.c_char_p, ip]
        for name in ("lhc_prop_stage", "lhc_prop_unstage", "lhc_batch", "lhc_combine_open", "lhc_combine_open_baryon", "lhc_set_projection", "lhc_wilson_apply", "lhc_wilson_solve", "lhc_set_tuning", "lhc_tuning_table", "lhc_tuning_load",
                     "lhc_create", "lhc_destroy", "lhc_set_gamma5", "lhc_momenta", "lhc_insertion",
                     "lhc_spectator", "lhc_combine", "lhc_profile", "lhc_profile_read", "lhc_sync", "lhc_release_workspace",
                     "lhc_selftest_timeout", "lhc_selftest_flag", "lhc_serve_start", "lhc_serve_stop", "lhc_prop_register",
                     "lhc_prop_release", "lhc_submit", "lhc_poll", "lhc_wait", "lhc_cancel", "lhc_job_times",
                     "lhc_job_device_times", "lhc_serve_stats"):
            getattr(L, name).restype = ci
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise LhcError(status, lib().lhc_last_error().decode())


def launch_count() -> int:
    """Kernel launches this library has issued since it was loaded (graph replays excluded)."""
    return int(lib().lhc_launch_count())


TUNE_OFF, TUNE_ON = 0, 1
PROJECTIONS = {"auto": 0, "gemm": 1, "dft": 2}


def tuning_table() -> np.ndarray:
    """The process-wide launch-shape table: int [n][8] rows (part, dtype, V3, n_r, nt,
    nrep, NH, nsplit)."""
    n = ctypes.c_int(0)
    _check(lib().lhc_tuning_table(None, 0, ctypes.byref(n)))
    t = np.zeros((max(n.value, 1), 8), dtype=np.int32)
    _check(lib().lhc_tuning_table(t.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n.value, ctypes.byref(n)))
    return t[:n.value]


def tuning_load(path: str) -> int:
    """Load a launch-shape table file into the process-wide table (no GPU needed)."""
    n = ctypes.c_int(0)
    _check(lib().lhc_tuning_load(str(path).encode(), ctypes.byref(n)))
    return n.value


def momenta(n2max: int, cmax: int = -1) -> np.ndarray:
    """Momentum set of the library (|k|^2 <= n2max, |k_j| <= cmax if cmax >= 0)."""
    nq = ctypes.c_int(0)
    _check(lib().lhc_momenta(n2max, cmax, None, 0, ctypes.byref(nq)))
    k = np.zeros((nq.value, 3), dtype=np.int32)
    _check(lib().lhc_momenta(n2max, cmax, k.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), nq.value,
                             ctypes.byref(nq)))
    return k


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _dtype_code(t):
    if t.dtype == torch.complex128:
        return C128
    if t.dtype == torch.complex64:
        return C64
    raise ValueError(f"unsupported dtype {t.dtype}")


def _ints(v, n=None):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(-1))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} integers")
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _stream(t, stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if t.is_cuda:
        return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return ctypes.c_void_p(0)


def _L_of(V3):
    L = int(round(V3 ** (1.0 / 3.0)))
    if L ** 3 != V3:
        raise ValueError(f"{V3} sites is not a cube")
    return L


class Context:
    """An lhc context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, gamma5=(1, 1, -1, -1)):
        self._h = ctypes.c_void_p()
        self._staged = {}   # staged propagators by address, kept alive while staged
        _check(lib().lhc_create(ctypes.byref(self._h), int(device), int(hbm_budget)))
        self.device = device
        self.set_gamma5(gamma5)

    def close(self):
        if self._h:
            lib().lhc_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._staged.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def sync(self, stream=None):
        """Wait for the stream; raise if a kernel of this context gave up a bounded wait."""
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        _check(lib().lhc_sync(self._h, ctypes.c_void_p(int(stream))))

    def profile(self, enable: bool):
        """Start (clearing old records) or stop CUDA-event timing of the kernels."""
        _check(lib().lhc_profile(self._h, 1 if enable else 0))

    def profile_read(self, kernel: int):
        """(total device ms, launches, algorithmic work) recorded for one kernel class."""
        ms, n, w = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
        _check(lib().lhc_profile_read(self._h, kernel, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)))
        return ms.value, n.value, w.value

    def batch(self, calls, stream=None):
        """Mixed-precision calls in one persistent fused launch per part kind and
        momentum-chunk width (up to 64 calls per launch): each call a dict with
        part ("ins", "spec" or "baryon"), S, vec, optional GB, t_lo, t_hi (t_lo = t_hi =
        t_sink for spectators), r, k and optional out (device tensors).  Returns the
        outputs, bitwise those of the same calls made one by one in "gemm" projection mode
        (a batch always projects on the tensor cores)."""
        arr = (Call * len(calls))()
        keep, outs = [], []
        for a, c in zip(arr, calls):
            S, vec = c["S"], c["vec"]
            T, V3 = S.shape[0], S.shape[1]
            n_r = vec.shape[0]
            part = {"ins": 0, "spec": 1, "baryon": 2}[c["part"]]
            ka, kp = _ints(c["k"])
            ra, _ = _ints(c["r"], 4)
            nq = ka.size // 3
            nt = c["t_hi"] - c["t_lo"] + 1
            cols = 3072 if part == 2 else 192
            out = c.get("out")
            if out is None:
                shape = (nt, nq, n_r, cols) if part == 0 else (nq, n_r, cols)
                out = torch.empty(shape, dtype=torch.complex128, device=S.device)
            keep += [ka, ra]
            outs.append(out)
            a.part = part
            a.lat = Lattice(_L_of(V3), T, _dtype_code(S))
            addr = lambda t: None if t is None else _ptr(t).value
            a.S, a.vec, a.out, a.GB = addr(S), addr(vec), addr(out), addr(c.get("GB"))
            a.n_r, a.t_lo, a.t_hi, a.nq = n_r, c["t_lo"], c["t_hi"], nq
            for e in range(4):
                a.r[e] = int(ra[e])
            a.k = kp
        _check(lib().lhc_batch(self._h, arr, len(calls), _stream(calls[0]["S"], stream)))
        return outs

    def stage_propagator(self, S, t_lo, t_hi, stream=None):
        """Narrow slices t_lo..t_hi of the complex128 propagator S [T][V3][12][12] (device)
        once; later mixed insertion and meson spectator calls on those slices read the
        copy (bitwise the same results).  S must not change while staged (or is staged
        again after a change).  The copy is found by S's address, so the context keeps S
        alive until unstage_propagator(S) or close()."""
        T, V3 = S.shape[0], S.shape[1]
        lat = Lattice(_L_of(V3), T, _dtype_code(S))
        _check(lib().lhc_prop_stage(self._h, ctypes.byref(lat), _ptr(S), int(t_lo), int(t_hi), _stream(S, stream)))
        self._staged[S.data_ptr()] = S

    def unstage_propagator(self, S):
        _check(lib().lhc_prop_unstage(self._h, _ptr(S)))
        self._staged.pop(S.data_ptr(), None)

    def set_projection(self, mode: str):
        """Momentum projection of single calls: "auto" (a DFT over the slice when
        nq >= L^3 / 2), "gemm" (always the direct projection) or "dft" (always the
        all-momenta transform).  batch() always projects on the tensor cores."""
        _check(lib().lhc_set_projection(self._h, PROJECTIONS[mode]))

    def set_tuning(self, enable: bool, path=None):
        """Autotune the launch shape of each new mixed-precision shape on its first call
        (which then synchronizes its stream); path: optional table file, loaded now and
        rewritten after each new entry."""
        _check(lib().lhc_set_tuning(self._h, TUNE_ON if enable else TUNE_OFF,
                                    None if path is None else str(path).encode()))

    def _wilson_args(self, field, gammas):
        if field.dtype != torch.complex128 or not field.is_cuda or field.dim() != 4 or field.shape[-1] != 12:
            raise ValueError("fields are complex128 CUDA tensors [nrhs][T][L^3][12]")
        nrhs, T, V3 = field.shape[0], field.shape[1], field.shape[2]
        L = round(V3 ** (1 / 3))
        if L ** 3 != V3:
            raise ValueError("L^3 sites per timeslice expected")
        g = np.ascontiguousarray(np.asarray(gammas, dtype=np.complex128).reshape(4, 4, 4))
        return Lattice(L, T, C128), nrhs, g

    def wilson_apply(self, field, mass, gammas, dagger=False, out=None, stream=None):
        """D field (or D^dagger field) for the free (unit-link) Wilson-Dirac operator."""
        lat, nrhs, g = self._wilson_args(field, gammas)
        field = field.contiguous()
        out = torch.empty_like(field) if out is None else out
        _check(lib().lhc_wilson_apply(self._h, ctypes.byref(lat), float(mass), g.ctypes.data, 1 if dagger else 0,
                                      _ptr(field), _ptr(out), nrhs, _stream(field, stream)))
        return out

    def wilson_solve(self, src, mass, gammas, tol=1e-12, maxiter=2000, stream=None):
        """D^{-1} src (free Wilson-Dirac operator, CG on the normal equations);
        returns (solution, iterations, max relative residual |src - D sol| / |src|)."""
        lat, nrhs, g = self._wilson_args(src, gammas)
        src = src.contiguous()
        sol = torch.empty_like(src)
        it, res = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(lib().lhc_wilson_solve(self._h, ctypes.byref(lat), float(mass), g.ctypes.data, _ptr(src), _ptr(sol),
                                      nrhs, float(tol), int(maxiter), ctypes.byref(it), ctypes.byref(res),
                                      _stream(src, stream)))
        return sol, it.value, res.value

    def set_gamma5(self, g5):
        self._g5, p = _ints(g5, 4)
        _check(lib().lhc_set_gamma5(self._h, p))

    def insertion(self, S3, psi, t_lo, t_hi, r, k, prec="mixed", out=None, stream=None):
        """Insertion part (Eq. 10).  S3: [T][V3][12][12]; psi: [n_r][T][V3][12];
        returns complex128 [t_hi - t_lo + 1][nq][n_r][192]."""
        T, V3 = S3.shape[0], S3.shape[1]
        n_r = psi.shape[0]
        lat = Lattice(_L_of(V3), T, _dtype_code(S3))
        ka, kp = _ints(k)
        nq = ka.size // 3
        ra, rp = _ints(r, 4)
        nt = t_hi - t_lo + 1
        if out is None:
            out = torch.empty((nt, nq, n_r, 192), dtype=torch.complex128, device=S3.device)
        _check(lib().lhc_insertion(self._h, ctypes.byref(lat), _ptr(S3), _ptr(psi), n_r, t_lo, t_hi,
                                   rp, kp, nq, PRECISIONS[prec], _ptr(out), _stream(S3, stream)))
        return out

    def spectator(self, S1, eta, t_sink, r, k, prec="mixed", GB=None, out=None, stream=None):
        """Spectator part on slice t_sink: meson (Eq. 9) when GB is None, else the
        baryon eps-eps spectator with GA = S1.  eta: [n_r][V3][12].
        Returns complex128 [nq][n_r][192 | 3072]."""
        T, V3 = S1.shape[0], S1.shape[1]
        n_r = eta.shape[0]
        lat = Lattice(_L_of(V3), T, _dtype_code(S1))
        ka, kp = _ints(k)
        nq = ka.size // 3
        ra, rp = _ints(r, 4)
        kind = MESON if GB is None else BARYON
        cols = 192 if GB is None else 3072
        if out is None:
            out = torch.empty((nq, n_r, cols), dtype=torch.complex128, device=S1.device)
        _check(lib().lhc_spectator(self._h, ctypes.byref(lat), kind, _ptr(S1), _ptr(GB), _ptr(eta), n_r,
                                   t_sink, rp, kp, nq, PRECISIONS[prec], _ptr(out), _stream(S1, stream)))
        return out

    def combine(self, spec, ins, snk, ins_g, src, prec="fp64", out=None, stream=None):
        """Noise-averaged combine.  spec: [np][n_r][192 | 3072]; ins: [nq][n_r][192] (one
        insertion slice) or [nt][nq][n_r][192]; snk/src: [ng][4][4] (meson) or
        [ng][4][4][4] (baryon); ins_g: [ng][4][4].
        Returns complex128 [ng][np][nq] for one slice, else [nt][ng][np][nq]."""
        np_, n_r = spec.shape[0], spec.shape[1]
        single = ins.dim() == 3
        nt = 1 if single else ins.shape[0]
        nq = ins.shape[-3]
        kind = MESON if spec.shape[2] == 192 else BARYON
        ng = ins_g.shape[0]
        shape = (ng, np_, nq) if single else (nt, ng, np_, nq)
        if out is None:
            out = torch.empty(shape, dtype=torch.complex128, device=spec.device)
        _check(lib().lhc_combine(self._h, kind, _ptr(spec), np_, _ptr(ins), nq, n_r, nt, _ptr(snk), _ptr(ins_g),
                                 _ptr(src), ng, PRECISIONS[prec], _ptr(out), _stream(spec, stream)))
        return out

    def combine_open(self, spec, ins, snk, ins_g, prec="fp64", out=None, stream=None):
        """Open-source-spin meson combine: spec [np][n_r][192], ins [nt][nq][n_r][192] (or
        one slice [nq][n_r][192]), snk [ngs][4][4], ins_g [ngi][4][4]; returns complex128
        [nt][ngs][ngi][np][nq][4 al][4 be] (no nt axis for one slice).  Contract with
        Gsrc[be][al] for any source structure."""
        single = ins.dim() == 3
        nt = 1 if single else ins.shape[0]
        np_, n_r, nq = spec.shape[0], spec.shape[1], ins.shape[-3]
        ngs, ngi = snk.shape[0], ins_g.shape[0]
        shape = (nt, ngs, ngi, np_, nq, 4, 4)
        if out is None:
            out = torch.empty(shape, dtype=torch.complex128, device=spec.device)
        _check(lib().lhc_combine_open(self._h, _ptr(spec), np_, _ptr(ins), nq, n_r, nt, _ptr(snk), ngs, _ptr(ins_g),
                                      ngi, PRECISIONS[prec], _ptr(out), _stream(spec, stream)))
        return out[0] if single else out

    def combine_open_baryon(self, spec, ins, wsnk, ins_g, prec="fp64", out=None, stream=None):
        """Open-source-spin baryon combine: spec [np][n_r][3072], ins [nt][nq][n_r][192] (or
        one slice [nq][n_r][192]), wsnk [ngs][4][4][4], ins_g [ngi][4][4]; returns complex128
        [nt][ngs][ngi][np][nq][4 a1][4 a2][4 b] (no nt axis for one slice).  Contract with
        Wsrc[a1][a2][b] for any source structure."""
        single = ins.dim() == 3
        nt = 1 if single else ins.shape[0]
        np_, n_r, nq = spec.shape[0], spec.shape[1], ins.shape[-3]
        ngs, ngi = wsnk.shape[0], ins_g.shape[0]
        shape = (nt, ngs, ngi, np_, nq, 4, 4, 4)
        if out is None:
            out = torch.empty(shape, dtype=torch.complex128, device=spec.device)
        _check(lib().lhc_combine_open_baryon(self._h, _ptr(spec), np_, _ptr(ins), nq, n_r, nt, _ptr(wsnk), ngs,
                                             _ptr(ins_g), ngi, PRECISIONS[prec], _ptr(out), _stream(spec, stream)))
        return out[0] if single else out

    # ------------------------------------------------------------------ job server
    def serve_start(self, slots: int = 4):
        _check(lib().lhc_serve_start(self._h, int(slots)))

    def serve_stop(self):
        _check(lib().lhc_serve_stop(self._h))

    def prop_register(self, S):
        """Register a resident device propagator [T][V3][12][12]; returns its handle."""
        if not S.is_cuda:
            raise ValueError("registered propagators must be device tensors")
        lat = Lattice(_L_of(S.shape[1]), S.shape[0], _dtype_code(S))
        h = ctypes.c_uint64()
        _check(lib().lhc_prop_register(self._h, _ptr(S), ctypes.byref(lat), ctypes.byref(h)))
        return h.value

    def prop_release(self, handle):
        _check(lib().lhc_prop_release(self._h, ctypes.c_uint64(handle)))

    def submit(self, type, prop, k, r=(0, 0, 0, 0), prec="mixed", kind=MESON, prop_b=0, psi=None, eta=None,
               n_r=None, t_lo=0, t_hi=0, t_sink=0, out_ins=None, out_spec=None):
        """Submit a job; returns its id.  Tensors must stay alive until the job finishes."""
        ka, kp = _ints(k)
        j = Job()
        j.type, j.kind, j.prec = type, kind, PRECISIONS[prec]
        j.prop, j.prop_b = prop, prop_b
        j.psi = psi.data_ptr() if psi is not None else None
        j.eta = eta.data_ptr() if eta is not None else None
        j.n_r = n_r if n_r is not None else (psi.shape[0] if psi is not None else eta.shape[0])
        j.t_lo, j.t_hi, j.t_sink = t_lo, t_hi, t_sink
        for a in range(4):
            j.r[a] = int(r[a])
        j.k, j.nq = kp, ka.size // 3
        j.out_ins = out_ins.data_ptr() if out_ins is not None else None
        j.out_spec = out_spec.data_ptr() if out_spec is not None else None
        jid = ctypes.c_uint64()
        _check(lib().lhc_submit(self._h, ctypes.byref(j), ctypes.byref(jid)))
        return jid.value

    def poll(self, jid):
        """(status, state): status LHC_EBUSY (6) while queued/running, else LHC_OK."""
        st = ctypes.c_int()
        s = lib().lhc_poll(self._h, ctypes.c_uint64(jid), ctypes.byref(st))
        return s, st.value

    def wait(self, jid, timeout_ms=60000):
        _check(lib().lhc_wait(self._h, ctypes.c_uint64(jid), int(timeout_ms)))

    def wait_status(self, jid, timeout_ms=60000):
        return lib().lhc_wait(self._h, ctypes.c_uint64(jid), int(timeout_ms))

    def cancel(self, jid):
        return lib().lhc_cancel(self._h, ctypes.c_uint64(jid))

    def job_times(self, jid):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().lhc_job_times(self._h, ctypes.c_uint64(jid), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def job_device_times(self, jid):
        """(ms_start, ms_done) of a finished job on the device, after the server's epoch event."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().lhc_job_device_times(self._h, ctypes.c_uint64(jid), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def serve_stats(self):
        b, q, r = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
        _check(lib().lhc_serve_stats(self._h, ctypes.byref(b), ctypes.byref(q), ctypes.byref(r)))
        return b.value, q.value, r.value

    def selftest_timeout(self, limit_us=200000, stream=None):
        """Run the bounded-wait self-test; returns the lhc_sync status (LHC_ETIMEOUT expected)."""
        st = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        return lib().lhc_selftest_timeout(self._h, int(limit_us), ctypes.c_void_p(int(st)))

    def selftest_flag(self, limit_us=1000, stream=None):
        """The same bounded wait, leaving the device error word set until the next sync."""
        st = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        _check(lib().lhc_selftest_flag(self._h, int(limit_us), ctypes.c_void_p(int(st))))
