"""Python binding of libeor21 (include/eor21.h): argument marshalling only.

Every step of the likelihood path runs in the library's CUDA kernels; this module
turns numpy arrays (host memory, EOR_HOST) and CUDA torch tensors (device memory,
EOR_DEVICE) into pointers and calls the C ABI by the same names. If the shared
library is missing it raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

EOR_OK, EOR_EINVAL, EOR_ENOMEM, EOR_ECUDA, EOR_ETIMEOUT, EOR_ESTATE, EOR_ENOTSUP = range(7)
EOR_HOST, EOR_DEVICE = 0, 1
MAX_Z, MAX_BINS, MAX_RADII = 8, 64, 64

# names exported by include/eor21.h
EXPORTS = ("eor_default_config", "eor_create", "eor_init_boxes", "eor_set_efficiency", "eor_set_params",
           "eor_run_ionization",
           "eor_power_spectrum", "eor_chi2", "eor_likelihood", "eor_filtered_density",
           "eor_density_spectrum", "eor_density_box", "eor_walker_ladder", "eor_box_power_spectrum", "eor_set_tuning", "eor_set_ps_split", "eor_set_ps_streams", "eor_get_tuning", "eor_autotune", "eor_noise_sigma", "eor_set_method", "eor_basis_info", "eor_basis_window", "eor_contraction_info", "eor_debug_withhold", "eor_trace",
           "eor_trace_read", "eor_kernel_class_name", "eor_launch_count", "eor_box_power_spectrum_noalloc",
           "eor_tensor_core_check", "eor_last_error", "eor_version", "eor_destroy",
           "eor_emu_default_config", "eor_emu_create", "eor_emu_n_params", "eor_emu_set_data", "eor_emu_train",
           "eor_emu_forward", "eor_emu_loss_grad", "eor_emu_train_batch", "eor_emu_get_weights",
           "eor_emu_set_weights", "eor_emu_get_normalization", "eor_emu_set_normalization", "eor_emu_predict",
           "eor_emu_calibrate", "eor_emu_set_threshold", "eor_emu_likelihood", "eor_emu_set_inference",
           "eor_emu_inference", "eor_emu_last_error",
           "eor_emu_destroy", "eor_mcmc_default_config", "eor_mcmc_create", "eor_mcmc_start", "eor_mcmc_run",
           "eor_mcmc_walkers", "eor_mcmc_last_error", "eor_mcmc_destroy")
EMU_MAX_HIDDEN, EMU_MAX_MEMBERS = 8, 8
KERNEL_CLASSES = 8
EOR_METHOD_BASIS, EOR_METHOD_DIRECT, EOR_METHOD_BASIS_SIMT, EOR_METHOD_BASIS_TF32 = 0, 1, 2, 3
EOR_CONTRACT_NONE, EOR_CONTRACT_FP32, EOR_CONTRACT_TF32, EOR_CONTRACT_FP16 = 0, 1, 2, 3

_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class EorConfig(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("box_mpc", ctypes.c_double), ("n_z", ctypes.c_int),
                ("z", ctypes.c_double * MAX_Z),
                ("h", ctypes.c_double), ("omega_m", ctypes.c_double), ("omega_b", ctypes.c_double),
                ("n_s", ctypes.c_double), ("sigma8", ctypes.c_double),
                ("r_factor", ctypes.c_double), ("r_cell_rule", ctypes.c_int), ("delta_c", ctypes.c_double),
                ("mu", ctypes.c_double), ("n_bins", ctypes.c_int), ("k_lo", ctypes.c_double),
                ("k_hi", ctypes.c_double), ("chi2_k_lo", ctypes.c_double), ("chi2_k_hi", ctypes.c_double),
                ("max_walkers", ctypes.c_int), ("r_mfp_max", ctypes.c_double),
                ("dev_alloc", _ALLOC), ("dev_free", _FREE), ("alloc_user", ctypes.c_void_p),
                ("rsd", ctypes.c_int), ("rsd_max_dvdr", ctypes.c_double), ("zeldovich", ctypes.c_int),
                ("efficiency_model", ctypes.c_int)]


class EmuConfig(ctypes.Structure):
    _fields_ = [("n_z", ctypes.c_int), ("z", ctypes.c_double * MAX_Z), ("n_bins", ctypes.c_int),
                ("hidden", ctypes.c_int), ("n_hidden", ctypes.c_int), ("members", ctypes.c_int),
                ("max_rows", ctypes.c_int), ("max_samples", ctypes.c_int),
                ("prior_lo", ctypes.c_double * 3), ("prior_hi", ctypes.c_double * 3),
                ("d2_floor", ctypes.c_double), ("err_tol", ctypes.c_double), ("seed", ctypes.c_ulonglong)]


class McmcConfig(ctypes.Structure):
    _fields_ = [("n_walkers", ctypes.c_int), ("a", ctypes.c_double), ("prior_lo", ctypes.c_double * 3),
                ("prior_hi", ctypes.c_double * 3), ("xhi_prior_z", ctypes.c_int), ("xhi_prior_min", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("gauss_target", ctypes.c_int), ("gauss_mean", ctypes.c_double * 3),
                ("gauss_precision", ctypes.c_double * 9)]


class EorError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libeor21 error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load (building first if allowed) the in-tree libeor21.so; raise if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if build_if_missing and _build.stale():
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libeor21 is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "eor_default_config": (None, [ctypes.POINTER(EorConfig)]),
        "eor_create": (I, [ctypes.POINTER(EorConfig), P, ctypes.POINTER(P)]),
        "eor_init_boxes": (I, [P, P, I]),
        "eor_set_params": (I, [P, P, I, I]),
        "eor_set_efficiency": (I, [P, P, I, I]),
        "eor_run_ionization": (I, [P, P, P, I]),
        "eor_power_spectrum": (I, [P, P, P, P, I]),
        "eor_chi2": (I, [P, P, P, P, I]),
        "eor_likelihood": (I, [P, P, I, P, P, P, P, I]),
        "eor_filtered_density": (I, [P, I, D, P, I]),
        "eor_density_spectrum": (I, [P, I, P, I]),
        "eor_density_box": (I, [P, I, P, I]),
        "eor_walker_ladder": (I, [P, I, P, ctypes.POINTER(I)]),
        "eor_box_power_spectrum": (I, [P, P, P, P, P, I]),
        "eor_set_tuning": (I, [P, I, I, I]),
        "eor_set_ps_split": (I, [P, I]),
        "eor_set_ps_streams": (I, [P, I]),
        "eor_get_tuning": (I, [P] + [ctypes.POINTER(I)] * 5),
        "eor_set_method": (I, [P, I]),
        "eor_autotune": (I, [P, P, I, P, P, I, P, P, P, P, I]),
        "eor_noise_sigma": (I, [P, P, P, D, P, I]),
        "eor_basis_info": (I, [P, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "eor_basis_window": (I, [P, D, P, I]),
        "eor_debug_withhold": (I, [P, I, D]),
        "eor_contraction_info": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "eor_trace": (I, [P, I]),
        "eor_trace_read": (I, [P, P, P, I]),
        "eor_kernel_class_name": (ctypes.c_char_p, [I]),
        "eor_launch_count": (ctypes.c_longlong, [P]),
        "eor_box_power_spectrum_noalloc": (I, [I, D, I, D, D, P, P, P, P]),
        "eor_tensor_core_check": (I, [P, P, P, I, P, P]),
        "eor_last_error": (ctypes.c_char_p, [P]),
        "eor_version": (ctypes.c_char_p, []),
        "eor_destroy": (None, [P]),
        "eor_emu_default_config": (None, [ctypes.POINTER(EmuConfig)]),
        "eor_emu_create": (I, [ctypes.POINTER(EmuConfig), P, ctypes.POINTER(P)]),
        "eor_emu_n_params": (ctypes.c_longlong, [P]),
        "eor_emu_set_data": (I, [P, P, P, I, I]),
        "eor_emu_train": (I, [P, I, I, D, ctypes.c_ulonglong, P]),
        "eor_emu_forward": (I, [P, P, I, P, I]),
        "eor_emu_loss_grad": (I, [P, P, P, I, P, P, I]),
        "eor_emu_train_batch": (I, [P, P, P, I, I, D, P, I]),
        "eor_emu_get_weights": (I, [P, P, I]),
        "eor_emu_set_weights": (I, [P, P, I]),
        "eor_emu_get_normalization": (I, [P, P]),
        "eor_emu_set_normalization": (I, [P, P]),
        "eor_emu_predict": (I, [P, P, I, P, P, P, I]),
        "eor_emu_calibrate": (I, [P, P, P, I, D, P, P, I]),
        "eor_emu_set_threshold": (I, [P, D]),
        "eor_emu_likelihood": (I, [P, P, P, I, P, P, P, P, P, I]),
        "eor_emu_set_inference": (I, [P, I]),
        "eor_emu_inference": (I, [P]),
        "eor_emu_last_error": (ctypes.c_char_p, [P]),
        "eor_emu_destroy": (None, [P]),
        "eor_mcmc_default_config": (None, [ctypes.POINTER(McmcConfig)]),
        "eor_mcmc_create": (I, [ctypes.POINTER(McmcConfig), P, ctypes.POINTER(P)]),
        "eor_mcmc_start": (I, [P, P, P, P, P, I]),
        "eor_mcmc_run": (I, [P, I, P, P, P, I]),
        "eor_mcmc_walkers": (I, [P, P, P, I]),
        "eor_mcmc_last_error": (ctypes.c_char_p, [P]),
        "eor_mcmc_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _lib = lib
    return lib


def default_config(**overrides) -> EorConfig:
    cfg = EorConfig()
    load_library().eor_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "z":
            cfg.n_z = len(v)
            for j, zv in enumerate(v):
                cfg.z[j] = float(zv)
        else:
            setattr(cfg, k, v)
    return cfg


def _is_torch_cuda(x) -> bool:
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


def _arg(x, dtype):
    """(pointer, mem, keepalive) for a numpy array or a CUDA torch tensor."""
    if x is None:
        return None, EOR_HOST, None
    if _is_torch_cuda(x):
        if not x.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), EOR_DEVICE, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(ctypes.c_void_p), EOR_HOST, a


class Context:
    """One libeor21 context (eor_create ... eor_destroy)."""

    def __init__(self, cfg: EorConfig | None = None, stream=None, torch_allocator: bool = False, **overrides):
        self.lib = load_library()
        self.cfg = cfg if cfg is not None else default_config(**overrides)
        self._cb = None
        if torch_allocator:
            import torch
            blocks = {}

            def _alloc(nbytes, _user):
                try:
                    ptr = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                             torch.cuda.current_stream().cuda_stream)
                except Exception:
                    return None
                blocks[ptr] = True
                return ptr

            def _free(ptr, _user):
                if ptr in blocks:
                    del blocks[ptr]
                    torch.cuda.caching_allocator_delete(ptr)

            self._cb = (_ALLOC(_alloc), _FREE(_free))
            self.cfg.dev_alloc, self.cfg.dev_free = self._cb
        handle = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else None
        rc = self.lib.eor_create(ctypes.byref(self.cfg), st, ctypes.byref(handle))
        if rc != EOR_OK:
            raise EorError(rc, self.lib.eor_last_error(None).decode())
        self.handle = handle
        self.n, self.n_z, self.n_bins = self.cfg.n, self.cfg.n_z, self.cfg.n_bins
        self.n_walkers = 0

    # ---------------------------------------------------------------- helpers
    def _check(self, rc: int):
        if rc != EOR_OK:
            raise EorError(rc, self.lib.eor_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.eor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _out(self, like_device: bool, shape, dtype):
        if like_device:
            import torch
            tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int64: torch.int64}[dtype]
            return torch.empty(shape, dtype=tdt, device="cuda")
        return np.empty(shape, dtype=dtype)

    # ---------------------------------------------------------------- C ABI
    def eor_init_boxes(self, delta):
        p, mem, keep = _arg(delta, np.float32)
        self._check(self.lib.eor_init_boxes(self.handle, p, mem))

    def eor_set_params(self, params):
        p, mem, keep = _arg(params, np.float64)
        nw = int(keep.shape[0])
        self._check(self.lib.eor_set_params(self.handle, p, nw, mem))
        self.n_walkers = nw

    def eor_set_efficiency(self, q):
        """Efficiency parameters [n_walkers][4] of efficiency_model 1 or 2."""
        p, mem, keep = _arg(q, np.float64)
        self._check(self.lib.eor_set_efficiency(self.handle, p, int(keep.shape[0]), mem))

    def eor_run_ionization(self, want_xhi: bool = False, device: bool = False):
        pairs = (self.n_walkers, self.n_z)
        xhi = self._out(device, pairs + (self.n,) * 3, np.float32) if want_xhi else None
        mean = self._out(device, pairs, np.float64)
        px = None if xhi is None else _arg(xhi, np.float32)[0]
        self._check(self.lib.eor_run_ionization(self.handle, px, _arg(mean, np.float64)[0],
                                                EOR_DEVICE if device else EOR_HOST))
        return xhi, mean

    def eor_power_spectrum(self, device: bool = False):
        shape = (self.n_walkers, self.n_z, self.n_bins)
        d2 = self._out(device, shape, np.float64)
        km = self._out(device, shape, np.float64)
        cnt = self._out(device, shape, np.int64)
        self._check(self.lib.eor_power_spectrum(self.handle, _arg(d2, np.float64)[0], _arg(km, np.float64)[0],
                                                _arg(cnt, np.int64)[0], EOR_DEVICE if device else EOR_HOST))
        return d2, km, cnt

    def eor_chi2(self, mock_d2, sigma):
        pm, mem, km = _arg(mock_d2, np.float64)
        ps, mem2, ks = _arg(sigma, np.float64)
        if mem != mem2:
            raise ValueError("mock and sigma must both be host or both device")
        out = self._out(mem == EOR_DEVICE, (self.n_walkers,), np.float64)
        self._check(self.lib.eor_chi2(self.handle, pm, ps, _arg(out, np.float64)[0], mem))
        return out

    def eor_likelihood(self, params, mock_d2, sigma, want_d2: bool = False):
        pp, mem, kp = _arg(params, np.float64)
        pm, _, km = _arg(mock_d2, np.float64)
        ps, _, ks = _arg(sigma, np.float64)
        nw = int(kp.shape[0])
        dev = mem == EOR_DEVICE
        chi2 = self._out(dev, (nw,), np.float64)
        d2 = self._out(dev, (nw, self.n_z, self.n_bins), np.float64) if want_d2 else None
        self._check(self.lib.eor_likelihood(self.handle, pp, nw, pm, ps, _arg(chi2, np.float64)[0],
                                            None if d2 is None else _arg(d2, np.float64)[0], mem))
        self.n_walkers = nw
        return (chi2, d2) if want_d2 else chi2

    def eor_filtered_density(self, z_index: int, r_mpc: float, device: bool = False):
        out = self._out(device, (self.n,) * 3, np.float32)
        self._check(self.lib.eor_filtered_density(self.handle, int(z_index), float(r_mpc),
                                                  _arg(out, np.float32)[0], EOR_DEVICE if device else EOR_HOST))
        return out

    def eor_density_spectrum(self, z_index: int) -> np.ndarray:
        """Half spectrum as complex64 [kz][kx][ky], kz = 0..n/2."""
        out = np.empty((self.n // 2 + 1, self.n, self.n), dtype=np.complex64)
        self._check(self.lib.eor_density_spectrum(self.handle, int(z_index), out.ctypes.data_as(ctypes.c_void_p),
                                                  EOR_HOST))
        return out

    def eor_density_box(self, z_index: int) -> np.ndarray:
        out = np.empty((self.n,) * 3, dtype=np.float32)
        self._check(self.lib.eor_density_box(self.handle, int(z_index), out.ctypes.data_as(ctypes.c_void_p), EOR_HOST))
        return out

    def eor_walker_ladder(self, walker: int) -> np.ndarray:
        radii = np.zeros(MAX_RADII, dtype=np.float64)
        cnt = ctypes.c_int()
        self._check(self.lib.eor_walker_ladder(self.handle, int(walker), radii.ctypes.data_as(ctypes.c_void_p),
                                               ctypes.byref(cnt)))
        return radii[:cnt.value].copy()

    def eor_box_power_spectrum(self, box):
        p, mem, keep = _arg(box, np.float32)
        dev = mem == EOR_DEVICE
        d2 = self._out(dev, (self.n_bins,), np.float64)
        km = self._out(dev, (self.n_bins,), np.float64)
        cnt = self._out(dev, (self.n_bins,), np.int64)
        self._check(self.lib.eor_box_power_spectrum(self.handle, p, _arg(d2, np.float64)[0], _arg(km, np.float64)[0],
                                                    _arg(cnt, np.int64)[0], mem))
        return d2, km, cnt

    def eor_set_tuning(self, group: int, pairs: int, plane_threads: int = 512):
        self._check(self.lib.eor_set_tuning(self.handle, int(group), int(pairs), int(plane_threads)))

    def eor_set_ps_split(self, split: int):
        self._check(self.lib.eor_set_ps_split(self.handle, int(split)))

    def eor_set_ps_streams(self, streams: int):
        self._check(self.lib.eor_set_ps_streams(self.handle, int(streams)))

    def eor_get_tuning(self) -> dict:
        v = [ctypes.c_int() for _ in range(5)]
        self._check(self.lib.eor_get_tuning(self.handle, *[ctypes.byref(x) for x in v]))
        return dict(zip(("group", "pairs", "plane_threads", "ps_split", "ps_streams"), (x.value for x in v)))

    def eor_autotune(self, params, mock_d2, sigma, reps: int = 3):
        """Pick the fastest launch schedule for these walkers; returns (group, pairs,
        plane_threads, ms per call)."""
        pp, mem, kp = _arg(params, np.float64)
        pm, _, km = _arg(mock_d2, np.float64)
        ps, _, ks = _arg(sigma, np.float64)
        g, p, t, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.eor_autotune(self.handle, pp, int(kp.shape[0]), pm, ps, int(reps), ctypes.byref(g),
                                          ctypes.byref(p), ctypes.byref(t), ctypes.byref(ms), mem))
        return g.value, p.value, t.value, ms.value

    def eor_noise_sigma(self, mock_d2, thermal=None, model_frac: float = 0.25) -> np.ndarray:
        """Total uncertainty [n_z][n_bins] of mock spectra: T+S mode sum plus modelling error."""
        pm, mem, _ = _arg(mock_d2, np.float64)
        pt, _, kt = _arg(thermal, np.float32)
        out = self._out(mem == EOR_DEVICE, (self.n_z, self.n_bins), np.float64)
        self._check(self.lib.eor_noise_sigma(self.handle, pm, pt, float(model_frac), _arg(out, np.float64)[0], mem))
        return out

    def eor_set_method(self, method: int):
        self._check(self.lib.eor_set_method(self.handle, int(method)))

    def eor_basis_info(self):
        """(basis size, largest residual of the top-hat projection)."""
        r, e = ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.eor_basis_info(self.handle, ctypes.byref(r), ctypes.byref(e)))
        return r.value, e.value

    def eor_basis_window(self, r_mpc: float) -> np.ndarray:
        """sum_b c_b(R) phi_b on every |m|^2 index 0 .. 3 (n/2)^2 (NaN where no mode has it)."""
        n = self.cfg.n
        out = np.empty(3 * (n // 2) ** 2 + 1, dtype=np.float64)
        self._check(self.lib.eor_basis_window(self.handle, float(r_mpc), out.ctypes.data_as(ctypes.c_void_p),
                                              EOR_HOST))
        return out

    def eor_contraction_info(self):
        """(kind, K slots) of the contraction the current method runs (EOR_CONTRACT_*)."""
        k, ks = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.eor_contraction_info(self.handle, ctypes.byref(k), ctypes.byref(ks)))
        return k.value, ks.value

    def eor_debug_withhold(self, step: int, wait_ms: float = 1.0):
        """Test-only: make the contraction withhold one accumulator release (step < 0: off)."""
        self._check(self.lib.eor_debug_withhold(self.handle, int(step), float(wait_ms)))

    def eor_trace(self, enable: bool = True):
        self._check(self.lib.eor_trace(self.handle, 1 if enable else 0))

    def eor_trace_read(self) -> dict:
        """{class name: (milliseconds, launches)} of the last call."""
        ms = np.zeros(KERNEL_CLASSES)
        cnt = np.zeros(KERNEL_CLASSES, dtype=np.int64)
        self._check(self.lib.eor_trace_read(self.handle, ms.ctypes.data_as(ctypes.c_void_p),
                                            cnt.ctypes.data_as(ctypes.c_void_p), KERNEL_CLASSES))
        return {self.lib.eor_kernel_class_name(k).decode(): (float(ms[k]), int(cnt[k]))
                for k in range(KERNEL_CLASSES)}

    def eor_launch_count(self) -> int:
        return int(self.lib.eor_launch_count(self.handle))

    # short aliases
    init_boxes = eor_init_boxes
    set_params = eor_set_params
    set_efficiency = eor_set_efficiency
    run_ionization = eor_run_ionization
    power_spectrum = eor_power_spectrum
    chi2 = eor_chi2
    likelihood = eor_likelihood
    filtered_density = eor_filtered_density
    density_spectrum = eor_density_spectrum
    walker_ladder = eor_walker_ladder
    density_box = eor_density_box
    box_power_spectrum = eor_box_power_spectrum
    trace = eor_trace
    set_tuning = eor_set_tuning
    set_method = eor_set_method
    autotune = eor_autotune
    set_ps_split = eor_set_ps_split
    set_ps_streams = eor_set_ps_streams
    get_tuning = eor_get_tuning
    noise_sigma = eor_noise_sigma
    basis_info = eor_basis_info
    basis_window = eor_basis_window
    debug_withhold = eor_debug_withhold
    contraction_info = eor_contraction_info
    trace_read = eor_trace_read
    launch_count = eor_launch_count


def emu_default_config(**overrides) -> EmuConfig:
    cfg = EmuConfig()
    load_library().eor_emu_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "z":
            cfg.n_z = len(v)
            for j, zv in enumerate(v):
                cfg.z[j] = float(zv)
        elif k in ("prior_lo", "prior_hi"):
            for c in range(3):
                getattr(cfg, k)[c] = float(v[c])
        else:
            setattr(cfg, k, v)
    return cfg


class Emulator:
    """The power-spectrum surrogate (eor_emu_create ... eor_emu_destroy): numpy arrays are
    host buffers, CUDA torch tensors device buffers."""

    def __init__(self, cfg: EmuConfig | None = None, stream=None, **overrides):
        self.lib = load_library()
        self.cfg = cfg if cfg is not None else emu_default_config(**overrides)
        handle = ctypes.c_void_p()
        rc = self.lib.eor_emu_create(ctypes.byref(self.cfg), ctypes.c_void_p(stream) if stream else None,
                                     ctypes.byref(handle))
        if rc != EOR_OK:
            raise EorError(rc, self.lib.eor_emu_last_error(None).decode())
        self.handle = handle
        self.members, self.n_z, self.n_bins = self.cfg.members, self.cfg.n_z, self.cfg.n_bins
        self.n_params = int(self.lib.eor_emu_n_params(handle))

    def _check(self, rc: int):
        if rc != EOR_OK:
            raise EorError(rc, self.lib.eor_emu_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.eor_emu_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def eor_emu_set_data(self, params, d2):
        pp, mem, kp = _arg(params, np.float64)
        pd, mem2, _ = _arg(d2, np.float64)
        if mem != mem2:
            raise ValueError("params and d2 must both be host or both device")
        self._check(self.lib.eor_emu_set_data(self.handle, pp, pd, int(kp.shape[0]), mem))

    def eor_emu_train(self, steps: int, batch: int, lr: float, seed: int = 0) -> np.ndarray:
        loss = np.zeros(self.members)
        self._check(self.lib.eor_emu_train(self.handle, int(steps), int(batch), float(lr), int(seed),
                                           loss.ctypes.data_as(ctypes.c_void_p)))
        return loss

    def eor_emu_forward(self, x) -> np.ndarray:
        px, mem, kx = _arg(x, np.float32)
        n = int(kx.shape[0])
        y = np.empty((self.members, n, self.n_bins), dtype=np.float32)
        if mem == EOR_DEVICE:
            raise ValueError("host arrays only")
        self._check(self.lib.eor_emu_forward(self.handle, px, n, y.ctypes.data_as(ctypes.c_void_p), EOR_HOST))
        return y

    def eor_emu_loss_grad(self, x, t):
        px, _, kx = _arg(x, np.float32)
        pt, _, _ = _arg(t, np.float32)
        loss = np.zeros(self.members)
        grad = np.empty((self.members, self.n_params), dtype=np.float32)
        self._check(self.lib.eor_emu_loss_grad(self.handle, px, pt, int(kx.shape[0]),
                                               loss.ctypes.data_as(ctypes.c_void_p),
                                               grad.ctypes.data_as(ctypes.c_void_p), EOR_HOST))
        return loss, grad

    def eor_emu_train_batch(self, x, t, steps: int, lr: float) -> np.ndarray:
        px, _, kx = _arg(x, np.float32)
        pt, _, _ = _arg(t, np.float32)
        loss = np.zeros(self.members)
        self._check(self.lib.eor_emu_train_batch(self.handle, px, pt, int(kx.shape[0]), int(steps), float(lr),
                                                 loss.ctypes.data_as(ctypes.c_void_p), EOR_HOST))
        return loss

    def eor_emu_get_weights(self) -> np.ndarray:
        w = np.empty((self.members, self.n_params), dtype=np.float32)
        self._check(self.lib.eor_emu_get_weights(self.handle, w.ctypes.data_as(ctypes.c_void_p), EOR_HOST))
        return w

    def eor_emu_set_weights(self, w):
        pw, mem, _ = _arg(w, np.float32)
        self._check(self.lib.eor_emu_set_weights(self.handle, pw, mem))

    def eor_emu_get_normalization(self) -> np.ndarray:
        out = np.empty((2, self.n_bins))
        self._check(self.lib.eor_emu_get_normalization(self.handle, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def eor_emu_set_normalization(self, mean_std):
        a = np.ascontiguousarray(mean_std, dtype=np.float64)
        self._check(self.lib.eor_emu_set_normalization(self.handle, a.ctypes.data_as(ctypes.c_void_p)))

    def eor_emu_predict(self, params):
        """(log10 Delta^2 [n][n_z][n_bins], spread [n][n_z], fallback [n])."""
        pp, mem, kp = _arg(params, np.float64)
        n = int(kp.shape[0])
        dev = mem == EOR_DEVICE
        if dev:
            import torch
            pred = torch.empty((n, self.n_z, self.n_bins), dtype=torch.float64, device="cuda")
            spread = torch.empty((n, self.n_z), dtype=torch.float64, device="cuda")
            fb = torch.empty((n,), dtype=torch.int32, device="cuda")
        else:
            pred = np.empty((n, self.n_z, self.n_bins))
            spread = np.empty((n, self.n_z))
            fb = np.empty((n,), dtype=np.int32)
        self._check(self.lib.eor_emu_predict(self.handle, pp, n, _arg(pred, np.float64)[0],
                                             _arg(spread, np.float64)[0], _arg(fb, np.int32)[0], mem))
        return pred, spread, fb

    def eor_emu_calibrate(self, params, d2, recall: float = 0.99):
        """(tau, fraction of these walkers sent to the simulation)."""
        pp, mem, kp = _arg(params, np.float64)
        pd, _, _ = _arg(d2, np.float64)
        tau, frac = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.eor_emu_calibrate(self.handle, pp, pd, int(kp.shape[0]), float(recall),
                                               ctypes.byref(tau), ctypes.byref(frac), mem))
        return tau.value, frac.value

    def eor_emu_set_threshold(self, tau: float):
        self._check(self.lib.eor_emu_set_threshold(self.handle, float(tau)))

    def eor_emu_likelihood(self, ctx: "Context", params, mock_d2, sigma, want_d2: bool = False):
        """(chi2 [n], d2 [n][n_z][n_bins] or None, fallback [n])."""
        pp, mem, kp = _arg(params, np.float64)
        pm, _, km = _arg(mock_d2, np.float64)
        ps, _, ks = _arg(sigma, np.float64)
        n = int(kp.shape[0])
        dev = mem == EOR_DEVICE
        if dev:
            import torch
            chi2 = torch.empty((n,), dtype=torch.float64, device="cuda")
            d2 = torch.empty((n, self.n_z, self.n_bins), dtype=torch.float64, device="cuda") if want_d2 else None
            fb = torch.empty((n,), dtype=torch.int32, device="cuda")
        else:
            chi2 = np.empty((n,))
            d2 = np.empty((n, self.n_z, self.n_bins)) if want_d2 else None
            fb = np.empty((n,), dtype=np.int32)
        self._check(self.lib.eor_emu_likelihood(self.handle, ctx.handle, pp, n, pm, ps, _arg(chi2, np.float64)[0],
                                                None if d2 is None else _arg(d2, np.float64)[0],
                                                _arg(fb, np.int32)[0], mem))
        return chi2, d2, fb

    def eor_emu_set_inference(self, tensor_cores: bool):
        self._check(self.lib.eor_emu_set_inference(self.handle, 1 if tensor_cores else 0))

    def eor_emu_inference(self) -> int:
        return int(self.lib.eor_emu_inference(self.handle))

    set_inference = eor_emu_set_inference
    inference = eor_emu_inference
    set_data = eor_emu_set_data
    train = eor_emu_train
    forward = eor_emu_forward
    loss_grad = eor_emu_loss_grad
    train_batch = eor_emu_train_batch
    get_weights = eor_emu_get_weights
    set_weights = eor_emu_set_weights
    get_normalization = eor_emu_get_normalization
    set_normalization = eor_emu_set_normalization
    predict = eor_emu_predict
    calibrate = eor_emu_calibrate
    set_threshold = eor_emu_set_threshold
    likelihood = eor_emu_likelihood


def mcmc_default_config(**overrides) -> McmcConfig:
    cfg = McmcConfig()
    load_library().eor_mcmc_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k in ("prior_lo", "prior_hi", "gauss_mean", "gauss_precision"):
            arr = getattr(cfg, k)
            for i, x in enumerate(np.ravel(v)):
                arr[i] = float(x)
        else:
            setattr(cfg, k, v)
    return cfg


class Sampler:
    """The device-side ensemble sampler (eor_mcmc_create ... eor_mcmc_destroy) on a Context
    (or, with ctx None and gauss_target=1, on a Gaussian test target)."""

    def __init__(self, ctx: "Context | None", cfg: McmcConfig | None = None, **overrides):
        self.lib = load_library()
        self.cfg = cfg if cfg is not None else mcmc_default_config(**overrides)
        self.ctx = ctx   # keeps the context alive
        handle = ctypes.c_void_p()
        rc = self.lib.eor_mcmc_create(ctypes.byref(self.cfg), None if ctx is None else ctx.handle,
                                      ctypes.byref(handle))
        if rc != EOR_OK:
            raise EorError(rc, self.lib.eor_mcmc_last_error(None).decode())
        self.handle = handle
        self.n_walkers = self.cfg.n_walkers

    def _check(self, rc: int):
        if rc != EOR_OK:
            raise EorError(rc, self.lib.eor_mcmc_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.eor_mcmc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def eor_mcmc_start(self, params, mock_d2=None, sigma=None) -> np.ndarray:
        pp, mem, _ = _arg(params, np.float64)
        pm, _, km = _arg(mock_d2, np.float64)
        ps, _, ks = _arg(sigma, np.float64)
        lnp = np.empty(self.n_walkers)
        if mem == EOR_DEVICE:
            raise ValueError("host arrays only")
        self._check(self.lib.eor_mcmc_start(self.handle, pp, pm, ps, lnp.ctypes.data_as(ctypes.c_void_p), EOR_HOST))
        return lnp

    def eor_mcmc_run(self, steps: int, want_chain: bool = True):
        """(chain [steps][W][3], lnp [steps][W], accepted [steps][W]) as numpy arrays."""
        w = self.n_walkers
        chain = np.empty((steps, w, 3)) if want_chain else None
        lnp = np.empty((steps, w)) if want_chain else None
        acc = np.empty((steps, w), dtype=np.int32) if want_chain else None
        self._check(self.lib.eor_mcmc_run(self.handle, int(steps),
                                          None if chain is None else chain.ctypes.data_as(ctypes.c_void_p),
                                          None if lnp is None else lnp.ctypes.data_as(ctypes.c_void_p),
                                          None if acc is None else acc.ctypes.data_as(ctypes.c_void_p), EOR_HOST))
        return chain, lnp, acc

    def eor_mcmc_walkers(self):
        x = np.empty((self.n_walkers, 3))
        lnp = np.empty(self.n_walkers)
        self._check(self.lib.eor_mcmc_walkers(self.handle, x.ctypes.data_as(ctypes.c_void_p),
                                              lnp.ctypes.data_as(ctypes.c_void_p), EOR_HOST))
        return x, lnp

    start = eor_mcmc_start
    run = eor_mcmc_run
    walkers = eor_mcmc_walkers


def check_noalloc_tensors(n: int, n_bins: int, box, d2, nmodes, device: int) -> None:
    """Refuse tensors that eor_box_power_spectrum_noalloc would misread: each must be a
    contiguous CUDA tensor on `device` with the dtype and element count the call reads or
    writes (box float32 with n^3 elements; d2 float64 and nmodes int64 with at least n_bins
    elements). Raises ValueError."""
    import torch
    need = [("box", box, torch.float32, n ** 3, True), ("d2", d2, torch.float64, n_bins, False)]
    if nmodes is not None:
        need.append(("nmodes", nmodes, torch.int64, n_bins, False))
    for name, t, dtype, count, exact in need:
        if not getattr(t, "is_cuda", False) or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, not {t.dtype}")
        if (t.numel() != count) if exact else (t.numel() < count):
            raise ValueError(f"{name} has {t.numel()} elements; {'exactly' if exact else 'at least'} {count} needed")
        if t.device.index != device:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{device}")


def box_power_spectrum_noalloc(n: int, box_mpc: float, box, d2, nmodes=None, n_bins: int = 14, k_lo: float = 0.1,
                               k_hi: float = 1.5, stream=None) -> None:
    """eor_box_power_spectrum_noalloc on CUDA tensors of the current device: box float32 with
    n^3 elements, d2 float64 with at least n_bins elements, nmodes int64 with at least n_bins
    elements or None. The work is ordered on `stream` (a cudaStream_t handle) and the call
    returns without waiting. The library checks only sizes and ranges, since it sees raw
    device pointers; this wrapper also checks each tensor's dtype, element count and device
    (check_noalloc_tensors), so that a mismatched tensor is refused here instead of being
    read or written out of bounds on the GPU. The first call for each (device, n) does the
    set-up that the header describes; make it before any stream capture."""
    import torch
    n, n_bins = int(n), int(n_bins)
    check_noalloc_tensors(n, n_bins, box, d2, nmodes, torch.cuda.current_device())
    lib = load_library()
    rc = lib.eor_box_power_spectrum_noalloc(n, float(box_mpc), n_bins, float(k_lo), float(k_hi),
                                            ctypes.c_void_p(box.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                                            None if nmodes is None else ctypes.c_void_p(nmodes.data_ptr()),
                                            ctypes.c_void_p(stream) if stream else None)
    if rc != EOR_OK:
        raise EorError(rc, lib.eor_last_error(None).decode())


def tensor_core_check(a, b, stream=None):
    """D = A B^T through the tcgen05 TF32 path (a: CUDA float32 [128, 32], b: [n, 32]);
    returns (D, err) as CUDA tensors after synchronising the stream."""
    import torch
    lib = load_library()
    n = int(b.shape[0])
    d = torch.zeros((128, n), dtype=torch.float32, device=a.device)
    err = torch.zeros(1, dtype=torch.int32, device=a.device)
    rc = lib.eor_tensor_core_check(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                   ctypes.c_void_p(d.data_ptr()), n, ctypes.c_void_p(err.data_ptr()),
                                   ctypes.c_void_p(stream) if stream else None)
    if rc != EOR_OK:
        raise EorError(rc, lib.eor_last_error(None).decode())
    torch.cuda.synchronize()
    return d, err


def version() -> str:
    return load_library().eor_version().decode()
