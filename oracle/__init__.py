"""Plain FP64 CPU oracle of the excursion-set 21-cm likelihood path (arXiv:1501.06576).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` (and its ``--impl reference`` arm) may import this
package. It shares no code with the CUDA library in ``paper_1501_06576_gb300``
and never calls it; the CUDA path never calls the oracle.

The numerics live in ``eor_oracle.c`` (plain C, FP64, textbook radix-2 FFT); this
module compiles it with gcc into ``oracle/_build/liboracle.so`` and wraps each
function with ctypes. See ``eor_oracle.h`` for the pin of every function.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eor_oracle.c")
_HDR = os.path.join(_HERE, "eor_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no host-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB_PATH) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cosmo(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double),
                ("omega_b", ctypes.c_double), ("n_s", ctypes.c_double), ("sigma8", ctypes.c_double),
                ("use_transfer", ctypes.c_int), ("amp", ctypes.c_double)]


class _IonCfg(ctypes.Structure):
    _fields_ = [("r_factor", ctypes.c_double), ("r_cell_rule", ctypes.c_int),
                ("delta_c", ctypes.c_double), ("mu", ctypes.c_double)]


_D = ctypes.c_double
_I = ctypes.c_int
_P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    sig = {
        "or_set_threads": (None, [_I]),
        "or_get_threads": (_I, []),
        "or_fft1d": (None, [_P, _I, _I]),
        "or_fft3d": (None, [_P, _I, _I]),
        "or_bbks_transfer": (_D, [_D]),
        "or_cosmo_init": (None, [ctypes.POINTER(_Cosmo)]),
        "or_pk": (_D, [ctypes.POINTER(_Cosmo), _D]),
        "or_tophat_w": (_D, [_D]),
        "or_sigma2": (_D, [ctypes.POINTER(_Cosmo), _D]),
        "or_growth": (_D, [ctypes.POINTER(_Cosmo), _D]),
        "or_growth_rate": (_D, [ctypes.POINTER(_Cosmo), _D]),
        "or_los_gradient": (None, [_I, _D, _P, _P]),
        "or_rho_mean": (_D, [ctypes.POINTER(_Cosmo)]),
        "or_mass_to_radius": (_D, [ctypes.POINTER(_Cosmo), _D]),
        "or_mmin": (_D, [ctypes.POINTER(_Cosmo), _D, _D, _D]),
        "or_t0_mk": (_D, [ctypes.POINTER(_Cosmo), _D]),
        "or_radius_ladder": (_I, [ctypes.POINTER(_IonCfg), _I, _D, _D, _P, _I]),
        "or_r_cell": (_D, [ctypes.POINTER(_IonCfg), _I, _D]),
        "or_fcoll": (_D, [_D, _D, _D, _D]),
        "or_filter_box": (None, [_I, _D, _P, _D, _P]),
        "or_ionize": (_I, [ctypes.POINTER(_Cosmo), ctypes.POINTER(_IonCfg), _I, _D, _D, _P,
                           _D, _D, _D, _P, _P, _P, _P]),
        "or_power_spectrum": (None, [_I, _D, _P, _I, _D, _D, _P, _P, _P]),
        "or_chi2": (_D, [_I, _D, _D, _D, _D, _P, _P, _P, _P]),
        "or_dsigma2_dlnr": (_D, [ctypes.POINTER(_Cosmo), _D]),
        "or_var_table_new": (_P, [ctypes.POINTER(_Cosmo), _D, _D, _D, _D]),
        "or_var_table_free": (None, [_P]),
        "or_var_s": (_D, [_P, _D, _P]),
        "or_fcoll_pops": (_D, [_P, _P, _I, _D, _D, _D]),
        "or_ionize_pops": (_I, [ctypes.POINTER(_Cosmo), ctypes.POINTER(_IonCfg), _I, _D, _D, _P, _P, _I,
                                _D, _P, _P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- parameters

@dataclass(frozen=True)
class Cosmology:
    """Flat LCDM parameters (Mpc units)."""
    h: float = 0.68
    omega_m: float = 0.31
    omega_b: float = 0.02254 / 0.68 ** 2
    n_s: float = 0.96
    sigma8: float = 0.82
    omega_l: float | None = None
    use_transfer: bool = True


PAPER_COSMOLOGY = Cosmology(h=0.70, omega_m=0.27, omega_b=0.046, n_s=0.96, sigma8=0.82, omega_l=0.73)


@dataclass(frozen=True)
class IonConfig:
    r_factor: float = 1.1
    r_cell_rule: int = 0          # 0: sphere of a cell's volume; 1: cell side
    delta_c: float = 1.686
    mu: float = 0.6


class Oracle:
    """ctypes front end of eor_oracle.c for one cosmology and ionization configuration."""

    def __init__(self, cosmo: Cosmology = Cosmology(), ion: IonConfig = IonConfig(), threads: int = 0):
        self.lib = _load()
        if threads:
            self.lib.or_set_threads(int(threads))
        om_l = cosmo.omega_l if cosmo.omega_l is not None else 1.0 - cosmo.omega_m
        self._c = _Cosmo(cosmo.h, cosmo.omega_m, om_l, cosmo.omega_b, cosmo.n_s, cosmo.sigma8,
                         1 if cosmo.use_transfer else 0, 0.0)
        self.lib.or_cosmo_init(ctypes.byref(self._c))
        self._ion = _IonCfg(ion.r_factor, ion.r_cell_rule, ion.delta_c, ion.mu)
        self.cosmo, self.ion = cosmo, ion

    @property
    def threads(self) -> int:
        return int(self.lib.or_get_threads())

    @property
    def amp(self) -> float:
        return float(self._c.amp)

    # cosmology
    def pk(self, k: float) -> float:
        return self.lib.or_pk(ctypes.byref(self._c), float(k))

    def sigma2(self, r: float) -> float:
        return self.lib.or_sigma2(ctypes.byref(self._c), float(r))

    def growth(self, z: float) -> float:
        return self.lib.or_growth(ctypes.byref(self._c), float(z))

    def growth_rate(self, z: float) -> float:
        return self.lib.or_growth_rate(ctypes.byref(self._c), float(z))

    def rho_mean(self) -> float:
        return self.lib.or_rho_mean(ctypes.byref(self._c))

    def mass_to_radius(self, m: float) -> float:
        return self.lib.or_mass_to_radius(ctypes.byref(self._c), float(m))

    def mmin(self, tvir: float, z: float, mu: float | None = None) -> float:
        return self.lib.or_mmin(ctypes.byref(self._c), float(tvir), float(z),
                                float(self.ion.mu if mu is None else mu))

    def t0_mk(self, z: float) -> float:
        return self.lib.or_t0_mk(ctypes.byref(self._c), float(z))

    # excursion set
    def r_cell(self, n: int, box_mpc: float) -> float:
        return self.lib.or_r_cell(ctypes.byref(self._ion), int(n), float(box_mpc))

    def radius_ladder(self, n: int, box_mpc: float, r_mfp: float) -> np.ndarray:
        cnt = self.lib.or_radius_ladder(ctypes.byref(self._ion), n, box_mpc, r_mfp, None, 0)
        out = np.zeros(cnt, dtype=np.float64)
        self.lib.or_radius_ladder(ctypes.byref(self._ion), n, box_mpc, r_mfp, _ptr(out), cnt)
        return out

    def fcoll(self, delta_r: float, sigma2_min: float, sigma2_r: float) -> float:
        return self.lib.or_fcoll(float(delta_r), float(sigma2_min), float(sigma2_r), self.ion.delta_c)

    def filter_box(self, delta: np.ndarray, box_mpc: float, r: float) -> np.ndarray:
        d = np.ascontiguousarray(delta, dtype=np.float32)
        n = d.shape[0]
        out = np.empty(d.shape, dtype=np.float64)
        self.lib.or_filter_box(n, float(box_mpc), _ptr(d), float(r), _ptr(out))
        return out

    def rsd_weight(self, delta: np.ndarray, box_mpc: float, z: float, max_dvdr: float) -> np.ndarray:
        """(1 + delta) H / (dv_r/dr + H) with linear velocities along the last axis:
        dv_r/dr / H = -f IDFT(k_z^2/k^2 delta_hat), clipped to [-max_dvdr, max_dvdr] (Sec. 2.2's
        velocity-gradient factor; the clip is a reading: the paper is silent where it diverges)."""
        d = np.ascontiguousarray(delta, dtype=np.float32)
        n = d.shape[0]
        g = np.empty(d.shape, dtype=np.float64)
        self.lib.or_los_gradient(n, float(box_mpc), _ptr(d), _ptr(g))
        dvdr = np.clip(-self.growth_rate(z) * g, -max_dvdr, max_dvdr)
        return (1.0 + d.astype(np.float64)) / (1.0 + dvdr)

    def ionize(self, delta: np.ndarray, box_mpc: float, z: float, zeta: float, r_mfp: float,
               log10_tvir: float, rsd_max_dvdr: float | None = None) -> dict:
        d = np.ascontiguousarray(delta, dtype=np.float32)
        n = d.shape[0]
        xhi = np.empty(d.shape, dtype=np.float64)
        flag = np.empty(d.shape, dtype=np.uint8)
        dtb = np.empty(d.shape, dtype=np.float64)
        mean = np.zeros(1, dtype=np.float64)
        nr = self.lib.or_ionize(ctypes.byref(self._c), ctypes.byref(self._ion), n, float(box_mpc),
                                float(z), _ptr(d), float(zeta), float(r_mfp), float(log10_tvir),
                                _ptr(xhi), _ptr(flag), _ptr(dtb), _ptr(mean))
        if rsd_max_dvdr is not None:
            # delta T_b = T0 x_HI (1 + delta) H / (dv_r/dr + H) (Sec. 2.2)
            dtb = self.t0_mk(z) * xhi * self.rsd_weight(d, box_mpc, z, rsd_max_dvdr)
        return {"xhi": xhi, "flag": flag, "dtb": dtb, "xhi_mean": float(mean[0]), "n_radii": nr}

    # mass-dependent efficiency (Sec. 5)
    def dsigma2_dlnr(self, r: float) -> float:
        return self.lib.or_dsigma2_dlnr(ctypes.byref(self._c), float(r))

    def var_table(self, growth: float, m_lo: float, m_hi: float, dlnm: float = 0.03) -> "VarTable":
        return VarTable(self, growth, m_lo, m_hi, dlnm)

    def populations(self, model: int, params, extra, z: float) -> np.ndarray:
        """Populations [n][5] = (zeta0, m_pivot, slope, m_lo, m_hi) of an efficiency model at z.
        model 1: two populations zeta_i0 (M / 1e10 Msun)^alpha_i above their own M_min(T_vir,i):
                 params = (zeta_10, R_mfp, log10 T_vir,1), extra = (alpha_1, zeta_20, alpha_2, log10 T_vir,2).
        model 2: Sec. 5's feedback form in T_vir, zeta0 (T/T_F)^alpha for 10^4 K <= T < T_F and
                 zeta0 (T/T_F)^beta above T_F; at fixed z T_vir ~ M^(2/3), so the mass slopes are
                 2 alpha / 3 and 2 beta / 3: params = (zeta0, R_mfp, log10 T_F), extra = (alpha, beta, -, -)."""
        if model == 1:
            return np.array([[params[0], 1e10, extra[0], self.mmin(10.0 ** params[2], z), 0.0],
                             [extra[1], 1e10, extra[2], self.mmin(10.0 ** extra[3], z), 0.0]], dtype=np.float64)
        if model == 2:
            m_f = self.mmin(10.0 ** params[2], z)
            m_cool = self.mmin(1e4, z)
            pops = []
            if m_cool < m_f:
                pops.append([params[0], m_f, 2.0 * extra[0] / 3.0, m_cool, m_f])
            pops.append([params[0], m_f, 2.0 * extra[1] / 3.0, max(m_f, m_cool), 0.0])
            return np.array(pops, dtype=np.float64)
        raise ValueError("model must be 1 or 2")

    def ionize_pops(self, delta: np.ndarray, box_mpc: float, z: float, pops: np.ndarray, r_mfp: float) -> dict:
        d = np.ascontiguousarray(delta, dtype=np.float32)
        p = np.ascontiguousarray(pops, dtype=np.float64).reshape(-1, 5)
        n = d.shape[0]
        xhi = np.empty(d.shape, dtype=np.float64)
        flag = np.empty(d.shape, dtype=np.uint8)
        dtb = np.empty(d.shape, dtype=np.float64)
        mean = np.zeros(1, dtype=np.float64)
        nr = self.lib.or_ionize_pops(ctypes.byref(self._c), ctypes.byref(self._ion), n, float(box_mpc), float(z),
                                     _ptr(d), _ptr(p), p.shape[0], float(r_mfp), _ptr(xhi), _ptr(flag), _ptr(dtb),
                                     _ptr(mean))
        return {"xhi": xhi, "flag": flag, "dtb": dtb, "xhi_mean": float(mean[0]), "n_radii": nr}


class VarTable:
    """S(M) = D^2 sigma^2(R(M)) on a ln M grid (cubic Hermite) and the populations' collapsed
    fraction over it (or_fcoll_pops)."""

    def __init__(self, oracle: Oracle, growth: float, m_lo: float, m_hi: float, dlnm: float):
        self._lib = oracle.lib
        self._t = oracle.lib.or_var_table_new(ctypes.byref(oracle._c), float(growth), float(m_lo), float(m_hi),
                                              float(dlnm))

    def __del__(self):
        if getattr(self, "_t", None):
            self._lib.or_var_table_free(self._t)
            self._t = None

    def s(self, m: float) -> tuple[float, float]:
        ds = np.zeros(1)
        v = self._lib.or_var_s(self._t, float(np.log(m)), _ptr(ds))
        return v, float(ds[0])

    def fcoll(self, pops, m_r: float, delta_r: float, delta_c: float = 1.686) -> float:
        p = np.ascontiguousarray(pops, dtype=np.float64).reshape(-1, 5)
        return self._lib.or_fcoll_pops(self._t, _ptr(p), p.shape[0], float(m_r), float(delta_r), float(delta_c))


# ---------------------------------------------------------------- free functions

def fft1d(a: np.ndarray, sign: int) -> np.ndarray:
    buf = np.ascontiguousarray(a, dtype=np.complex128).copy()
    _load().or_fft1d(_ptr(buf), buf.shape[0], int(sign))
    return buf


def fft3d(a: np.ndarray, sign: int) -> np.ndarray:
    buf = np.ascontiguousarray(a, dtype=np.complex128).copy()
    _load().or_fft3d(_ptr(buf), buf.shape[0], int(sign))
    return buf


def bbks_transfer(q: float) -> float:
    return _load().or_bbks_transfer(float(q))


def tophat_w(x: float) -> float:
    return _load().or_tophat_w(float(x))


def power_spectrum(box: np.ndarray, box_mpc: float, nbins: int = 14, k_lo: float = 0.1,
                   k_hi: float = 1.5):
    b = np.ascontiguousarray(box, dtype=np.float64)
    n = b.shape[0]
    d2 = np.empty(nbins); km = np.empty(nbins); cnt = np.empty(nbins, dtype=np.int64)
    _load().or_power_spectrum(n, float(box_mpc), _ptr(b), nbins, float(k_lo), float(k_hi),
                              _ptr(d2), _ptr(km), _ptr(cnt))
    return d2, km, cnt


def chi2(d2: np.ndarray, nmodes: np.ndarray | None, mock: np.ndarray, sigma: np.ndarray,
         k_lo: float = 0.1, k_hi: float = 1.5, chi_lo: float = 0.15, chi_hi: float = 1.0) -> float:
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    mock = np.ascontiguousarray(mock, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    nb = d2.shape[0]
    cnt = None if nmodes is None else np.ascontiguousarray(nmodes, dtype=np.int64)
    return _load().or_chi2(nb, float(k_lo), float(k_hi), float(chi_lo), float(chi_hi), _ptr(d2),
                           None if cnt is None else _ptr(cnt), _ptr(mock), _ptr(sigma))


def likelihood(oracle: Oracle, boxes, box_mpc: float, zs, zeta: float, r_mfp: float,
               log10_tvir: float, mock_d2, sigma, nbins: int = 14, k_lo: float = 0.1,
               k_hi: float = 1.5, chi_lo: float = 0.15, chi_hi: float = 1.0) -> dict:
    """One walker's likelihood: per redshift ionize -> Delta^2 -> chi^2, summed linearly over
    redshifts (Sec. 3.4)."""
    total = 0.0
    per_z = []
    for j, z in enumerate(zs):
        ion = oracle.ionize(boxes[j], box_mpc, z, zeta, r_mfp, log10_tvir)
        d2, km, cnt = power_spectrum(ion["dtb"], box_mpc, nbins, k_lo, k_hi)
        c = chi2(d2, cnt, mock_d2[j], sigma[j], k_lo, k_hi, chi_lo, chi_hi)
        total += c
        per_z.append({"xhi_mean": ion["xhi_mean"], "d2": d2, "kmean": km, "nmodes": cnt, "chi2": c,
                      "n_radii": ion["n_radii"]})
    return {"chi2": total, "per_z": per_z}
