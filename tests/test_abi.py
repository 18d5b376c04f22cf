"""The C ABI without a GPU: the library builds, loads, exports every function that
include/eor21.h declares, its struct layout matches the binding, and calls fail cleanly
(error code + message, no crash) where no CUDA device is present."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_1501_06576_gb300 import eor21

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eor21.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|long long|const char\s*\*)\s+(eor_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["eor_create", "eor_init_boxes", "eor_set_params", "eor_run_ionization",
                     "eor_power_spectrum", "eor_chi2", "eor_destroy", "eor_last_error"]:
        assert required in names
    assert sorted(eor21.EXPORTS) == names


def test_library_exports_every_declared_symbol():
    lib = eor21.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", eor21.library_path()], capture_output=True, text=True)
    exported = set(re.findall(r" T (eor_\w+)", out.stdout))
    assert set(declared_functions()) <= exported


def test_config_layout_matches_c():
    fields = [f[0] for f in eor21.EorConfig._fields_]
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"eor21.h\"\nint main(void){\n"
    prog += 'printf("size %zu\\n", sizeof(eor_config));\n'
    for f in fields:
        prog += f'printf("{f} %zu\\n", offsetof(eor_config, {f}));\n'
    prog += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in lines if line)
    assert int(got["size"]) == ctypes.sizeof(eor21.EorConfig)
    for f in fields:
        assert int(got[f]) == getattr(eor21.EorConfig, f).offset, f


def test_default_config_values():
    cfg = eor21.default_config()
    assert (cfg.n, cfg.box_mpc, cfg.n_z) == (128, 250.0, 3)
    assert list(cfg.z)[:3] == [8.0, 9.0, 10.0]
    assert (cfg.r_factor, cfg.delta_c, cfg.mu, cfg.n_bins) == (1.1, 1.686, 0.6, 14)
    assert (cfg.k_lo, cfg.k_hi, cfg.chi2_k_lo, cfg.chi2_k_hi) == (0.1, 1.5, 0.15, 1.0)
    assert cfg.omega_b == pytest.approx(0.02254 / 0.68 ** 2)


def test_create_rejects_bad_config_before_touching_cuda():
    lib = eor21.load_library()
    h = ctypes.c_void_p()
    cfg = eor21.default_config(n=48)
    assert lib.eor_create(ctypes.byref(cfg), None, ctypes.byref(h)) == eor21.EOR_ENOTSUP
    assert h.value is None
    assert b"n must be" in lib.eor_last_error(None)
    cfg = eor21.default_config(box_mpc=-1.0)
    assert lib.eor_create(ctypes.byref(cfg), None, ctypes.byref(h)) == eor21.EOR_EINVAL
    cfg = eor21.default_config(r_mfp_max=1e6)
    rc = lib.eor_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert rc in (eor21.EOR_EINVAL, eor21.EOR_ECUDA)
    assert lib.eor_create(None, None, ctypes.byref(h)) == eor21.EOR_EINVAL
    cfg = eor21.default_config(efficiency_model=3)
    assert lib.eor_create(ctypes.byref(cfg), None, ctypes.byref(h)) == eor21.EOR_EINVAL
    assert b"efficiency_model" in lib.eor_last_error(None)


def test_null_context_calls_fail_cleanly():
    lib = eor21.load_library()
    assert lib.eor_init_boxes(None, None, 0) == eor21.EOR_EINVAL
    assert lib.eor_set_params(None, None, 1, 0) == eor21.EOR_EINVAL
    assert lib.eor_run_ionization(None, None, None, 0) == eor21.EOR_EINVAL
    assert lib.eor_chi2(None, None, None, None, 0) == eor21.EOR_EINVAL
    lib.eor_destroy(None)


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="checks the no-GPU error path")
def test_create_without_gpu_reports_cuda_error():
    lib = eor21.load_library()
    h = ctypes.c_void_p()
    cfg = eor21.default_config()
    rc = lib.eor_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert rc == eor21.EOR_ECUDA and h.value is None
    assert len(lib.eor_last_error(None)) > 0
