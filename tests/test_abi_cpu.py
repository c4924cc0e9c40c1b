"""CPU checks of the C-ABI library: it loads, exports every entry point of include/lmvd.h, and its
host-side argument validation rejects bad configurations before any CUDA work."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_09878_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2206_09878_gb300 import lmvd
    return lmvd


def declared():
    src = open(os.path.join(ROOT, "include", "lmvd.h")).read()
    return sorted(set(re.findall(r"\b(lmvd_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines()}
    missing = [s for s in declared() if s not in syms]
    assert not missing, missing
    assert set(declared()) == set(lib.EXPORTED)


def test_config_struct_layout_matches(lib, tmp_path):
    """ctypes offsets of lmvd_config equal the C compiler's, field by field (host gcc on the header)."""
    names = [f[0] for f in lib.lmvd_config._fields_]
    body = "".join('printf("%%s %%zu\\n", "%s", offsetof(lmvd_config, %s));' % (n, n) for n in names)
    src = tmp_path / "probe.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lmvd.h"\nint main(void){%s'
                   'printf("sizeof %%zu\\n", sizeof(lmvd_config));return 0;}\n' % body)
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for n in names:
        assert int(out[n]) == getattr(lib.lmvd_config, n).offset, n
    assert int(out["sizeof"]) == ctypes.sizeof(lib.lmvd_config)
    cfg = lib.lmvd_default_config(32, 33, 32)
    assert (cfg.spline_order, cfg.kf, cfg.n_startup, cfg.precision, cfg.bc_mode) == (6, 4, 20, 0, 0)
    assert cfg.beta_n == 0.0 and cfg.beta_p == -4.0 and abs(cfg.rho_light - 1 / 3) < 1e-16


@pytest.mark.parametrize("bad", [dict(nx=7), dict(ny=5), dict(spline_order=3), dict(dt=0.0), dict(re=-1.0),
                                 dict(y1=-2.0), dict(kf=-1), dict(precision=2),
                                 dict(bc_mode=2), dict(bc_mode=-1), dict(memory_layout=3)])
def test_invalid_configs_rejected_without_gpu(lib, bad):
    cfg = lib.lmvd_default_config(32, 33, 32)
    for k, v in bad.items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p()
    rc = lib._lib.lmvd_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert rc == -1 and not h.value


def test_null_arguments(lib):
    L = lib._lib
    assert L.lmvd_create(None, None, None) == -1
    assert L.lmvd_advance_substage(None) == -1
    assert L.lmvd_step(None, 1) == -1
    assert L.lmvd_history_bytes(None) == 0
    assert L.lmvd_state_bytes(None) == 0
    assert L.lmvd_device_bytes(None) == 0
    assert L.lmvd_field_bytes(None, 0) == 0
    assert L.lmvd_substage_index(None) == -1
    assert L.lmvd_status(None) == -1
    assert L.lmvd_synchronize(None) == -1
    assert L.lmvd_kernel_launches(None) == -1
    assert L.lmvd_profile_enable(None, 1) == -1
    assert L.lmvd_diagnostics_enable(None, 1) == -1
    assert L.lmvd_graphs_enable(None, 1) == -1
    assert L.lmvd_graph_count(None) == -1
    assert L.lmvd_set_state(None, None, None, None, None, None, None) == -1
    assert L.lmvd_adjoint_substage(None, None, None, None, None) == -1
    assert L.lmvd_adjoint_startup(None, None, None, None) == -1
    assert L.lmvd_inverse_transform(None, None, None, 1) == -1
    assert L.lmvd_forward_transform(None, None, None, 1) == -1
    assert lib.lmvd_strerror(-3) == "device out of memory"


def test_error_strings_and_class_names(lib):
    msgs = [lib.lmvd_strerror(c) for c in range(0, -7, -1)]
    assert msgs[0] == "ok" and len(set(msgs)) == 7 and "unknown" not in " ".join(msgs)
    assert lib.lmvd_strerror(-99) == "unknown error"
    names = [lib.lmvd_kernel_class_name(c) for c in range(lib.LMVD_KERNEL_CLASSES)]
    assert len(set(names)) == lib.LMVD_KERNEL_CLASSES and "unknown" not in names
    assert names[:4] == ["fft_z_inverse", "fft_x_inverse", "fft_x_forward", "fft_z_forward"]
    assert lib.lmvd_kernel_class_name(lib.LMVD_KERNEL_CLASSES) == "unknown"


def test_host_side_argument_checks_without_gpu(lib):
    """Checks that return before any CUDA call: the allocation-free transform's sizes and radices, and the
    conversion self-test's empty and NULL cases."""
    L = lib._lib
    fake = ctypes.c_void_p(16)          # never dereferenced: every case below returns before device work
    assert L.lmvd_inverse_transform_noalloc(2, 9, 8, fake, fake, 1, None) == -1       # nx < 4
    assert L.lmvd_inverse_transform_noalloc(9, 9, 8, fake, fake, 1, None) == -1       # odd nx
    assert L.lmvd_inverse_transform_noalloc(8, 9, 8, None, fake, 1, None) == -1       # NULL spec
    assert L.lmvd_inverse_transform_noalloc(8, 9, 8, ctypes.c_void_p(24), fake, 1, None) == -1  # spec unaligned
    assert L.lmvd_inverse_transform_noalloc(8, 9, 8, fake, fake, -1, None) == -1      # nfields < 0
    assert L.lmvd_inverse_transform_noalloc(10, 9, 8, fake, fake, 1, None) == -5      # 3nx/2 = 15 = 3 * 5
    assert L.lmvd_inverse_transform_noalloc(4, 70000, 4, fake, fake, 1, None) == -1   # ny > 65535 (fits the array)
    out = ctypes.c_double(0.0)
    assert L.lmvd_rate_probe(0, 10, None, None) == -1                                  # NULL output
    assert L.lmvd_rate_probe(4, 10, ctypes.byref(out), None) == -1                     # unknown op
    assert L.lmvd_rate_probe(0, 0, ctypes.byref(out), None) == -1                      # no iterations
    assert L.lmvd_tile_wait_probe(None, 0, fake, None) == -1                          # NULL source
    assert L.lmvd_tile_wait_probe(ctypes.c_void_p(24), 0, fake, None) == -1           # source not 16-byte aligned
    assert L.lmvd_tile_wait_probe(fake, 8, fake, None) == -1                          # extra not a multiple of 16
    assert L.lmvd_tile_wait_probe(fake, 2048, fake, None) == -1                       # extra beyond 1024
    assert L.lmvd_tile_wait_probe(fake, 16, None, None) == -1                         # NULL status
    assert L.lmvd_df64_convert(None, None, None, None, None, None, 0, None) == 0      # nothing to do
    assert L.lmvd_df64_convert(None, None, None, None, None, None, 4, None) == -1


def test_every_exported_function_has_a_ctypes_signature(lib):
    """Pointers and sizes are 64-bit: a function without argtypes / restype would be called with C int
    conversions. lmvd_destroy returns void (restype None by design)."""
    for name in lib.EXPORTED:
        fn = getattr(lib._lib, name)
        assert fn.argtypes is not None, name
        if name != "lmvd_destroy":
            assert fn.restype is not None, name


def test_checked_build_reports_itself(lib):
    """liblmvd.so is the normal build; liblmvd_check.so (built beside it) has the kernels' index checks."""
    import ctypes
    import os
    assert lib._lib.lmvd_checked_build() == 0
    chk = ctypes.CDLL(os.path.join(os.path.dirname(lib.LIB_PATH), "liblmvd_check.so"))
    chk.lmvd_checked_build.restype = ctypes.c_int
    assert chk.lmvd_checked_build() == 1
    chk.lmvd_strerror.restype = ctypes.c_char_p
    assert b"bounds" in chk.lmvd_strerror(-7)
