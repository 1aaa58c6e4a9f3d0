"""The C-ABI library: exports, argument checks and error reporting."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2009_08500_gb300 import rr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rr.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rr_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(rr.LIB_PATH):
        from paper_2009_08500_gb300 import build
        build.build()
    return rr.load_library()


def test_library_exports_every_declared_entry_point(lib):
    declared = _declared()
    assert set(declared) == set(rr.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_null_handles_are_rejected_without_a_device(lib):
    assert lib.rr_nparam(None) == -1
    assert lib.rr_workspace_bytes(None, 4, 4, 0) == 0
    assert lib.rr_destroy(None) == 0
    assert lib.rr_build_weights(None, None) == 1
    assert lib.rr_read_table(None, 0, None, 0) == -1
    assert lib.rr_launch_count(None) == 0
    out = ctypes.c_void_p()
    assert lib.rr_create(None, ctypes.byref(out)) == 1
    assert b"cfg" in lib.rr_last_error(None)
    assert lib.rr_host_path(None) == 0
    assert lib.rr_request_bytes(None, 4, 4, 0) == 0
    # the server's entry points refuse a null server before any CUDA call
    ss, ex = (ctypes.c_int32 * 1)(1), (ctypes.c_double * 1)(0.0)
    assert lib.rr_server_submit_at(None, None, None, None, 4, None, 1, ss, ex, None, None, None, None, 0) == -1
    ids, sts = (ctypes.c_int64 * 1)(), (ctypes.c_int32 * 1)()
    assert lib.rr_server_poll(None, ids, sts, None, 1, 0) == -1
    assert lib.rr_server_pending(None) == -1
    assert lib.rr_server_destroy(None) == 0


@pytest.mark.parametrize("field,value,msg", [("zcut", 1.5, b"zcut"), ("nzin", 0, b"nzin"), ("ng", 1, b"ng"),
                                             ("k1", 0.001, b"k0"), ("npb", 40, b"npb"), ("ld_model", 11, b"ld_model"),
                                             ("precision", 5, b"precision"), ("chromatic", 2, b"chromatic"),
                                             ("direct", 2, b"direct"), ("shared_weights", 3, b"shared_weights"),
                                             ("k_small", -0.1, b"k_small"), ("k_small", float("nan"), b"k_small")])
def test_create_rejects_bad_config_before_touching_the_device(lib, field, value, msg):
    cfg = rr.RRConfig(0.7, 200, 300, 200, 60, 0.005, 0.3, 1, 1, 0, 1, 0)
    setattr(cfg, field, value)
    out = ctypes.c_void_p()
    assert lib.rr_create(ctypes.byref(cfg), ctypes.byref(out)) == 1
    assert out.value is None
    assert msg in lib.rr_last_error(None)


def test_direct_model_does_not_check_the_k_grid(lib):
    # the direct model has no k table: nk, k0, k1 are ignored (validation passes on to the device)
    cfg = rr.RRConfig(0.7, 200, 300, 200, 0, 0.0, 0.0, 1, 1, 0, 1, 0, 0, 1)
    out = ctypes.c_void_p()
    st = lib.rr_create(ctypes.byref(cfg), ctypes.byref(out))
    msg = lib.rr_last_error(None)
    assert b"nk" not in msg and b"k0" not in msg
    if st == 0:
        lib.rr_destroy(out)


@pytest.mark.parametrize("ld_model", [9, 10])
def test_power2_laws_need_the_direct_model(lib, ld_model):
    cfg = rr.RRConfig(0.7, 200, 300, 200, 60, 0.005, 0.3, 1, ld_model, 0, 1, 0, 0, 0)
    out = ctypes.c_void_p()
    assert lib.rr_create(ctypes.byref(cfg), ctypes.byref(out)) == 1
    assert b"direct" in lib.rr_last_error(None)
    cfg.direct, cfg.k_small = 1, 0.05
    assert lib.rr_create(ctypes.byref(cfg), ctypes.byref(out)) == 1


@pytest.mark.parametrize("ld_model,ncoef", [(6, 0), (6, 5), (1, 2), (8, 1)])
def test_create_checks_the_general_law_term_count(lib, ld_model, ncoef):
    cfg = rr.RRConfig(0.7, 200, 300, 200, 60, 0.005, 0.3, 1, ld_model, 0, 1, 0, ncoef)
    out = ctypes.c_void_p()
    assert lib.rr_create(ctypes.byref(cfg), ctypes.byref(out)) == 1
    assert b"ncoef" in lib.rr_last_error(None)


def test_status_bits_match_the_oracle():
    from oracle import model as om
    assert (rr.PV_K_RANGE, rr.PV_E_RANGE, rr.PV_B_RANGE, rr.PV_P_RANGE, rr.PV_NONFINITE, rr.PV_LD_INVALID,
            rr.PV_A_RANGE, rr.PV_KEPLER) == (om.ST_K_RANGE, om.ST_E_RANGE, om.ST_B_RANGE, om.ST_P_RANGE,
                                             om.ST_NONFINITE, om.ST_LD_INVALID, om.ST_A_RANGE, om.ST_KEPLER)
    hdr = open(HEADER).read()
    for name, val in [("RR_PV_K_RANGE", 1), ("RR_PV_KEPLER", 128), ("RR_MAX_PB", 32)]:
        assert re.search(rf"#define {name}\s+{val}\b", hdr)


def test_config_struct_layout_matches_header(tmp_path):
    """The ctypes mirror of rr_config has the size and field offsets a C compiler gives the header's struct."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = [f[0] for f in rr.RRConfig._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"rr.h\"\nint main(void) {\n"
                   '  printf("%zu\\n", sizeof(rr_config));\n' +
                   "".join(f'  printf("%zu\\n", offsetof(rr_config, {n}));\n' for n in names) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got[0] == ctypes.sizeof(rr.RRConfig)
    assert got[1:] == [getattr(rr.RRConfig, n).offset for n in names]


def test_no_cpu_fallback_without_cuda(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    with pytest.raises(RuntimeError, match="CUDA"):
        rr.Model("quadratic")


def test_paper_heterogeneous_example_shapes():
    # lcids / pbids of Sect. 4.2 flatten to one passband index per exposure
    lcids = np.array([0, 0, 1, 1, 1, 2])
    pbids = np.array([0, 1, 0])
    assert list(pbids[lcids]) == [0, 0, 1, 1, 1, 0]
