"""The C ABI library loads and exports every entry point include/*.h
declares; host-side parameter validation runs without a GPU."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_1904_03618_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lbm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ("lbm_create", "lbm_init_fields", "lbm_step", "lbm_moments",
                 "lbm_diagnostics", "lbm_destroy", "lbm_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(lbm.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_struct_layout_matches_header(tmp_path):
    """Compile a probe against include/lbm.h with the host C compiler and
    compare sizeof and every field offset with the ctypes mirror."""
    fields = [f[0] for f in lbm.LbmParams._fields_]
    src = tmp_path / "probe.c"
    body = "".join('printf("%%s %%zu\\n", "%s", offsetof(lbm_params, %s));' % (f, f)
                   for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\n'
                   'int main(void){printf("sizeof %%zu\\n", sizeof(lbm_params));%s'
                   'return 0;}\n' % body)
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = dict(line.split() for line in
               subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(out["sizeof"]) == ctypes.sizeof(lbm.LbmParams)
    for f in fields:
        assert int(out[f]) == getattr(lbm.LbmParams, f).offset, f


@pytest.mark.parametrize("field,value,msg", [
    ("tau_R", 0.5, "tau_R"), ("tau_q", 0.2, "tau_q"), ("beta", 1.5, "beta"),
    ("delta", 0.0, "delta"), ("alpha_B", 1.0, "alpha"), ("rho_in_R", 0.0, "rho_in"),
    ("nx", 0, "nx"), ("storage", 7, "storage"), ("kernel", 5, "kernel"),
])
def test_invalid_parameters_are_rejected_on_the_host(field, value, msg):
    p = lbm.make_params(8, 8, 8)
    setattr(p, field, value)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(p)
    assert ei.value.status == lbm.LBM_ERR_ARG
    assert msg in str(ei.value)


def test_null_context_calls_do_not_crash():
    assert lbm._lib.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert lbm._lib.lbm_moments(None, None, None, None) == lbm.LBM_ERR_ARG
    assert lbm._lib.lbm_population_bytes(None) == 0
    lbm.lbm_destroy(None)


def test_batch_creation_validates_every_case_on_the_host():
    good = lbm.make_params(8, 8, 8)
    bad = lbm.make_params(8, 8, 8, tau_R=0.3)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create_batch([good, bad])
    assert ei.value.status == lbm.LBM_ERR_ARG and "case 1" in str(ei.value)
    mixed = lbm.make_params(8, 8, 8, storage="f16")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create_batch([good, mixed])
    assert "same storage" in str(ei.value)
    two_pass = lbm.make_params(8, 8, 8, kernel="two_pass")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create_batch([two_pass, two_pass])
    assert "fused kernel only" in str(ei.value)


def test_inplace_calls_validate_arguments_on_the_host():
    """The in-place entry points reject bad arguments before any CUDA call;
    they take lattices beyond the two-buffer kernels' 32-bit pair offsets
    (the check that stops lbm_create there)."""
    big = lbm.make_params(1024, 1024, 1024)          # 1.07e9 cells
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(big)
    assert "too large" in str(ei.value)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_step_inplace(big, None, 0, 1, None)
    assert ei.value.status == lbm.LBM_ERR_ARG and "NULL array" in str(ei.value)

    p = lbm.make_params(8, 8, 8)
    cases = [
        (lambda: lbm.lbm_step_inplace(p, 4096, 2, 1, 8192), "parity"),
        (lambda: lbm.lbm_step_inplace(p, 4096, 0, -1, 8192), "nsteps"),
        (lambda: lbm.lbm_step_inplace(p, 4096, 0, 1, 8200), "16-byte"),
        (lambda: lbm.lbm_inplace_read(p, 4096, 0), "no output"),
        (lambda: lbm.lbm_inplace_read(p, 4096, 3, f_out=8192), "parity"),
        (lambda: lbm.lbm_inplace_init(p, None, 4096, 8192, 16384), "NULL array"),
        # rho_R (512 floats) at 1 << 20 overlaps u starting 1 KB later
        (lambda: lbm.lbm_inplace_read(p, 4096, 0, rho_R=1 << 20, u=(1 << 20) + 1024),
         "two outputs overlap"),
    ]
    for call, msg in cases:
        with pytest.raises(lbm.LbmError) as ei:
            call()
        assert ei.value.status == lbm.LBM_ERR_ARG and msg in str(ei.value), (msg, str(ei.value))
    plates = lbm.make_params(8, 8, 8, wall=(0, 0, 2))
    for call in (lambda: lbm.lbm_step_inplace(plates, 4096, 0, 1, 8192),
                 lambda: lbm.lbm_inplace_init(plates, 4096, 8192, 12288, 16384),
                 lambda: lbm.lbm_inplace_read(plates, 4096, 0, f_out=8192)):
        with pytest.raises(lbm.LbmError) as ei:
            call()
        assert "wall = 2" in str(ei.value)
    bad = lbm.make_params(8, 8, 8, tau_R=0.3)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_step_inplace(bad, 4096, 0, 1, 8192)
    assert "tau_R" in str(ei.value)


def test_pointers_of_another_gpu_are_refused_before_any_launch():
    """The calls that hand caller pointers to kernels refuse device memory
    of a GPU other than the one the work runs on (a kernel reading it
    without peer access faults).  The attribute lookup is faked, so no
    second GPU -- and no GPU at all -- is needed: every pointer is taken to
    be device memory of GPU 1 while GPU 0 is current."""
    fake = lbm._lib.lbm_test_fake_pointer_attributes
    fake.argtypes = [ctypes.c_int] * 4
    fake.restype = None
    p = lbm.make_params(8, 8, 8)
    n = 8 * 8 * 8
    f_in, f_out = 1 << 24, (1 << 24) + 38 * 4 * n + 4096
    fld = [(1 << 26) + k * 4 * 3 * n for k in range(4)]
    calls = [
        (lambda: lbm.lbm_step_noalloc(p, f_in, f_out), "lbm_step_noalloc: f_in"),
        (lambda: lbm.lbm_inplace_init(p, fld[0], fld[1], fld[2], f_in),
         "lbm_inplace_init: rho_R"),
        (lambda: lbm.lbm_step_inplace(p, f_in, 0, 1, fld[3]), "lbm_step_inplace: f"),
        (lambda: lbm.lbm_inplace_read(p, f_in, 0, rho_R=fld[0]), "lbm_inplace_read: f"),
    ]
    fake(1, 2, 1, 0)
    try:
        for call, what in calls:
            with pytest.raises(lbm.LbmError) as ei:
                call()
            msg = str(ei.value)
            assert ei.value.status == lbm.LBM_ERR_ARG, msg
            assert what in msg and "device memory of GPU 1" in msg and "GPU 0 is current" in msg
        # host memory is refused by the same calls with its own message
        fake(1, 1, 0, 0)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_step_noalloc(p, f_in, f_out)
        assert "f_in must be device memory" in str(ei.value)
    finally:
        fake(0, 0, 0, 0)
