"""Host-only checks of the C ABI: the library loads, exports every entry
point include/cunbody.h declares, and rejects bad arguments on the host
before any CUDA call (so these run without a GPU)."""

import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "cunbody.h")


@pytest.fixture(scope="module")
def lib():
    from paper_astro_ph_0703100_gb300 import _build, _lib

    _build.build()
    return _lib.load()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^CN_API\s+[^(]*?\b(cn_[a-z0-9_]+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("cn_force", "cn_force_dd", "cn_force_batched", "cn_force_adjoint", "cn_potential_energy",
                     "cn_workspace_bytes", "cn_get_device_status", "cn_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_astro_ph_0703100_gb300 import _lib

    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True, check=True)
    exported = {line.split()[-1] for line in out.stdout.splitlines() if line.strip()}
    declared = set(declared_symbols())
    assert declared <= exported, declared - exported
    # nothing else with the ABI prefix leaks out
    assert {s for s in exported if s.startswith("cn_")} == declared
    # and the binding declares a signature for each of them
    assert set(_lib.SIGNATURES) == declared
    for name in declared:
        assert getattr(lib, name) is not None


def test_status_strings_and_version(lib):
    for code, name in {0: "CN_OK", 1: "CN_ERR_INVALID_ARG", 2: "CN_ERR_MISALIGNED", 3: "CN_ERR_CUDA",
                       4: "CN_ERR_TIMEOUT", 5: "CN_ERR_UNSUPPORTED_DEVICE", 6: "CN_ERR_WORKSPACE",
                       7: "CN_ERR_HOST"}.items():
        assert lib.cn_status_string(code).decode() == name
    assert b"sm_103a" in lib.cn_version()


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "cunbody.h"\nint main(void){ return (int)CN_OK; }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", str(src),
                    "-o", str(tmp_path / "t.o")], check=True)


FAKE = 0x10000  # never dereferenced: every call below fails validation first
V = ctypes.c_void_p


def test_force_rejects_bad_arguments_on_host(lib):
    st = lambda *a: lib.cn_force(*a)
    # negative sizes
    assert st(-1, V(FAKE), 4, V(FAKE), 0.01, V(FAKE * 4), None, None) == 1
    # eps2 negative / NaN / inf
    assert st(4, V(FAKE), 4, V(FAKE), -1.0, V(FAKE * 4), None, None) == 1
    assert st(4, V(FAKE), 4, V(FAKE), float("nan"), V(FAKE * 4), None, None) == 1
    assert st(4, V(FAKE), 4, V(FAKE), float("inf"), V(FAKE * 4), None, None) == 1
    # NULL inputs / outputs
    assert st(4, None, 4, V(FAKE), 0.01, V(FAKE * 4), None, None) == 1
    assert st(4, V(FAKE), 4, None, 0.01, V(FAKE * 4), None, None) == 1
    assert st(4, V(FAKE), 4, V(FAKE), 0.01, None, None, None) == 1
    # misaligned records (not 16-byte aligned)
    assert st(4, V(FAKE + 4), 4, V(FAKE), 0.01, V(FAKE * 4), None, None) == 2
    assert st(4, V(FAKE), 4, V(FAKE + 8), 0.01, V(FAKE * 4), None, None) == 2
    # misaligned outputs
    assert st(4, V(FAKE), 4, V(FAKE), 0.01, V(FAKE * 4 + 2), None, None) == 2
    assert lib.cn_force_dd(4, V(FAKE), 4, V(FAKE), 0.01, V(FAKE * 4 + 4), None, None) == 2
    # outputs overlapping inputs
    assert st(4, V(FAKE), 4, V(FAKE * 2), 0.01, V(FAKE + 16), None, None) == 1
    assert st(4, V(FAKE), 4, V(FAKE * 2), 0.01, V(FAKE * 4), V(FAKE * 4 + 16), None) == 1
    assert b"overlap" in lib.cn_last_error_message()


def test_empty_i_set_is_a_noop_without_cuda(lib):
    assert lib.cn_force(0, None, 0, None, 0.01, None, None, None) == 0
    assert lib.cn_force_dd(0, None, 5, V(FAKE), 0.01, None, None, None) == 0
    assert lib.cn_force_adjoint(0, None, 0.01, None, None, None, None) == 0


def test_adjoint_and_energy_validation(lib):
    assert lib.cn_force_adjoint(-3, V(FAKE), 0.01, V(FAKE), V(FAKE), V(FAKE), None) == 1
    assert lib.cn_force_adjoint(8, V(FAKE + 4), 0.01, V(FAKE * 8), V(FAKE * 16), V(FAKE * 32), None) == 2
    assert lib.cn_force_adjoint(8, V(FAKE), 0.01, None, V(FAKE * 16), V(FAKE * 32), None) == 1
    assert lib.cn_potential_energy(8, V(FAKE), V(FAKE * 8), None, None) == 1
    assert lib.cn_potential_energy(-1, V(FAKE), V(FAKE * 8), V(FAKE * 16), None) == 1


def test_batch_plan_validation(lib):
    from paper_astro_ph_0703100_gb300._lib import cn_tune

    h = ctypes.c_void_p()
    offs = (ctypes.c_int64 * 3)(0, 10, 5)  # decreasing
    eps = (ctypes.c_float * 2)(0.1, 0.1)
    assert lib.cn_batch_plan_create(2, offs, eps, None, 0, ctypes.byref(h)) == 1
    offs = (ctypes.c_int64 * 3)(1, 10, 20)  # must start at 0
    assert lib.cn_batch_plan_create(2, offs, eps, None, 0, ctypes.byref(h)) == 1
    offs = (ctypes.c_int64 * 3)(0, 10, 20)
    bad = (ctypes.c_float * 2)(0.1, -1.0)
    assert lib.cn_batch_plan_create(2, offs, bad, None, 0, ctypes.byref(h)) == 1
    assert lib.cn_force_batched(None, V(FAKE), V(FAKE), None, None, 0, None) == 1
    assert lib.cn_batch_plan_launch(None, None) == 1
    t = cn_tune(3, 128, 256, 4, 0, 0)  # 3 i-particles per thread is not offered
    assert lib.cn_tune_set(0, 1024, 1024, ctypes.byref(t)) == 1
    t = cn_tune(4, 96, 256, 4, 0, 0)
    assert lib.cn_tune_set(0, 1024, 1024, ctypes.byref(t)) == 1
    t = cn_tune(4, 128, 100, 4, 0, 0)
    assert lib.cn_tune_set(0, 1024, 1024, ctypes.byref(t)) == 1
    t = cn_tune(4, 128, 8, 4, 0, 0)  # below the 16-record minimum
    assert lib.cn_tune_set(0, 1024, 1024, ctypes.byref(t)) == 1
    t = cn_tune(1, 128, 256, 4, 0, 0, 3)  # j_lanes must be a power of two
    assert lib.cn_tune_set(0, 1024, 1024, ctypes.byref(t)) == 1
    t = cn_tune(4, 128, 256, 4, 0, 0, 8)  # per-i softening with j_lanes > 1: one or two i-particles per thread
    assert lib.cn_tune_set(10, 1024, 1024, ctypes.byref(t)) == 1
    assert lib.cn_tune_set(4, 1024, 1024, ctypes.byref(t)) == 1  # the adjoint with j_lanes > 1: exactly two
    t = cn_tune(8, 128, 256, 4, 0, 0, 8)  # the compensated form takes no j_lanes
    assert lib.cn_tune_set(2, 1024, 1024, ctypes.byref(t)) == 1
    t = cn_tune(1, 128, 96, 4, 0, 0, 8)  # j_tile not a multiple of 8 x j_lanes
    assert lib.cn_tune_set(0, 1024, 1024, ctypes.byref(t)) == 1


def test_indexed_list_plan_validation(lib):
    """The gathering list plan checks its index array on the host, before any
    device work: an entry outside 0 .. n_src - 1 that a group with
    i-particles reaches, a list running past the end of j_index, a NULL
    j_index with entries, or n_src beyond 32 bits is CN_ERR_INVALID_ARG."""
    h = ctypes.c_void_p()
    i_off = (ctypes.c_int64 * 3)(0, 4, 8)
    eps = (ctypes.c_float * 2)(0.01, 0.01)
    create = lambda jb, jc, idx, n_index, n_src, i=i_off: lib.cn_list_plan_create_indexed(
        2, i, (ctypes.c_int64 * 2)(*jb), (ctypes.c_int64 * 2)(*jc), eps, idx, n_index, n_src, None, 0,
        ctypes.byref(h))
    idx = (ctypes.c_int32 * 6)(0, 1, 2, 7, 3, 9)
    assert create((0, 3), (3, 3), idx, 6, 9) == 1      # entry 9 outside 0 .. 8
    assert create((0, 3), (3, 3), idx, 6, 5) == 1      # entries 7 and 9 outside 0 .. 4
    neg = (ctypes.c_int32 * 6)(0, 1, -2, 3, 3, 3)
    assert create((0, 3), (3, 3), neg, 6, 10) == 1     # negative entry
    assert create((0, 4), (3, 3), idx, 6, 10) == 1     # the second list runs past the end
    assert create((0, 3), (3, 3), None, 6, 10) == 1    # NULL index array with entries
    assert create((0, 3), (3, 3), idx, -1, 10) == 1    # negative counts
    assert create((0, 3), (3, 3), idx, 6, 1 << 31) == 1  # n_src beyond the 32-bit index range
    assert create((-1, 3), (3, 3), idx, 6, 10) == 1    # negative list begin
    assert lib.cn_list_plan_create_indexed(2, (ctypes.c_int64 * 3)(0, 4, 2), (ctypes.c_int64 * 2)(0, 3),
                                           (ctypes.c_int64 * 2)(3, 3), eps, idx, 6, 10, None, 0,
                                           ctypes.byref(h)) == 1  # decreasing i_offsets
    assert lib.cn_list_plan_create_indexed(2, i_off, (ctypes.c_int64 * 2)(0, 3), (ctypes.c_int64 * 2)(3, 3), eps,
                                           idx, 6, 10, None, 0, None) == 1  # NULL plan_out
    assert h.value is None


def test_no_exception_leaves_the_library(lib, monkeypatch):
    """Host memory exhausted while a plan is built (CN_FAULT_INJECT=hostmem
    throws std::bad_alloc inside the library, after the arguments were
    checked and before any device work) comes back as CN_ERR_HOST with a
    message; no plan is returned and the process carries on."""
    h = ctypes.c_void_p()
    offs = (ctypes.c_int64 * 3)(0, 10, 20)
    eps = (ctypes.c_float * 2)(0.1, 0.1)
    jb, jc = (ctypes.c_int64 * 2)(0, 5), (ctypes.c_int64 * 2)(5, 5)
    idx = (ctypes.c_int32 * 10)(*range(10))
    monkeypatch.setenv("CN_FAULT_INJECT", "hostmem")
    assert lib.cn_batch_plan_create(2, offs, eps, None, 0, ctypes.byref(h)) == 7
    assert b"host memory" in lib.cn_last_error_message()
    assert lib.cn_list_plan_create(2, offs, jb, jc, eps, None, 0, ctypes.byref(h)) == 7
    assert lib.cn_list_plan_create_indexed(2, offs, jb, jc, eps, idx, 10, 10, None, 0, ctypes.byref(h)) == 7
    assert h.value is None
    # argument errors are still reported as such, before the injected failure
    bad = (ctypes.c_int64 * 3)(0, 10, 5)
    assert lib.cn_batch_plan_create(2, bad, eps, None, 0, ctypes.byref(h)) == 1
    monkeypatch.delenv("CN_FAULT_INJECT")
    assert lib.cn_status_string(7) == b"CN_ERR_HOST"


def test_host_f64_form_validation(lib):
    assert lib.cn_force_host_f64(None, None, None, 0.01, None, -1, 0) == 1
    assert lib.cn_force_host_f64(None, None, V(FAKE), 0.01, V(FAKE), 0, 0) == 0
    assert lib.cn_force_host(4, None, 4, V(FAKE), 0.01, V(FAKE), None, None) == 1


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_astro_ph_0703100_gb300 import _lib

    with pytest.raises((RuntimeError, OSError)):
        # a path that does not exist must raise, never fall back
        _lib._lib_saved = _lib._lib
        try:
            _lib._lib = None
            _lib.load(str(tmp_path / "missing.so"))
        finally:
            _lib._lib = _lib._lib_saved


def test_binding_has_every_entry_point_by_name():
    """The Python binding offers each C entry point under the same name."""
    import re

    import paper_astro_ph_0703100_gb300 as cn

    with open(os.path.join(ROOT, "include", "cunbody.h")) as f:
        names = re.findall(r"CN_API\s+[\w\s\*]+?\b(cn_\w+)\s*\(", f.read())
    assert len(names) >= 30
    assert [n for n in names if not hasattr(cn, n)] == []


def test_tuning_file_is_checked_before_any_device_work(lib, tmp_path):
    """cn_tune_load parses and validates the whole file on the host first:
    a missing, malformed or foreign-format file, or an entry with an invalid
    field, is refused with CN_ERR_INVALID_ARG and nothing is stored."""
    n = ctypes.c_int32(7)
    assert lib.cn_tune_load(str(tmp_path / "missing.json").encode(), ctypes.byref(n)) == 1
    assert n.value == 0
    assert lib.cn_tune_load(None, None) == 1
    assert lib.cn_tune_save(None) == 1
    head = '{"format": "cunbody-tune-1", "device": "X", "arch": "sm_103", "sms": 152, "entries": ['
    entry = ('{"variant": "f32", "n_i_class": 17, "n_j_class": 17, "i_per_thread": %d, "threads": 256, '
             '"j_tile": 1024, "stages": 4, "ctas_per_sm": 0, "chunk_units": 0, "j_lanes": 1}')
    bad = {
        "not json": "{not json",
        "trailing": head + "]} x",
        "format": '{"format": "other", "device": "X", "arch": "sm_103", "sms": 152, "entries": []}',
        "no entries": '{"format": "cunbody-tune-1", "device": "X", "arch": "sm_103", "sms": 152}',
        "unknown variant": head + entry.replace('"f32"', '"nope"') % 8 + "]}",
        "k = 3": head + entry % 3 + "]}",
        "missing field": head + '{"variant": "f32", "n_i_class": 17}' + "]}",
        "deep": "[" * 40 + "]" * 40,
    }
    for name, text in bad.items():
        p = tmp_path / (name.replace(" ", "_") + ".json")
        p.write_text(text)
        assert lib.cn_tune_load(str(p).encode(), ctypes.byref(n)) == 1, name
        assert n.value == 0, name
