"""The C-ABI library builds, loads and exports every entry point that
include/dt.h declares; argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2107_03368_gb300 import dt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*\(", src, re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    lib = dt.load()
    names = declared_functions()
    for required in ("dt_build", "dt_search", "bf_search", "retrieve_objects", "dt_free",
                     "dt_status_string", "dt_last_error", "dt_export", "dt_get_info",
                     "dt_sync_status"):
        assert required in names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings():
    assert dt.dt_status_string(0) == "DT_OK"
    assert dt.dt_status_string(-1) == "DT_EINVAL"
    assert dt.dt_status_string(-4) == "DT_ETIMEOUT"
    assert dt.dt_status_string(12345) == "DT_UNKNOWN"


@pytest.mark.parametrize("k", [0, -1, 33])
def test_bad_k_is_rejected_before_any_device_work(k):
    lib = dt.load()
    assert lib.bf_search(None, 10, None, 5, k, None, None, None, 0, None) == dt.DT_EINVAL
    assert "k must be" in dt.dt_last_error()
    assert lib.dt_search(None, None, 5, 1, None, None, None, None, None) == dt.DT_EINVAL


def test_bad_sizes_are_rejected():
    lib = dt.load()
    out = ctypes.c_void_p()
    assert lib.dt_build(None, 10, None, None, None) == dt.DT_EINVAL
    assert lib.dt_build(None, 0, None, None, ctypes.byref(out)) == dt.DT_EINVAL
    assert lib.bf_search(None, 0, None, 5, 1, None, None, None, 0, None) == dt.DT_EINVAL
    assert lib.bf_search(None, 10, None, 5, 1, None, None, None, 7, None) == dt.DT_EINVAL
    assert lib.retrieve_objects(None, None, 3, None, None, 1, 10, 0, 0, None, None, None, 0,
                                None) == dt.DT_EINVAL
    assert lib.dt_get_info(None, None) == dt.DT_EINVAL
    assert lib.dt_keep_widened(None, 1, None) == dt.DT_EINVAL


def test_new_entry_points_check_their_arguments_first():
    """Warm-started search, inverted-file search, embedding, insertion and QUICCI reject bad
    arguments with DT_EINVAL before touching the device."""
    from paper_2107_03368_gb300 import learned
    lib = learned._lib()
    assert lib.dt_search_seeded(None, None, 5, 1, None, 0, None, None, None, None,
                                None) == dt.DT_EINVAL
    dummy = ctypes.c_void_p(16)
    # n_seed out of range, on a non-null (never dereferenced) index handle
    assert lib.dt_search_seeded(dummy, None, 5, 1, None, 5000, None, None, None, None,
                                None) == dt.DT_EINVAL
    assert "n_seed" in dt.dt_last_error()
    assert dt.load().dt_search_path(dummy, None, 5, 1, None, 0, None, None, None, None, 3,
                                    None) == dt.DT_EINVAL
    assert "path" in dt.dt_last_error()
    assert lib.ivf_search(None, None, None, 5, 1, 1, None, None, None, 0, None) == dt.DT_EINVAL
    assert lib.enc_embed(None, None, 5, None, None, 0, None) == dt.DT_EINVAL
    assert dt.load().dt_insert(None, None, 5, None) == dt.DT_EINVAL
    assert dt.load().quicci_generate(None, 10, None, 5, None, None, 4, 0.0, 0, None,
                                     None) == dt.DT_EINVAL
    assert dt.load().quicci_generate(None, 0, None, 5, None, None, 4, 100.0, 0, None,
                                     None) == dt.DT_EINVAL


def test_tune_table_file_roundtrip(tmp_path):
    p = tmp_path / "tune.txt"
    p.write_text("0 23 13 10 152 256 3\n1 23 13 10 152 8 0\nbad line\n")
    dt.dt_tune_clear()
    assert dt.dt_tune_load(p) == 2
    out = tmp_path / "out.txt"
    dt.dt_tune_save(out)
    assert sorted(out.read_text().split("\n")[:2]) == ["0 23 13 10 152 256 3", "1 23 13 10 152 8 0"]
    dt.dt_tune_clear()
    with pytest.raises(dt.DtError):
        dt.dt_tune_load(tmp_path / "missing.txt")
