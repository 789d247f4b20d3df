"""The C-ABI library loads and exports every symbol include/mc.h declares.
No compute calls: these run without a GPU."""
import ctypes
import re

import pytest


@pytest.fixture(scope="module")
def mc():
    from paper_2106_08150_gb300 import _build
    _build.build()
    from paper_2106_08150_gb300 import mc as m
    return m


def test_every_declared_symbol_is_exported(mc):
    names = mc.declared_symbols()
    assert len(names) >= 15
    for core in ["mc_db_create", "mc_db_add_targets", "mc_db_finalize", "mc_classify", "mc_db_free"]:
        assert core in names
    lib = ctypes.CDLL(mc.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_header_is_plain_c(mc):
    text = open(mc.HEADER).read()
    assert 'extern "C"' in text
    assert not re.search(r"\btorch\b|\bat::|\bstd::", text)


def test_version_and_status_strings(mc):
    assert mc.mc_version() == 2
    lib = ctypes.CDLL(mc.LIB_PATH)
    lib.mc_status_string.restype = ctypes.c_char_p
    assert lib.mc_status_string(0) == b"MC_OK"
    assert lib.mc_status_string(7) == b"MC_ERR_CAPACITY"


@pytest.mark.parametrize("bad", [dict(k=0), dict(k=17), dict(sketch_size=0), dict(sketch_size=33),
                                 dict(window_len=8, k=16), dict(window_len=513), dict(window_stride=0),
                                 dict(window_stride=114), dict(bucket_cap=0), dict(bucket_cap=70000)])
def test_invalid_parameters_are_rejected_before_any_device_call(mc, bad):
    import numpy as np
    p = dict(k=16, sketch_size=16, window_len=128, window_stride=113, bucket_cap=254)
    p.update(bad)
    with pytest.raises(mc.McError) as e:
        mc.mc_db_create(mc.db_params(**p), 1, np.zeros(1, np.uint32), stream=0)
    assert e.value.code == mc.MC_ERR_ARG


def test_invalid_taxonomy_is_rejected(mc):
    import numpy as np
    with pytest.raises(mc.McError) as e:
        mc.mc_db_create(mc.db_params(), 3, np.array([0, 5, 1], np.uint32), stream=0)
    assert e.value.code == mc.MC_ERR_ARG


def test_load_rejects_missing_and_foreign_files(mc, tmp_path):
    with pytest.raises(mc.McError) as e:
        mc.mc_db_load(str(tmp_path / "nope.mcdb"), stream=0)
    assert e.value.code == mc.MC_ERR_ARG
    junk = tmp_path / "junk.mcdb"
    junk.write_bytes(b"not a database" * 10)
    with pytest.raises(mc.McError) as e:
        mc.mc_db_load(str(junk), stream=0)
    assert e.value.code == mc.MC_ERR_ARG
