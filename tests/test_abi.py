"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/adanns.h declares; argument checks that need no device
memory return the documented error codes."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "adanns.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(adanns_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2305_19435_gb300 as P
    P.build()
    return P.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("adanns_build_ivf", "adanns_search_ivf", "adanns_index_create", "adanns_last_error"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    import paper_2305_19435_gb300 as P
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_version_and_argument_errors_without_device(lib):
    assert lib.adanns_version() == 100
    fake = ctypes.c_void_p(16)
    h = ctypes.c_void_p()
    # d_c = 17 is not an MR granularity
    rc = lib.adanns_build_ivf(fake, 100, 64, 17, 4, 2, 50, 1, 1, 1, None, None, ctypes.byref(h))
    assert rc == -2 and b"granularity" in lib.adanns_last_error()
    # train_n below nlist
    rc = lib.adanns_build_ivf(fake, 100, 64, 16, 40, 2, 20, 1, 1, 1, None, None, ctypes.byref(h))
    assert rc == -1
    # d_c beyond d
    rc = lib.adanns_build_ivf(fake, 100, 8, 16, 4, 2, 50, 1, 1, 1, None, None, ctypes.byref(h))
    assert rc == -2
    # unknown metric
    rc = lib.adanns_build_ivf(fake, 100, 64, 16, 4, 2, 50, 1, 7, 1, None, None, ctypes.byref(h))
    assert rc == -1
    # NULL index
    rc = lib.adanns_search_ivf(None, fake, 1, 16, 64, 1, 10, 1, 0, fake, fake, None, None)
    assert rc == -1
    # shard merge: G, k, batch size out of range; map with negative sizes
    rc = lib.adanns_merge_shards(fake, fake, 0, 4, 10, fake, fake, None)
    assert rc == -1 and b"G" in lib.adanns_last_error()
    rc = lib.adanns_merge_shards(fake, fake, 129, 4, 10, fake, fake, None)
    assert rc == -1
    rc = lib.adanns_merge_shards(fake, fake, 2, 4, 0, fake, fake, None)
    assert rc == -1
    rc = lib.adanns_merge_shards(fake, fake, 2, -1, 10, fake, fake, None)
    assert rc == -1
    rc = lib.adanns_merge_shards(None, fake, 2, 4, 10, fake, fake, None)
    assert rc == -1
    assert lib.adanns_merge_shards(None, None, 2, 0, 10, None, None, None) == 0
    assert lib.adanns_map_ids(fake, -1, fake, 4, None) == -1
    assert lib.adanns_map_ids(fake, 4, None, 4, None) == -1
    assert lib.adanns_map_ids(None, 0, None, 0, None) == 0


def test_runtime_options_without_device(lib):
    v = ctypes.c_int64()
    assert lib.adanns_get_option(5, ctypes.byref(v)) == 0 and v.value == 2_000_000_000
    assert lib.adanns_set_option(5, 10) == -1           # wait limit below 1e5 ns
    assert lib.adanns_set_option(0, 2) == -1            # switches take 0 or 1
    assert lib.adanns_set_option(99, 1) == -1           # unknown option
    assert lib.adanns_get_option(99, ctypes.byref(v)) == -1
    assert lib.adanns_set_option(4, 1 << 30) == 0       # scratch budget 1 GiB
    assert lib.adanns_get_option(4, ctypes.byref(v)) == 0 and v.value == 1 << 30
    assert lib.adanns_set_option(4, 12 << 30) == 0
    assert lib.adanns_get_option(6, ctypes.byref(v)) == 0 and v.value == -1
    assert lib.adanns_get_option(8, ctypes.byref(v)) == 0 and v.value == 1  # narrow tiles: auto
    assert lib.adanns_set_option(8, 3) == -1            # 0, 1 or 2
    assert lib.adanns_set_option(8, 2) == 0 and lib.adanns_set_option(8, 1) == 0


def test_index_import_rejects_bad_files_without_device(lib, tmp_path):
    import indexfile
    h = ctypes.c_void_p()
    missing = str(tmp_path / "missing.idx").encode()
    assert lib.adanns_index_import(missing, None, ctypes.byref(h)) == -1
    bad = tmp_path / "bad.idx"
    bad.write_bytes(b"NOTANIDX" + bytes(200))
    assert lib.adanns_index_import(str(bad).encode(), None, ctypes.byref(h)) == -6
    assert b"not an AdANNS index file" in lib.adanns_last_error()
    short = tmp_path / "short.idx"
    short.write_bytes(b"ADANNSIX" + bytes(20))
    assert lib.adanns_index_import(str(short).encode(), None, ctypes.byref(h)) == -6
    # a valid header with inconsistent sizes (d_c > d)
    odd = tmp_path / "odd.idx"
    odd.write_bytes(indexfile.HEADER.pack(b"ADANNSIX", 1, 96, 10, 8, 16, 2, 1, 1, 0, 0, 0,
                                          *([0] * 10)))
    assert lib.adanns_index_import(str(odd).encode(), None, ctypes.byref(h)) == -6
    ver = tmp_path / "ver.idx"
    ver.write_bytes(indexfile.HEADER.pack(b"ADANNSIX", 7, 96, 10, 8, 8, 2, 1, 1, 0, 0, 0,
                                          *([0] * 10)))
    assert lib.adanns_index_import(str(ver).encode(), None, ctypes.byref(h)) == -6
    assert not h.value
