"""The C-ABI library builds, loads and exports exactly what include/fsparse.h
declares; host-only entry points behave as documented (no GPU needed)."""
import ctypes
import json
import os
import re
import subprocess

import pytest

from paper_1406_1066_gb300 import build as libbuild
from paper_1406_1066_gb300 import fsparse

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(fsparse_[a-z_0-9]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return fsparse.lib()


def test_header_declares_the_boundary():
    names = declared()
    for must in ("fsparse_symbolic", "fsparse_numeric", "fsparse_assemble",
                 "fsparse_numeric_adjoint", "fsparse_batch_numeric", "fsparse_autotune"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_no_undeclared_exports(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", libbuild.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(fsparse_[a-z_0-9]+)\b", out))
    assert exported == declared()


def test_status_strings(lib):
    for k, name in enumerate(fsparse.STATUS_NAMES):
        assert fsparse.fsparse_status_string(k) == "FSPARSE_" + name


def test_argument_errors_without_device(lib):
    with pytest.raises(fsparse.FsparseError) as e:
        fsparse.fsparse_symbolic(0, 0, -1, 3, 3, 0, 0)
    assert e.value.status == fsparse.ERR_ARG
    with pytest.raises(fsparse.FsparseError) as e:
        fsparse.fsparse_symbolic(0, 0, 10, 3, 3, 0, 0)   # NULL arrays with len > 0
    assert e.value.status == fsparse.ERR_ARG
    with pytest.raises(fsparse.FsparseError) as e:
        fsparse.fsparse_symbolic(8, 8, 2**30, 3, 3, 0, 0)
    assert e.value.status == fsparse.ERR_SIZE
    with pytest.raises(fsparse.FsparseError) as e:
        fsparse.fsparse_symbolic(8, 8, 4, -3, 3, 0, 0)
    assert e.value.status == fsparse.ERR_ARG
    with pytest.raises(fsparse.FsparseError) as e:
        fsparse.fsparse_symbolic(8, 8, 4, 3, 3, -1, 0)
    assert e.value.status == fsparse.ERR_ARG
    assert lib.fsparse_plan_info(None, None, None, None, None, None) == fsparse.ERR_ARG
    assert lib.fsparse_numeric(None, None, None, None) == fsparse.ERR_ARG
    assert lib.fsparse_plan_destroy(None) == fsparse.OK
    assert lib.fsparse_batch_destroy(None) == fsparse.OK
    assert lib.fsparse_assemble(None, None, None, 0, 0, 0, 0, None, 0, None, None) == fsparse.ERR_ARG
    # double-index entry points validate before touching the device
    for args, status in (((0, 0, -1, 3, 3, 0, 0), fsparse.ERR_ARG), ((0, 0, 10, 3, 3, 0, 0), fsparse.ERR_ARG),
                         ((8, 8, 2**30, 3, 3, 0, 0), fsparse.ERR_SIZE), ((8, 8, 4, -3, 3, 0, 0), fsparse.ERR_ARG),
                         ((8, 8, 4, 3, 3, -1, 0), fsparse.ERR_ARG)):
        with pytest.raises(fsparse.FsparseError) as e:
            fsparse.fsparse_symbolic_f64(*args)
        assert e.value.status == status
    assert lib.fsparse_symbolic_f64(None, None, 0, 0, 0, 0, None, None) == fsparse.ERR_ARG
    assert lib.fsparse_assemble_f64(None, None, None, 0, 0, 0, 0, None, 0, None, None) == fsparse.ERR_ARG
    assert lib.fsparse_plan_append(None, None, None, 0, None, None) == fsparse.ERR_ARG
    # plan images are checked before any device access
    assert lib.fsparse_plan_export(None, None, 0, ctypes.byref(fsparse._I64())) == fsparse.ERR_ARG
    out = fsparse._P()
    for image in (b"", b"x" * 200, b"FSPPLAN1" + b"\0" * 120, b"FSPPLAN1" + b"\xff" * 120):
        assert lib.fsparse_plan_import(image, len(image), None, ctypes.byref(out)) == fsparse.ERR_ARG
    assert lib.fsparse_plan_import(None, 0, None, None) == fsparse.ERR_ARG
    assert lib.fsparse_plan_append(None, None, None, 0, None, ctypes.byref(fsparse._P())) == fsparse.ERR_ARG
    assert lib.fsparse_assemble_f64(8, 8, None, 4, 3, 3, 0, None, 0, None,
                                    ctypes.byref(fsparse._P())) == fsparse.ERR_ARG   # NULL values


def test_config_resolution_is_host_logic(lib):
    fsparse.fsparse_set_config(None)
    c = fsparse.fsparse_get_config(93148704, 10**6, 10**6)
    assert c["strategy"] in (fsparse.SORT_ONESWEEP, fsparse.SORT_BUCKET)
    assert 6 <= c["radix_bits"] <= 8 and c["numeric_tile"] in (1024, 2048, 4096)
    fsparse.fsparse_set_config({"strategy": fsparse.SORT_ONESWEEP, "radix_bits": 7, "sweep_items": 0,
                                "sweep_threads": 512, "bucket_target": 0, "numeric_tile": 1024})
    c2 = fsparse.fsparse_get_config(93148704, 10**6, 10**6)
    assert (c2["strategy"], c2["radix_bits"], c2["sweep_threads"], c2["numeric_tile"]) == \
        (fsparse.SORT_ONESWEEP, 7, 512, 1024)
    assert c2["sweep_items"] == c["sweep_items"]
    with pytest.raises(fsparse.FsparseError):
        fsparse.fsparse_set_config({"strategy": 1, "radix_bits": 3, "sweep_items": 8,
                                    "sweep_threads": 256, "bucket_target": 8192, "numeric_tile": 4096})
    # 9- and 10-bit digits only with 256-thread passes
    for bits, threads, ok in [(9, 256, True), (10, 256, True), (9, 512, False), (11, 256, False)]:
        cfg = {"strategy": 1, "radix_bits": bits, "sweep_items": 16, "sweep_threads": threads,
               "bucket_target": 8192, "numeric_tile": 1024}
        if ok:
            fsparse.fsparse_set_config(cfg)
        else:
            with pytest.raises(fsparse.FsparseError):
                fsparse.fsparse_set_config(cfg)
    fsparse.fsparse_set_config(None)
    assert fsparse.fsparse_get_config(93148704, 10**6, 10**6) == c


@pytest.mark.parametrize("strategy,ok", [(fsparse.SORT_AUTO, True), (fsparse.SORT_ONESWEEP, True),
                                         (fsparse.SORT_BUCKET, True), (fsparse.SORT_BUCKET_RADIX, True),
                                         (4, False), (-1, True)])
def test_strategy_override_range(lib, strategy, ok):
    """The four strategies are accepted as overrides (a value <= 0 leaves the
    strategy to the tuner); anything above is an argument error."""
    cfg = {"strategy": strategy, "radix_bits": 0, "sweep_items": 0, "sweep_threads": 0,
           "bucket_target": 0, "numeric_tile": 0}
    try:
        if ok:
            fsparse.fsparse_set_config(cfg)
            c = fsparse.fsparse_get_config(93148704, 10**6, 10**6)
            if strategy > 0:
                assert c["strategy"] == strategy
        else:
            with pytest.raises(fsparse.FsparseError):
                fsparse.fsparse_set_config(cfg)
    finally:
        fsparse.fsparse_set_config(None)


def test_tuning_table_roundtrip(lib, tmp_path):
    fsparse.fsparse_tune_clear()
    key = "L%d_K%d_D%d" % ((1000000).bit_length(), (999).bit_length() + (499).bit_length(),
                           (1000000 >> (499).bit_length()).bit_length())
    entry = {"class": key, "strategy": 1, "radix_bits": 6, "sweep_items": 12, "sweep_threads": 512,
             "bucket_target": 4096, "numeric_tile": 1024}
    src = tmp_path / "in.json"
    src.write_text(json.dumps({"version": 1, "entries": [entry]}))
    fsparse.fsparse_tune_load(str(src))
    c = fsparse.fsparse_get_config(1000000, 1000, 500)
    assert {k: c[k] for k in c} == {k: v for k, v in entry.items() if k != "class"}
    out = tmp_path / "out.json"
    fsparse.fsparse_tune_save(str(out))
    saved = json.loads(out.read_text())
    assert saved["entries"] == [entry]
    radix = dict(entry, strategy=fsparse.SORT_BUCKET_RADIX, bucket_target=8192)
    src.write_text(json.dumps({"version": 1, "entries": [radix]}))
    fsparse.fsparse_tune_load(str(src))
    assert fsparse.fsparse_get_config(1000000, 1000, 500)["strategy"] == fsparse.SORT_BUCKET_RADIX
    bad = tmp_path / "bad.json"
    bad.write_text('{"entries": [{"class": "L1_K1", "strategy": 9}]}')
    with pytest.raises(fsparse.FsparseError):
        fsparse.fsparse_tune_load(str(bad))
    fsparse.fsparse_tune_clear()
    assert fsparse.fsparse_get_config(1000000, 1000, 500)["radix_bits"] == 8
