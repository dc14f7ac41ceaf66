"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/pg.h declares; the Python binding carries the same names. No
compute call is made here (no GPU needed)."""

import ctypes
import re
import subprocess

import pytest

import paper_1203_4037_gb300 as pg


@pytest.fixture(scope="module")
def lib():
    pg.build()
    return pg.lib()


def test_header_declares_expected_calls():
    names = pg.exported_symbols()
    for must in ["pg_create", "pg_destroy", "pg_set_eps", "pg_set_table", "pg_set_j", "pg_set_i",
                 "pg_run", "pg_get_force", "pg_set_n", "pg_set_groups", "pg_backward_dev"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", pg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pg_[a-z_]+)$", out, flags=re.M))
    missing = set(pg.exported_symbols()) - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for name in pg.exported_symbols():
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_names_match_header():
    assert set(pg.SIGNATURES) == set(pg.exported_symbols())
    for name in pg.SIGNATURES:
        assert callable(getattr(pg, name))


def test_version_and_no_device_behaviour():
    assert "sm_103a" in pg.pg_version()
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pg.PGError) as ei:
        pg.pg_create(0)
    assert ei.value.code in (pg.PG_ECUDA, pg.PG_EINVAL)
