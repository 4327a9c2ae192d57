"""Host-side checks of the C-ABI library that need no GPU: it builds, loads, exports every
entry point declared in include/ldpc.h, and rejects invalid parity matrices before any
device work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "ldpc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2507_10424_gb300 import build, ldpc
    build.build()
    return ldpc.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ldpc_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ldpc_create", "ldpc_decode", "ldpc_decode_ex", "ldpc_destroy", "ldpc_decode_host"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2507_10424_gb300 import ldpc
    out = subprocess.run(["nm", "-D", "--defined-only", ldpc.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b[TW] (ldpc_\w+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(ldpc.SIGNATURES) == set(declared_functions())


def test_strerror_and_status_codes(lib):
    from paper_2507_10424_gb300 import ldpc
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert ldpc.ldpc_strerror(code) != "unknown status"
    assert ldpc.ldpc_strerror(12345) == "unknown status"


@pytest.mark.parametrize("H,why", [
    (np.array([[1, 2, 0], [0, 1, 1]], np.uint8), "entry not 0/1"),
    (np.array([[1, 0, 0], [0, 1, 1]], np.uint8), "row of weight 1"),
])
def test_invalid_dense_h_is_rejected_on_host(lib, H, why):
    from paper_2507_10424_gb300 import ldpc
    h = ldpc.ldpc_create(H.shape[0], H.shape[1], H)
    assert not h, why
    assert ldpc.ldpc_last_error() == ldpc.LDPC_ERR_INVALID_H


def test_invalid_csr_and_packed_are_rejected_on_host(lib):
    from paper_2507_10424_gb300 import ldpc
    P = ldpc._host
    rp = np.array([0, 2, 4], np.int64)
    dup = np.array([0, 0, 1, 2], np.int32)  # duplicate column in row 0
    h = ldpc.ldpc_create_ex(2, 3, ldpc.LDPC_H_CSR, P(rp), P(dup), 0, 0)
    assert not h and ldpc.ldpc_last_error() == ldpc.LDPC_ERR_INVALID_H
    oob = np.array([0, 3, 1, 2], np.int32)  # column 3 >= N
    h = ldpc.ldpc_create_ex(2, 3, ldpc.LDPC_H_CSR, P(rp), P(oob), 0, 0)
    assert not h and ldpc.ldpc_last_error() == ldpc.LDPC_ERR_INVALID_H
    packed = np.array([[0b1011], [0b110]], np.uint32)  # bit 3 lies past N = 3
    h = ldpc.ldpc_create_ex(2, 3, ldpc.LDPC_H_PACKED_U32, P(packed), None, 0, 0)
    assert not h and ldpc.ldpc_last_error() == ldpc.LDPC_ERR_INVALID_H
    h = ldpc.ldpc_create_ex(0, 3, ldpc.LDPC_H_DENSE_U8, None, None, 0, 0)
    assert not h and ldpc.ldpc_last_error() == ldpc.LDPC_ERR_INVALID_H
    h = ldpc.ldpc_create_ex(2, 3, 7, P(rp), None, 0, 0)
    assert not h and ldpc.ldpc_last_error() == ldpc.LDPC_ERR_INVALID_ARG
    h = ldpc.ldpc_create_ex(2, 3, ldpc.LDPC_H_DENSE_U8, P(np.ones((2, 3), np.uint8)), None, 5, 0)
    assert not h and ldpc.ldpc_last_error() == ldpc.LDPC_ERR_INVALID_ARG


def test_decode_rejects_null_handle(lib):
    from paper_2507_10424_gb300 import ldpc
    assert ldpc.ldpc_decode(None, None, 1, 1, None, None) == ldpc.LDPC_ERR_BAD_POINTER
    assert ldpc.ldpc_set_mode(None, 0) == ldpc.LDPC_ERR_BAD_POINTER
    ldpc.ldpc_destroy(None)  # ignored
