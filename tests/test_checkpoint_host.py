"""Checkpoint files are read and checked on the host before any device work:
missing, foreign, truncated and inconsistent files come back as error codes
(no GPU needed)."""
import ctypes as C
import struct

import pytest

from paper_2606_04771_b300._lib import Opts, lib


def _load(path):
    h = C.c_void_p()
    t = C.c_double()
    return lib().tdvp_load(str(path).encode(), None, C.byref(h), C.byref(t)), h


def _header(L=4, center=0, version=1):
    return b"TDVPCKP1" + struct.pack("<6i3d", version, L, 1, center, 0, 0, 1.0, 4.0, 0.5)


def test_missing_file_is_an_io_error(tmp_path):
    rc, h = _load(tmp_path / "nope.ckpt")
    assert rc == -9 and not h


def test_foreign_and_broken_files_are_rejected(tmp_path):
    cases = {
        "foreign": b"NOTACKPT" + b"\0" * 64,
        "truncated_header": b"TDVPCKP1" + b"\0" * 5,
        "bad_version": _header(version=7),
        "bad_centre": _header(center=9),
        "truncated_bonds": _header() + struct.pack("<i", 1),
        "zero_degeneracy": _header() + struct.pack("<4i", 1, 0, 0, 0),
        "duplicate_sector": _header() + struct.pack("<7i", 2, 0, 0, 1, 0, 0, 1),
    }
    for name, data in cases.items():
        p = tmp_path / f"{name}.ckpt"
        p.write_bytes(data)
        rc, h = _load(p)
        assert rc == -1 and not h, name
        assert b"checkpoint" in lib().tdvp_last_error(), name


def test_missing_trailer_is_rejected(tmp_path):
    # a complete L = 2 file whose sites are empty except for the trailer
    body = _header(L=2)
    for _ in range(3):  # bonds 0..2, one sector each
        body += struct.pack("<4i", 1, 0, 0, 1)
    body += struct.pack("<q", 0) * 2
    p = tmp_path / "notrailer.ckpt"
    p.write_bytes(body + b"TDVPEND0")
    rc, h = _load(p)
    assert rc == -1 and b"trailer" in lib().tdvp_last_error()


def test_null_arguments():
    h = C.c_void_p()
    assert lib().tdvp_load(None, None, C.byref(h), None) == -1
    assert lib().tdvp_save(None, b"x", 0.0) == -1
    assert Opts  # the options struct is the one tdvp_create takes
