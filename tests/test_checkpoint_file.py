"""The checkpoint file check (sgdg_checkpoint_verify), host only: files
written here from the layout the header documents, with the FNV-1a 64
checksum computed from its published definition (offset basis
14695981039346656037, prime 1099511628211, xor then multiply per byte).

A complete file is accepted and its header read back; a flipped byte
anywhere, a truncation, a trailing byte, a wrong magic, and header sizes
larger than the file are refused with SGDG_EIO (the check runs before
sgdg_restore touches a handle, so none of these reaches the device)."""
import os
import struct

import numpy as np
import pytest

import paper_2204_05988_gb300 as P

EIO = 7   # SGDG_EIO


def _fnv1a64(data: bytes) -> int:
    h = 14695981039346656037
    for b in data:
        h ^= b
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _file(nc=6, ns=3, prev2=True, guess=False, field=None, t_now=0.375, nsolved=3, hsh=0x1234ABCD):
    rng = np.random.default_rng(9)
    flags = [1, 0, 1, nsolved, 2, int(prev2), int(guess), int(field is not None)]
    body = b"SGDGCKP2" + struct.pack("<Qqq", hsh, nc, ns) + struct.pack("<8i", *flags) + struct.pack("<d", t_now)
    for n in [nc, nc, ns] + ([nc] if prev2 else []) + ([nc] if guess else []):
        body += rng.standard_normal(n).tobytes()
    if field is not None:
        d, ncell, nvert = field
        body += struct.pack("<4i", d, ncell, nvert, 1) + rng.standard_normal(d * ncell + 2 * nvert).tobytes()
    return body + struct.pack("<Q", _fnv1a64(body))


def _code(path):
    with pytest.raises(P.SgdgError) as e:
        P.checkpoint_verify(str(path))
    return e.value.code


def test_fnv1a64_reference_values():
    # the empty input is the offset basis; "a" is the published test value
    assert _fnv1a64(b"") == 0xCBF29CE484222325
    assert _fnv1a64(b"a") == 0xAF63DC4C8601EC8C


@pytest.mark.parametrize("kw", [{}, {"guess": True}, {"field": (2, 5, 4)}], ids=["plain", "guess", "field"])
def test_complete_file_is_accepted(tmp_path, kw):
    p = tmp_path / "ok.ckp"
    p.write_bytes(_file(**kw))
    info = P.checkpoint_verify(str(p))
    assert (info.problem_hash, info.n_coeffs, info.n_spatial) == (0x1234ABCD, 6, 3)
    assert info.t_now == 0.375 and info.strips_solved == 3
    assert info.has_field == (1 if "field" in kw else 0)


def test_every_flipped_byte_is_refused(tmp_path):
    good = _file(field=(1, 4, 5))
    p = tmp_path / "bad.ckp"
    for i in range(len(good)):
        b = bytearray(good)
        b[i] ^= 0x10
        p.write_bytes(bytes(b))
        assert _code(p) == EIO, i


def test_truncated_extended_and_foreign_files_are_refused(tmp_path):
    good = _file()
    p = tmp_path / "x.ckp"
    for data in (good[:-1], good[:len(good) // 2], good[:8], b"", good + b"\0",
                 b"SGDGCKP1" + good[8:], b"NOTACKPT" * 4):
        p.write_bytes(data)
        assert _code(p) == EIO
    assert _code(tmp_path / "missing.ckp") == EIO


def test_header_sizes_beyond_the_file_are_refused(tmp_path):
    """A header that claims 2^40 coefficients is refused from the file length,
    before any buffer is sized from it."""
    body = b"SGDGCKP2" + struct.pack("<Qqq", 1, 1 << 40, 3) + struct.pack("<8i", 1, 0, 1, 0, 0, 0, 0, 0) \
        + struct.pack("<d", 0.0)
    p = tmp_path / "huge.ckp"
    p.write_bytes(body + struct.pack("<Q", _fnv1a64(body)))
    assert _code(p) == EIO
    body = b"SGDGCKP2" + struct.pack("<Qqq", 1, -4, 3) + struct.pack("<8i", 1, 0, 1, 0, 0, 0, 0, 0) \
        + struct.pack("<d", 0.0)
    p.write_bytes(body + struct.pack("<Q", _fnv1a64(body)))
    assert _code(p) == EIO
