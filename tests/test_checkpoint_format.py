"""The checkpoint file format of gs_save / gs_load (layout documented in include/gs.h), checked on
the CPU through gs_checkpoint_info, which validates a file exactly as gs_load does before it
touches a context: files written here by the documented layout are accepted with their n, and
every kind of damage (magic, version, rows, size, truncation, trailing bytes, one flipped payload
bit) is rejected with GS_ERR_IO."""
import struct

import numpy as np
import pytest

from paper_2504_02437_gb300 import _native as N
from paper_2504_02437_gb300 import build as B
from paper_2504_02437_gb300.api import checkpoint_info


def fnv1a64(data: bytes) -> int:
    h = 0xcbf29ce484222325
    for b in data:
        h ^= b
        h = (h * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def write_ckpt(path, n, seed=0, magic=b"GSMAPCK1", version=1, rows=14, payload_fix=None, size_fix=0, tail=b""):
    rng = np.random.default_rng(seed)
    arrays = [rng.standard_normal((3, 14, n)).astype(np.float32).tobytes(),
              rng.random((2, n)).astype(np.float32).tobytes(),
              rng.integers(0, 50, n).astype(np.uint32).tobytes()]
    payload = b"".join(arrays)
    if payload_fix is not None:
        payload = payload_fix(payload)
    header = struct.pack("<8sIIIIiIddQQ", magic, version, rows, n, 7, 7, 0, 0.9 ** 7, 0.999 ** 7,
                         180 * n + size_fix, fnv1a64(payload))
    assert len(header) == 64
    path.write_bytes(header + payload + tail)
    return path


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    N.load()


def code_of(path):
    lib = N.load()
    return lib.gs_checkpoint_info(str(path).encode(), None, None)


@pytest.mark.parametrize("n", [0, 1, 37, 1000])
def test_valid_files_are_accepted(tmp_path, n):
    p = write_ckpt(tmp_path / "a.ckpt", n)
    assert checkpoint_info(str(p)) == {"n": n, "version": 1}


def test_damaged_files_are_rejected(tmp_path):
    n = 40
    flip = lambda b: b[:123] + bytes([b[123] ^ 0x10]) + b[124:]
    cases = {
        "magic": write_ckpt(tmp_path / "m", n, magic=b"GSMAPCK0"),
        "version": write_ckpt(tmp_path / "v", n, version=2),
        "rows": write_ckpt(tmp_path / "r", n, rows=13),
        "size field": write_ckpt(tmp_path / "s", n, size_fix=4),
        "trailing bytes": write_ckpt(tmp_path / "t", n, tail=b"\0"),
    }
    good = write_ckpt(tmp_path / "g", n).read_bytes()
    # checksum of the undamaged payload, one payload bit flipped afterwards
    (tmp_path / "f").write_bytes(good[:64] + flip(good[64:]))
    cases["flipped bit"] = tmp_path / "f"
    (tmp_path / "c").write_bytes(good[:-1])
    cases["truncated payload"] = tmp_path / "c"
    (tmp_path / "h").write_bytes(good[:40])
    cases["truncated header"] = tmp_path / "h"
    cases["missing"] = tmp_path / "does-not-exist"
    for what, p in cases.items():
        assert code_of(p) == N.GS_ERR_IO, what
    assert code_of(tmp_path / "g") == N.GS_OK
    with pytest.raises(N.GSError):
        checkpoint_info(str(tmp_path / "m"))


def test_null_path_is_an_argument_error():
    assert N.load().gs_checkpoint_info(None, None, None) == N.GS_ERR_ARG


def test_checksum_is_fnv1a64():
    """The published FNV-1a test vectors pin the checksum written into the header."""
    assert fnv1a64(b"") == 0xcbf29ce484222325
    assert fnv1a64(b"a") == 0xaf63dc4c8601ec8c
    assert fnv1a64(b"foobar") == 0x85944171f73967e8
