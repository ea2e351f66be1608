"""The index file read by dt_load is checked before anything reaches the
device (no GPU needed here): files crafted byte by byte from the documented
layout pass the checks when they describe a valid tree — the call then stops
at the database pointer — and every kind of damage is rejected with a
message naming the check."""
import ctypes
import struct

import numpy as np
import pytest

from paper_2107_03368_gb300 import dt

MASK = (1 << 64) - 1


def checksum(data: bytes) -> int:
    h = 0x9E3779B97F4A7C15
    pad = data + b"\0" * (-len(data) % 8)
    for (w,) in struct.iter_unpack("<Q", pad):
        h ^= w
        h = (h * 0x100000001B3) & MASK
        h ^= h >> 29
    return h


def index_file(nodes, n, perm=None, leaf_size=32, depth=None, n_leaves=None, use_and=0,
               magic=b"DTINDEX\0", version=1, bad_sum=False, truncate=0, reserved=0):
    nn = len(nodes)
    depth = max(r[3] for r in nodes) if depth is None else depth
    n_leaves = sum(1 for r in nodes if r[0] < 0) if n_leaves is None else n_leaves
    perm = list(range(n)) if perm is None else perm
    header = magic + struct.pack("<II", version, 64) + struct.pack("<qqq", n, nn, n_leaves) + \
        struct.pack("<iiii", depth, leaf_size, use_and, reserved) + struct.pack("<q", 0)
    assert len(header) == 64
    body = b"".join(struct.pack("<iiii", *r) for r in nodes)
    body += np.full(nn * 64 * (1 + use_and), 0x0F0F, np.uint64).tobytes()
    body += np.asarray(perm, np.uint32).tobytes()
    s = checksum(body) ^ (1 if bad_sum else 0)
    data = header + body + struct.pack("<Q", s)
    return data[:len(data) - truncate] if truncate else data


def load(tmp_path, data, n):
    p = tmp_path / "ix.bin"
    p.write_bytes(data)
    out = ctypes.c_void_p()
    rc = dt.load().dt_load(str(p).encode(), None, n, None, ctypes.byref(out))
    return rc, dt.dt_last_error()


TWO_LEVEL = [(1, 0, 40, 0), (-1, 0, 20, 1), (-1, 20, 20, 1)]


@pytest.mark.parametrize("nodes,n,extra", [
    ([(-1, 0, 3, 0)], 3, {}),                     # a single leaf
    (TWO_LEVEL, 40, {}),
    (TWO_LEVEL, 40, {"use_and": 1}),
    # a grown tree: the rebuilt children of node 2 come after node 4's children
    ([(1, 0, 80, 0), (3, 0, 40, 1), (5, 40, 40, 1), (-1, 0, 20, 2), (-1, 20, 20, 2),
      (-1, 40, 30, 2), (-1, 70, 10, 2)], 80, {}),
])
def test_valid_files_pass_the_checks(tmp_path, nodes, n, extra):
    rc, msg = load(tmp_path, index_file(nodes, n, **extra), n)
    assert rc == dt.DT_EINVAL and "d_db" in msg          # stopped at the database pointer


@pytest.mark.parametrize("kwargs,nodes,n,expect", [
    ({"bad_sum": True}, TWO_LEVEL, 40, "checksum"),
    ({"truncate": 3}, TWO_LEVEL, 40, "file size"),
    ({"magic": b"DTINDEY\0"}, TWO_LEVEL, 40, "not an index file"),
    ({"version": 2}, TWO_LEVEL, 40, "version"),
    ({"reserved": 1}, TWO_LEVEL, 40, "reserved"),
    ({}, [(-1, 0, 40, 0)], 40, "a leaf"),                                  # leaf over leaf_size
    ({}, [(0, 0, 40, 0), (-1, 0, 20, 1), (-1, 20, 20, 1)], 40, "a child id"),
    ({}, [(1, 0, 40, 0), (-1, 0, 20, 1), (-1, 19, 21, 1)], 40, "split their parent"),
    ({}, [(1, 0, 40, 0), (-1, 0, 20, 1), (-1, 20, 20, 2)], 40, "child level"),
    ({"leaf_size": 64}, [(1, 0, 40, 0), (-1, 0, 40, 1), (-1, 40, 0, 1)], 40,
     "out of range"),                                                    # an empty child
    ({}, [(-1, 0, 30, 0), (-1, 0, 30, 1)], 30, "without a parent"),
    ({"depth": 3}, TWO_LEVEL, 40, "shape"),
    ({"depth": 0}, TWO_LEVEL, 40, "depth"),
    ({"n_leaves": 1}, TWO_LEVEL, 40, "leaf count"),
    ({"perm": [0] * 40}, TWO_LEVEL, 40, "permutation"),
    ({"perm": list(range(1, 41))}, TWO_LEVEL, 40, "permutation"),
    ({}, [(1, 1, 40, 0), (-1, 1, 20, 1), (-1, 21, 20, 1)], 40, "root"),
])
def test_damaged_files_are_rejected(tmp_path, kwargs, nodes, n, expect):
    rc, msg = load(tmp_path, index_file(nodes, n, **kwargs), n)
    assert rc == dt.DT_EINVAL
    assert expect in msg


def test_wrong_database_size_and_missing_file(tmp_path):
    rc, msg = load(tmp_path, index_file(TWO_LEVEL, 40), 41)
    assert rc == dt.DT_EINVAL and "built over 40" in msg
    out = ctypes.c_void_p()
    rc = dt.load().dt_load(str(tmp_path / "none.bin").encode(), None, 40, None, ctypes.byref(out))
    assert rc == dt.DT_EIO and dt.dt_status_string(rc) == "DT_EIO"
    assert dt.load().dt_save(None, b"x") == dt.DT_EINVAL
    assert dt.load().dt_load(None, None, 40, None, ctypes.byref(out)) == dt.DT_EINVAL
