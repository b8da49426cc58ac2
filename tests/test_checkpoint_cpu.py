"""Checkpoints of a constructed representation (h2_save / h2_load), on the
CPU with host-only handles: a saved and reloaded construction is the same one
(statistics, tree order, every pivot, and the file written again byte for
byte), and truncated or corrupted files are rejected with an error code."""

import ctypes
import os

import numpy as np
import pytest

import paper_2309_14085_gb300 as pkg
from paper_2309_14085_gb300 import H2Error, H2Matrix, inputs

CASES = [
    dict(kernel="invr", d=3, N=3000, variant="h2star", storage="f64"),
    dict(kernel="log2d", d=2, N=4096, variant="h2plush", storage="f32"),
    dict(kernel="imq", d=2, N=2500, variant="h2sqrt", storage="df64", kparam=0.5),
    dict(kernel="log2d", d=2, N=3000, variant="h2star_t", storage="bf16"),
    dict(kernel="invr", d=3, N=3000, variant="h2sqrt_t", storage="f32", m2l="fly"),
    dict(kernel="matern12", d=3, N=2000, variant="h2star_b", storage="f64", m2l="device"),
]


def _build(c):
    c = dict(c)
    P = inputs.points(c.pop("N"), c.pop("d"), 91)
    return H2Matrix(P, c.pop("kernel"), leaf_size=32, tol=1e-6, host_only=True, **c)


def _pivots(A):
    i = A.info()
    out = []
    for b in range(i["nbases"]):
        for l in range(i["kappa"] + 1):
            for X in range(1 << (i["d"] * l)):
                out.append(A.pivots(b, l, X))
    return out


@pytest.mark.parametrize("case", CASES, ids=[f"{c['variant']}-{c['storage']}" for c in CASES])
def test_saved_and_loaded_construction_is_the_same(tmp_path, case):
    A = _build(case)
    f1, f2 = str(tmp_path / "a.h2"), str(tmp_path / "b.h2")
    A.save(f1)
    B = H2Matrix.load(f1, host_only=True)
    assert (B.N, B.d, B.kernel, B.variant, B.storage) == (A.N, A.d, case["kernel"],
                                                          case["variant"], case["storage"])
    ia, ib = A.info(), B.info()
    assert ia == ib
    assert np.array_equal(A.tree_order(), B.tree_order())
    for (ta, sa), (tb, sb) in zip(_pivots(A), _pivots(B)):
        assert np.array_equal(ta, tb) and np.array_equal(sa, sb)
    B.save(f2)
    assert open(f1, "rb").read() == open(f2, "rb").read()


def _degenerate():
    yield H2Matrix(inputs.points(10, 2, 3), "log2d", leaf_size=64, tol=1e-8, host_only=True)
    yield H2Matrix(np.array([[0.25, -0.5, 0.125]]), "invr", leaf_size=4, tol=1e-8, host_only=True)
    yield H2Matrix(inputs.points(100, 2, 4), "log2d", leaf_size=30, tol=1e-8, host_only=True)
    P = inputs.points(500, 3, 5, lo=0.0, hi=0.2)
    yield H2Matrix(P, "invr", leaf_size=8, tol=1e-6, domain=((0.0, 0.0, 0.0), 1.0), host_only=True)
    Q = np.repeat(inputs.points(40, 2, 6), 3, axis=0)                     # coincident points
    yield H2Matrix(Q, "imq", leaf_size=8, tol=1e-8, variant="h2plush", host_only=True)
    yield H2Matrix(inputs.points(700, 3, 7), "matern12", leaf_size=16, tol=1e-6,
                   variant="h2sqrt", near="stored", storage="f32", host_only=True)
    C = np.vstack([inputs.points(1500, 2, 803), inputs.points(300, 2, 813, lo=0.0, hi=0.3)])
    yield H2Matrix(C, "invr", leaf_size=32, tol=1e-6, kappa="strict", host_only=True)  # depth 5


def test_degenerate_constructions_round_trip(tmp_path):
    """The loaded-state checks accept every layout the construction makes,
    including one leaf, one point, no far field, empty boxes, coincident
    points and a strict-depth tree over clustered points (each file is also
    written again byte for byte)."""
    for k, A in enumerate(_degenerate()):
        f1, f2 = str(tmp_path / f"{k}a.h2"), str(tmp_path / f"{k}b.h2")
        A.save(f1)
        B = H2Matrix.load(f1, host_only=True)
        assert A.info() == B.info()
        B.save(f2)
        assert open(f1, "rb").read() == open(f2, "rb").read()


def test_truncated_and_corrupted_files_are_rejected(tmp_path):
    A = _build(CASES[0])
    path = str(tmp_path / "a.h2")
    A.save(path)
    data = open(path, "rb").read()
    bad = str(tmp_path / "bad.h2")

    def load(blob):
        with open(bad, "wb") as f:
            f.write(blob)
        return H2Matrix.load(bad, host_only=True)

    for cut in (0, 7, 8, 100, len(data) // 2, len(data) - 1):
        with pytest.raises(H2Error) as e:
            load(data[:cut])
        assert e.value.code == -1
    for blob in (b"X" + data[1:], data + b"\0"):
        with pytest.raises(H2Error) as e:
            load(blob)
        assert e.value.code == -1
    # single-byte corruptions anywhere (the checksum covers every byte)
    rng = np.random.default_rng(93)
    for pos in rng.integers(0, len(data), size=60):
        blob = bytearray(data)
        blob[int(pos)] ^= 1 << int(rng.integers(0, 8))
        with pytest.raises(H2Error) as e:
            load(bytes(blob))
        assert e.value.code == -1
    # another format version is named in the message
    blob = bytearray(data)
    blob[7] = 9
    with pytest.raises(H2Error) as e:
        load(bytes(blob))
    assert "version 9" in str(e.value)
    with pytest.raises(H2Error) as e:
        H2Matrix.load(str(tmp_path / "missing.h2"), host_only=True)
    assert e.value.code == -1


def test_abi_arguments(tmp_path):
    L = pkg.lib()
    h = ctypes.c_void_p()
    assert L.h2_load(None, 1, ctypes.byref(h)) == -1
    assert L.h2_load(b"x", 2, ctypes.byref(h)) == -1
    assert L.h2_save(None, b"x") == -1
    A = _build(CASES[0])
    assert L.h2_save(A._h, os.fsencode(str(tmp_path / "no-such-dir" / "x.h2"))) == -1


def test_construction_is_independent_of_the_thread_count(tmp_path):
    """The whole construction (every pivot, operator and offset, as written by
    h2_save) is the same with one host thread and with four: the parallel
    loops split independent clusters and no sum crosses threads.  Bytes 60-75
    hold the recorded build and pivot-search times and the last 8 the file's
    checksum."""
    P = inputs.points(6000, 3, 98)
    files = []
    for threads in (1, 4):
        A = H2Matrix(P, "invr", leaf_size=32, tol=1e-6, variant="h2plush", threads=threads,
                     host_only=True)
        files.append(str(tmp_path / f"t{threads}.h2"))
        A.save(files[-1])
    a, b = (open(f, "rb").read() for f in files)
    assert len(a) == len(b) and a[:60] == b[:60] and a[76:-8] == b[76:-8]


def _checksum(b):
    """The checkpoint's checksum, written out from its definition in the
    loader's header: little-endian 64-bit words (the last one zero-padded)
    folded by h <- (h xor w) * P with P the 64-bit FNV prime, from the FNV
    offset basis, then the byte length folded the same way."""
    P, M = 0x100000001b3, (1 << 64) - 1
    h = 0xcbf29ce484222325
    pad = bytes(b) + b"\0" * ((-len(b)) % 8)
    for w in np.frombuffer(pad, dtype="<u8").tolist():
        h = ((h ^ w) * P) & M
    return ((h ^ len(b)) * P) & M


def test_crafted_low_rank_fields_are_rejected(tmp_path):
    """A file whose checksum is right but whose (H2+H)* level pointers are
    missing, or whose scratch length is negative, is refused: the product reads
    lr_level_ptr[0 .. kappa + 1] even when there are no low-rank blocks.  The
    tail of an H2*(b+t) file is lr_level_ptr (length kappa + 2, all zero),
    eight empty arrays, lr_tlen and the checksum."""
    A = _build(CASES[0])
    f = str(tmp_path / "a.h2")
    A.save(f)
    data = open(f, "rb").read()
    assert _checksum(data[:-8]) == int.from_bytes(data[-8:], "little")    # the definition holds
    K = A.info()["kappa"]
    body = data[:-8]
    tail = 8 + 8 * (K + 2) + 8 * 8 + 8
    head, old = body[:-tail], body[-tail:]
    assert int.from_bytes(old[:8], "little") == K + 2 and old[8:] == b"\0" * (tail - 8)

    def load(blob):
        g = str(tmp_path / "b.h2")
        open(g, "wb").write(blob + _checksum(blob).to_bytes(8, "little"))
        return H2Matrix.load(g, host_only=True)

    load(body)                                                  # unchanged: accepted
    empty_ptr = head + (0).to_bytes(8, "little") + b"\0" * (8 * 8) + (0).to_bytes(8, "little")
    with pytest.raises(H2Error) as e:
        load(empty_ptr)
    assert e.value.code == -1 and "low-rank level pointers" in str(e.value)
    neg_tlen = body[:-8] + (-1).to_bytes(8, "little", signed=True)
    with pytest.raises(H2Error) as e:
        load(neg_tlen)
    assert e.value.code == -1 and "scratch" in str(e.value)


def test_crafted_option_combinations_are_rejected(tmp_path):
    """Options h2_build refuses are refused in a loaded file too (with a valid
    checksum), and so is a near-field mode that disagrees with the packed near
    field: either would make a product skip a stage.  Header bytes (after the
    8-byte magic): kernel kind 8-11, parameter 12-19, variant 20-23, storage
    24-27, near mode 28-31, tensor cores 32-35."""
    A = _build(CASES[0])                          # fp64, stored near field
    f = str(tmp_path / "a.h2")
    A.save(f)
    body = bytearray(open(f, "rb").read()[:-8])

    def load(blob):
        g = str(tmp_path / "b.h2")
        open(g, "wb").write(bytes(blob) + _checksum(blob).to_bytes(8, "little"))
        return H2Matrix.load(g, host_only=True)

    tc = bytearray(body)
    tc[32:36] = (1).to_bytes(4, "little")         # tensor cores with fp64 storage
    with pytest.raises(H2Error) as e:
        load(tc)
    assert e.value.code == -1 and "combination" in str(e.value)
    near = bytearray(body)
    near[28:32] = (1).to_bytes(4, "little")       # "on the fly" over stored blocks
    with pytest.raises(H2Error) as e:
        load(near)
    assert e.value.code == -1 and "near-field mode" in str(e.value)
    df = bytearray(body)
    df[24:28] = (2).to_bytes(4, "little")         # double-float, consistent: accepted
    load(df)
