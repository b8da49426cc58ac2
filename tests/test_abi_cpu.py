"""The C ABI library on the CPU: it loads, exports every symbol its header
declares, validates arguments, and its host construction (tree, lists, ACA,
B2T / T2B pivots) agrees index for index with the oracle.  No compute call
needs a GPU here (host-only handles)."""

import ctypes
import os
import re

import numpy as np
import pytest

import paper_2309_14085_gb300 as pkg
from oracle import h2 as oh2
from oracle import tree as otree
from paper_2309_14085_gb300 import H2Error, H2Matrix, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session", autouse=True)
def built_library():
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2309_14085_gb300 import build_lib
        build_lib.build()
    return pkg.lib()


def test_library_exports_every_declared_symbol():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        text = open(os.path.join(ROOT, "include", hdr)).read()
        names |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(h2_\w+)\s*\(", text, re.M))
    assert {"h2_build", "h2_matvec", "h2_info", "h2_destroy", "h2_last_error"} <= names
    L = ctypes.CDLL(pkg.LIB_PATH)
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(pkg.EXPORTED) <= names


def test_status_names_match_the_header():
    text = open(os.path.join(ROOT, "include", "h2star.h")).read()
    codes = {int(v): n for n, v in re.findall(r"^#define\s+H2_(?:E_)?(\w+)\s+(-?\d+)\b", text, re.M)
             if n in set(pkg.STATUS.values())}
    assert codes == pkg.STATUS
    assert H2Error(-7, "x").status == "TIMEOUT"


def test_invalid_arguments_return_error_codes():
    P = inputs.points(100, 2, 1)
    with pytest.raises(H2Error) as e:
        H2Matrix(P, "log2d", leaf_size=0, tol=1e-6, host_only=True)
    assert e.value.code == -1
    with pytest.raises(H2Error):
        H2Matrix(P, "log2d", leaf_size=8, tol=2.0, host_only=True)
    with pytest.raises(H2Error):
        H2Matrix(np.zeros((10, 4)), "log2d", host_only=True)
    with pytest.raises(H2Error):
        H2Matrix(P, "log2d", domain=((0.0, 0.0), 0.5), host_only=True)   # points outside
    bad = P.copy()
    bad[3, 1] = np.nan
    with pytest.raises(H2Error):
        H2Matrix(bad, "log2d", host_only=True)
    h = ctypes.c_void_p()
    assert pkg.lib().h2_build(None, 10, 2, 0, 8, 1e-6, 0, None, ctypes.byref(h)) == -1
    assert b"NULL" in pkg.lib().h2_last_error()


def test_device_pivot_option_is_checked_before_any_device_use():
    """pivots = 1 asks for the device pivot search: refused with host_only
    (no device may be touched) and, without a CUDA device, NO_DEVICE before
    any construction work."""
    P = inputs.points(300, 2, 2)
    with pytest.raises(H2Error) as e:
        H2Matrix(P, "invr", leaf_size=16, tol=1e-6, pivots="device", host_only=True)
    assert e.value.code == -1
    o = pkg.BuildOpts()
    o.pivots = 3
    h = ctypes.c_void_p()
    assert pkg.lib().h2_build(P.ctypes.data, 300, 2, 1, 16, 1e-6, 0, ctypes.byref(o),
                              ctypes.byref(h)) == -1
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except ImportError:
        has_gpu = False
    if not has_gpu:
        with pytest.raises(H2Error) as e:
            H2Matrix(P, "invr", leaf_size=16, tol=1e-6, pivots="device")
        assert e.value.code == -6
    # host_only takes the host search by default; forcing it is accepted too
    A = H2Matrix(P, "invr", leaf_size=16, tol=1e-6, host_only=True)
    B = H2Matrix(P, "invr", leaf_size=16, tol=1e-6, host_only=True, pivots="host")
    assert A.info()["pivot_problems_device"] == 0 and A.info()["pivot_problems_host"] > 0
    assert np.array_equal(A.pivots(0, 2, 5)[0], B.pivots(0, 2, 5)[0])


def test_unsupported_combinations_are_rejected():
    P = inputs.points(300, 2, 2)
    with pytest.raises(H2Error) as e:
        H2Matrix(P, "log2d", leaf_size=16, tol=1e-6, storage="df64", near="fly", host_only=True)
    assert e.value.code == -5
    with pytest.raises(H2Error) as e:
        H2Matrix(P, "log2d", leaf_size=16, tol=1e-6, storage="df64", variant="h2plush",
                 host_only=True)
    assert e.value.code == -5


def test_convert_rejects_before_touching_a_device():
    P = inputs.points(300, 2, 2)
    fly = H2Matrix(P, "log2d", leaf_size=16, tol=1e-6, near="fly", host_only=True)
    with pytest.raises(H2Error) as e:
        fly.convert("df64")                       # double-float needs stored near blocks
    assert e.value.code == -5
    hp = H2Matrix(P, "log2d", leaf_size=16, tol=1e-6, variant="h2plush", host_only=True)
    with pytest.raises(H2Error) as e:
        hp.convert("df64")
    assert e.value.code == -5
    h = ctypes.c_void_p()
    assert pkg.lib().h2_convert(fly._h, 7, ctypes.byref(h)) == -1
    assert pkg.lib().h2_convert(None, 0, ctypes.byref(h)) == -1
    if not _has_gpu():
        with pytest.raises(H2Error) as e:
            fly.convert("f32")
        assert e.value.code == -6


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_bf16_and_tensor_core_options_are_validated():
    P = inputs.points(300, 2, 2)
    with pytest.raises(H2Error) as e:
        H2Matrix(P, "log2d", leaf_size=16, tol=1e-6, storage="bf16", near="fly", host_only=True)
    assert e.value.code == -5
    with pytest.raises(H2Error) as e:
        H2Matrix(P, "log2d", leaf_size=16, tol=1e-6, storage="bf16", variant="h2plush",
                 host_only=True)
    assert e.value.code == -5
    with pytest.raises(H2Error) as e:
        H2Matrix(P, "log2d", leaf_size=16, tol=1e-6, tensor_cores=True, host_only=True)
    assert e.value.code == -1                     # tf32 tensor cores are for fp32 storage
    A = H2Matrix(P, "log2d", leaf_size=16, tol=1e-6, storage="bf16", host_only=True)
    B = H2Matrix(P, "log2d", leaf_size=16, tol=1e-6, storage="f32", tensor_cores=True,
                 host_only=True)
    a, b = A.info(), B.info()
    assert a["near_stored"] == 1 and b["near_stored"] == 0
    assert a["bytes_m2l"] * 4 == H2Matrix(P, "log2d", leaf_size=16, tol=1e-6,
                                          host_only=True).info()["bytes_m2l"]


def test_m2l_on_the_fly_stores_no_coupling_blocks():
    P = inputs.points(3000, 3, 5)
    with pytest.raises(H2Error) as e:
        H2Matrix(P, "invr", leaf_size=32, tol=1e-6, m2l="fly", host_only=True)   # fp64
    assert e.value.code == -5
    S = H2Matrix(P, "invr", leaf_size=32, tol=1e-6, storage="f32", host_only=True).info()
    F = H2Matrix(P, "invr", leaf_size=32, tol=1e-6, storage="f32", m2l="fly", host_only=True).info()
    assert S["bytes_m2l"] > 0 and F["bytes_m2l"] == 0
    assert F["m2l_src_coeffs"] == S["m2l_src_coeffs"] and F["vlen"] == S["vlen"]
    assert F["ranks"] == S["ranks"]


def test_device_formed_m2l_keeps_the_construction_and_the_accounting():
    """m2l_mode 2 changes where the coupling blocks are formed, not what is
    built: the same pivots and the same stored M2L entries as mode 0."""
    P = inputs.points(3000, 3, 6)
    kw = dict(leaf_size=32, tol=1e-6, host_only=True)
    o = pkg.BuildOpts()
    o.host_only, o.m2l_mode = 1, 3
    h = ctypes.c_void_p()
    Pc = np.ascontiguousarray(P)
    assert pkg.lib().h2_build(Pc.ctypes.data, 3000, 3, 1, 32, 1e-6, 0, ctypes.byref(o),
                              ctypes.byref(h)) == -1
    for variant, storage in [("h2star", "f64"), ("h2sqrt", "f32"), ("h2plush", "f64"),
                             ("h2star_t", "bf16")]:
        S = H2Matrix(P, "invr", variant=variant, storage=storage, **kw)
        D = H2Matrix(P, "invr", variant=variant, storage=storage, m2l="device", **kw)
        a, b = S.info(), D.info()
        assert a["m2l_fly"] == 0 and b["m2l_fly"] == 2
        for k in ("bytes_m2l", "m2l_pairs", "m2l_src_coeffs", "m2l_dst_coeffs", "vlen",
                  "bytes_basis", "bytes_transfer"):
            assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
        for basis in range(a["nbases"]):
            for l in range(1, a["kappa"] + 1):
                for X in (0, 5):
                    assert all(np.array_equal(u, v) for u, v in
                               zip(S.pivots(basis, l, X), D.pivots(basis, l, X)))
    # a host-only handle of this mode holds no M2L values: batches refuse it
    D = H2Matrix(P, "invr", near="stored", m2l="device", **kw)
    hs = (ctypes.c_void_p * 1)(D._h.value)
    out = ctypes.c_void_p()
    assert pkg.lib().h2_batch_create(hs, 1, None, ctypes.byref(out)) == -5
    assert b"host-only" in pkg.lib().h2_last_error()


def test_near_field_storage_accounting():
    P = inputs.points(4096, 2, 1001)
    S = H2Matrix(P, "log2d", leaf_size=64, tol=1e-6, host_only=True).info()
    F = H2Matrix(P, "log2d", leaf_size=64, tol=1e-6, near="fly", host_only=True).info()
    assert S["near_stored"] == 1 and F["near_stored"] == 0
    # stored rows hold every near-field kernel value plus the fused leaf bases
    assert S["bytes_leaf_rows"] >= 8 * (S["near_evals"]) + S["bytes_basis"]
    assert F["bytes_leaf_rows"] == 0
    assert S["bytes_m2l"] == F["bytes_m2l"]


def test_matvec_on_host_only_handle_is_rejected():
    A = H2Matrix(inputs.points(300, 2, 2), "log2d", leaf_size=16, tol=1e-6, host_only=True)
    rc = pkg.lib().h2_matvec(A._h, ctypes.c_void_p(16), 300, ctypes.c_void_p(16), 300, 1, None)
    assert rc == -6
    assert A.info()["bytes_device"] == 0


def test_wait_expiry_injection_validates_before_any_launch():
    L = pkg.lib()
    assert L.h2_inject_wait_expiry(None, 16, None) == -1
    A = H2Matrix(inputs.points(300, 2, 2), "log2d", leaf_size=16, tol=1e-6, storage="bf16",
                 host_only=True)
    assert L.h2_inject_wait_expiry(A._h, -1, None) == -1
    assert L.h2_inject_wait_expiry(A._h, (1 << 22) + 1, None) == -1
    assert L.h2_inject_wait_expiry(A._h, 16, None) == -6
    assert pkg.STATUS[-6] == "NO_DEVICE"


@pytest.mark.parametrize("variant", ["h2star", "h2sqrt", "h2plush", "h2star_t", "h2sqrt_t", "h2star_b"])
@pytest.mark.parametrize("kind,d,N,n_max,eps", [("log2d", 2, 4096, 64, 1e-8),
                                                ("invr", 3, 6000, 32, 1e-6),
                                                ("imq", 2, 3000, 32, 1e-8)])
def test_host_pivots_match_oracle(variant, kind, d, N, n_max, eps):
    """B2T / T2B pivots are integer decisions taken in fp64 on both sides with
    the same reading of ACA: they must agree index for index."""
    P = inputs.points(N, d, 1000 + N)
    A = H2Matrix(P, kind, leaf_size=n_max, tol=eps, variant=variant, host_only=True)
    O = oh2.H2(P, kind, variant=variant, n_max=n_max, eps=eps)
    assert np.array_equal(A.tree_order(), O.tree.order)
    names = ["far", "ver"] if variant == "h2star" else ["far"]
    total = 0
    for b, name in enumerate(names):
        B = O.bases[name]
        for (l, X), ti in B.ti.items():
            gti, gsi = A.pivots(b, l, X)
            assert np.array_equal(gti, ti), (name, l, X)
            assert np.array_equal(gsi, B.si[(l, X)]), (name, l, X)
            total += 1
    assert total > 0
    info = A.info()
    if variant == "h2plush":
        assert info["lowrank_pairs"] == len(O.lowrank)


def test_list_counts_on_full_grids():
    """Stored M2L pairs and near-field blocks on full uniform grids: 2D kappa 3
    has 672 far / 196 vertex-sharing pairs and 288 near-field blocks; strong
    admissibility 1272 pairs and 484 near blocks (the same counts the oracle's
    lists give, which its own tests pin to the paper's closed forms)."""
    P = inputs.points(4096, 2, 1001)
    A = H2Matrix(P, "log2d", leaf_size=64, tol=1e-4, host_only=True)
    info = A.info()
    assert info["kappa"] == 3 and info["m2l_pairs"] == [672, 196] and info["near_pairs"] == 288
    S = H2Matrix(P, "log2d", leaf_size=64, tol=1e-4, variant="h2sqrt", host_only=True)
    si = S.info()
    assert si["m2l_pairs"][0] == 1272 and si["near_pairs"] == 484
    t = otree.Tree(P, n_max=64)
    assert sum(len(t.near_star(3, X)) for X in range(64)) == 288


def test_degenerate_trees_build():
    # fewer points than a leaf holds: kappa 0, everything is near field
    A = H2Matrix(inputs.points(10, 2, 3), "log2d", leaf_size=64, tol=1e-8, host_only=True)
    assert A.info()["kappa"] == 0 and A.info()["near_pairs"] == 1
    # one point
    B = H2Matrix(np.array([[0.25, -0.5, 0.125]]), "invr", leaf_size=4, tol=1e-8, host_only=True)
    assert B.info()["N"] == 1
    # kappa 1: no far field, vertex-sharing only
    C = H2Matrix(inputs.points(100, 2, 4), "log2d", leaf_size=30, tol=1e-8, host_only=True)
    assert C.info()["kappa"] == 1 and C.info()["m2l_pairs"] == [0, 4]
    # points in one corner of a forced domain: most boxes are empty
    P = inputs.points(500, 3, 5, lo=0.0, hi=0.2)
    D = H2Matrix(P, "invr", leaf_size=8, tol=1e-6, domain=((0.0, 0.0, 0.0), 1.0), host_only=True)
    assert D.info()["kappa"] >= 2


@pytest.mark.parametrize("kind,d", [("log2d", 2), ("invr", 3)])
def test_strict_tree_depth_matches_oracle(kind, d):
    """kappa = -1 (the strict reading of §3.1) on clustered points: the same
    depth, tree order and B2T / T2B pivots as the oracle's strict tree; more
    coincident points than leaf_size are refused."""
    nu, nc, side = (1500, 300, 0.3) if d == 2 else (1850, 150, 0.5)
    P = np.vstack([inputs.points(nu, d, 801 + d), inputs.points(nc, d, 811 + d, lo=0.0, hi=side)])
    A = H2Matrix(P, kind, leaf_size=32, tol=1e-6, kappa="strict", host_only=True)
    O = oh2.H2(P, kind, n_max=32, eps=1e-6, kappa="strict")
    assert A.info()["kappa"] == O.tree.kappa == (5 if d == 2 else 3)
    assert np.array_equal(A.tree_order(), O.tree.order)
    for b, name in enumerate(["far", "ver"]):
        B = O.bases[name]
        for (l, X), ti in B.ti.items():
            gti, gsi = A.pivots(b, l, X)
            assert np.array_equal(gti, ti), (name, l, X)
            assert np.array_equal(gsi, B.si[(l, X)]), (name, l, X)
    with pytest.raises(H2Error) as e:
        H2Matrix(np.repeat(inputs.points(4, d, 5), 40, axis=0), kind, leaf_size=32, tol=1e-6,
                 kappa="strict", host_only=True)
    assert e.value.code == -1


def test_header_is_plain_c_and_links(tmp_path):
    """include/h2star.h is a C header: a C99 program compiles against it with
    -pedantic -Werror, links against the library and gets INVALID_ARG and a
    message from h2_build with no points (no device is touched)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "abi.c"
    src.write_text(
        '#include <stdio.h>\n#include "h2star.h"\n'
        "int main(void) {\n"
        "    h2_build_opts o = {0};\n"
        "    h2_handle h = 0;\n"
        "    int rc = h2_build(0, 10, 2, H2_KERNEL_LOG2D, 8, 1e-6, H2_STAR_BT, &o, &h);\n"
        '    printf("%d %s\\n", rc, h2_last_error());\n'
        "    return rc == H2_E_INVALID_ARG && h == 0 ? 0 : 1;\n"
        "}\n")
    exe = tmp_path / "abi"
    lib_dir = os.path.dirname(pkg.lib()._name)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L" + lib_dir, "-lh2star", "-Wl,-rpath," + lib_dir], check=True)
    out = subprocess.run([str(exe)], stdout=subprocess.PIPE, text=True)
    assert out.returncode == 0, out.stdout
    assert out.stdout.startswith("-1 ") and len(out.stdout.strip()) > 3
