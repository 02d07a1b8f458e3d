"""The C ABI without a GPU: the library loads, exports every function include/pauli.h
declares, and rejects bad arguments with the documented status before touching the device.

Only arguments that fail validation are passed with fabricated pointer values; the one call
with valid-looking fabricated pointers arms the host failure hook first, so nothing is ever
enqueued.
"""
import ctypes
import os
import re

import pytest

from paper_2401_16378_gb300 import _build, _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pauli.h")

OK, ARG, NULL, ALIGN, ALIAS, DTYPE, NOMEM, CUDA, TIMEOUT, UNSUP = range(10)
C64, C128 = 0, 1


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pauli_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("pauli_decompose", "pauli_compose", "pauli_coeffs_at", "pauli_plan_create", "pauli_plan_execute",
                 "pauli_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_version(lib):
    assert lib.pauli_version() >= 100


def P(v):
    return ctypes.c_void_p(v)


A, B = 0x10000000, 0x20000000  # fabricated, 16-byte aligned, far apart


def test_decompose_rejects_bad_arguments(lib):
    assert lib.pauli_decompose(P(A), 4, 1, 7, P(B), 0, None) == DTYPE
    assert lib.pauli_decompose(P(A), 0, 1, C128, P(B), 0, None) == ARG
    assert lib.pauli_decompose(P(A), 17, 1, C128, P(B), 0, None) == ARG
    assert lib.pauli_decompose(P(A), 4, 0, C128, P(B), 0, None) == ARG
    assert lib.pauli_decompose(None, 4, 1, C128, P(B), 0, None) == NULL
    assert lib.pauli_decompose(P(A), 4, 1, C128, None, 0, None) == NULL
    assert lib.pauli_decompose(P(A + 8), 4, 1, C128, P(B), 0, None) == ALIGN
    assert lib.pauli_decompose(P(A + 4), 4, 1, C64, P(B), 0, None) == ALIGN
    assert lib.pauli_decompose(P(A), 4, 1, C128, P(A + 16 * 255), 0, None) == ALIAS
    assert lib.pauli_decompose(P(A), 4, 1, C128, P(B), 9, None) == ARG
    assert lib.pauli_decompose(P(A), 3, 1, C128, P(B), 2, None) == UNSUP  # no XOR-diagonal kernel at N=3
    assert lib.pauli_set_variant(5, C128, 0, 1) == UNSUP
    assert lib.pauli_set_variant(14, C128, 4, 1) == ARG
    assert lib.pauli_get_variant(10, C128, 0) == 1  # one matrix: 8192-element units
    assert lib.pauli_get_variant(10, C128, 2) == 2  # a batch: 4096-element units, two CTAs per SM
    assert lib.pauli_get_variant(14, C128, 2) == 7
    assert lib.pauli_set_variant(14, C128, 3, 5) == UNSUP
    assert lib.pauli_get_variant(3, C128, 0) == 0
    assert lib.pauli_get_variant(14, C128, 0) == 7  # decompose at N = 14: the two-stage kernel
    assert lib.pauli_get_variant(14, C128, 1) == 1  # compose: single-pass 8192-element units
    assert lib.pauli_get_variant(12, C128, 0) == 7
    assert lib.pauli_set_variant(14, C128, 1, 5) == UNSUP  # tiled is decompose-only


def test_error_message_names_the_problem(lib):
    assert lib.pauli_decompose(P(A), 17, 1, C128, P(B), 0, None) == ARG
    assert b"N = 17" in lib.pauli_last_error()
    assert lib.pauli_decompose(None, 4, 1, C128, P(B), 0, None) == NULL
    assert b"G is NULL" in lib.pauli_last_error()


def test_compose_rejects_bad_arguments(lib):
    assert lib.pauli_compose(P(A), 4, 1, C128, P(B), 65, None) == ARG
    assert lib.pauli_compose(P(A), 4, 1, C128, P(A), 0, None) == ALIAS
    assert lib.pauli_compose(P(A), 4, 1, 3, P(B), 0, None) == DTYPE


def test_hermitian_and_norm_reject_bad_arguments(lib):
    assert lib.pauli_decompose_hermitian(P(A), 4, 1, C128, None, 0, None) == NULL
    assert lib.pauli_decompose_hermitian(P(A), 4, 1, C128, P(B + 4), 0, None) == ALIGN
    assert lib.pauli_decompose_hermitian(P(A), 4, 1, C64, P(B + 2), 0, None) == ALIGN
    assert lib.pauli_decompose_hermitian(P(A), 4, 1, C128, P(A + 8 * 255), 0, None) == ALIAS
    assert lib.pauli_decompose_hermitian(P(A), 4, 0, C128, P(B), 0, None) == ARG
    assert lib.pauli_decompose_hermitian(P(A), 3, 1, C128, P(B), 2, None) == UNSUP
    assert lib.pauli_decompose_hermitian_upper(P(A), 6, 1, C128, P(B), 2, None) == UNSUP
    assert lib.pauli_decompose_hermitian_upper(P(1 << 36), 15, 1, C128, P(2 << 36), 0, None) == UNSUP  # N > 14
    assert lib.pauli_decompose_hermitian_upper(P(1 << 32), 13, 1025, C128, P(1 << 44), 0, None) == UNSUP  # count
    assert lib.pauli_decompose_hermitian_upper(P(A), 4, 1, C128, P(A + 8), 0, None) == ALIAS
    assert lib.pauli_decompose_hermitian_upper(P(A), 4, 1, C128, P(B), 7, None) == ARG
    assert lib.pauli_decompose_real(P(A), 4, 1, C64, P(B), 0, None) == UNSUP
    assert lib.pauli_decompose_real(P(A + 4), 4, 1, C128, P(B), 0, None) == ALIGN
    assert lib.pauli_decompose_real(P(A), 4, 1, C128, P(A + 8 * 255), 0, None) == ALIAS
    assert lib.pauli_decompose_real(P(A), 3, 1, C128, P(B), 2, None) == UNSUP
    assert lib.pauli_weighted_norm(P(A), 4, 1, C128, None, P(B), None) == NULL
    assert lib.pauli_weighted_norm(P(A), 4, 1, C128, P(B), P(A + 8), None) == ALIAS  # loss inside c
    assert lib.pauli_weighted_norm(P(A), 4, 1, C128, P(B + 4), P(B + 4096), None) == ALIGN
    assert lib.pauli_weighted_norm_grad(P(A), 4, 1, C128, P(B), None, P(A + 16), None) == ALIAS
    assert lib.pauli_weighted_norm_grad(P(A), 4, 1, C128, P(B), None, P(B + 16), None) == ALIAS  # over w
    assert lib.pauli_weighted_norm_grad(P(A), 4, 1, C128, P(B), P(B + 4), P(B + 65536), None) == ALIGN
    # fused forms: c at B, w at B + 1 MiB, loss at B + 2 MiB
    W, L = B + (1 << 20), B + (2 << 20)
    assert lib.pauli_decompose_weighted_norm(P(A), 4, 1, C128, P(B), None, P(L), 0, None) == NULL
    assert lib.pauli_decompose_weighted_norm(P(A), 4, 1, C128, P(B), P(W), None, 0, None) == NULL
    assert lib.pauli_decompose_weighted_norm(P(A), 4, 1, C128, P(B), P(W), P(B + 64), 0, None) == ALIAS
    assert lib.pauli_decompose_weighted_norm(P(A), 4, 1, C128, P(B), P(B + 16), P(L), 0, None) == ALIAS
    assert lib.pauli_decompose_weighted_norm(P(A), 4, 1, C128, P(B), P(W + 4), P(L), 0, None) == ALIGN
    assert lib.pauli_compose_weighted(P(1 << 32), 13, 1, C128, P(3 << 32), None, P(2 << 32), 0, None) == UNSUP
    assert lib.pauli_compose_weighted(P(A), 4, 1, C128, None, None, P(B), 0, None) == NULL
    assert lib.pauli_compose_weighted(P(A), 4, 1, C128, P(W), None, P(B), 65, None) == ARG
    assert lib.pauli_compose_weighted(P(A), 4, 1, C128, P(B + 32), None, P(B), 0, None) == ALIAS


def test_host_stream_rejects_bad_arguments(lib):
    arr = lambda *v: (ctypes.c_void_p * len(v))(*[ctypes.c_void_p(x) for x in v])  # noqa: E731
    hosts, outs = arr(A), arr(A + (1 << 20))
    devs_g, devs_o = arr(B, B + 8192), arr(B + 16384, B + 24576)
    assert lib.pauli_decompose_host_stream(None, outs, 1, 4, C128, devs_g, devs_o, 0, None) == NULL
    assert lib.pauli_decompose_host_stream(hosts, outs, 0, 4, C128, devs_g, devs_o, 0, None) == ARG
    assert lib.pauli_decompose_host_stream(hosts, outs, 1, 4, C128, arr(B, B + 16), devs_o, 0, None) == ALIAS
    assert lib.pauli_decompose_host_stream(hosts, arr(A + 16), 1, 4, C128, devs_g, devs_o, 0, None) == ALIAS
    assert lib.pauli_decompose_host_stream(hosts, outs, 1, 4, C128, devs_g, devs_o, 9, None) == ARG


def test_coeffs_at_rejects_bad_arguments(lib):
    assert lib.pauli_coeffs_at(P(A), 4, C128, P(B), 0, P(B + 4096), None) == OK  # k = 0: nothing to do
    assert lib.pauli_coeffs_at(P(A), 4, C128, P(B), -1, P(B + 4096), None) == ARG
    assert lib.pauli_coeffs_at(P(A), 4, C128, None, 5, P(B + 4096), None) == NULL
    assert lib.pauli_coeffs_at(P(A), 4, C128, P(B + 4), 5, P(B + 4096), None) == ALIGN
    assert lib.pauli_coeffs_at(P(A), 4, C128, P(B), 5, P(A + 32), None) == ALIAS


def test_list_and_plan_argument_errors(lib):
    ns = (ctypes.c_int * 2)(3, 11)
    h = ctypes.c_void_p()
    assert lib.pauli_plan_create(ns, 2, C128, 0, 0, ctypes.byref(h)) == ARG
    assert lib.pauli_plan_create(ns, 0, C128, 0, 0, ctypes.byref(h)) == ARG
    assert lib.pauli_plan_create(None, 2, C128, 0, 0, ctypes.byref(h)) == NULL
    assert lib.pauli_plan_create_hermitian(ns, 2, C128, 0, 0, ctypes.byref(h)) == ARG  # N = 11 > 10
    assert lib.pauli_plan_create_hermitian(ns, 2, C128, 384, 0, ctypes.byref(h)) == ARG
    assert lib.pauli_plan_create_hermitian(ns, 2, 7, 0, 0, ctypes.byref(h)) == DTYPE
    assert lib.pauli_plan_execute(None, None) == NULL
    assert lib.pauli_decompose_list(None, ns, 2, C128, None, 0, None) == NULL
    assert lib.pauli_decompose_list(None, None, 0, C128, None, 0, None) == OK


def _ptr_list(vals):
    arr = (ctypes.c_void_p * len(vals))(*vals)
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


def test_compose_batched_rejects_bad_arguments(lib):
    cs, k1 = _ptr_list([A, A + 0x100000])
    gs, k2 = _ptr_list([B, B + 0x100000])
    ns = (ctypes.c_int * 2)(3, 5)
    assert lib.pauli_compose_batched(cs, ns, 2, 7, gs, 0, None) == DTYPE
    assert lib.pauli_compose_batched(cs, ns, -1, C128, gs, 0, None) == ARG
    assert lib.pauli_compose_batched(cs, ns, 0, C128, gs, 0, None) == OK  # nothing to do
    assert lib.pauli_compose_batched(None, ns, 2, C128, gs, 0, None) == NULL
    assert lib.pauli_compose_batched(cs, ns, 2, C128, gs, 65, None) == ARG
    bad = (ctypes.c_int * 2)(3, 12)
    assert lib.pauli_compose_batched(cs, bad, 2, C128, gs, 0, None) == ARG  # N above 11
    assert b"11" in lib.pauli_last_error()
    alias, k3 = _ptr_list([A, B])
    assert lib.pauli_compose_batched(cs, ns, 2, C128, alias, 0, None) == ALIAS  # entry 0: c and G overlap
    unal, k4 = _ptr_list([A + 8, A + 0x100000])
    assert lib.pauli_compose_batched(unal, ns, 2, C128, gs, 0, None) == ALIGN


def test_workspace_entry_points_reject_bad_arguments(lib):
    n = ctypes.c_size_t(123)
    assert lib.pauli_decompose_workspace_size(14, 1, C128, 0, None) == NULL
    assert lib.pauli_decompose_workspace_size(0, 1, C128, 0, ctypes.byref(n)) == ARG
    assert lib.pauli_decompose_workspace_size(14, 0, C128, 0, ctypes.byref(n)) == ARG
    assert lib.pauli_decompose_workspace_size(14, 1, 3, 0, ctypes.byref(n)) == DTYPE
    # the built-in shape at N = 14 is the tiled kernel: it needs scratch; PLAIN and N = 10 need none
    assert lib.pauli_decompose_workspace_size(14, 1, C128, 0, ctypes.byref(n)) == OK and n.value > (1 << 20)
    need = n.value
    assert lib.pauli_decompose_workspace_size(14, 1, C128, 1, ctypes.byref(n)) == OK and n.value == 0
    assert lib.pauli_decompose_workspace_size(10, 1, C128, 0, ctypes.byref(n)) == OK and n.value == 0
    assert lib.pauli_decompose_workspace_size(14, 2000, C128, 0, ctypes.byref(n)) == OK and n.value == 0
    W = 0x40000000
    assert lib.pauli_decompose_ws(P(A), 14, 1, C128, P(B), 0, None, need, None) == ALIAS  # G, out overlap
    G14, O14 = 0x100000000, 0x300000000  # 4 GiB each, apart
    assert lib.pauli_decompose_ws(P(G14), 14, 1, C128, P(O14), 0, None, need, None) == NULL
    assert lib.pauli_decompose_ws(P(G14), 14, 1, C128, P(O14), 0, P(W + 16), need, None) == ALIGN
    assert lib.pauli_decompose_ws(P(G14), 14, 1, C128, P(O14), 0, P(W), need - 1, None) == ARG
    assert lib.pauli_decompose_ws(P(G14), 14, 1, C128, P(O14), 0, P(G14 + 4096), need, None) == ALIAS
    assert lib.pauli_workspace_status(None, None) == NULL


def test_xhi_entry_points_reject_bad_arguments(lib):
    # N = 8, k = 2: G holds 4^8 = 65536 elements (1 MiB complex128), a shard 16384 (256 KiB)
    assert lib.pauli_xhi_layout(P(A), 8, 2, 1, 7, P(B), None) == DTYPE
    assert lib.pauli_xhi_layout(P(A), 8, 8, 0, C128, P(B), None) == ARG  # k = N
    assert lib.pauli_xhi_layout(P(A), 8, -1, 0, C128, P(B), None) == ARG
    assert lib.pauli_xhi_layout(P(A), 8, 2, 4, C128, P(B), None) == ARG  # x_hi = 2^k
    assert b"x_hi" in lib.pauli_last_error()
    assert lib.pauli_xhi_layout(None, 8, 2, 1, C128, P(B), None) == NULL
    assert lib.pauli_xhi_layout(P(A + 8), 8, 2, 1, C128, P(B), None) == ALIGN
    assert lib.pauli_xhi_layout(P(A), 8, 2, 1, C128, P(A + 0x80000), None) == ALIAS
    assert lib.pauli_decompose_xhi(P(A), 8, 2, 1, 7, P(B), 0, None) == DTYPE
    assert lib.pauli_decompose_xhi(P(A), 0, 0, 0, C128, P(B), 0, None) == ARG
    assert lib.pauli_decompose_xhi(P(A), 8, 9, 0, C128, P(B), 0, None) == ARG
    assert lib.pauli_decompose_xhi(P(A), 8, 2, -1, C128, P(B), 0, None) == ARG
    assert lib.pauli_decompose_xhi(P(A), 8, 2, 1, C128, None, 0, None) == NULL
    assert lib.pauli_decompose_xhi(P(A), 8, 2, 1, C128, P(A + 0x20000), 0, None) == ALIAS  # 256 KiB shard
    assert lib.pauli_decompose_xhi(P(A), 8, 2, 1, C128, P(B), 9, None) == ARG  # method
    lib.pauli_debug_fail_next_launches(2)
    assert lib.pauli_decompose_xhi(P(A), 8, 2, 1, C128, P(B), 0, None) == CUDA
    assert lib.pauli_xhi_layout(P(A), 8, 2, 1, C128, P(B), None) == CUDA
    lib.pauli_debug_fail_next_launches(0)


def test_injected_launch_failure_is_reported(lib):
    lib.pauli_debug_fail_next_launches(1)
    assert lib.pauli_decompose(P(A), 4, 1, C128, P(B), 0, None) == CUDA
    assert b"injected" in lib.pauli_last_error()
    lib.pauli_debug_fail_next_launches(0)


def test_header_is_plain_c(tmp_path):
    """include/pauli.h compiles as C99 (no C++ or torch types at the boundary)."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "pauli.h"\nint main(void) { return pauli_version() < 0; }\n')
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                          "-I", os.path.join(root, "include"), str(src)], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr


def test_autotune_cache_entries_reach_the_variant_tables(lib):
    """autotune.apply sets the one-matrix and the batch launch shapes separately (host only)."""
    from paper_2401_16378_gb300 import autotune

    cache = {"variants": {"10/c128/decompose": {"best": 4}, "10/c128/decompose_batched": {"best": 3},
                          "10/c64/compose_batched": {"best": 1}}}
    try:
        assert autotune.apply(cache) == 3
        assert lib.pauli_get_variant(10, C128, 0) == 4
        assert lib.pauli_get_variant(10, C128, 2) == 3
        assert lib.pauli_get_variant(10, 0, 3) == 1
    finally:
        for op in range(4):
            lib.pauli_set_variant(10, C128, op, 0)
            lib.pauli_set_variant(10, 0, op, 0)
    assert lib.pauli_get_variant(10, C128, 2) == 2  # built-in batch shape: 4096-element units
