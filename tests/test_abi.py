"""C-ABI contract checks that need no GPU: the library loads, exports every
function declared in include/tlbm.h, and validates host-side arguments."""
import math
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"TLBM_API\s+[\w\s\*]+?\b(tlbm_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def T():
    from paper_2211_03160_gb300 import tlbm
    tlbm.lib()
    return tlbm


def test_library_exports_every_declared_symbol(T):
    names = _declared("tlbm.h")
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", T.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (tlbm_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = T.lib()
    for n in names:
        assert getattr(L, n) is not None


def test_binding_has_every_c_name(T):
    for n in _declared("tlbm.h"):
        if n == "tlbm_default_params":
            continue
        assert hasattr(T, n), n


def test_default_params_are_nan(T):
    p = T.tlbm_default_params()
    assert p.walls == T.TLBM_RB and p.periodic_mask == 0
    for k in ("a_T", "nu", "alpha", "gbeta", "s_q", "q_e", "Th", "Tc", "store_scale"):
        assert math.isnan(getattr(p, k))


@pytest.mark.parametrize("args,code", [
    ((2, 10, 1, 0, 1e5, 0.71, 0.1, 1), -1),
    ((10, 2, 1, 0, 1e5, 0.71, 0.1, 1), -1),
    ((10, 10, 2, 1, 1e5, 0.71, 0.1, 1), -1),
    ((10, 10, 1, 0, 0.0, 0.71, 0.1, 1), -1),
    ((10, 10, 1, 0, 1e5, -1.0, 0.1, 1), -1),
    ((10, 10, 1, 0, 1e5, 0.71, 0.0, 1), -1),
    ((10, 10, 1, 7, 1e5, 0.71, 0.1, 1), -1),
    ((10, 10, 1, 0, 1e5, 0.71, 0.1, 9), -7),
])
def test_create_rejects_invalid(T, args, code):
    with pytest.raises(T.TlbmError) as ei:
        T.tlbm_create(*args)
    assert ei.value.code == code
    assert T.tlbm_last_error(None)


def test_create_rejects_tiny_relaxation(T):
    p = T.tlbm_default_params(nu=1e-8)
    with pytest.raises(T.TlbmError):
        T.tlbm_create(10, 10, 1, 0, 1e5, 0.71, 0.1, 1, p)


def test_unbound_handle_refuses_work(T):
    h = T.tlbm_create(33, 17, 1, 0, 1e5, 0.71, 0.1, 1)
    try:
        for fn in (lambda: T.tlbm_step(h, 1), lambda: T.tlbm_init(h, 1, 1e-3), T.tlbm_nusselt and
                   (lambda: T.tlbm_nusselt(h))):
            with pytest.raises(T.TlbmError) as ei:
                fn()
            assert ei.value.code == T.TLBM_ERR_UNBOUND
        assert T.tlbm_required_bytes(h) > 0
        assert T.tlbm_launch_count(h) == 0
    finally:
        T.tlbm_destroy(h)


def test_required_bytes_cover_both_buffers(T):
    for lattice, shape, prec, elem, q in ((0, (8193, 8193, 1), 1, 4, 14), (1, (385, 385, 385), 2, 2, 26),
                                           (0, (129, 129, 1), 0, 8, 14)):
        h = T.tlbm_create(*shape, lattice, 1e7, 0.71, 0.1, prec)
        try:
            n = T.tlbm_required_bytes(h)
            nodes = shape[0] * shape[1] * shape[2]
            assert n >= 2 * q * nodes * elem
            assert n < 2 * q * nodes * elem * 1.25 + (64 << 20)
            assert n % 256 == 0
        finally:
            T.tlbm_destroy(h)


def test_derived_parameters_match_oracle(T, O):
    """Both sides map (Ra, Pr, Ma) to the same lattice parameters and rates."""
    for lattice, shape in ((0, (129, 129, 1)), (1, (17, 19, 23))):
        h = T.tlbm_create(*shape, lattice, 1e5, 0.71, 0.1, 0)
        try:
            d = T.tlbm_derived(h)
        finally:
            T.tlbm_destroy(h)
        o = O.Sim(*shape, lattice=lattice, Ra=1e5, Pr=0.71, Ma=0.1).derived()
        ref = [o["U"], o["H"], o["nu"], o["alpha"], o["gbeta"], o["a_T"], o["omega"], *o["S"], *o["Q"]]
        assert len(d) == len(ref)
        for a, b in zip(d, ref):
            assert a == pytest.approx(b, rel=1e-15, abs=1e-300)


def test_bind_rejects_null_and_small(T):
    h = T.tlbm_create(33, 17, 1, 0, 1e5, 0.71, 0.1, 1)
    try:
        with pytest.raises(T.TlbmError) as ei:
            T.tlbm_bind_memory(h, 0, 1 << 30)
        assert ei.value.code == T.TLBM_ERR_ARG
        with pytest.raises(T.TlbmError) as ei:
            T.tlbm_bind_memory(h, 1 << 20, 16)
        assert ei.value.code == T.TLBM_ERR_OOM
    finally:
        T.tlbm_destroy(h)


def _declared_arity(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"TLBM_API\s+[\w\s\*]+?\b(tlbm_\w+)\s*\(([^)]*)\)", src):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else len(args.split(","))
    return out


def test_binding_argument_counts_match_the_header(T):
    """Every ctypes signature has exactly as many arguments as the C declaration,
    and every Python wrapper passes that many."""
    import inspect

    arity = _declared_arity("tlbm.h")
    for name, (res, args) in T._SIGS.items():
        assert arity[name] == len(args), name
    for name, n in arity.items():
        src = inspect.getsource(getattr(T, name)) if hasattr(T, name) else ""
        call = re.search(r"lib\(\)\." + name + r"\((.*)\)\)", src.replace("\n", " "))
        if call and "*" not in call.group(1):
            depth, count = 0, 1
            for ch in call.group(1):
                depth += ch in "([{"
                depth -= ch in ")]}"
                count += ch == "," and depth == 0
            assert count == n, (name, count, n)


def test_inplace_streaming_needs_one_buffer(T):
    p = T.tlbm_default_params()
    assert p.streaming == T.TLBM_STREAM_PULL
    h2 = T.tlbm_create(8193, 8193, 1, 0, 1e8, 0.71, 0.1, 1, p)
    h1 = T.tlbm_create(8193, 8193, 1, 0, 1e8, 0.71, 0.1, 1, T.tlbm_default_params(streaming=T.TLBM_STREAM_INPLACE))
    try:
        b2, b1 = T.tlbm_required_bytes(h2), T.tlbm_required_bytes(h1)
        pop = 14 * 4 * 8193 * 8193
        assert pop <= b2 - b1 < 1.2 * pop
    finally:
        T.tlbm_destroy(h2)
        T.tlbm_destroy(h1)
    with pytest.raises(T.TlbmError) as ei:
        T.tlbm_create(10, 10, 1, 0, 1e5, 0.71, 0.1, 1, T.tlbm_default_params(streaming=2))
    assert ei.value.code == T.TLBM_ERR_ARG


def test_wait_limits_are_validated(T):
    h = T.tlbm_create(33, 17, 1, 0, 1e5, 0.71, 0.1, 2)
    try:
        T.tlbm_set_wait_limit(h, 0.0)
        T.tlbm_set_wait_limit(h, 10.0)
        for bad in (-1e-9, 10.5, float("nan")):
            with pytest.raises(T.TlbmError) as ei:
                T.tlbm_set_wait_limit(h, bad)
            assert ei.value.code == T.TLBM_ERR_ARG
    finally:
        T.tlbm_destroy(h)
    b = T.tlbm_batch_create([(33, 33, 1, 1e5, 0.71, 0.1, 1), (17, 17, 1, 1e5, 0.71, 0.1, 2)], 0, 1)
    try:
        T.tlbm_batch_set_wait_limit(b, 0.0)
        for bad in (-1.0, 11.0, float("nan")):
            with pytest.raises(T.TlbmError) as ei:
                T.tlbm_batch_set_wait_limit(b, bad)
            assert ei.value.code == T.TLBM_ERR_ARG
    finally:
        T.tlbm_batch_destroy(b)


def test_checkpoint_needs_bound_memory_and_a_path(T):
    h = T.tlbm_create(33, 17, 1, 0, 1e5, 0.71, 0.1, 1)
    try:
        for fn in (T.lib().tlbm_save, T.lib().tlbm_load):
            assert fn(h, b"/nonexistent/x.ckpt") == T.TLBM_ERR_UNBOUND
            assert fn(h, None) == T.TLBM_ERR_UNBOUND
    finally:
        T.tlbm_destroy(h)


def test_staged_query_and_batch_rows_on_host(T):
    h = T.tlbm_create(33, 17, 1, 0, 1e5, 0.71, 0.1, 2)
    try:
        assert T.tlbm_get_staged(h) == (0, 0, 0)  # not bound: the register kernels
    finally:
        T.tlbm_destroy(h)
    b = T.tlbm_batch_create([(33, 33, 1, 1e5, 0.71, 0.1, 1)], 0, 1)
    try:
        assert T.tlbm_batch_get_rows(b) == 1
        for bad in (0, 3, -1):
            with pytest.raises(T.TlbmError) as ei:
                T.tlbm_batch_set_rows(b, bad)
            assert ei.value.code == T.TLBM_ERR_ARG
        T.tlbm_batch_set_rows(b, 2)
        assert T.tlbm_batch_get_rows(b) == 2
    finally:
        T.tlbm_batch_destroy(b)


def test_staged_batch_arguments_on_host(T):
    """tlbm_batch_set_staged checks its arguments before any device call:
    consumer warps 4 or 8 in 2D (4 or 7 in 3D), stages 0 or 2..8, no FP64
    storage, not with the persistent form; a fresh batch reports the register
    kernels."""
    b = T.tlbm_batch_create([(33, 33, 1, 1e5, 0.71, 0.1, 1)], 0, T.TLBM_FP16_OFFSET)
    try:
        assert T.tlbm_batch_get_staged(b) == (0, 0, 0)
        for nc, ns, code in ((7, 0, T.TLBM_ERR_ARG), (5, 0, T.TLBM_ERR_ARG), (-1, 0, T.TLBM_ERR_ARG),
                             (8, 1, T.TLBM_ERR_ARG), (4, 9, T.TLBM_ERR_ARG)):
            with pytest.raises(T.TlbmError) as ei:
                T.tlbm_batch_set_staged(b, nc, ns)
            assert ei.value.code == code, (nc, ns)
        T.tlbm_batch_set_staged(b, 0, 0)  # off: nothing to check
        assert T.tlbm_batch_get_staged(b) == (0, 0, 0)
    finally:
        T.tlbm_batch_destroy(b)
    b3 = T.tlbm_batch_create([(9, 11, 7, 1e5, 0.71, 0.1, 1)], 1, T.TLBM_BF16_OFFSET)
    try:
        with pytest.raises(T.TlbmError) as ei:
            T.tlbm_batch_set_staged(b3, 8, 0)  # 4 or 7 in 3D
        assert ei.value.code == T.TLBM_ERR_ARG
    finally:
        T.tlbm_batch_destroy(b3)
    b64 = T.tlbm_batch_create([(33, 33, 1, 1e5, 0.71, 0.1, 1)], 0, T.TLBM_FP64)
    try:
        with pytest.raises(T.TlbmError) as ei:
            T.tlbm_batch_set_staged(b64, 8, 0)
        assert ei.value.code == T.TLBM_ERR_UNSUPPORTED
    finally:
        T.tlbm_batch_destroy(b64)


def test_conv_weight_operand_size(T):
    """The packed convolution weights hold 9 taps x ceil(cin / 16) tiles of
    32 x 16 BF16 elements; channel counts outside 1..32 have no operand."""
    for cin, n in ((1, 4608), (5, 4608), (16, 4608), (17, 9216), (32, 9216)):
        assert T.tlbm_conv3x3_weight_elems(cin) == n
    for bad in (0, -3, 33):
        assert T.tlbm_conv3x3_weight_elems(bad) == 0
