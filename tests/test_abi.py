"""The C-ABI library loads and exports every entry point include/rbgs.h declares, and its
argument checking works without a GPU (host logic only: no CUDA work is issued)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2607_01735_gb300 as rb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rbgs.h")
HEADERS = sorted(os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include"))
                 if h.endswith(".h"))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_01735_gb300 import build
    build.build_library()
    return rb.load_library()


def _declared(path=HEADER):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rbgs[a-z0-9]*_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_names():
    assert set(_declared()) == set(rb.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", rb.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rbgs\w*)", out))
    assert len(HEADERS) >= 2
    for h in HEADERS:
        names = _declared(h)
        assert names, h
        for name in names:
            assert hasattr(lib, name), name
        assert set(names) <= exported, (h, set(names) - exported)


CITATION = re.compile(r"Section \d|Eq\. \(\d|Algorithm \d|not in the paper|no counterpart", re.I)


def _declaration_comments(path):
    """(name, comment) for every function declared in a header: the block comment that
    precedes the declaration, or, for declarations grouped under one comment, that one."""
    text = open(path).read()
    out, last_comment = [], ""
    for m in re.finditer(r"/\*.*?\*/|\b(rbgs[a-z0-9]*_[a-z0-9_]+)\s*\(", text, flags=re.S):
        if m.group(0).startswith("/*"):
            last_comment = m.group(0)
        else:
            out.append((m.group(1), last_comment))
    return out


def test_every_declaration_cites_its_passage_or_says_it_has_none():
    """Each entry point's comment names the paper's passage it implements (section,
    equation, algorithm) or states that the paper has no counterpart."""
    for h in HEADERS:
        decls = _declaration_comments(h)
        assert {n for n, _ in decls} == set(_declared(h)), h
        for name, comment in decls:
            flat = " ".join(comment.replace("/*", " ").replace("*/", " ").replace("*", " ").split())
            assert CITATION.search(flat), (h, name, flat[:120])


def test_default_opts(lib):
    o = rb.default_opts()
    assert (o.precision, o.kernel, o.check_every, o.fp64_emulate) == (rb.RBGS_FP64, rb.RBGS_KERNEL_AUTO, 100, -1)
    assert o.max_sweeps == 1000000000
    assert (o.fma, o.stall_checks, o.max_seconds) == (0, 0, 0.0)


def test_struct_layouts_match_header(lib):
    # rbgs_opts: 3 ints (+4 padding), a long, 10 ints, a double -> 72 bytes on LP64
    assert ctypes.sizeof(rb.Opts) == 72
    assert ctypes.sizeof(rb.Problem) == 32
    assert ctypes.sizeof(rb.Result) == 32


def test_argument_errors_without_gpu(lib):
    f = np.zeros((4, 4))
    u = np.zeros((6, 6))
    h = ctypes.c_void_p()
    assert lib.rbgs_create(0, 0.04, f.ctypes.data, u.ctypes.data, None, None, ctypes.byref(h)) == rb.RBGS_EINVAL
    assert "n = 0" in rb.rbgs_last_error()
    assert lib.rbgs_create(4, -1.0, f.ctypes.data, u.ctypes.data, None, None, ctypes.byref(h)) == rb.RBGS_EINVAL
    assert lib.rbgs_create(4, 0.04, None, u.ctypes.data, None, None, ctypes.byref(h)) == rb.RBGS_EINVAL
    assert lib.rbgs_create(4, 0.04, f.ctypes.data, u.ctypes.data, None, None, None) == rb.RBGS_EINVAL
    bad = rb.default_opts(precision=7)
    assert lib.rbgs_create(4, 0.04, f.ctypes.data, u.ctypes.data, ctypes.byref(bad), None,
                           ctypes.byref(h)) == rb.RBGS_EINVAL
    bad = rb.default_opts(fp64_emulate=0x33)
    assert lib.rbgs_create(4, 0.04, f.ctypes.data, u.ctypes.data, ctypes.byref(bad), None,
                           ctypes.byref(h)) == rb.RBGS_EINVAL
    # kernel choice and the depths each kernel supports
    for bad in (rb.default_opts(kernel=5), rb.default_opts(kernel=rb.RBGS_KERNEL_WAVEFRONT, tblock_k=3),
                rb.default_opts(kernel=rb.RBGS_KERNEL_WAVEFRONT, tblock_k=1),
                rb.default_opts(kernel=rb.RBGS_KERNEL_WAVEFRONT, precision=rb.RBGS_FP32_REFINE, tblock_k=8),
                rb.default_opts(kernel=rb.RBGS_KERNEL_TEMPORAL, tblock_k=6)):
        assert lib.rbgs_create(4, 0.04, f.ctypes.data, u.ctypes.data, ctypes.byref(bad), None,
                               ctypes.byref(h)) == rb.RBGS_EINVAL
    # the cooperative FP64 launch indexes its items in 32 bits: n <= 32768 (the arrays are
    # never read: options are checked first)
    big = rb.default_opts(kernel=rb.RBGS_KERNEL_PERSISTENT)
    assert lib.rbgs_create(40000, 1e-9, f.ctypes.data, u.ctypes.data, ctypes.byref(big), None,
                           ctypes.byref(h)) == rb.RBGS_EINVAL
    assert "32768" in rb.rbgs_last_error()
    # the fused update (fma = 1): FP64 sweeps, one launch per colour; stall and time options
    for bad in (rb.default_opts(fma=2), rb.default_opts(fma=-1),
                rb.default_opts(fma=1, precision=rb.RBGS_FP32_REFINE),
                rb.default_opts(fma=1, kernel=rb.RBGS_KERNEL_PERSISTENT),
                rb.default_opts(fma=1, kernel=rb.RBGS_KERNEL_WAVEFRONT),
                rb.default_opts(stall_checks=-2), rb.default_opts(max_seconds=-1.0),
                rb.default_opts(max_seconds=float("nan")), rb.default_opts(max_seconds=float("inf"))):
        assert lib.rbgs_create(4, 0.04, f.ctypes.data, u.ctypes.data, ctypes.byref(bad), None,
                               ctypes.byref(h)) == rb.RBGS_EINVAL
    vpa = ctypes.c_void_p * 1
    assert lib.rbgs_run_stream(None, 1, vpa(f.ctypes.data), vpa(u.ctypes.data), 1, vpa(u.ctypes.data),
                               None) == rb.RBGS_EINVAL
    # the 3D variant checks its arguments on the host too
    f3, u3 = np.zeros((2, 2, 2)), np.zeros((4, 4, 4))
    assert lib.rbgs3d_create(0, 0.1, f3.ctypes.data, u3.ctypes.data, None, ctypes.byref(h)) == rb.RBGS_EINVAL
    assert lib.rbgs3d_create(4096, 0.1, f3.ctypes.data, u3.ctypes.data, None, ctypes.byref(h)) == rb.RBGS_EINVAL
    assert lib.rbgs3d_create(2, -0.1, f3.ctypes.data, u3.ctypes.data, None, ctypes.byref(h)) == rb.RBGS_EINVAL
    assert lib.rbgs3d_create(2, 0.1, None, u3.ctypes.data, None, ctypes.byref(h)) == rb.RBGS_EINVAL
    assert lib.rbgs3d_sweep(None, 1) == rb.RBGS_EINVAL
    assert lib.rbgs3d_residual(None, None) == rb.RBGS_EINVAL
    assert lib.rbgs3d_get_solution(None, None) == rb.RBGS_EINVAL
    lib.rbgs3d_destroy(None)
    assert lib.rbgs_sweep(None, 1) == rb.RBGS_EINVAL
    assert lib.rbgs_residual(None, None) == rb.RBGS_EINVAL
    assert lib.rbgs_solve(None, 1e-8, None, None) == rb.RBGS_EINVAL
    assert lib.rbgs_get_solution(None, None) == rb.RBGS_EINVAL
    assert lib.rbgs_set_problem(None, None, None) == rb.RBGS_EINVAL
    lib.rbgs_destroy(None)  # ignored


def test_batched_argument_errors_without_gpu(lib):
    """rbgs_solve_batched checks its arguments on the host before any CUDA call."""
    f = np.zeros((4, 4))
    u = np.zeros((6, 6))
    out = np.zeros((6, 6))
    probs = (rb.Problem * 1)(rb.Problem(4, 0.04, f.ctypes.data, u.ctypes.data))
    outs = (ctypes.c_void_p * 1)(out.ctypes.data)
    res = (rb.Result * 1)()
    ok_args = (probs, 1e-8, None, None, outs, res)
    assert lib.rbgs_solve_batched(0, None, 1e-8, None, None, None, None) == rb.RBGS_OK  # nothing to do
    assert lib.rbgs_solve_batched(-1, *ok_args) == rb.RBGS_EINVAL
    assert lib.rbgs_solve_batched(1, None, 1e-8, None, None, outs, res) == rb.RBGS_EINVAL
    assert lib.rbgs_solve_batched(1, probs, 1e-8, None, None, None, res) == rb.RBGS_EINVAL
    assert lib.rbgs_solve_batched(1, probs, 1e-8, None, None, outs, None) == rb.RBGS_EINVAL
    assert lib.rbgs_solve_batched(1, probs, -1.0, None, None, outs, res) == rb.RBGS_EINVAL
    assert lib.rbgs_solve_batched(1, probs, float("nan"), None, None, outs, res) == rb.RBGS_EINVAL
    bad = rb.default_opts(precision=7)
    assert lib.rbgs_solve_batched(1, probs, 1e-8, ctypes.byref(bad), None, outs, res) == rb.RBGS_EINVAL
    for n, h2, fp, up in ((0, 0.04, f, u), (40000, 1e-9, f, u), (4, 0.0, f, u), (4, 0.04, None, u),
                          (4, 0.04, f, None)):
        bad_p = (rb.Problem * 1)(rb.Problem(n, h2, fp.ctypes.data if fp is not None else None,
                                            up.ctypes.data if up is not None else None))
        assert lib.rbgs_solve_batched(1, bad_p, 1e-8, None, None, outs, res) == rb.RBGS_EINVAL
        assert "problem 0" in rb.rbgs_last_error()
    null_out = (ctypes.c_void_p * 1)(None)
    assert lib.rbgs_solve_batched(1, probs, 1e-8, None, None, null_out, res) == rb.RBGS_EINVAL


def test_unet_and_conv_argument_errors_without_gpu(lib):
    """The convolution and network entry points check their arguments on the host."""
    vp, i32 = ctypes.c_void_p, ctypes.c_int
    buf = np.zeros(4096, dtype=np.uint16)
    base = buf.ctypes.data + (-buf.ctypes.data) % 16         # a 16-byte aligned address
    x, w, y = vp(base), vp(base + 1024), vp(base + 2048)

    def fwd(X, Wt, Y, B=1, H=8, W=8, cin=8, cout=8, ks=3):
        return lib.rbgs_conv_forward(X, Wt, None, Y, i32(B), i32(H), i32(W), i32(cin), i32(cout),
                                     i32(ks), i32(0), i32(0), None)

    assert fwd(None, w, y) == rb.RBGS_EINVAL
    assert fwd(x, None, y) == rb.RBGS_EINVAL
    assert fwd(x, w, None) == rb.RBGS_EINVAL
    assert fwd(x, w, y, cin=12) == rb.RBGS_EINVAL            # channels: multiples of 8
    assert fwd(x, w, y, cout=4) == rb.RBGS_EINVAL
    assert fwd(x, w, y, ks=2) == rb.RBGS_EINVAL              # 3x3 or 1x1 only
    assert fwd(x, w, y, B=0) == rb.RBGS_EINVAL
    assert fwd(vp(base + 2), w, y) == rb.RBGS_EINVAL         # operands 16-byte aligned
    assert "bad arguments" in rb.rbgs_last_error()
    dx = vp(base + 3072)
    # a data gradient needs the transposed-weight scratch
    assert lib.rbgs_conv_backward(x, w, y, dx, dx, None, None, i32(1), i32(8), i32(8), i32(8), i32(8),
                                  i32(3), i32(0), None) == rb.RBGS_EINVAL
    engine = lib.rbgs_conv_get_engine()
    assert lib.rbgs_conv_set_engine(i32(7)) == rb.RBGS_EINVAL
    assert lib.rbgs_conv_get_engine() == engine              # unchanged by a refused value
    kind = lib.rbgs_conv_get_wgrad_kernel()
    assert kind == 0                                         # RBGS_WGRAD_AUTO by default
    assert lib.rbgs_conv_set_wgrad_kernel(i32(4)) == rb.RBGS_EINVAL
    assert lib.rbgs_conv_set_wgrad_kernel(i32(-1)) == rb.RBGS_EINVAL
    assert lib.rbgs_conv_get_wgrad_kernel() == kind
    assert lib.rbgs_conv_set_wgrad_kernel(i32(2)) == rb.RBGS_OK
    assert lib.rbgs_conv_get_wgrad_kernel() == 2
    assert lib.rbgs_conv_set_wgrad_kernel(i32(0)) == rb.RBGS_OK
    assert lib.rbgs_unet_create(ctypes.c_uint64(1), None, None) == rb.RBGS_EINVAL
    lib.rbgs_unet_num_params.restype = ctypes.c_long
    assert lib.rbgs_unet_num_params(None) == 0
    p = vp(base)
    assert lib.rbgs_unet_get_params(None, p) == rb.RBGS_EINVAL
    assert lib.rbgs_unet_set_params(None, p) == rb.RBGS_EINVAL
    assert lib.rbgs_unet_forward(None, p, p, i32(1), i32(8), i32(8)) == rb.RBGS_EINVAL
    assert lib.rbgs_unet_train_step(None, p, p, p, i32(1), i32(8), i32(8), ctypes.c_float(1e-3), None,
                                    None) == rb.RBGS_EINVAL
    lib.rbgs_unet_destroy(None)  # ignored


def test_static_residual_binding_checks_sizes_without_gpu(lib):
    """The library cannot see buffer sizes; the binding refuses mismatched ones (and host
    arrays) before any call, so no kernel reads past a caller's allocation."""
    for f, u, out, word in ((np.zeros((3, 3)), np.zeros((6, 6)), np.zeros(1), "f holds 9"),
                            (np.zeros((4, 4)), np.zeros((4, 4)), np.zeros(1), "u holds 16"),
                            (np.zeros((4, 4)), np.zeros((6, 6)), np.zeros(0), "rel_out holds 0"),
                            (np.zeros((4, 4)), np.zeros((6, 6)), np.zeros(1), "CUDA tensors")):
        with pytest.raises(rb.RbgsError) as e:
            rb.rbgs_residual_static(4, 0.04, f, u, out)
        assert e.value.status == rb.RBGS_EINVAL and word in str(e.value)


def test_binding_rejects_wrong_dtypes(lib):
    with pytest.raises(TypeError):
        rb._ptr(np.zeros(4, dtype=np.float32))
    with pytest.raises(TypeError):
        rb._ptr(np.zeros((4, 4))[:, ::2])
